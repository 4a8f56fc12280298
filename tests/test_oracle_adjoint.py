"""Pins of the oracle's reverse-mode derivatives (force VJP and leapfrog adjoint)
against central finite differences of the oracle's own forward functions, a
hand-derived two-body Jacobian and translation invariance."""
import numpy as np
import pytest

import nbody_inputs as ni


def test_two_body_jacobian_closed_form(oracle_mod):
    """Bodies 0 at the origin and 1 at (d,0,0): a_0 = m_1 (d,0,0)/s^{3/2}, so
    d(lam.a_0)/dr_1 = m_1 T lam with T = diag(s^-3/2 - 3 d^2 s^-5/2, s^-3/2, s^-3/2),
    and d(lam.a_0)/dm_1 = lam.(d,0,0) s^-3/2."""
    d, m0, m1, eps = 0.8, 0.3, 1.7, 0.2
    s = d * d + eps * eps
    pos = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
    mass = np.array([m0, m1])
    lam = np.array([[0.4, -1.1, 0.7], [0.0, 0.0, 0.0]])
    g, gm = oracle_mod.accel_vjp(pos, mass, eps, lam)
    T = np.diag([s ** -1.5 - 3 * d * d * s ** -2.5, s ** -1.5, s ** -1.5])
    np.testing.assert_allclose(g[1], m1 * T @ lam[0], rtol=1e-14)
    np.testing.assert_allclose(g[0], -m1 * T @ lam[0], rtol=1e-14)
    np.testing.assert_allclose(gm[1], lam[0, 0] * d * s ** -1.5, rtol=1e-14)
    assert gm[0] == 0.0


@pytest.mark.parametrize("with_mu", [False, True])
def test_force_vjp_matches_finite_differences(oracle_mod, with_mu):
    n, eps, h = 9, 0.07, 1e-6
    p, _, m = ni.plummer(n, 300, masses="loguniform")
    lam = ni.gaussian((n, 3), 301)
    mu = ni.gaussian((n,), 302) if with_mu else None

    def L(pos, mass):
        a, phi = oracle_mod.accel(pos, mass, eps)
        return float((lam * a).sum() + ((mu * phi).sum() if with_mu else 0.0))

    g, gm = oracle_mod.accel_vjp(p, m, eps, lam, mu)
    for k in range(n):
        for c in range(3):
            pp, pm = p.copy(), p.copy()
            pp[k, c] += h
            pm[k, c] -= h
            fd = (L(pp, m) - L(pm, m)) / (2 * h)
            assert abs(fd - g[k, c]) <= 1e-6 * max(1.0, abs(g).max())
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (L(p, mp) - L(p, mm)) / (2 * h)
        assert abs(fd - gm[k]) <= 1e-6 * max(1.0, abs(gm).max())


def test_force_vjp_translation_invariance(oracle_mod):
    """The force depends on differences only, so the position gradients of any
    cotangent sum to zero."""
    n = 200
    p, _, m = ni.plummer(n, 310, masses="loguniform")
    g, _ = oracle_mod.accel_vjp(p, m, 0.01, ni.gaussian((n, 3), 311), ni.gaussian((n,), 312))
    assert np.abs(g.sum(axis=0)).max() <= 1e-10 * np.abs(g).sum()


def test_leapfrog_adjoint_matches_finite_differences(oracle_mod):
    """L = sum_i m_i |x_i(T) - y_i|^2 + c.v(T) over 20 KDK steps: every
    coordinate of dL/dx0, dL/dv0 and the dynamics part of dL/dm against central
    differences of the oracle's forward leapfrog (the direct mass term of L is
    added on both sides)."""
    n, K, eps, dt, h = 7, 20, 0.05, 2.0 ** -6, 1e-6
    p0, v0, m = ni.plummer(n, 320, masses="loguniform")
    y = p0 + ni.gaussian((n, 3), 321, 0.05)
    c = ni.gaussian((n, 3), 322)

    def L(x0, v0_, mass):
        xT, vT, _ = oracle_mod.leapfrog(x0, v0_, mass, eps, dt, K)
        return float((mass[:, None] * (xT - y) ** 2).sum() + (c * vT).sum())

    xT, vT, _ = oracle_mod.leapfrog(p0, v0, m, eps, dt, K)
    gx, gv, gm = oracle_mod.leapfrog_vjp(p0, v0, m, eps, dt, K, 2 * m[:, None] * (xT - y), c)
    gm = gm + ((xT - y) ** 2).sum(axis=1)
    scale = max(abs(gx).max(), abs(gv).max(), abs(gm).max())
    for k in range(n):
        for comp in range(3):
            for arr, grad in ((0, gx), (1, gv)):
                a0, a1 = p0.copy(), v0.copy()
                b0, b1 = p0.copy(), v0.copy()
                (a0 if arr == 0 else a1)[k, comp] += h
                (b0 if arr == 0 else b1)[k, comp] -= h
                fd = (L(a0, a1, m) - L(b0, b1, m)) / (2 * h)
                assert abs(fd - grad[k, comp]) <= 1e-6 * scale, (arr, k, comp, fd, grad[k, comp])
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (L(p0, v0, mp) - L(p0, v0, mm)) / (2 * h)
        assert abs(fd - gm[k]) <= 1e-6 * scale


def test_leapfrog_adjoint_zero_steps(oracle_mod):
    p0, v0, m = ni.plummer(5, 330)
    gxT = ni.gaussian((5, 3), 331)
    gvT = ni.gaussian((5, 3), 332)
    gx, gv, gm = oracle_mod.leapfrog_vjp(p0, v0, m, 0.1, 0.01, 0, gxT, gvT)
    assert np.array_equal(gx, gxT) and np.array_equal(gv, gvT) and np.all(gm == 0)
