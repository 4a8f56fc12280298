"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test fixes a case whose answer follows from geometry, a closed form, a
conservation law or an independent high-precision evaluation, chosen so that a
plausible slip in the oracle (a dropped term, a sign, a wrong exponent, a
transposed index, the self term kept) fails at least one of them.  Eq. 1 of
Miki & Hanawa (Sec. III.A) is the force law; the potential is the negative
softened potential with the self term removed.
"""
import math

import numpy as np
import pytest

import nbody_inputs as ni


def rot(seed):
    """A fixed proper rotation (QR of a seeded matrix)."""
    g = ni.gaussian((3, 3), seed)
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("eps", [0.0, 0.05, 0.7])
def test_two_body_closed_form(oracle_mod, eps):
    """Two bodies at separation d along a rotated axis: |a_0| = m_1 d/(d^2+eps^2)^{3/2}
    toward body 1, a_1 = -(m_0/m_1) a_0 direction-reversed, phi_0 = -m_1/sqrt(d^2+eps^2)."""
    R = rot(11)
    d, m0, m1 = 1.7, 0.3, 0.9
    u = R @ np.array([1.0, 0.0, 0.0])
    x0 = np.array([0.2, -0.4, 1.1])
    pos = np.stack([x0, x0 + d * u])
    mass = np.array([m0, m1])
    acc, pot = oracle_mod.accel(pos, mass, eps)
    s = d * d + eps * eps
    np.testing.assert_allclose(acc[0], m1 * d / s ** 1.5 * u, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(acc[1], -m0 * d / s ** 1.5 * u, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(pot, [-m1 / math.sqrt(s), -m0 / math.sqrt(s)], rtol=1e-14)


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_cube_vertices_and_centre(oracle_mod, eps):
    """Unit cube of 8 equal masses m plus a centre body of mass mc.

    Centre: zero force by symmetry.  Vertex at the origin: its 3 edge, 3
    face-diagonal and 1 body-diagonal neighbours each pull along (1,1,1), giving
    per component m[(1+e2)^-3/2 + 2(2+e2)^-3/2 + (3+e2)^-3/2] + mc/2 (3/4+e2)^-3/2,
    and potential -m[3(1+e2)^-1/2 + 3(2+e2)^-1/2 + (3+e2)^-1/2] - mc (3/4+e2)^-1/2.
    """
    m, mc = 0.125, 0.4
    e2 = eps * eps
    verts = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    pos = np.vstack([verts, [[0.5, 0.5, 0.5]]])
    mass = np.array([m] * 8 + [mc])
    acc, pot = oracle_mod.accel(pos, mass, eps)
    comp = m * ((1 + e2) ** -1.5 + 2 * (2 + e2) ** -1.5 + (3 + e2) ** -1.5) + mc * 0.5 * (0.75 + e2) ** -1.5
    phiv = -m * (3 * (1 + e2) ** -0.5 + 3 * (2 + e2) ** -0.5 + (3 + e2) ** -0.5) - mc * (0.75 + e2) ** -0.5
    np.testing.assert_allclose(acc[0], [comp, comp, comp], rtol=1e-14)
    # every vertex is pulled toward the centre with the same magnitude
    toward = 0.5 - verts
    np.testing.assert_allclose(acc[:8], 2 * comp * toward, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(acc[8], 0.0, atol=1e-15)
    np.testing.assert_allclose(pot[:8], phiv, rtol=1e-14)
    np.testing.assert_allclose(pot[8], -8 * m * (0.75 + e2) ** -0.5, rtol=1e-14)


@pytest.mark.parametrize("k", [3, 7, 12])
def test_regular_polygon_ring(oracle_mod, k):
    """k equal masses on a circle of radius R around a central mass: the centre
    feels no force; each ring body is pulled radially inward by
    mc R/(R^2+e2)^{3/2} + sum_l m 2R sin^2(pi l/k) / (4R^2 sin^2(pi l/k) + e2)^{3/2}."""
    R, m, mc, eps = 1.3, 0.01, 1.0, 0.02
    e2 = eps * eps
    th = 2 * math.pi * np.arange(k) / k
    ring = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(k)], axis=1)
    pos = np.vstack([ring, [[0.0, 0.0, 0.0]]]) @ rot(5).T + np.array([3.0, -2.0, 0.5])
    mass = np.array([m] * k + [mc])
    acc, _ = oracle_mod.accel(pos, mass, eps)
    s = np.sin(math.pi * np.arange(1, k) / k)
    mag = mc * R / (R * R + e2) ** 1.5 + np.sum(m * 2 * R * s * s / (4 * R * R * s * s + e2) ** 1.5)
    centre = pos[k]
    for i in range(k):
        inward = (centre - pos[i]) / np.linalg.norm(centre - pos[i])
        np.testing.assert_allclose(acc[i], mag * inward, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(acc[k], 0.0, atol=1e-15)


# ---------------------------------------------------------------- invariants
def test_newton_third_law(oracle_mod):
    """sum_i m_i a_i = 0 for any configuration (pairwise-antisymmetric forces)."""
    p, v, m = ni.plummer(777, 21, masses="loguniform")
    acc, _ = oracle_mod.accel(p, m, 2.0 ** -7)
    net = (m[:, None] * acc).sum(axis=0)
    scale = np.abs(m[:, None] * acc).sum()
    assert np.all(np.abs(net) <= 1e-14 * scale)


def test_potential_is_force_potential(oracle_mod):
    """a_i = -(1/m_i) dW/dr_i with W = (1/2) sum m_i phi_i: central differences of
    the oracle's W reproduce its force (exponents and signs of both agree)."""
    p, v, m = ni.plummer(24, 31, masses="loguniform")
    eps = 0.05
    acc, _ = oracle_mod.accel(p, m, eps)
    h = 1e-5
    for i in (0, 5, 23):
        for c in range(3):
            pp = p.copy(); pp[i, c] += h
            pm = p.copy(); pm[i, c] -= h
            Wp = oracle_mod.energy(pp, v, m, eps)["W"]
            Wm = oracle_mod.energy(pm, v, m, eps)["W"]
            fd = -(Wp - Wm) / (2 * h) / m[i]
            assert abs(fd - acc[i, c]) <= 1e-6 * np.abs(acc[i]).max()


def test_translation_rotation_permutation(oracle_mod):
    p, v, m = ni.plummer(200, 41, masses="loguniform")
    eps = 2.0 ** -7
    a0, f0 = oracle_mod.accel(p, m, eps)
    # rigid translation by the precision workload's offset
    a1, f1 = oracle_mod.accel(p + np.array([1e4, -3e3, 7e2]), m, eps)
    np.testing.assert_allclose(a1, a0, rtol=0, atol=1e-8 * np.abs(a0).max())
    np.testing.assert_allclose(f1, f0, rtol=1e-10)
    # rotation: a(Rx) = R a(x); phi invariant
    R = rot(3)
    a2, f2 = oracle_mod.accel(p @ R.T, m, eps)
    np.testing.assert_allclose(a2, a0 @ R.T, rtol=0, atol=1e-12 * np.abs(a0).max())
    np.testing.assert_allclose(f2, f0, rtol=1e-12)
    # permutation: outputs permute with the bodies
    perm = np.argsort(ni.gaussian((200,), 9))
    a3, f3 = oracle_mod.accel(p[perm], m[perm], eps)
    np.testing.assert_allclose(a3, a0[perm], rtol=0, atol=1e-13 * np.abs(a0).max())
    np.testing.assert_allclose(f3, f0[perm], rtol=1e-13)


def test_self_term_excluded(oracle_mod):
    """A lone body feels nothing; two coincident bodies (eps>0) exert no force
    and potential -m/eps on each other; a massless body feels but exerts nothing."""
    a, f = oracle_mod.accel(np.array([[1.0, 2.0, 3.0]]), np.array([5.0]), 0.1)
    assert np.all(a == 0) and np.all(f == 0)
    pos = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]])
    a, f = oracle_mod.accel(pos, np.array([2.0, 3.0]), 0.25)
    assert np.all(a == 0)
    np.testing.assert_allclose(f, [-3.0 / 0.25, -2.0 / 0.25], rtol=1e-15)
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    a_with, f_with = oracle_mod.accel(pos, np.array([1.0, 0.5, 0.0]), 0.0)
    a_wo, f_wo = oracle_mod.accel(pos[:2], np.array([1.0, 0.5]), 0.0)
    np.testing.assert_allclose(a_with[:2], a_wo, rtol=1e-15)
    np.testing.assert_allclose(f_with[:2], f_wo, rtol=1e-15)
    assert np.linalg.norm(a_with[2]) > 0


def test_bruteforce_high_precision(oracle_mod):
    """N <= 8: an independent 40-digit evaluation with mpmath of each pair term."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for n, seed in ((2, 1), (5, 2), (8, 3)):
        p, v, m = ni.plummer(n, 100 + seed, masses="loguniform")
        eps = 0.01 * seed
        acc, pot = oracle_mod.accel(p, m, eps)
        for i in range(n):
            ai = [mp.mpf(0)] * 3
            phi = mp.mpf(0)
            for j in range(n):
                if j == i:
                    continue
                d = [mp.mpf(p[j, c]) - mp.mpf(p[i, c]) for c in range(3)]
                s = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + mp.mpf(eps) ** 2
                ai = [ai[c] + mp.mpf(m[j]) * d[c] / s ** mp.mpf(1.5) for c in range(3)]
                phi -= mp.mpf(m[j]) / mp.sqrt(s)
            scale = max(abs(float(x)) for x in ai)
            for c in range(3):
                assert abs(acc[i, c] - float(ai[c])) <= 1e-14 * scale
            assert abs(pot[i] - float(phi)) <= 1e-14 * abs(float(phi))


def test_subset_matches_full_bitwise(oracle_mod):
    p, v, m = ni.plummer(300, 51, masses="loguniform")
    idx = ni.subsample(300, 37, 5)
    a, f = oracle_mod.accel(p, m, 0.01)
    a2, f2 = oracle_mod.accel_subset(p, m, 0.01, idx)
    assert np.array_equal(a[idx], a2) and np.array_equal(f[idx], f2)


# ---------------------------------------------------------------- Plummer statistics
def _trunc_plummer():
    from scipy.integrate import quad
    a = ni.PLUMMER_A
    R = 10 * a
    Mr = lambda r: r ** 3 / (r * r + a * a) ** 1.5
    MR = Mr(R)
    dM = lambda r: 3 * a * a * r * r / (r * r + a * a) ** 2.5
    W = -quad(lambda r: (Mr(r) / MR) * (dM(r) / MR) / r, 0, R, limit=200)[0]
    return W, (lambda r: Mr(r) / MR)


def test_plummer_potential_energy_and_mean_field(oracle_mod):
    """Sampled Plummer sphere (truncated at 10a, renormalised to M=1): the
    oracle's W matches the continuum integral -int M(r) dM / r, the sphere is
    near virial equilibrium, and the mean radial force in shells matches
    -M(<r)/r^2 (Newton's shell theorem)."""
    pytest.importorskip("scipy")
    Wc, Mfrac = _trunc_plummer()
    n = 16384
    p, v, m = ni.plummer(n, 7)
    e = oracle_mod.energy(p, v, m, 1e-5)
    assert abs(e["W"] - Wc) <= 0.02 * abs(Wc)
    assert 0.95 <= 2 * e["T"] / abs(e["W"]) <= 1.02
    acc, _ = oracle_mod.accel(p, m, 1e-5, with_pot=False)
    r = np.linalg.norm(p, axis=1)
    ar = -(acc * p).sum(axis=1) / r
    a = ni.PLUMMER_A
    for lo, hi in ((0.3 * a, 0.7 * a), (0.7 * a, 1.5 * a), (1.5 * a, 3 * a)):
        sel = (r > lo) & (r < hi)
        ratio = np.mean(ar[sel] / (Mfrac(r[sel]) / r[sel] ** 2))
        assert abs(ratio - 1) < 0.03


# ---------------------------------------------------------------- sinks and sources
def test_sink_source_split(oracle_mod):
    """Listing 4's form (separate sinks and sources, no pair excluded): linear in
    the sources; one source gives the two-body closed form; sinks taken from the
    sources agree with the self-excluding sum except for the self pair's -m_i/eps
    in the potential."""
    p, _, m = ni.plummer(400, 90, masses="loguniform")
    sinks = p[ni.subsample(400, 50, 91)] + 0.01
    a12, f12 = oracle_mod.accel_ij(sinks, p, m, 0.03)
    a1, f1 = oracle_mod.accel_ij(sinks, p[:150], m[:150], 0.03)
    a2, f2 = oracle_mod.accel_ij(sinks, p[150:], m[150:], 0.03)
    np.testing.assert_allclose(a12, a1 + a2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(f12, f1 + f2, rtol=1e-12)
    d = np.array([0.3, -0.4, 1.2])
    a, f = oracle_mod.accel_ij(np.zeros((1, 3)), d[None, :], np.array([2.5]), 0.1)
    s = d @ d + 0.01
    np.testing.assert_allclose(a[0], 2.5 * d / s ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(f[0], -2.5 / s ** 0.5, rtol=1e-14)
    idx = ni.subsample(400, 30, 92)
    aij, fij = oracle_mod.accel_ij(p[idx], p, m, 0.03)
    asub, fsub = oracle_mod.accel_subset(p, m, 0.03, idx)
    np.testing.assert_allclose(aij, asub, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(fij, fsub - m[idx] / 0.03, rtol=1e-12)
