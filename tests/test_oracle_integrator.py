"""Pins of the oracle's kick-drift-kick leapfrog and energy diagnostics.

Kepler's two-body problem gives the exact orbit (Kepler's equation, solved
here by Newton iteration); the leapfrog must approach it at second order in dt.
Time reversibility, momentum conservation and the dt^2 scaling of the energy
error are properties of the KDK scheme itself.
"""
import math

import numpy as np
import pytest

import nbody_inputs as ni


def kepler_state(e, t, m0=0.4, m1=0.6, a_k=1.0):
    """Exact two-body positions at time t, started at pericentre on the x axis
    (G=1, mu = m0+m1), from the eccentric anomaly E - e sin E = n t."""
    mu = m0 + m1
    nmot = math.sqrt(mu / a_k ** 3)
    M = nmot * t
    E = M if e < 0.8 else math.pi
    for _ in range(100):
        dE = (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
        E -= dE
        if abs(dE) < 1e-16:
            break
    rel = np.array([a_k * (math.cos(E) - e), a_k * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    return np.stack([-m1 / mu * rel, m0 / mu * rel])


def kepler_initial(e, m0=0.4, m1=0.6, a_k=1.0):
    mu = m0 + m1
    rp = a_k * (1 - e)
    vp = math.sqrt(mu * (1 + e) / rp)
    rel = np.array([rp, 0.0, 0.0])
    vrel = np.array([0.0, vp, 0.0])
    pos = np.stack([-m1 / mu * rel, m0 / mu * rel])
    vel = np.stack([-m1 / mu * vrel, m0 / mu * vrel])
    return pos, vel, np.array([m0, m1])


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kepler_orbit_second_order(oracle_mod, e):
    """After one period the leapfrog orbit matches Kepler's equation, and the
    error drops by ~4x when dt halves."""
    pos0, vel0, m = kepler_initial(e)
    T = 2 * math.pi
    errs = []
    for nsteps in (2000, 4000):
        dt = T / nsteps
        t_end = 0.37 * T
        k = int(round(t_end / dt))
        p, v, _ = oracle_mod.leapfrog(pos0, vel0, m, 1e-9, dt, k)
        exact = kepler_state(e, k * dt)
        errs.append(np.abs(p - exact).max())
    assert errs[0] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_kepler_circular_force_closed_form(oracle_mod):
    """Circular binary: the force is mu/d^2 (eps -> 0) and the leapfrog keeps the
    separation constant to O(dt^2)."""
    pos0, vel0, m = kepler_initial(0.0)
    _, _, acc = oracle_mod.leapfrog(pos0, vel0, m, 1e-9, 0.01, 0)
    np.testing.assert_allclose(np.linalg.norm(acc[1]), m[0] / 1.0 ** 2, rtol=1e-12)
    p, v, _ = oracle_mod.leapfrog(pos0, vel0, m, 1e-9, 2 * math.pi / 1000, 1000)
    d = np.linalg.norm(p[1] - p[0])
    assert abs(d - 1.0) < 1e-4


def test_two_body_energy_closed_form(oracle_mod):
    pos = np.array([[0.1, 0.2, -0.3], [1.0, -0.5, 0.4]])
    vel = np.array([[0.3, -0.1, 0.2], [-0.2, 0.05, 0.1]])
    m = np.array([0.7, 0.2])
    eps = 0.1
    d2 = ((pos[1] - pos[0]) ** 2).sum()
    T = 0.5 * (m[:, None] * vel ** 2).sum()
    W = -m[0] * m[1] / math.sqrt(d2 + eps * eps)
    e = oracle_mod.energy(pos, vel, m, eps)
    np.testing.assert_allclose([e["T"], e["W"], e["E"]], [T, W, T + W], rtol=1e-15)
    np.testing.assert_allclose(e["P"], (m[:, None] * vel).sum(0), rtol=1e-15)


def test_energy_error_scales_as_dt2(oracle_mod):
    """Eccentric binary over a fixed time: max |dE| shrinks ~4x per halving of dt."""
    pos0, vel0, m = kepler_initial(0.6)
    E0 = oracle_mod.energy(pos0, vel0, m, 1e-9)["E"]
    res = []
    for nsteps in (400, 800):
        dt = 2 * math.pi / nsteps
        p, v = pos0.copy(), vel0.copy()
        worst = 0.0
        for _ in range(nsteps // 40):
            p, v, _ = oracle_mod.leapfrog(p, v, m, 1e-9, dt, 40)
            worst = max(worst, abs(oracle_mod.energy(p, v, m, 1e-9)["E"] - E0))
        res.append(worst)
    assert 3.3 < res[0] / res[1] < 4.7


def test_time_reversibility(oracle_mod):
    p0, v0, m = ni.plummer(64, 61)
    p1, v1, _ = oracle_mod.leapfrog(p0, v0, m, 0.05, 2.0 ** -7, 40)
    p2, v2, _ = oracle_mod.leapfrog(p1, -v1, m, 0.05, 2.0 ** -7, 40)
    np.testing.assert_allclose(p2, p0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-v2, v0, rtol=0, atol=1e-11)


def test_momentum_conserved_and_energy_bounded(oracle_mod):
    p0, v0, m = ni.plummer(256, 71, masses="loguniform")
    eps = 2.0 ** -5
    e0 = oracle_mod.energy(p0, v0, m, eps)
    p1, v1, _ = oracle_mod.leapfrog(p0, v0, m, eps, 2.0 ** -8, 64)
    e1 = oracle_mod.energy(p1, v1, m, eps)
    assert np.abs(e1["P"] - e0["P"]).max() < 1e-14
    assert abs(e1["E"] - e0["E"]) / abs(e0["E"]) < 1e-4


def test_zero_steps_is_identity(oracle_mod):
    p0, v0, m = ni.plummer(16, 81)
    p1, v1, a = oracle_mod.leapfrog(p0, v0, m, 0.01, 0.1, 0)
    assert np.array_equal(p1, p0) and np.array_equal(v1, v0)
    a2, _ = oracle_mod.accel(p0, m, 0.01)
    assert np.array_equal(a, a2)
