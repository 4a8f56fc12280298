"""Parity at the benchmark's full sizes, on outputs the oracle can compute one
by one (seeded subsamples), in the launch configuration the benchmark times
(default options: mixed precision, compensated sums, tuned kernel shape).

Precision workload: N = 2^20 Plummer sphere offset to (1e4,-3e3,7e2),
log-uniform masses in [1e-3, 1] renormalised to 1, eps = 2^-9, one force
evaluation plus 4 KDK steps with dt = 2^-9.  Throughput workload: N = 65536
equal-mass Plummer, eps = dt = 2^-8, FP32 state.
"""
import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu


def t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def rel(a, ref):
    return np.linalg.norm(np.asarray(a, np.float64) - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


@pytest.fixture(scope="module")
def c3():
    return ni.precision_offset()


def test_precision_workload_force(nb, oracle_mod, c3):
    import torch
    w = c3
    n = w.n
    m32 = w.mass.astype(np.float32)
    P, M = t(w.pos, np.float64), t(m32, np.float32)
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((n,), dtype=torch.float32, device="cuda")
    nb.nbody_accel(P, M, w.eps, acc, pot)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    idx = w.extra["subsample"]
    ra, rp = oracle_mod.accel_subset(w.pos, w.mass, w.eps, idx)
    e = rel(acc.cpu().numpy()[idx], ra)
    ep = np.abs(pot.cpu().numpy()[idx] - rp) / np.abs(rp)
    print(f"mixed N=2^20: median {np.median(e):.3g} max {e.max():.3g} pot max {ep.max():.3g}")
    assert np.median(e) <= 2e-6 and e.max() <= 1e-4
    assert ep.max() <= 1e-5
    # without the potential: the kernel shape the benchmark's leapfrog runs
    nb.nbody_accel(P, M, w.eps, acc, None)
    torch.cuda.synchronize()
    e_np = rel(acc.cpu().numpy()[idx], ra)
    print(f"mixed N=2^20 no potential: median {np.median(e_np):.3g} max {e_np.max():.3g}")
    assert np.median(e_np) <= 2e-6 and e_np.max() <= 1e-4
    # one FP32 running sum over 2^20 terms instead of per-tile compensation
    nb.nbody_accel(P, M, w.eps, acc, None, accumulate=nb.NBODY_ACC_FP32)
    torch.cuda.synchronize()
    e_fp32 = rel(acc.cpu().numpy()[idx], ra)
    print(f"fp32 running sum N=2^20: median {np.median(e_fp32):.3g} max {e_fp32.max():.3g}")
    assert np.median(e_fp32) > 2 * np.median(e)
    # plain FP32 absolute coordinates, same launch otherwise: fails by design
    nb.nbody_accel(P, M, w.eps, acc, None, precision=nb.NBODY_PREC_PLAIN)
    torch.cuda.synchronize()
    e_plain = rel(acc.cpu().numpy()[idx], ra)
    print(f"plain N=2^20: median {np.median(e_plain):.3g} max {e_plain.max():.3g}")
    assert np.median(e_plain) > 50 * 2e-6 and e_plain.max() > 1e-2  # misses the target by >50x


def test_precision_workload_steps(nb, oracle_mod, c3):
    """Four KDK steps at N=2^20, each checked from the GPU's own state on a
    512-body sample: v_{k+1} = v_k + dt/2 (a(x_k) + a(x_{k+1})) and
    x_{k+1} = x_k + dt (v_k + dt/2 a(x_k)) with the oracle's a on the sample.
    Then the 4-step call (merged kicks, the benchmark's launch) reproduces the
    four single steps."""
    import torch
    w = c3
    m32 = w.mass.astype(np.float32)
    M = t(m32, np.float32)
    idx = ni.subsample(w.n, 512, 33)
    x = w.pos.copy()
    v = w.vel.copy()
    a_prev, _ = oracle_mod.accel_subset(x, w.mass, w.eps, idx, with_pot=False)
    P, V = t(x, np.float64), t(v, np.float64)
    kicks = np.zeros(len(idx))  # sum over the steps of |dt/2 (a_k + a_{k+1})| on the sample
    for k in range(w.steps):
        nb.nbody_leapfrog(P, V, M, w.eps, w.dt, 1)
        torch.cuda.synchronize()
        x1, v1 = P.cpu().numpy(), V.cpu().numpy()
        a_next, _ = oracle_mod.accel_subset(x1, w.mass, w.eps, idx, with_pot=False)
        x_pred = x[idx] + w.dt * (v[idx] + 0.5 * w.dt * a_prev)
        v_pred = v[idx] + 0.5 * w.dt * (a_prev + a_next)
        kick = 0.5 * w.dt * np.linalg.norm(a_prev + a_next, axis=1)
        kicks += kick
        ev = np.linalg.norm(v1[idx] - v_pred, axis=1) / kick
        assert np.median(ev) <= 2e-6 and ev.max() <= 1e-4, (k, np.median(ev), ev.max())
        assert np.abs(x1[idx] - x_pred).max() <= 1e-9
        x, v, a_prev = x1, v1, a_next
    P4, V4 = t(w.pos, np.float64), t(w.vel, np.float64)
    nb.nbody_leapfrog(P4, V4, M, w.eps, w.dt, w.steps)
    torch.cuda.synchronize()
    # Each one-step call took its own Morton order and cell centres from its
    # starting positions; the 4-step call keeps one order and centres its cells
    # on the positions one step earlier.  The two runs differ only by the FP32
    # rounding of their packed offsets: on the sample, within twice the
    # per-step tolerance relative to the velocity change (two results, each
    # within it of the exact one).
    assert np.abs(P4.cpu().numpy() - x).max() <= 1e-9
    d4 = np.linalg.norm(V4.cpu().numpy()[idx] - v[idx], axis=1) / kicks
    assert np.median(d4) <= 4e-6 and d4.max() <= 2e-4, (np.median(d4), d4.max())
    assert nb.nbody_last_device_error() == 0


def test_throughput_workload_energy(nb, oracle_mod):
    """N=65536 FP32-state run: energy after 4 steps agrees with the oracle's
    4-step run to 1e-5 relative."""
    import torch
    w = ni.throughput_plain()
    m32 = w.mass.astype(np.float32)
    P, V, M = t(w.pos, np.float32), t(w.vel, np.float32), t(m32, np.float32)
    nb.nbody_leapfrog_f32(P, V, M, np.float32(w.eps), np.float32(w.dt), 4)
    torch.cuda.synchronize()
    p_ref, v_ref, _ = oracle_mod.leapfrog(w.pos, w.vel, w.mass, w.eps, w.dt, 4)
    e0 = oracle_mod.energy(w.pos, w.vel, w.mass, w.eps)["E"]
    e_ref = oracle_mod.energy(p_ref, v_ref, w.mass, w.eps)["E"]
    e_dev = nb.nbody_energy_f32(P, V, M, np.float32(w.eps))["E"]
    assert abs(e_dev - e_ref) <= 1e-5 * abs(e0)
    assert np.abs(P.cpu().numpy() - p_ref).max() <= 1e-5


def test_four_million_bodies(nb, oracle_mod):
    """Beyond the benchmark's size: N = 2^22 + 777 (a ragged last cell) with the
    precision recipe (offset centre, log-uniform masses), one mixed-precision
    force evaluation with the potential and one leapfrog step, checked on 512
    seeded bodies against the oracle: the 64-bit indexing of the grids, the
    Morton order and the result stores at 4.2 million bodies."""
    import torch
    n = (1 << 22) + 777
    p, v, m = ni.plummer(n, 31, masses="loguniform", offset=ni.plummer_offset())
    m32 = m.astype(np.float32)
    P, M = t(p, np.float64), t(m32, np.float32)
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((n,), dtype=torch.float32, device="cuda")
    nb.nbody_accel(P, M, 2.0 ** -9, acc, pot)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    idx = ni.subsample(n, 512, 32)
    ra, rp = oracle_mod.accel_subset(p, m32.astype(np.float64), 2.0 ** -9, idx)
    e = rel(acc.cpu().numpy()[idx], ra)
    ep = np.abs(pot.cpu().numpy()[idx] - rp) / np.abs(rp)
    assert np.median(e) <= 2e-6 and e.max() <= 1e-4, (np.median(e), e.max())
    assert ep.max() <= 1e-5
    V = t(v, np.float64)
    nb.nbody_leapfrog(P, V, M, 2.0 ** -9, 2.0 ** -9, 1)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    # one KDK step: x1 = x0 + dt v0 + dt^2/2 a(x0), so the sampled bodies moved
    # as their oracle accelerations say, to the accelerations' accuracy and a
    # few FP64 ulps of the offset coordinates
    x1 = P.cpu().numpy()[idx]
    h2 = 0.5 * 2.0 ** -18
    expect = p[idx] + 2.0 ** -9 * v[idx] + h2 * ra
    tol = h2 * 2e-4 * np.linalg.norm(ra, axis=1)[:, None] + 8 * np.spacing(np.abs(p[idx]))
    assert np.all(np.abs(x1 - expect) <= tol)
