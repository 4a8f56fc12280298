"""GPU leapfrog against the oracle's leapfrog, and one-step checks from the
GPU's own state where a full oracle trajectory would be too slow."""
import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu


def t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def test_small_plain_16_steps(nb, oracle_mod):
    """N=1024 equal-mass Plummer, eps=dt=2^-7, 16 KDK steps with FP32 state:
    positions track the FP64 oracle and the energy agrees to 1e-5."""
    import torch
    w = ni.small_plain()
    m32 = w.mass.astype(np.float32)
    P, V = t(w.pos, np.float32), t(w.vel, np.float32)
    nb.nbody_leapfrog_f32(P, V, t(m32, np.float32), np.float32(w.eps), np.float32(w.dt), w.steps)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    p_ref, v_ref, _ = oracle_mod.leapfrog(w.pos, w.vel, w.mass, w.eps, w.dt, w.steps)
    pg, vg = P.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    assert np.abs(pg - p_ref).max() <= 2e-5
    assert np.abs(vg - v_ref).max() <= 2e-4
    e0 = oracle_mod.energy(w.pos, w.vel, w.mass, w.eps)["E"]
    e_ref = oracle_mod.energy(p_ref, v_ref, w.mass, w.eps)["E"]
    e_gpu = oracle_mod.energy(pg, vg, w.mass, w.eps)["E"]
    assert abs(e_gpu - e_ref) <= 1e-5 * abs(e0)
    e_dev = nb.nbody_energy_f32(P, V, t(m32, np.float32), np.float32(w.eps))["E"]
    assert abs(e_dev - e_ref) <= 1e-5 * abs(e0)


@pytest.mark.parametrize("prec", ["mixed", "plain"])
def test_fp64_state_trajectory(nb, oracle_mod, prec):
    import torch
    p, v, m = ni.plummer(3000, 12, masses="loguniform")
    m32 = m.astype(np.float32)
    eps, dt, steps = 2.0 ** -7, 2.0 ** -8, 8
    P, V = t(p, np.float64), t(v, np.float64)
    pr = nb.NBODY_PREC_MIXED if prec == "mixed" else nb.NBODY_PREC_PLAIN
    nb.nbody_leapfrog(P, V, t(m32, np.float32), eps, dt, steps, precision=pr)
    torch.cuda.synchronize()
    p_ref, v_ref, _ = oracle_mod.leapfrog(p, v, m32.astype(np.float64), eps, dt, steps)
    vs = np.abs(v_ref).max()
    assert np.abs(P.cpu().numpy() - p_ref).max() <= 1e-8 * 8
    assert np.abs(V.cpu().numpy() - v_ref).max() <= 1e-6 * vs


def test_steps_compose(nb):
    """One call of k steps equals k calls of one step (FP64 state) up to the
    FP32 rounding of the packed offsets.  Besides the merged kick's rounding,
    the calls differ in the FP64 centres the offsets are taken from: the first
    pack of a call centres each cell on its current positions, the later packs
    of a call on its positions one step earlier; and the default Morton order
    is taken afresh by each call from its own starting positions, so bodies
    that changed cells round their offsets differently.  Either moves the
    force of a body with a very close neighbour by up to ~1e-5 of itself,
    times dt."""
    import torch
    p, v, m = ni.plummer(2000, 13)
    m32 = t(m.astype(np.float32), np.float32)
    for prec in (nb.NBODY_PREC_MIXED_UNSORTED, nb.NBODY_PREC_MIXED):
        P1, V1 = t(p, np.float64), t(v, np.float64)
        P2, V2 = t(p, np.float64), t(v, np.float64)
        nb.nbody_leapfrog(P1, V1, m32, 0.01, 2.0 ** -8, 4, precision=prec)
        for _ in range(4):
            nb.nbody_leapfrog(P2, V2, m32, 0.01, 2.0 ** -8, 1, precision=prec)
        torch.cuda.synchronize()
        dx = float((P1 - P2).abs().max())
        dv = float((V1 - V2).abs().max())
        assert dx <= 1e-8 and dv <= 1e-6, (prec, dx, dv)


def test_zero_steps_and_momentum(nb):
    import torch
    p, v, m = ni.plummer(1500, 14, masses="loguniform")
    m32 = m.astype(np.float32)
    P, V = t(p, np.float64), t(v, np.float64)
    nb.nbody_leapfrog(P, V, t(m32, np.float32), 0.01, 0.01, 0)
    torch.cuda.synchronize()
    assert np.array_equal(P.cpu().numpy(), p) and np.array_equal(V.cpu().numpy(), v)
    mom0 = (m32[:, None].astype(np.float64) * v).sum(0)
    nb.nbody_leapfrog(P, V, t(m32, np.float32), 0.01, 2.0 ** -8, 16)
    torch.cuda.synchronize()
    mom1 = (m32[:, None].astype(np.float64) * V.cpu().numpy()).sum(0)
    # sum m a vanishes up to FP32 pair rounding: drift stays tiny
    assert np.abs(mom1 - mom0).max() <= 1e-7


def test_host_state_roundtrip(nb):
    """Host (numpy) state is staged through the device and written back."""
    import torch
    p, v, m = ni.plummer(1024, 15)
    m32 = m.astype(np.float32)
    ph, vh = p.copy(), v.copy()
    nb.nbody_leapfrog(ph, vh, m32, 0.01, 2.0 ** -8, 3)
    P, V = t(p, np.float64), t(v, np.float64)
    nb.nbody_leapfrog(P, V, t(m32, np.float32), 0.01, 2.0 ** -8, 3)
    torch.cuda.synchronize()
    assert np.array_equal(ph, P.cpu().numpy()) and np.array_equal(vh, V.cpu().numpy())


@pytest.mark.parametrize("n", [1024, 20011, 65536])
def test_chained_launches_repeatable(nb, n):
    """The kernels of a step are chained by programmatic dependent launch, so
    each may start before its predecessor finishes; whatever the timing, the
    same call gives the same bits (five device runs from fresh arrays, one
    host run).  Reading the chain's data through the read-only path instead of
    L2 once made these runs differ.  The sizes take the pack variant for fewer
    CTAs than SMs (1024, 20011) and the one for more (65536)."""
    import torch
    p, v, m = ni.plummer(n, 16, masses="loguniform")
    m32 = m.astype(np.float32)
    runs = []
    for _ in range(5):
        P, V = t(p, np.float64), t(v, np.float64)
        nb.nbody_leapfrog(P, V, t(m32, np.float32), 2.0 ** -8, 2.0 ** -8, 3)
        torch.cuda.synchronize()
        runs.append((P.cpu().numpy(), V.cpu().numpy()))
    ph, vh = p.copy(), v.copy()
    nb.nbody_leapfrog(ph, vh, m32, 2.0 ** -8, 2.0 ** -8, 3)
    runs.append((ph, vh))
    assert nb.nbody_last_device_error() == 0
    for k, (pk_, vk_) in enumerate(runs[1:], 1):
        assert np.array_equal(pk_, runs[0][0]) and np.array_equal(vk_, runs[0][1]), k


def test_kepler_orbit_second_order(nb):
    """Eccentric binary (e=0.5, FP64 state) after 0.37 of a period matches
    Kepler's equation, with the error falling ~4x per halving of dt: the FP32
    force error stays far below the integrator's."""
    import math
    import torch
    from test_oracle_integrator import kepler_initial, kepler_state
    pos0, vel0, m = kepler_initial(0.5)
    T = 2 * math.pi
    errs = []
    for nsteps in (2000, 4000):
        dt = T / nsteps
        k = int(round(0.37 * T / dt))
        P, V = t(pos0, np.float64), t(vel0, np.float64)
        nb.nbody_leapfrog(P, V, t(m.astype(np.float32), np.float32), 1e-9, dt, k)
        torch.cuda.synchronize()
        errs.append(np.abs(P.cpu().numpy() - kepler_state(0.5, k * dt)).max())
    assert errs[0] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_repeated_calls_replay_a_cuda_graph(nb):
    """The second identical call is captured into a CUDA graph that later calls
    launch; the results stay bit-identical to direct launches (the tape-recording
    call never uses graphs)."""
    import torch
    p, v, m = ni.plummer(3000, 17, masses="loguniform")
    m32 = t(m.astype(np.float32), np.float32)
    P1, V1 = t(p, np.float64), t(v, np.float64)
    P2, V2 = t(p, np.float64), t(v, np.float64)
    tape = torch.empty(nb.nbody_tape_bytes(3000, 3, 3), dtype=torch.uint8, device="cuda")
    for _ in range(5):
        nb.nbody_leapfrog(P1, V1, m32, 0.01, 2.0 ** -8, 3)
        nb.nbody_leapfrog_record(P2, V2, m32, 0.01, 2.0 ** -8, 3, 3, tape)
    torch.cuda.synchronize()
    assert torch.equal(P1, P2) and torch.equal(V1, V2)
    # FP32 state as well
    Q1, W1 = t(p, np.float32), t(v, np.float32)
    Q2, W2 = t(p, np.float32), t(v, np.float32)
    for _ in range(4):
        nb.nbody_leapfrog_f32(Q1, W1, m32, 0.01, 2.0 ** -8, 2)
    nb.nbody_leapfrog_f32(Q2, W2, m32, 0.01, 2.0 ** -8, 2)
    for _ in range(3):  # a different array each time: never the same arguments twice
        Q2, W2 = Q2.clone(), W2.clone()
        nb.nbody_leapfrog_f32(Q2, W2, m32, 0.01, 2.0 ** -8, 2)
    torch.cuda.synchronize()
    assert torch.equal(Q1, Q2) and torch.equal(W1, W2)


def test_graph_replay_rechecks_equal_masses(nb):
    """The equal-mass check runs inside the captured sequence: when the caller
    changes the masses in place between two identical calls, the replayed
    graph takes the general loop (and back), bit-identical to calls that
    never repeat their arguments."""
    import torch
    n = 3000
    p, v, m = ni.plummer(n, 18)
    equal = m.astype(np.float32)
    mixed = equal.copy()
    mixed[::7] *= np.float32(3.0)
    M = t(equal, np.float32)
    P1, V1 = t(p, np.float64), t(v, np.float64)
    for masses in (equal, equal, mixed, mixed, equal):  # calls 2.. replay the graph of call 2
        M.copy_(torch.from_numpy(masses))
        nb.nbody_leapfrog(P1, V1, M, 0.01, 2.0 ** -8, 2)
    P2, V2 = t(p, np.float64), t(v, np.float64)
    for masses in (equal, equal, mixed, mixed, equal):
        P2, V2 = P2.clone(), V2.clone()  # new arrays: never captured
        nb.nbody_leapfrog(P2, V2, t(masses, np.float32), 0.01, 2.0 ** -8, 2)
    torch.cuda.synchronize()
    assert torch.equal(P1, P2) and torch.equal(V1, V2)
    assert nb.nbody_last_device_error() == 0
