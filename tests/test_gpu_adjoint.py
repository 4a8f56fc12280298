"""Reverse mode on the GPU: the force VJP against the oracle's, the
checkpointed leapfrog adjoint against the oracle's FP64 adjoint and against
FP64 central finite differences of the oracle's forward run, and the
torch.autograd binding end to end."""
import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu


def t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def rel_rows(a, ref):
    """Per-body error of a gradient, relative to that body's gradient but never
    to less than a tenth of the median body's: a gradient is a sum of terms of
    both signs and a few bodies' sums land near zero by chance, where a purely
    relative error says nothing about the arithmetic."""
    a = np.asarray(a, np.float64)
    if ref.ndim == 2:
        err, mag = np.linalg.norm(a - ref, axis=1), np.linalg.norm(ref, axis=1)
    else:
        err, mag = np.abs(a - ref), np.abs(ref)
    return err / np.maximum(mag, 0.1 * np.median(mag))


def gpu_vjp(nb, pos, mass32, eps, lam32, mu32=None, **kw):
    import torch
    n = pos.shape[0]
    gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gm = torch.empty((n,), dtype=torch.float32, device="cuda")
    nb.nbody_accel_vjp(t(pos, np.float64), t(mass32, np.float32), eps, t(lam32, np.float32),
                       t(mu32, np.float32) if mu32 is not None else None, gp, gm, **kw)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    return gp.cpu().numpy(), gm.cpu().numpy()


@pytest.mark.parametrize("masses", ["loguniform", "equal"])
@pytest.mark.parametrize("with_mu", [False, True])
@pytest.mark.parametrize("n", [2, 33, 1000, 3001])
def test_force_vjp_matches_oracle(nb, oracle_mod, n, with_mu, masses):
    """Equal masses take the VJP's loop that forms u = mu (lam_j - lam_k)
    without the masses; distinct masses the general loop."""
    p, _, m = ni.plummer(n, 700 + n, masses=masses)
    m32 = m.astype(np.float32)
    lam = ni.gaussian((n, 3), 701).astype(np.float32)
    mu = ni.gaussian((n,), 702).astype(np.float32) if with_mu else None
    eps = 2.0 ** -7
    gp, gm = gpu_vjp(nb, p, m32, eps, lam, mu)
    rp, rm = oracle_mod.accel_vjp(p, m32.astype(np.float64), eps, lam.astype(np.float64),
                                  mu.astype(np.float64) if with_mu else None)
    e = rel_rows(gp, rp)
    em = rel_rows(gm, rm)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-3, (np.median(e), e.max())
    assert np.median(em) <= 1e-5 and em.max() <= 1e-3, (np.median(em), em.max())


@pytest.mark.parametrize("k", range(4))
def test_every_vjp_shape(nb, oracle_mod, k):
    lib = nb.load()
    if k >= 4:
        pytest.skip()
    n = 1500 + 37 * k
    p, _, m = ni.plummer(n, 720 + k, masses="loguniform", offset=(1e4, -3e3, 7e2))
    m32 = m.astype(np.float32)
    lam = ni.gaussian((n, 3), 721).astype(np.float32)
    gp, gm = gpu_vjp(nb, p, m32, 2.0 ** -8, lam, config=k)
    rp, rm = oracle_mod.accel_vjp(p, m32.astype(np.float64), 2.0 ** -8, lam.astype(np.float64))
    e = rel_rows(gp, rp)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-3, (k, np.median(e), e.max())


def record_and_vjp(nb, pos, vel, m32, eps, dt, steps, ckpt, gxT, gvT, **kw):
    import torch
    n = pos.shape[0]
    P, V, M = t(pos, np.float64), t(vel, np.float64), t(m32, np.float32)
    tape = torch.empty(nb.nbody_tape_bytes(n, steps, ckpt), dtype=torch.uint8, device="cuda")
    nb.nbody_leapfrog_record(P, V, M, eps, dt, steps, ckpt, tape, **kw)
    gx0 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gv0 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gm = torch.empty((n,), dtype=torch.float64, device="cuda")
    gX = gxT(P.cpu().numpy()) if callable(gxT) else gxT
    nb.nbody_leapfrog_vjp_tape(M, eps, dt, steps, ckpt, tape, t(gX, np.float64), t(gvT, np.float64), gx0, gv0, gm, **kw)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    return P.cpu().numpy(), V.cpu().numpy(), gx0.cpu().numpy(), gv0.cpu().numpy(), gm.cpu().numpy()


def test_record_matches_leapfrog(nb):
    import torch
    p, v, m = ni.plummer(2000, 730)
    m32 = m.astype(np.float32)
    P, V = t(p, np.float64), t(v, np.float64)
    nb.nbody_leapfrog(P, V, t(m32, np.float32), 0.01, 2.0 ** -8, 10)
    torch.cuda.synchronize()
    P2, V2, *_ = record_and_vjp(nb, p, v, m32, 0.01, 2.0 ** -8, 10, 3, np.zeros((2000, 3)), np.zeros((2000, 3)))
    assert np.array_equal(P.cpu().numpy(), P2) and np.array_equal(V.cpu().numpy(), V2)


@pytest.mark.parametrize("ckpt", [1, 4, 5, 16])
def test_leapfrog_adjoint_matches_oracle_adjoint(nb, oracle_mod, ckpt):
    """Cotangents of L = sum m |x(T) - y|^2 + c.v(T): the GPU adjoint against the
    oracle's FP64 adjoint of its own FP64 run (median 1e-5 relative)."""
    n, K, eps, dt = 1024, 16, 2.0 ** -7, 2.0 ** -8
    p, v, m = ni.plummer(n, 740, masses="loguniform")
    m32 = m.astype(np.float32)
    m64 = m32.astype(np.float64)
    y = p + ni.gaussian((n, 3), 741, 0.05)
    c = ni.gaussian((n, 3), 742)
    xT_ref, vT_ref, _ = oracle_mod.leapfrog(p, v, m64, eps, dt, K)
    gxT_ref = 2 * m64[:, None] * (xT_ref - y)
    rx, rv, rm = oracle_mod.leapfrog_vjp(p, v, m64, eps, dt, K, gxT_ref, c)
    xT, vT, gx, gv, gm = record_and_vjp(nb, p, v, m32, eps, dt, K, ckpt,
                                        lambda xT: 2 * m64[:, None] * (xT - y), c)
    for g, r in ((gx, rx), (gv, rv)):
        e = rel_rows(g, r)
        assert np.median(e) <= 1e-5 and e.max() <= 1e-3, (ckpt, np.median(e), e.max())
    em = rel_rows(gm, rm)
    assert np.median(em) <= 1e-5 and em.max() <= 1e-3, (ckpt, np.median(em), em.max())


def _fd_check(nb, oracle_mod, n, K, ncoord, seed):
    """The adjoint workload's recipe (eps=2^-7, dt=2^-8, checkpoints every 8
    steps, y = x0 + N(0,0.05^2)) at n bodies: GPU gradients of
    L = sum m |x(T) - y|^2 against FP64 central differences (h = 1e-6) of the
    oracle's forward run on ncoord seeded coordinates of x0, v0 and m."""
    eps, dt, ckpt, h = 2.0 ** -7, 2.0 ** -8, 8, 1e-6
    p, v, m = ni.plummer(n, seed)
    m32 = m.astype(np.float32)
    m64 = m32.astype(np.float64)
    y = p + ni.gaussian((n, 3), seed + 1, 0.05)
    xT, vT, gx, gv, gm = record_and_vjp(nb, p, v, m32, eps, dt, K, ckpt,
                                        lambda xT: 2 * m64[:, None] * (xT - y), np.zeros((n, 3)))
    gm = gm + ((xT - y) ** 2).sum(axis=1)  # direct mass term of L

    def L(x0, v0, mass):
        xT_, _, _ = oracle_mod.leapfrog(x0, v0, mass, eps, dt, K)
        return float((mass[:, None] * (xT_ - y) ** 2).sum())

    pick = ni.subsample(7 * n, ncoord, seed + 2)
    worst = 0.0
    for q in pick:
        kind, rest = divmod(int(q), n)  # 0,1,2: x0 comps; 3,4,5: v0 comps; 6: m
        x0, v0, mm = p.copy(), v.copy(), m64.copy()
        x1, v1, m1 = p.copy(), v.copy(), m64.copy()
        if kind < 3:
            x0[rest, kind] += h; x1[rest, kind] -= h; g = gx[rest, kind]
        elif kind < 6:
            v0[rest, kind - 3] += h; v1[rest, kind - 3] -= h; g = gv[rest, kind - 3]
        else:
            mm[rest] += h; m1[rest] -= h; g = gm[rest]
        fd = (L(x0, v0, mm) - L(x1, v1, m1)) / (2 * h)
        err = abs(g - fd) / abs(fd)
        worst = max(worst, err)
        assert err <= 1e-4, (kind, rest, g, fd, err)
    return worst


def test_adjoint_recipe_finite_differences_32_coordinates(nb, oracle_mod):
    """32 seeded coordinates at n = 2048, K = 64."""
    _fd_check(nb, oracle_mod, 2048, 64, 32, 750)


def workload_fd_errors(nb):
    """The adjoint workload (N = 16384, eps = 2^-7, dt = 2^-8, K = 64,
    checkpoints every 8, L = sum m |x(T) - y|^2): the GPU gradient against the
    FP64 central differences stored in tests/golden/adjoint_fd_n16384.json
    (32 seeded coordinates of x0, v0 and m, written by
    tests/golden/make_adjoint_fd.py from the oracle alone).  Returns the
    relative error per coordinate."""
    import json
    import os
    doc = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "adjoint_fd_n16384.json")))
    w = ni.adjoint_case()
    # The generator's transcendental functions may round differently on
    # another machine (last bit), so the inputs are compared to 1e-12, not bit
    # for bit; the gradient moves by ~1e-14 relative under such a change.
    for name, arr in (("pos", w.pos), ("vel", w.vel), ("mass", w.mass), ("target", w.extra["target"])):
        fp, a = doc["inputs_fingerprint"][name], np.asarray(arr, dtype=np.float64).reshape(-1)
        assert abs(np.abs(a).sum() - fp["sum_abs"]) <= 1e-12 * fp["sum_abs"], name
        for got, want in zip(np.concatenate([a[:4], a[-4:]]), fp["head"] + fp["tail"]):
            assert abs(got - want) <= 1e-12 * max(abs(want), 1e-300), name
    n, y = w.n, w.extra["target"]
    m64 = w.mass
    xT, vT, gx, gv, gm = record_and_vjp(nb, w.pos, w.vel, m64.astype(np.float32), w.eps, w.dt, w.steps,
                                        w.extra["ckpt_every"], lambda xT_: 2 * m64[:, None] * (xT_ - y),
                                        np.zeros((n, 3)))
    gm = gm + ((xT - y) ** 2).sum(axis=1)  # direct mass term of L
    errs = []
    for r in doc["rows"]:
        g = {"x0": gx, "v0": gv}[r["kind"]][r["body"], r["component"]] if r["kind"] != "m" else gm[r["body"]]
        errs.append(abs(g - r["fd"]) / abs(r["fd"]))
    return np.asarray(errs)


def test_adjoint_workload_finite_differences(nb):
    """All 32 stored coordinates of the full adjoint workload within 1e-4."""
    e = workload_fd_errors(nb)
    assert e.size == 32
    assert e.max() <= 1e-4, (np.round(e, 8).tolist())


def test_one_call_adjoint_equals_record_and_sweep(nb):
    """nbody_leapfrog_vjp(n, pos0, vel0, ...) records the run on copies in the
    library's workspace and sweeps it: the same kernels in the same order as
    nbody_leapfrog_record + nbody_leapfrog_vjp_tape, so the same bits; the
    inputs are left untouched, and host arrays work as well as device ones."""
    import torch
    n, K, ck, eps, dt = 1500, 12, 5, 2.0 ** -7, 2.0 ** -8
    p, v, m = ni.plummer(n, 790, masses="loguniform")
    m32 = m.astype(np.float32)
    gxT = ni.gaussian((n, 3), 791)
    gvT = ni.gaussian((n, 3), 792)
    _, _, rx, rv, rm = record_and_vjp(nb, p, v, m32, eps, dt, K, ck, gxT, gvT)
    P, V, M = t(p, np.float64), t(v, np.float64), t(m32, np.float32)
    gx = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gv = torch.empty_like(gx)
    gm = torch.empty((n,), dtype=torch.float64, device="cuda")
    nb.nbody_leapfrog_vjp(P, V, M, eps, dt, K, ck, t(gxT, np.float64), t(gvT, np.float64), gx, gv, gm)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    assert np.array_equal(gx.cpu().numpy(), rx) and np.array_equal(gv.cpu().numpy(), rv)
    assert np.array_equal(gm.cpu().numpy(), rm)
    assert np.array_equal(P.cpu().numpy(), p) and np.array_equal(V.cpu().numpy(), v)
    hx, hv, hm = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    nb.nbody_leapfrog_vjp(np.ascontiguousarray(p), np.ascontiguousarray(v), m32, eps, dt, K, ck, gxT, gvT, hx, hv, hm)
    assert np.array_equal(hx, rx) and np.array_equal(hv, rv) and np.array_equal(hm, rm)


def test_adjoint_sweep_repeatable(nb):
    """The sweep's kernels are chained by programmatic dependent launch like
    the forward's: three record + sweep runs give the same bits."""
    n, K, ck, eps, dt = 6000, 10, 4, 2.0 ** -7, 2.0 ** -8
    p, v, m = ni.plummer(n, 793)
    m32 = m.astype(np.float32)
    gxT = ni.gaussian((n, 3), 794)
    gvT = ni.gaussian((n, 3), 795)
    first = record_and_vjp(nb, p, v, m32, eps, dt, K, ck, gxT, gvT)
    for _ in range(2):
        again = record_and_vjp(nb, p, v, m32, eps, dt, K, ck, gxT, gvT)
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
    assert nb.nbody_last_device_error() == 0


def test_autograd_trajectory(nb):
    import torch
    n, K, eps, dt = 700, 12, 2.0 ** -7, 2.0 ** -8
    p, v, m = ni.plummer(n, 760, masses="loguniform")
    y = t(p + ni.gaussian((n, 3), 761, 0.05), np.float64)
    x0 = t(p, np.float64).requires_grad_(True)
    v0 = t(v, np.float64).requires_grad_(True)
    mm = t(m.astype(np.float32), np.float64).requires_grad_(True)
    xT, vT = nb.Trajectory.apply(x0, v0, mm, eps, dt, K, 4)
    loss = (mm[:, None] * (xT - y) ** 2).sum() + (0.1 * vT).sum()
    loss.backward()
    # the same through the C ABI
    m32 = m.astype(np.float32)
    xr, vr, gx, gv, gm = record_and_vjp(nb, p, v, m32, eps, dt, K, 4,
                                        lambda xT_: 2 * m32.astype(np.float64)[:, None] * (xT_ - y.cpu().numpy()),
                                        np.full((n, 3), 0.1))
    assert np.allclose(xT.detach().cpu().numpy(), xr, rtol=0, atol=0)
    assert np.allclose(x0.grad.cpu().numpy(), gx, rtol=1e-12, atol=1e-14)
    assert np.allclose(v0.grad.cpu().numpy(), gv, rtol=1e-12, atol=1e-14)
    direct = ((xr - y.cpu().numpy()) ** 2).sum(axis=1)
    assert np.allclose(mm.grad.cpu().numpy(), gm + direct, rtol=1e-10, atol=1e-14)
