"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (per body, vector 2-norm): median relative acceleration error
<= 2e-6 and max <= 1e-4; max relative potential error <= 1e-5.  The FP32 pair
arithmetic with the approximate MUFU reciprocal square root has per-pair
relative error of a few 1e-7 and the compensated per-tile summation keeps the
sum's rounding below that, so these bounds leave an order of magnitude of
margin while failing any arithmetic slip.
"""
import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu

ACC_MED, ACC_MAX, POT_MAX = 2e-6, 1e-4, 1e-5


def t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def rel_err(a, ref):
    num = np.linalg.norm(np.asarray(a, dtype=np.float64) - ref, axis=-1) if ref.ndim == 2 else \
        np.abs(np.asarray(a, dtype=np.float64) - ref)
    den = np.linalg.norm(ref, axis=-1) if ref.ndim == 2 else np.abs(ref)
    return num / den


def gpu_accel(nb, api, pos, mass32, eps, with_pot=True, **kw):
    import torch
    n = pos.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((n,), dtype=torch.float32, device="cuda") if with_pot else None
    if api == "f32":
        nb.nbody_accel_f32(t(pos, np.float32), t(mass32, np.float32), np.float32(eps), acc, pot, **kw)
    else:
        prec = {"mixed": nb.NBODY_PREC_MIXED, "plain": nb.NBODY_PREC_PLAIN,
                "unsorted": nb.NBODY_PREC_MIXED_UNSORTED}[api]
        nb.nbody_accel(t(pos, np.float64), t(mass32, np.float32), eps, acc, pot, precision=prec, **kw)
    torch.cuda.synchronize()
    assert nb.nbody_last_device_error() == 0
    return acc.cpu().numpy(), (pot.cpu().numpy() if with_pot else None)


def reference_inputs(api, p):
    return p.astype(np.float32).astype(np.float64) if api == "f32" else p


def check(acc, pot, ra, rp, med=ACC_MED, mx=ACC_MAX, pmx=POT_MAX):
    e = rel_err(acc, ra)
    assert np.all(np.isfinite(acc))
    assert np.median(e) <= med, f"median rel acc err {np.median(e):.3g}"
    assert e.max() <= mx, f"max rel acc err {e.max():.3g}"
    if pot is not None:
        ep = rel_err(pot, rp)
        assert ep.max() <= pmx, f"max rel pot err {ep.max():.3g}"


@pytest.mark.parametrize("api", ["f32", "mixed", "plain", "unsorted"])
@pytest.mark.parametrize("n", [2, 3, 31, 257, 1000, 2500, 4097])
def test_accel_matches_oracle(nb, oracle_mod, api, n):
    p, _, m = ni.plummer(n, 1000 + n, masses="loguniform")
    m32 = m.astype(np.float32)
    eps = 2.0 ** -7
    acc, pot = gpu_accel(nb, api, p, m32, eps)
    ra, rp = oracle_mod.accel(reference_inputs(api, p), m32.astype(np.float64), eps)
    check(acc, pot, ra, rp)


def test_single_body_and_pair(nb, oracle_mod):
    acc, pot = gpu_accel(nb, "mixed", np.array([[0.3, -0.2, 5.0]]), np.array([2.0], np.float32), 0.1)
    assert np.all(acc == 0) and np.all(pot == 0)
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 1.5, 0.0]])
    m = np.array([0.25, 0.75], np.float32)
    acc, pot = gpu_accel(nb, "mixed", pos, m, 0.5)
    s = 1.5 ** 2 + 0.25
    np.testing.assert_allclose(acc[0], [0, 0.75 * 1.5 / s ** 1.5, 0], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(acc[1], [0, -0.25 * 1.5 / s ** 1.5, 0], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(pot, [-0.75 / s ** 0.5, -0.25 / s ** 0.5], rtol=1e-6)


def test_zero_softening_distinct_positions(nb, oracle_mod):
    p, _, m = ni.plummer(700, 77)
    m32 = m.astype(np.float32)
    acc, pot = gpu_accel(nb, "f32", p, m32, 0.0)
    ra, rp = oracle_mod.accel(reference_inputs("f32", p), m32.astype(np.float64), 0.0)
    check(acc, pot, ra, rp, med=1e-5, mx=1e-3, pmx=1e-4)


def test_coincident_bodies_with_softening(nb, oracle_mod):
    p, _, m = ni.plummer(300, 78)
    p[10] = p[20]
    p[200] = p[20]
    m32 = m.astype(np.float32)
    acc, pot = gpu_accel(nb, "f32", p, m32, 0.05)
    ra, rp = oracle_mod.accel(reference_inputs("f32", p), m32.astype(np.float64), 0.05)
    check(acc, pot, ra, rp)


def test_massless_and_padding_bodies(nb, oracle_mod):
    """Massless bodies feel but exert nothing; n just above a block boundary
    leaves a nearly empty last block of padding."""
    blk = nb.nbody_config_block(0)
    n = blk + 1
    p, _, m = ni.plummer(n, 79)
    m32 = m.astype(np.float32)
    m32[::7] = 0.0
    acc, pot = gpu_accel(nb, "mixed", p, m32, 2.0 ** -7, config=0)
    ra, rp = oracle_mod.accel(p, m32.astype(np.float64), 2.0 ** -7)
    check(acc, pot, ra, rp)


@pytest.mark.parametrize("k", range(5))
@pytest.mark.parametrize("with_pot", [True, False])
def test_every_kernel_shape(nb, oracle_mod, k, with_pot):
    if k >= nb.nbody_num_configs():
        pytest.skip("shape not compiled")
    blk = nb.nbody_config_block(k)
    n = 3 * blk + 37  # several i-blocks, several j-tiles, ragged tail
    p, _, m = ni.plummer(n, 500 + k, masses="loguniform")
    m32 = m.astype(np.float32)
    for api in ("mixed", "f32"):
        acc, pot = gpu_accel(nb, api, p, m32, 2.0 ** -8, with_pot=with_pot, config=k)
        ra, rp = oracle_mod.accel(reference_inputs(api, p), m32.astype(np.float64), 2.0 ** -8)
        check(acc, pot, ra, rp)


def test_fp32_running_sum_mode(nb, oracle_mod):
    """accumulate=FP32 keeps one FP32 running sum: less accurate, still close."""
    p, _, m = ni.plummer(4096, 90)
    m32 = m.astype(np.float32)
    acc, pot = gpu_accel(nb, "f32", p, m32, 2.0 ** -7, accumulate=nb.NBODY_ACC_FP32)
    ra, rp = oracle_mod.accel(reference_inputs("f32", p), m32.astype(np.float64), 2.0 ** -7)
    check(acc, pot, ra, rp, med=2e-5, mx=1e-3, pmx=1e-4)


def test_offset_sphere_mixed_vs_plain(nb, oracle_mod):
    """Offset to (1e4,-3e3,7e2): tile-centred FP32 math meets the tolerance;
    FP32 absolute coordinates (ulp ~1e-3 there) cannot."""
    n = 8192
    p, _, m = ni.plummer(n, 91, masses="loguniform", offset=(1e4, -3e3, 7e2))
    m32 = m.astype(np.float32)
    eps = 2.0 ** -9
    ra, rp = oracle_mod.accel(p, m32.astype(np.float64), eps)
    acc, pot = gpu_accel(nb, "mixed", p, m32, eps)
    check(acc, pot, ra, rp)
    acc_p, _ = gpu_accel(nb, "plain", p, m32, eps, with_pot=False)
    assert np.median(rel_err(acc_p, ra)) > 50 * ACC_MED  # misses the target by >50x


def test_deterministic(nb):
    p, _, m = ni.plummer(5000, 92, masses="loguniform")
    m32 = m.astype(np.float32)
    a1, f1 = gpu_accel(nb, "mixed", p, m32, 0.01)
    a2, f2 = gpu_accel(nb, "mixed", p, m32, 0.01)
    assert np.array_equal(a1, a2) and np.array_equal(f1, f2)


def test_host_arrays_are_staged(nb, oracle_mod):
    """numpy (host) arrays go through the same kernels and give the same bits."""
    p, _, m = ni.plummer(3000, 93)
    m32 = m.astype(np.float32)
    acc_h = np.zeros((3000, 3), np.float32)
    pot_h = np.zeros(3000, np.float32)
    nb.nbody_accel(np.ascontiguousarray(p), m32, 0.01, acc_h, pot_h)
    acc_d, pot_d = gpu_accel(nb, "mixed", p, m32, 0.01)
    assert np.array_equal(acc_h, acc_d) and np.array_equal(pot_h, pot_d)


def test_energy_diagnostics(nb, oracle_mod):
    w = ni.small_plain()
    m32 = w.mass.astype(np.float32)
    e_ref = oracle_mod.energy(w.pos, w.vel, w.mass, w.eps)
    e32 = nb.nbody_energy_f32(t(w.pos, np.float32), t(w.vel, np.float32), t(m32, np.float32), w.eps)
    e64 = nb.nbody_energy(t(w.pos, np.float64), t(w.vel, np.float64), t(m32, np.float32), w.eps)
    for e in (e32, e64):
        assert abs(e["T"] - e_ref["T"]) <= 1e-12 * abs(e_ref["T"])
        assert abs(e["W"] - e_ref["W"]) <= 2e-6 * abs(e_ref["W"])
        assert abs(e["E"] - e_ref["E"]) <= 1e-5 * abs(e_ref["E"])
        assert np.abs(e["P"] - e_ref["P"]).max() <= 1e-12
        # Newton's third law up to FP32 pair rounding
        assert np.abs(e["F"]).max() <= 1e-5


def test_streams_are_independent(nb, oracle_mod):
    import torch
    p, _, m = ni.plummer(2048, 94)
    m32 = m.astype(np.float32)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    P, M = t(p, np.float64), t(m32, np.float32)
    torch.cuda.synchronize()
    outs = []
    for s, eps in ((s1, 0.01), (s2, 0.02)):
        acc = torch.empty((2048, 3), dtype=torch.float32, device="cuda")
        nb.nbody_accel(P, M, eps, acc, None, stream=s)
        outs.append((acc, eps))
    torch.cuda.synchronize()
    for acc, eps in outs:
        ra, _ = oracle_mod.accel(p, m32.astype(np.float64), eps, with_pot=False)
        check(acc.cpu().numpy(), None, ra, None)


@pytest.mark.parametrize("api", ["f32", "mixed", "plain"])
@pytest.mark.parametrize("ni_,nj_", [(1, 1), (37, 500), (1000, 4097), (3000, 257), (5, 0)])
def test_sink_source_split_matches_oracle(nb, oracle_mod, api, ni_, nj_):
    import torch
    p, _, m = ni.plummer(max(nj_, 1), 900 + nj_, masses="loguniform", offset=(0.0, 0.0, 0.0))
    p, m = p[:nj_], m[:nj_]
    sinks, _, _ = ni.plummer(ni_, 901 + ni_)
    sinks = sinks + np.array([0.11, -0.07, 0.05])  # a lone sink and a lone source both sit at the origin
    m32 = m.astype(np.float32)
    eps = 2.0 ** -7
    acc = torch.empty((ni_, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((ni_,), dtype=torch.float32, device="cuda")
    if api == "f32":
        nb.nbody_accel_ij_f32(t(sinks, np.float32), t(p, np.float32), t(m32, np.float32), np.float32(eps), acc, pot)
        si, pj = sinks.astype(np.float32).astype(np.float64), p.astype(np.float32).astype(np.float64)
    else:
        prec = nb.NBODY_PREC_MIXED if api == "mixed" else nb.NBODY_PREC_PLAIN
        nb.nbody_accel_ij(t(sinks, np.float64), t(p, np.float64), t(m32, np.float32), eps, acc, pot, precision=prec)
        si, pj = sinks, p
    torch.cuda.synchronize()
    a, f = acc.cpu().numpy(), pot.cpu().numpy()
    if nj_ == 0:
        assert np.all(a == 0) and np.all(f == 0)
        return
    ra, rp = oracle_mod.accel_ij(si, pj, m32.astype(np.float64), eps)
    check(a, f, ra, rp)


def test_kahan_per_pair_mode(nb, oracle_mod):
    """accumulate=KAHAN_PAIR compensates every pair term: within tolerance, and
    no less accurate than the default per-tile compensation."""
    p, _, m = ni.plummer(8192, 95, masses="loguniform", offset=(1e4, -3e3, 7e2))
    m32 = m.astype(np.float32)
    ra, rp = oracle_mod.accel(p, m32.astype(np.float64), 2.0 ** -8)
    errs = {}
    for mode in (nb.NBODY_ACC_KAHAN_PAIR, nb.NBODY_ACC_COMPENSATED, nb.NBODY_ACC_FP32):
        acc, pot = gpu_accel(nb, "mixed", p, m32, 2.0 ** -8, accumulate=mode)
        errs[mode] = np.median(rel_err(acc, ra))
        if mode != nb.NBODY_ACC_FP32:
            check(acc, pot, ra, rp)
    assert errs[nb.NBODY_ACC_KAHAN_PAIR] <= 1.2 * errs[nb.NBODY_ACC_COMPENSATED]
    # at this size the sums' rounding is below the pair arithmetic's, so the
    # three modes differ by noise; the FP32 running sum's gap shows at large n
    assert errs[nb.NBODY_ACC_COMPENSATED] <= 1.2 * errs[nb.NBODY_ACC_FP32]


def test_morton_order_shrinks_close_pair_errors(nb, oracle_mod):
    """All 65536 bodies of an offset sphere: in the caller's order a cell spans
    the system and close pairs carry FP32 offset rounding of the system's size
    (worst body ~1.8e-4 relative); in the default Morton order cells are compact
    and the worst body stays within the 1e-4 bound."""
    n = 65536
    p, _, m = ni.plummer(n, 4242 + n, masses="loguniform", offset=(1e4, -3e3, 7e2))
    m32 = m.astype(np.float32)
    ra, rp = oracle_mod.accel(p, m32.astype(np.float64), 2.0 ** -9)
    acc_s, pot_s = gpu_accel(nb, "mixed", p, m32, 2.0 ** -9)
    acc_u, _ = gpu_accel(nb, "unsorted", p, m32, 2.0 ** -9, with_pot=False)
    es, eu = rel_err(acc_s, ra), rel_err(acc_u, ra)
    print(f"all bodies: sorted median {np.median(es):.3g} max {es.max():.3g}; "
          f"caller's order median {np.median(eu):.3g} max {eu.max():.3g}")
    check(acc_s, pot_s, ra, rp)
    assert es.max() < 0.5 * eu.max()


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_equal_mass_loop_matches_general_loop(nb, precision):
    """Equal masses take the pair loops without m_j (force and VJP, the sums
    scaled once); raising one body's mass by one FP32 ulp sends the same
    inputs through the general loops.  The two agree to FP32 rounding."""
    import torch
    n = 5000
    p, _, m = ni.plummer(n, 7100)
    m32 = m.astype(np.float32)
    assert np.all(m32 == m32[0])
    m_gen = m32.copy()
    m_gen[-1] = np.nextafter(m_gen[-1], np.float32(1.0))
    prec = nb.NBODY_PREC_MIXED if precision == "mixed" else nb.NBODY_PREC_PLAIN
    P = torch.from_numpy(p).cuda()
    out = []
    for mm in (m32, m_gen):
        acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        pot = torch.empty((n,), dtype=torch.float32, device="cuda")
        nb.nbody_accel(P, torch.from_numpy(mm).cuda(), 2.0 ** -8, acc, pot, precision=prec)
        lam = torch.from_numpy(ni.gaussian((n, 3), 7101).astype(np.float32)).cuda()
        gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        gm = torch.empty((n,), dtype=torch.float32, device="cuda")
        nb.nbody_accel_vjp(P, torch.from_numpy(mm).cuda(), 2.0 ** -8, lam, None, gp, gm, precision=prec)
        torch.cuda.synchronize()
        out.append([x.cpu().numpy().astype(np.float64) for x in (acc, pot, gp, gm)])
    (a0, p0, g0, h0), (a1, p1, g1, h1) = out
    ea = np.linalg.norm(a0 - a1, axis=1) / np.linalg.norm(a1, axis=1)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-4, (np.median(ea), ea.max())
    assert (np.abs(p0 - p1) / np.abs(p1)).max() <= 1e-5
    eg = np.linalg.norm(g0 - g1, axis=1)
    assert np.median(eg / np.linalg.norm(g1, axis=1)) <= 1e-5, np.median(eg / np.linalg.norm(g1, axis=1))
    assert np.median(np.abs(h0 - h1) / np.abs(h1)) <= 1e-5
    assert nb.nbody_last_device_error() == 0


@pytest.mark.parametrize("accumulate", ["compensated", "fp32"])
@pytest.mark.parametrize("n,masses,eps", [(1000, "equal", 2.0 ** -7), (4096, "loguniform", 2.0 ** -7),
                                          (20011, "equal", 2.0 ** -8)])
def test_fp32_path_at_least_as_accurate_as_listing(nb, oracle_mod, n, masses, eps, accumulate):
    """The plain FP32 path (nbody_accel_f32) against the oracle's correctly
    rounded FP32 restatement of Listing 4: per body, both are compared with the
    FP64 oracle on the same FP32 inputs, and the GPU's error must be no larger
    than the listing's own (median) and at most 1.5 times its largest (max).
    The kernel replaces the listing's exact 1/sqrt by the MUFU approximation
    but sums in shorter FP32 runs (per j-tile, folded by Kahan summation, or
    split across the stream-K slices), so it is expected to be more accurate,
    not only within a loose bound; a slip in its per-pair arithmetic would show
    as an error well above the listing's."""
    p, _, m = ni.plummer(n, 300 + n, masses=masses)
    p = p.astype(np.float32).astype(np.float64)
    m = m.astype(np.float32).astype(np.float64)
    eps = float(np.float32(eps))
    idx = np.arange(n) if n <= 4096 else ni.subsample(n, 2048, 5)
    ra, _ = oracle_mod.accel_subset(p, m, eps, idx)
    la, _ = oracle_mod.accel_listing_f32(p, m, eps, idx=idx)
    kw = {} if accumulate == "compensated" else {"accumulate": nb.NBODY_ACC_FP32}
    acc, _ = gpu_accel(nb, "f32", p, m.astype(np.float32), eps, with_pot=False, **kw)
    eg, el = rel_err(acc[idx], ra), rel_err(la, ra)
    assert np.median(eg) <= np.median(el), (np.median(eg), np.median(el))
    assert eg.max() <= 1.5 * el.max(), (eg.max(), el.max())
