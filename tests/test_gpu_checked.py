"""Checked build: every kernel's computed global indices tested in range.

compute-sanitizer is not available for these runs, so the library has a
second build (-DNBODY_CHECKS) in which each global load and store of the
force, VJP, batched and packing kernels first tests its index against the
buffer it addresses; an index out of range records NBODY_EBOUNDS in the
library's device error word and skips the access.  This module builds that
variant beside the normal one, drives every entry point through it at ragged
sizes, every kernel shape, every precision and summation mode, asserts that
no kernel met an index out of range, and that the checked results equal the
normal build's (the checks change no arithmetic).
"""
import contextlib
import os

import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked_lib(nb):
    from paper_2411_18889_gb300 import _lib, build
    path = build.build(extra=["-DNBODY_CHECKS"], lib_path=os.path.join(build.BUILD, "libnbody_checked.so"))
    return _lib.open_library(path)


@contextlib.contextmanager
def using(lib):
    from paper_2411_18889_gb300 import _lib
    saved = _lib.load()
    _lib._lib = lib
    try:
        yield
    finally:
        _lib._lib = saved


def t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def both(nb, checked_lib, fn):
    """fn() under the normal build, then under the checked build; the checked
    run must report no device error and return the same arrays."""
    import torch
    ref = [np.asarray(x) for x in fn()]
    with using(checked_lib):
        got = [np.asarray(x) for x in fn()]
        torch.cuda.synchronize()
        code = int(checked_lib.nbody_last_device_error())
    assert code == 0, checked_lib.nbody_strerror(code).decode()
    for g, r in zip(got, ref):
        scale = float(np.abs(r).max()) if r.size else 0.0
        np.testing.assert_allclose(g, r, rtol=1e-6, atol=1e-6 * scale)


def accel_f64(nb, p, m, eps, **kw):
    import torch
    n = p.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((n,), dtype=torch.float32, device="cuda")
    nb.nbody_accel(t(p, np.float64), t(m, np.float32), eps, acc, pot, **kw)
    return acc.cpu().numpy(), pot.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 3, 1000, 4099, 20011])
def test_accel_every_shape_in_bounds(nb, checked_lib, n, precision):
    p, _, m = ni.plummer(n, 900 + n, masses="loguniform", offset=ni.plummer_offset())
    for k in range(nb.nbody_num_configs()):
        both(nb, checked_lib, lambda: accel_f64(nb, p, m, 2.0 ** -9, config=k, precision=precision))


@pytest.mark.parametrize("precision", [0, 1])
def test_equal_mass_loops_in_bounds(nb, checked_lib, precision):
    """Equal masses: the force and VJP kernels take their loops without m_j."""
    import torch
    n = 4099
    p, _, m = ni.plummer(n, 915)
    lam = ni.gaussian((n, 3), 916)
    for k in range(nb.nbody_num_configs()):
        both(nb, checked_lib, lambda: accel_f64(nb, p, m, 2.0 ** -9, config=k, precision=precision))
    for k in range(4):
        def run():
            gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
            gm = torch.empty((n,), dtype=torch.float32, device="cuda")
            nb.nbody_accel_vjp(t(p, np.float64), t(m, np.float32), 2.0 ** -7, t(lam, np.float32), None, gp, gm,
                               config=k, precision=precision)
            return gp.cpu().numpy(), gm.cpu().numpy()

        both(nb, checked_lib, run)


@pytest.mark.parametrize("accumulate", [1, 2])
def test_accel_summation_modes_in_bounds(nb, checked_lib, accumulate):
    p, _, m = ni.plummer(5003, 910, masses="loguniform")
    both(nb, checked_lib, lambda: accel_f64(nb, p, m, 2.0 ** -8, accumulate=accumulate))


def test_accel_f32_and_ij_in_bounds(nb, checked_lib):
    import torch
    n = 4099
    p, _, m = ni.plummer(n, 911, masses="loguniform")

    def f32():
        acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        pot = torch.empty((n,), dtype=torch.float32, device="cuda")
        nb.nbody_accel_f32(t(p, np.float32), t(m, np.float32), 2.0 ** -8, acc, pot)
        return acc.cpu().numpy(), pot.cpu().numpy()

    both(nb, checked_lib, f32)
    q = ni.plummer(777, 912)[0] + 0.01

    def ij():
        acc = torch.empty((777, 3), dtype=torch.float32, device="cuda")
        pot = torch.empty((777,), dtype=torch.float32, device="cuda")
        nb.nbody_accel_ij(t(q, np.float64), t(p, np.float64), t(m, np.float32), 2.0 ** -8, acc, pot)
        return acc.cpu().numpy(), pot.cpu().numpy()

    both(nb, checked_lib, ij)


@pytest.mark.parametrize("precision", [0, 1])
def test_leapfrog_in_bounds(nb, checked_lib, precision):
    n = 3001
    p, v, m = ni.plummer(n, 913)

    def run():
        P, V = t(p, np.float64), t(v, np.float64)
        for _ in range(3):  # the repeats take the captured-graph path
            nb.nbody_leapfrog(P, V, t(m, np.float32), 0.01, 2.0 ** -8, 2, precision=precision)
        return P.cpu().numpy(), V.cpu().numpy()

    both(nb, checked_lib, run)

    def run32():
        P, V = t(p, np.float32), t(v, np.float32)
        nb.nbody_leapfrog_f32(P, V, t(m, np.float32), 0.01, 2.0 ** -8, 3)
        return P.cpu().numpy(), V.cpu().numpy()

    both(nb, checked_lib, run32)


@pytest.mark.parametrize("shape", range(6))
def test_batched_in_bounds(nb, checked_lib, shape):
    import torch
    # 15001 bodies: more than one CTA's image, so split over several CTAs
    sizes = [1, 2, 3, 0, 63, 64, 65, 127, 511, 513, 1000, 2049, 5, 0, 777, 15001]
    P, V, M = [], [], []
    for s, n in enumerate(sizes):
        p, v, m = ni.plummer(n, 920 + s)
        P.append(p); V.append(v); M.append(m)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    pos, vel, mass = np.concatenate(P), np.concatenate(V), np.concatenate(M)
    eps = np.asarray([4.0 / np.sqrt(max(n, 1)) for n in sizes])
    eps[2] = 0.0  # an unsoftened system takes the masked self-pair path
    ntot = int(off[-1])

    def acc():
        a = torch.empty((ntot, 3), dtype=torch.float32, device="cuda")
        u = torch.empty((ntot,), dtype=torch.float32, device="cuda")
        nb.nbody_accel_batched(t(off, np.int64), t(pos, np.float32), t(mass, np.float32), t(eps, np.float32), a, u,
                               config=shape)
        return a.cpu().numpy(), u.cpu().numpy()

    def leap():
        x, w = t(pos, np.float32), t(vel, np.float32)
        e = t(np.maximum(eps, 0.01), np.float32)
        nb.nbody_leapfrog_batched(t(off, np.int64), x, w, t(mass, np.float32), e, 2.0 ** -8, 3, config=shape)
        return x.cpu().numpy(), w.cpu().numpy()

    both(nb, checked_lib, acc)
    both(nb, checked_lib, leap)


@pytest.mark.parametrize("n", [2, 1500, 20011])
def test_vjp_every_shape_in_bounds(nb, checked_lib, n):
    import torch
    p, _, m = ni.plummer(n, 930 + n, masses="loguniform")
    lam = ni.gaussian((n, 3), 931)
    mu = ni.gaussian((n,), 932)

    for k in range(4):
        def run():
            gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
            gm = torch.empty((n,), dtype=torch.float32, device="cuda")
            nb.nbody_accel_vjp(t(p, np.float64), t(m, np.float32), 2.0 ** -7, t(lam, np.float32), t(mu, np.float32),
                               gp, gm, config=k)
            return gp.cpu().numpy(), gm.cpu().numpy()

        both(nb, checked_lib, run)


def test_adjoint_in_bounds(nb, checked_lib):
    import torch
    n, K, ck = 1024, 8, 3
    p, v, m = ni.plummer(n, 940, masses="loguniform")
    gx = ni.gaussian((n, 3), 941)
    gv = ni.gaussian((n, 3), 942)

    def run():
        P, V, M = t(p, np.float64), t(v, np.float64), t(m, np.float32)
        tape = torch.empty(nb.nbody_tape_bytes(n, K, ck), dtype=torch.uint8, device="cuda")
        nb.nbody_leapfrog_record(P, V, M, 2.0 ** -7, 2.0 ** -8, K, ck, tape)
        g0 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        h0 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gm = torch.empty((n,), dtype=torch.float64, device="cuda")
        nb.nbody_leapfrog_vjp_tape(M, 2.0 ** -7, 2.0 ** -8, K, ck, tape, t(gx, np.float64), t(gv, np.float64), g0, h0, gm)
        return P.cpu().numpy(), g0.cpu().numpy(), h0.cpu().numpy(), gm.cpu().numpy()

    both(nb, checked_lib, run)


def test_energy_and_noalloc_in_bounds(nb, checked_lib):
    import torch
    n = 5000
    p, v, m = ni.plummer(n, 950)

    def energy():
        e = nb.nbody_energy(t(p, np.float64), t(v, np.float64), t(m, np.float32), 0.01)
        return [np.concatenate([[e["T"], e["W"], e["E"]], e["P"], e["F"]])]

    both(nb, checked_lib, energy)

    def noalloc():
        from paper_2411_18889_gb300 import _lib
        lib = _lib.load()
        P, M = t(p, np.float64), t(m, np.float32)
        a = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        u = torch.empty((n,), dtype=torch.float32, device="cuda")
        st = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        rc = lib.nbody_accel_noalloc(n, P.data_ptr(), M.data_ptr(), 0.01, a.data_ptr(), u.data_ptr(), st.data_ptr(),
                                     None)
        torch.cuda.synchronize()
        assert rc == 0 and int(st.item()) == 0, (rc, int(st.item()))
        return a.cpu().numpy(), u.cpu().numpy()

    both(nb, checked_lib, noalloc)
