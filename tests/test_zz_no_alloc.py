"""nbody_accel_noalloc: the force evaluation for callers that cannot allocate
GPU memory (allocator callbacks, real-time loops, fully pre-reserved
processes), with all scratch in the library's fixed device array.

Called through the C ABI (ctypes) on device arrays, on two calls in a row:
its output must equal, bit for bit, that of the allocating entry point
nbody_accel with the same options (default precision and summation, kernel
shape 1) -- both queue the same kernels, so any difference would be a wrong
layout of the fixed scratch -- and it is checked against the FP64 oracle
(Eq. 1) within the parity tolerances of the other GPU tests.  The file sorts
last so that a run stopping at the first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest

import nbody_inputs as ni

pytestmark = pytest.mark.gpu

ACC_MED, ACC_MAX, POT_MAX = 2e-6, 1e-4, 1e-5
MAX_N = 65536
NOALLOC_SHAPE = 1  # 256 threads x 2 packed i-pairs, 1024-body i-blocks


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim == 2:
        return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    return np.abs(a - b) / np.abs(b)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@pytest.mark.parametrize("n,with_pot,masses", [(MAX_N, True, "loguniform"), (5000, False, "equal"),
                                                (4099, True, "equal"), (1, True, "equal")])
def test_noalloc_matches_accel_and_oracle_twice(nb, oracle_mod, n, with_pot, masses):
    import torch
    lib = nb.load()
    p, _, m = ni.plummer(n, 4242 + n, masses=masses, offset=(1e4, -3e3, 7e2))
    m = m.astype(np.float32).astype(np.float64)
    P = torch.from_numpy(p).cuda()
    M = torch.from_numpy(m.astype(np.float32)).cuda()
    eps = 2.0 ** -9
    # the allocating entry point with the same options
    acc_ref = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot_ref = torch.empty((n,), dtype=torch.float32, device="cuda") if with_pot else None
    nb.nbody_accel(P, M, eps, acc_ref, pot_ref, config=NOALLOC_SHAPE)
    torch.cuda.synchronize()
    acc_ref = acc_ref.cpu().numpy()
    pot_ref = pot_ref.cpu().numpy() if with_pot else None
    # the FP64 oracle on a seeded subsample (every body for small n)
    idx = np.arange(n) if n <= 8192 else ni.subsample(n, 2048, 77)
    ra, rp = oracle_mod.accel_subset(p, m, eps, idx)

    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty((n,), dtype=torch.float32, device="cuda") if with_pot else None
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        acc.fill_(float("nan"))
        if pot is not None:
            pot.fill_(float("nan"))
        rc = lib.nbody_accel_noalloc(n, _ptr(P), _ptr(M), eps, _ptr(acc), _ptr(pot), _ptr(status),
                                     ctypes.c_void_p(stream))
        assert rc == 0, nb._lib.strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        a = acc.cpu().numpy()
        assert np.array_equal(a, acc_ref), (call, np.abs(a - acc_ref).max())
        if with_pot:
            assert np.array_equal(pot.cpu().numpy(), pot_ref), call
        if n == 1:
            assert np.all(a == 0)
            assert float(pot.cpu()[0]) == 0.0
            continue
        e = _rel(a[idx], ra)
        assert np.median(e) <= ACC_MED and e.max() <= ACC_MAX, (call, np.median(e), e.max())
        if with_pot:
            ep = _rel(pot.cpu().numpy()[idx], rp)
            assert ep.max() <= POT_MAX, (call, ep.max())


def test_noalloc_allocates_nothing_and_rejects_out_of_range(nb):
    import torch
    lib = nb.load()
    n = 3000
    p, _, m = ni.plummer(n, 99)
    P = torch.from_numpy(p).cuda()
    M = torch.from_numpy(m.astype(np.float32)).cuda()
    acc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.nbody_accel_noalloc(n, _ptr(P), _ptr(M), 0.01, _ptr(acc), None, None, s) == 0  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert lib.nbody_accel_noalloc(n, _ptr(P), _ptr(M), 0.01, _ptr(acc), None, None, s) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # beyond the stated maximum: rejected before any work is queued
    big = MAX_N + 1
    assert lib.nbody_accel_noalloc(big, _ptr(P), _ptr(M), 0.01, _ptr(acc), None, None, s) == nb.NBODY_EINVAL
    # host arrays would need staging buffers: rejected
    ph = np.ascontiguousarray(p)
    assert lib.nbody_accel_noalloc(n, ctypes.c_void_p(ph.ctypes.data), _ptr(M), 0.01, _ptr(acc), None, None,
                                   s) == nb.NBODY_EINVAL
    assert lib.nbody_accel_noalloc(n, _ptr(P), _ptr(M), -1.0, _ptr(acc), None, None, s) == nb.NBODY_EINVAL
