"""Failure paths on the GPU without faulting it: the bounded device wait,
host-side fault injection, invalid arguments with device arrays."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounded_wait_times_out_and_context_survives(nb):
    import torch
    assert nb.nbody_selftest_wait(0.01) == nb.NBODY_ETIMEOUT
    assert nb.nbody_selftest_wait(0.001) == nb.NBODY_ETIMEOUT
    # the context is still usable and the flag was cleared
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0
    assert nb.nbody_last_device_error() == 0
    pos = torch.rand((100, 3), dtype=torch.float32, device="cuda")
    m = torch.full((100,), 0.01, dtype=torch.float32, device="cuda")
    acc = torch.empty((100, 3), dtype=torch.float32, device="cuda")
    nb.nbody_accel_f32(pos, m, 0.1, acc)
    torch.cuda.synchronize()
    assert torch.isfinite(acc).all()
    with pytest.raises(nb.NbodyError):
        nb.api.check(nb.load().nbody_selftest_wait(5.0, None), "limit")


@pytest.mark.parametrize("fault,code", [("alloc", -2), ("launch", -3)])
def test_host_fault_injection(fault, code):
    """NBODY_FAULT makes the library report the error without GPU work; run in
    a child so the variable does not leak into other tests."""
    prog = (
        "import numpy as np, torch, paper_2411_18889_gb300 as nb, ctypes\n"
        "p=torch.rand((64,3),dtype=torch.float32,device='cuda'); m=torch.ones(64,device='cuda')\n"
        "a=torch.empty((64,3),device='cuda')\n"
        "try:\n  nb.nbody_accel_f32(p,m,0.1,a)\nexcept nb.NbodyError as e:\n  print('CODE', e.code)\n"
    )
    env = dict(os.environ, NBODY_FAULT=fault)
    r = subprocess.run([sys.executable, "-c", prog], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert f"CODE {code}" in r.stdout, r.stdout + r.stderr


def test_wrong_arguments_with_device_arrays(nb):
    import torch
    pos = torch.rand((10, 3), dtype=torch.float64, device="cuda")
    m = torch.ones(10, dtype=torch.float32, device="cuda")
    acc = torch.empty((10, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(nb.NbodyError) as ei:
        nb.nbody_accel(pos, m, -1.0, acc)
    assert ei.value.code == nb.NBODY_EINVAL
    with pytest.raises(nb.NbodyError):
        nb.nbody_leapfrog(pos, pos.clone(), m, 0.1, float("inf"), 3)
