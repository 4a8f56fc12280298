"""torch.autograd binding of the checkpointed leapfrog adjoint.

``Trajectory.apply(x0, v0, m, eps, dt, steps, ckpt_every)`` integrates the
kick-drift-kick leapfrog driven by Eq. 1 (Miki & Hanawa, Sec. III.A) with
nbody_leapfrog_record and returns (x(T), v(T)); its backward calls
nbody_leapfrog_vjp_tape on the recorded tape, so the gradients of any loss of (x(T), v(T)) with respect
to x0, v0 and m come from the library's adjoint kernels.  A loss that also uses
m directly gets that term from torch's own graph.
"""
from __future__ import annotations

import torch

from . import api


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, eps, dt, steps, ckpt_every):
        if not (x0.is_cuda and v0.is_cuda and m.is_cuda):
            raise TypeError("Trajectory: x0, v0 and m must be CUDA tensors")
        n = int(x0.shape[0])
        x = x0.detach().to(torch.float64).contiguous().clone()
        v = v0.detach().to(torch.float64).contiguous().clone()
        m32 = m.detach().to(torch.float32).contiguous()
        tape = torch.empty(api.nbody_tape_bytes(n, steps, ckpt_every), dtype=torch.uint8, device=x.device)
        api.nbody_leapfrog_record(x, v, m32, eps, dt, steps, ckpt_every, tape)
        ctx.save_for_backward(m32, tape)
        ctx.params = (float(eps), float(dt), int(steps), int(ckpt_every), m.dtype, x0.dtype, v0.dtype)
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        m32, tape = ctx.saved_tensors
        eps, dt, steps, ckpt, mdt, xdt, vdt = ctx.params
        n = int(m32.shape[0])
        z = lambda: torch.zeros((n, 3), dtype=torch.float64, device=m32.device)
        gx = z() if gx is None else gx.to(torch.float64).contiguous()
        gv = z() if gv is None else gv.to(torch.float64).contiguous()
        g_x0, g_v0 = z(), z()
        g_m = torch.zeros((n,), dtype=torch.float64, device=m32.device)
        api.nbody_leapfrog_vjp_tape(m32, eps, dt, steps, ckpt, tape, gx, gv, g_x0, g_v0, g_m)
        return g_x0.to(xdt), g_v0.to(vdt), g_m.to(mdt), None, None, None, None
