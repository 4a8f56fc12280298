"""Python binding of libnbody with the C ABI's names (argument marshalling only).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; each must be
C-contiguous with the dtype and shape the C call expects.  CUDA tensors are
passed in place and the call is queued on the tensor's current torch stream
(or ``stream=``); host arrays are staged by the library and the call returns
when results are back.  Every computation happens in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import NbodyOpts, check, load

try:  # torch is only plumbing (device memory and streams)
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_torch(a):
    return torch is not None and isinstance(a, torch.Tensor)


_TORCH_DT = {"f32": "float32", "f64": "float64"}


def _ptr(a, dtype: str, shape, name: str):
    """Data pointer of ``a`` after checking dtype, shape and contiguity."""
    if a is None:
        return None
    if _is_torch(a):
        if str(a.dtype) != "torch." + _TORCH_DT[dtype]:
            raise TypeError(f"{name}: expected torch.{_TORCH_DT[dtype]}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(a.shape)}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(_TORCH_DT[dtype]):
            raise TypeError(f"{name}: expected {_TORCH_DT[dtype]}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: must be C-contiguous")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(a.shape)}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name}: expected a torch tensor or numpy array")


def make_opts(arrays=(), stream=None, precision=_lib.NBODY_PREC_MIXED, accumulate=_lib.NBODY_ACC_COMPENSATED,
              config=-1):
    o = NbodyOpts()
    load().nbody_opts_default(ctypes.byref(o))
    if stream is None:
        for a in arrays:
            if _is_torch(a) and a.is_cuda:
                stream = torch.cuda.current_stream(a.device)
                break
    if stream is not None:
        o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    o.precision = int(precision)
    o.accumulate = int(accumulate)
    o.config = int(config)
    return o


def _n(pos):
    return int(pos.shape[0])


def nbody_accel(pos, mass, eps, acc, pot=None, **kw):
    """nbody_accel: pos (n,3) f64, mass (n,) f32, acc (n,3) f32 out, pot (n,) f32 out or None."""
    n = _n(pos)
    o = make_opts((pos, mass, acc, pot), **kw)
    check(load().nbody_accel(n, _ptr(pos, "f64", (n, 3), "pos"), _ptr(mass, "f32", (n,), "mass"), float(eps),
                             _ptr(acc, "f32", (n, 3), "acc"), _ptr(pot, "f32", (n,), "pot"), ctypes.byref(o)),
          "nbody_accel")


def nbody_accel_f32(pos, mass, eps, acc, pot=None, **kw):
    """nbody_accel_f32: pos (n,3) f32, mass (n,) f32, acc (n,3) f32 out, pot (n,) f32 out or None."""
    n = _n(pos)
    o = make_opts((pos, mass, acc, pot), **kw)
    check(load().nbody_accel_f32(n, _ptr(pos, "f32", (n, 3), "pos"), _ptr(mass, "f32", (n,), "mass"), float(eps),
                                 _ptr(acc, "f32", (n, 3), "acc"), _ptr(pot, "f32", (n,), "pot"), ctypes.byref(o)),
          "nbody_accel_f32")


def nbody_leapfrog(pos, vel, mass, eps, dt, steps, **kw):
    """nbody_leapfrog: pos, vel (n,3) f64 updated in place; mass (n,) f32."""
    n = _n(pos)
    o = make_opts((pos, vel, mass), **kw)
    check(load().nbody_leapfrog(n, _ptr(pos, "f64", (n, 3), "pos"), _ptr(vel, "f64", (n, 3), "vel"),
                                _ptr(mass, "f32", (n,), "mass"), float(eps), float(dt), int(steps), ctypes.byref(o)),
          "nbody_leapfrog")


def nbody_leapfrog_f32(pos, vel, mass, eps, dt, steps, **kw):
    """nbody_leapfrog_f32: pos, vel (n,3) f32 updated in place; mass (n,) f32."""
    n = _n(pos)
    o = make_opts((pos, vel, mass), **kw)
    check(load().nbody_leapfrog_f32(n, _ptr(pos, "f32", (n, 3), "pos"), _ptr(vel, "f32", (n, 3), "vel"),
                                    _ptr(mass, "f32", (n,), "mass"), float(eps), float(dt), int(steps),
                                    ctypes.byref(o)),
          "nbody_leapfrog_f32")


def _i64ptr(a, shape, name):
    if _is_torch(a):
        if str(a.dtype) != "torch.int64" or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: expected contiguous torch.int64 of shape {tuple(shape)}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != np.int64 or not a.flags["C_CONTIGUOUS"] or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: expected C-contiguous int64 of shape {tuple(shape)}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name}: expected a torch tensor or numpy array")


def nbody_accel_batched(offsets, pos, mass, eps, acc, pot=None, **kw):
    """nbody_accel_batched: offsets (nsys+1,) int64, pos (N,3) f32, mass (N,) f32, eps (nsys,) f32,
    acc (N,3) f32 out, pot (N,) f32 out or None."""
    nsys = int(offsets.shape[0]) - 1
    n = int(pos.shape[0])
    o = make_opts((pos, mass, acc, pot), **kw)
    check(load().nbody_accel_batched(nsys, _i64ptr(offsets, (nsys + 1,), "offsets"), _ptr(pos, "f32", (n, 3), "pos"),
                                     _ptr(mass, "f32", (n,), "mass"), _ptr(eps, "f32", (nsys,), "eps"),
                                     _ptr(acc, "f32", (n, 3), "acc"), _ptr(pot, "f32", (n,), "pot"), ctypes.byref(o)),
          "nbody_accel_batched")


def nbody_leapfrog_batched(offsets, pos, vel, mass, eps, dt, steps, **kw):
    """nbody_leapfrog_batched: pos, vel (N,3) f32 updated in place."""
    nsys = int(offsets.shape[0]) - 1
    n = int(pos.shape[0])
    o = make_opts((pos, vel, mass), **kw)
    check(load().nbody_leapfrog_batched(nsys, _i64ptr(offsets, (nsys + 1,), "offsets"),
                                        _ptr(pos, "f32", (n, 3), "pos"), _ptr(vel, "f32", (n, 3), "vel"),
                                        _ptr(mass, "f32", (n,), "mass"), _ptr(eps, "f32", (nsys,), "eps"),
                                        float(dt), int(steps), ctypes.byref(o)),
          "nbody_leapfrog_batched")


def _accel_ij(fn, name, dt, ipos, jpos, jmass, eps, acc, pot, **kw):
    ni, nj = _n(ipos), _n(jpos)
    o = make_opts((ipos, jpos, acc, pot), **kw)
    check(fn(ni, _ptr(ipos, dt, (ni, 3), "ipos"), nj, _ptr(jpos, dt, (nj, 3), "jpos"),
             _ptr(jmass, "f32", (nj,), "jmass"), float(eps), _ptr(acc, "f32", (ni, 3), "acc"),
             _ptr(pot, "f32", (ni,), "pot"), ctypes.byref(o)), name)


def nbody_accel_ij(ipos, jpos, jmass, eps, acc, pot=None, **kw):
    """nbody_accel_ij: sinks ipos (ni,3) f64, sources jpos (nj,3) f64 with jmass (nj,) f32."""
    _accel_ij(load().nbody_accel_ij, "nbody_accel_ij", "f64", ipos, jpos, jmass, eps, acc, pot, **kw)


def nbody_accel_ij_f32(ipos, jpos, jmass, eps, acc, pot=None, **kw):
    """nbody_accel_ij_f32: as nbody_accel_ij with FP32 positions."""
    _accel_ij(load().nbody_accel_ij_f32, "nbody_accel_ij_f32", "f32", ipos, jpos, jmass, eps, acc, pot, **kw)


def nbody_accel_vjp(pos, mass, eps, g_acc, g_pot, g_pos, g_mass, **kw):
    """nbody_accel_vjp: pos (n,3) f64, mass (n,) f32, g_acc (n,3) f32, g_pot (n,) f32 or None;
    g_pos (n,3) f32 and g_mass (n,) f32 are overwritten."""
    n = _n(pos)
    o = make_opts((pos, mass, g_acc, g_pos), **kw)
    check(load().nbody_accel_vjp(n, _ptr(pos, "f64", (n, 3), "pos"), _ptr(mass, "f32", (n,), "mass"), float(eps),
                                 _ptr(g_acc, "f32", (n, 3), "g_acc"), _ptr(g_pot, "f32", (n,), "g_pot"),
                                 _ptr(g_pos, "f32", (n, 3), "g_pos"), _ptr(g_mass, "f32", (n,), "g_mass"),
                                 ctypes.byref(o)),
          "nbody_accel_vjp")


def nbody_tape_bytes(n, steps, ckpt_every):
    b = int(load().nbody_tape_bytes(int(n), int(steps), int(ckpt_every)))
    if b < 0:
        raise ValueError("invalid tape size arguments")
    return b


def _tape_ptr(tape):
    if not (_is_torch(tape) and tape.is_cuda and tape.is_contiguous()):
        raise TypeError("tape: expected a contiguous CUDA tensor")
    return ctypes.c_void_p(tape.data_ptr())


def nbody_leapfrog_record(pos, vel, mass, eps, dt, steps, ckpt_every, tape, **kw):
    """nbody_leapfrog_record: pos, vel (n,3) f64 on the device, in place; tape: CUDA byte tensor of
    nbody_tape_bytes(n, steps, ckpt_every) bytes."""
    n = _n(pos)
    if tape.numel() * tape.element_size() < nbody_tape_bytes(n, steps, ckpt_every):
        raise ValueError("tape too small")
    o = make_opts((pos, vel, mass), **kw)
    check(load().nbody_leapfrog_record(n, _ptr(pos, "f64", (n, 3), "pos"), _ptr(vel, "f64", (n, 3), "vel"),
                                       _ptr(mass, "f32", (n,), "mass"), float(eps), float(dt), int(steps),
                                       int(ckpt_every), _tape_ptr(tape), ctypes.byref(o)),
          "nbody_leapfrog_record")


def nbody_leapfrog_vjp_tape(mass, eps, dt, steps, ckpt_every, tape, g_posT, g_velT, g_pos0, g_vel0, g_mass, **kw):
    """nbody_leapfrog_vjp_tape: the reverse sweep from a tape of nbody_leapfrog_record; cotangents
    g_posT, g_velT (n,3) f64; outputs g_pos0, g_vel0 (n,3) f64 and g_mass (n,) f64 (the dynamics'
    part of dL/dm)."""
    n = int(mass.shape[0])
    o = make_opts((mass, g_posT, g_pos0), **kw)
    check(load().nbody_leapfrog_vjp_tape(n, _ptr(mass, "f32", (n,), "mass"), float(eps), float(dt), int(steps),
                                         int(ckpt_every), _tape_ptr(tape), _ptr(g_posT, "f64", (n, 3), "g_posT"),
                                         _ptr(g_velT, "f64", (n, 3), "g_velT"), _ptr(g_pos0, "f64", (n, 3), "g_pos0"),
                                         _ptr(g_vel0, "f64", (n, 3), "g_vel0"), _ptr(g_mass, "f64", (n,), "g_mass"),
                                         ctypes.byref(o)),
          "nbody_leapfrog_vjp_tape")


def nbody_leapfrog_vjp(pos0, vel0, mass, eps, dt, steps, ckpt_every, g_posT, g_velT, g_pos0, g_vel0, g_mass, **kw):
    """nbody_leapfrog_vjp: gradients of a loss of (x(T), v(T)) with respect to pos0, vel0 (n,3) f64
    and mass (n,) f32 in one call (forward run recorded in the library's workspace, then swept);
    outputs g_pos0, g_vel0 (n,3) f64 and g_mass (n,) f64."""
    n = _n(pos0)
    o = make_opts((pos0, vel0, mass, g_posT, g_pos0), **kw)
    check(load().nbody_leapfrog_vjp(n, _ptr(pos0, "f64", (n, 3), "pos0"), _ptr(vel0, "f64", (n, 3), "vel0"),
                                    _ptr(mass, "f32", (n,), "mass"), float(eps), float(dt), int(steps),
                                    int(ckpt_every), _ptr(g_posT, "f64", (n, 3), "g_posT"),
                                    _ptr(g_velT, "f64", (n, 3), "g_velT"), _ptr(g_pos0, "f64", (n, 3), "g_pos0"),
                                    _ptr(g_vel0, "f64", (n, 3), "g_vel0"), _ptr(g_mass, "f64", (n,), "g_mass"),
                                    ctypes.byref(o)),
          "nbody_leapfrog_vjp")


def _energy(fn, name, dt, pos, vel, mass, eps, **kw):
    n = _n(pos)
    o = make_opts((pos, vel, mass), **kw)
    out = np.zeros(9, dtype=np.float64)
    check(fn(n, _ptr(pos, dt, (n, 3), "pos"), _ptr(vel, dt, (n, 3), "vel"), _ptr(mass, "f32", (n,), "mass"),
             float(eps), ctypes.c_void_p(out.ctypes.data), ctypes.byref(o)), name)
    return {"T": out[0], "W": out[1], "E": out[2], "P": out[3:6].copy(), "F": out[6:9].copy()}


def nbody_energy(pos, vel, mass, eps, **kw):
    """nbody_energy (FP64 state): dict T, W, E, P (3,), F (3,)."""
    return _energy(load().nbody_energy, "nbody_energy", "f64", pos, vel, mass, eps, **kw)


def nbody_energy_f32(pos, vel, mass, eps, **kw):
    """nbody_energy_f32 (FP32 state): dict T, W, E, P (3,), F (3,)."""
    return _energy(load().nbody_energy_f32, "nbody_energy_f32", "f32", pos, vel, mass, eps, **kw)


def nbody_last_device_error():
    return int(load().nbody_last_device_error())


def nbody_num_configs():
    return int(load().nbody_num_configs())


def nbody_num_batched_configs():
    return int(load().nbody_num_batched_configs())


def nbody_config_block(k):
    return int(load().nbody_config_block(int(k)))


def nbody_selftest_wait(limit_seconds, **kw):
    """Returns the library code (NBODY_ETIMEOUT when the bounded wait works)."""
    o = make_opts((), **kw)
    return int(load().nbody_selftest_wait(float(limit_seconds), ctypes.byref(o)))


def nbody_profile_enable(on=True):
    load().nbody_profile_enable(1 if on else 0)


def nbody_profile_read():
    """(force-kernel ms, force-kernel launches, all kernel launches) since the last read."""
    ms, k, allk = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    check(load().nbody_profile_read(ctypes.byref(ms), ctypes.byref(k), ctypes.byref(allk)), "nbody_profile_read")
    return ms.value, k.value, allk.value


PROFILE_KINDS = {"force": 0, "pack": 1, "kick": 2, "vjp": 3}


def nbody_profile_read_kind(kind):
    """(ms, launches) of one timed kernel kind since its last read: "force", "pack" (kick, drift
    and packed j-array of a leapfrog step), "kick" (the closing half kick) or "vjp" (the force
    VJP kernel)."""
    ms, k = ctypes.c_double(), ctypes.c_int64()
    check(load().nbody_profile_read_kind(PROFILE_KINDS[kind], ctypes.byref(ms), ctypes.byref(k)),
          "nbody_profile_read_kind")
    return ms.value, k.value


def nbody_finalize():
    load().nbody_finalize()


def nbody_version():
    return int(load().nbody_version())


# ---------------------------------------------------------------------------
# Convenience: allocate outputs with torch on the inputs' device.
# ---------------------------------------------------------------------------
def accel(pos, mass, eps, with_pot=True, **kw):
    """(acc, pot) for torch tensors; pos f64 uses nbody_accel, f32 nbody_accel_f32."""
    n = _n(pos)
    acc = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
    pot = torch.empty((n,), dtype=torch.float32, device=pos.device) if with_pot else None
    if pos.dtype == torch.float64:
        nbody_accel(pos, mass, eps, acc, pot, **kw)
    else:
        nbody_accel_f32(pos, mass, eps, acc, pot, **kw)
    return acc, pot
