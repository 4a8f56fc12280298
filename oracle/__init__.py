"""FP64 CPU oracle for the all-pairs softened N-body force (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package; the CUDA library neither imports nor links it, and it
shares no code with the library.  The arithmetic lives in ``oracle.c``
(Eq. 1 of Miki & Hanawa, Sec. III.A, summed directly in double precision); this
module compiles it with gcc and wraps it for numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_accel.argtypes = [i64, vp, vp, dbl, vp, vp]
        lib.oracle_accel_subset.argtypes = [i64, vp, vp, dbl, i64, vp, vp, vp]
        lib.oracle_leapfrog.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, vp]
        lib.oracle_energy.argtypes = [i64, vp, vp, vp, dbl, vp]
        lib.oracle_accel_ij.argtypes = [i64, vp, i64, vp, vp, dbl, vp, vp]
        lib.oracle_accel_vjp.argtypes = [i64, vp, vp, dbl, vp, vp, vp, vp]
        lib.oracle_leapfrog_vjp.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, vp, vp, vp, vp, vp]
        flt = ctypes.c_float
        lib.oracle_accel_listing_f32.argtypes = [i64, vp, vp, flt, vp, vp]
        lib.oracle_accel_listing_f32_subset.argtypes = [i64, vp, vp, flt, i64, vp, vp, vp]
        _lib = lib
    return _lib


def _c(a, dtype=np.float64, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(nt: int) -> None:
    _load().oracle_set_threads(int(nt))


def accel(pos, mass, eps, with_pot: bool = True):
    """Eq. 1 for all bodies: returns (acc (n,3), pot (n,) or None), float64."""
    pos = _c(pos)
    n = pos.shape[0]
    pos = _c(pos, shape=(n, 3))
    mass = _c(mass, shape=(n,))
    acc = np.zeros((n, 3))
    pot = np.zeros(n) if with_pot else None
    _load().oracle_accel(n, _p(pos), _p(mass), float(eps), _p(acc), _p(pot))
    return acc, pot


def accel_subset(pos, mass, eps, idx, with_pot: bool = True):
    """Eq. 1 for the bodies listed in ``idx`` against all bodies."""
    pos = _c(pos)
    n = pos.shape[0]
    mass = _c(mass, shape=(n,))
    idx = _c(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise IndexError("subset index out of range")
    ns = idx.shape[0]
    acc = np.zeros((ns, 3))
    pot = np.zeros(ns) if with_pot else None
    _load().oracle_accel_subset(n, _p(pos), _p(mass), float(eps), ns, _p(idx), _p(acc), _p(pot))
    return acc, pot


def accel_listing_f32(pos, mass, eps, with_pot: bool = True, idx=None):
    """Listing 4's FP32 arithmetic, every operation correctly rounded, one
    running FP32 sum per body in j order, self pair skipped: (acc (n,3),
    pot (n,) or None) as float32.  Positions, masses and eps are rounded to
    FP32 first.  With ``idx``, only the listed bodies (each against all)."""
    pos = _c(pos, dtype=np.float32)
    n = pos.shape[0]
    pos = _c(pos, dtype=np.float32, shape=(n, 3))
    mass = _c(mass, dtype=np.float32, shape=(n,))
    if idx is None:
        acc = np.zeros((n, 3), np.float32)
        pot = np.zeros(n, np.float32) if with_pot else None
        _load().oracle_accel_listing_f32(n, _p(pos), _p(mass), float(np.float32(eps)), _p(acc), _p(pot))
        return acc, pot
    idx = _c(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise IndexError("subset index out of range")
    ns = idx.shape[0]
    acc = np.zeros((ns, 3), np.float32)
    pot = np.zeros(ns, np.float32) if with_pot else None
    _load().oracle_accel_listing_f32_subset(n, _p(pos), _p(mass), float(np.float32(eps)), ns, _p(idx), _p(acc),
                                            _p(pot))
    return acc, pot


def accel_ij(ipos, jpos, jmass, eps, with_pot=True):
    """Listing 4's form: every sink against every source, no pair excluded."""
    ipos = _c(ipos)
    jpos = _c(jpos)
    ni, nj = ipos.shape[0], jpos.shape[0]
    jmass = _c(jmass, shape=(nj,))
    acc = np.zeros((ni, 3))
    pot = np.zeros(ni) if with_pot else None
    _load().oracle_accel_ij(ni, _p(ipos), nj, _p(jpos), _p(jmass), float(eps), _p(acc), _p(pot))
    return acc, pot


def leapfrog(pos, vel, mass, eps, dt, steps):
    """KDK leapfrog for ``steps`` steps: returns (pos, vel, acc) at the end (copies)."""
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    vel = np.array(vel, dtype=np.float64, order="C", copy=True)
    n = pos.shape[0]
    mass = _c(mass, shape=(n,))
    acc = np.zeros((n, 3))
    _load().oracle_leapfrog(n, _p(pos), _p(vel), _p(mass), float(eps), float(dt), int(steps), _p(acc))
    return pos, vel, acc


def energy(pos, vel, mass, eps):
    """Returns dict T, W, E, P (3,), F (3,) = sum m a."""
    pos = _c(pos)
    n = pos.shape[0]
    vel = _c(vel, shape=(n, 3))
    mass = _c(mass, shape=(n,))
    out = np.zeros(9)
    _load().oracle_energy(n, _p(pos), _p(vel), _p(mass), float(eps), _p(out))
    return {"T": out[0], "W": out[1], "E": out[2], "P": out[3:6].copy(), "F": out[6:9].copy()}


def accel_vjp(pos, mass, eps, lam, mu=None):
    """Reverse mode of Eq. 1: (g_pos (n,3), g_mass (n,)) = gradients of
    sum_i lam_i.a_i (+ mu_i phi_i) with respect to positions and masses."""
    pos = _c(pos)
    n = pos.shape[0]
    mass = _c(mass, shape=(n,))
    lam = _c(lam, shape=(n, 3))
    mu = _c(mu, shape=(n,)) if mu is not None else None
    g = np.zeros((n, 3))
    gm = np.zeros(n)
    _load().oracle_accel_vjp(n, _p(pos), _p(mass), float(eps), _p(lam), _p(mu), _p(g), _p(gm))
    return g, gm


def leapfrog_vjp(pos0, vel0, mass, eps, dt, steps, gx_T, gv_T):
    """Reverse mode of ``leapfrog``: (dL/dx0, dL/dv0, dL/dm through the dynamics)."""
    pos0 = _c(pos0)
    n = pos0.shape[0]
    vel0 = _c(vel0, shape=(n, 3))
    mass = _c(mass, shape=(n,))
    gx_T = _c(gx_T, shape=(n, 3))
    gv_T = _c(gv_T, shape=(n, 3))
    gx0 = np.zeros((n, 3))
    gv0 = np.zeros((n, 3))
    gm = np.zeros(n)
    _load().oracle_leapfrog_vjp(n, _p(pos0), _p(vel0), _p(mass), float(eps), float(dt), int(steps), _p(gx_T),
                                _p(gv_T), _p(gx0), _p(gv0), _p(gm))
    return gx0, gv0, gm
