"""Seeded Plummer spheres and the workload configurations built from them.

The N-body demonstration of Miki & Hanawa (§III.A, Eq. 1) states the force law
but gives no initial conditions; the ones here are the standard
Aarseth-Henon-Wielen (1974) construction of a Plummer model in Henon units
(G = M = 1, total energy -1/4, Plummer scale a = 3*pi/16):

* radius from the cumulative mass fraction X: r = a (X^(-2/3) - 1)^(-1/2),
  redrawn when r > 10 a;
* isotropic direction;
* speed q * v_esc(r) with v_esc = sqrt(2) (r^2 + a^2)^(-1/4) and q drawn by von
  Neumann rejection from g(q) = q^2 (1 - q^2)^(7/2) under the bound 0.1;
* isotropic velocity direction;
* centre-of-mass position and velocity removed, no energy rescaling.

Every random number comes from ``rng.uniform`` on a named sub-stream, with a
counter that encodes (body, attempt, draw), so the arrays depend only on the
seed and N.  No force, potential or integrator arithmetic lives here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import rng

PLUMMER_A = 3.0 * math.pi / 16.0
R_CUT = 10.0
_MAX_ATTEMPTS = 1 << 10
# sub-stream ids
_S_RADIUS, _S_POSDIR, _S_SPEED, _S_VELDIR, _S_MASS, _S_SUBSAMPLE, _S_NSYS, _S_GAUSS = range(8)


def _rejection(key, n, ndraw, accept_fn):
    """Vectorised rejection sampling: body i, attempt t uses draws
    (i * _MAX_ATTEMPTS + t) * ndraw + d, d < ndraw.  Returns the accepted draws
    (n, ndraw)."""
    out = np.empty((n, ndraw), dtype=np.float64)
    pending = np.arange(n, dtype=np.int64)
    for t in range(_MAX_ATTEMPTS):
        if pending.size == 0:
            return out
        base = (pending.astype(np.uint64) * np.uint64(_MAX_ATTEMPTS) + np.uint64(t)) * np.uint64(ndraw)
        u = np.stack([rng.uniform(key, base + np.uint64(d)) for d in range(ndraw)], axis=1)
        ok = accept_fn(u)
        out[pending[ok]] = u[ok]
        pending = pending[~ok]
    raise RuntimeError("rejection sampling did not converge")


def _isotropic(key, n, scale):
    c = np.arange(n, dtype=np.uint64) * np.uint64(2)
    u1 = rng.uniform(key, c)
    u2 = rng.uniform(key, c + np.uint64(1))
    cos_t = 2.0 * u1 - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * u2
    return np.stack([scale * sin_t * np.cos(phi), scale * sin_t * np.sin(phi), scale * cos_t], axis=1)


def plummer(n: int, seed: int, a: float = PLUMMER_A, masses: str = "equal",
            mass_range=(1e-3, 1.0), offset=(0.0, 0.0, 0.0)):
    """Plummer sphere of ``n`` bodies: returns (pos (n,3) f64, vel (n,3) f64, mass (n,) f64).

    ``masses``: "equal" (1/n each) or "loguniform" (log-uniform over
    ``mass_range``, renormalised to total 1).  ``offset`` is added to every
    position after the centre of mass is removed.
    """
    if n <= 0:
        z = np.zeros((0, 3))
        return z, z.copy(), np.zeros(0)
    k_r = rng.stream_key(seed, _S_RADIUS)
    k_pd = rng.stream_key(seed, _S_POSDIR)
    k_sp = rng.stream_key(seed, _S_SPEED)
    k_vd = rng.stream_key(seed, _S_VELDIR)
    k_m = rng.stream_key(seed, _S_MASS)

    def radius(u):
        x = u[:, 0]
        r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        return r <= R_CUT * a

    x1 = _rejection(k_r, n, 1, radius)[:, 0]
    r = a / np.sqrt(x1 ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(k_pd, n, r)

    def speed(u):
        q = u[:, 0]
        y = 0.1 * u[:, 1]
        return y < q * q * (1.0 - q * q) ** 3.5

    q = _rejection(k_sp, n, 2, speed)[:, 0]
    v = q * math.sqrt(2.0) * (r * r + a * a) ** (-0.25)
    vel = _isotropic(k_vd, n, v)

    if masses == "equal":
        mass = np.full(n, 1.0 / n)
    elif masses == "loguniform":
        lo, hi = mass_range
        u = rng.uniform(k_m, np.arange(n, dtype=np.uint64))
        mass = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
        mass = mass / mass.sum()
    else:
        raise ValueError(masses)

    mt = mass.sum()
    pos -= (mass[:, None] * pos).sum(axis=0) / mt
    vel -= (mass[:, None] * vel).sum(axis=0) / mt
    pos += np.asarray(offset, dtype=np.float64)[None, :]
    return pos, vel, mass


def subsample(n: int, k: int, seed: int) -> np.ndarray:
    """Sorted, distinct indices of ``k`` of ``n`` bodies (seeded)."""
    k = min(k, n)
    key = rng.stream_key(seed, _S_SUBSAMPLE)
    order = np.argsort(rng.raw(key, np.arange(n, dtype=np.uint64)), kind="stable")
    return np.sort(order[:k]).astype(np.int64)


def gaussian(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    """N(0, sigma^2) draws by Box-Muller on one seeded stream."""
    m = int(np.prod(shape))
    key = rng.stream_key(seed, _S_GAUSS)
    c = np.arange(m, dtype=np.uint64) * np.uint64(2)
    u1 = rng.uniform(key, c)
    u2 = rng.uniform(key, c + np.uint64(1))
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return (sigma * g).reshape(shape)


def ragged_sizes(nsys: int, nmin: int, nmax: int, seed: int) -> np.ndarray:
    """System sizes drawn log-uniformly from [nmin, nmax] (integers, seeded)."""
    key = rng.stream_key(seed, _S_NSYS)
    u = rng.uniform(key, np.arange(nsys, dtype=np.uint64))
    n = np.floor(np.exp(math.log(nmin) + u * (math.log(nmax + 1) - math.log(nmin))))
    return np.clip(n, nmin, nmax).astype(np.int64)


# ---------------------------------------------------------------------------
# workload configurations
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n: int
    pos: np.ndarray          # (n,3) f64
    vel: np.ndarray          # (n,3) f64
    mass: np.ndarray         # (n,) f64, exactly representable in f32
    eps: float
    dt: float
    steps: int
    state: str               # "f32" (FP32 state) or "f64" (FP64 positions)
    extra: dict = field(default_factory=dict)


def _f32_exact(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def small_plain(n: int = 1024, seed: int = 1) -> Workload:
    """N=1024 equal-mass Plummer, eps=2^-7, dt=2^-7, 16 steps, FP32 state."""
    p, v, m = plummer(n, seed)
    return Workload("plummer_n1024_fp32", n, _f32_exact(p), _f32_exact(v), _f32_exact(m),
                    2.0 ** -7, 2.0 ** -7, 16, "f32")


def throughput_plain(n: int = 65536, seed: int = 2) -> Workload:
    """N=65536 equal-mass Plummer, eps=2^-8, dt=2^-8, 128 steps, FP32 state."""
    p, v, m = plummer(n, seed)
    return Workload("plummer_n65536_fp32", n, _f32_exact(p), _f32_exact(v), _f32_exact(m),
                    2.0 ** -8, 2.0 ** -8, 128, "f32")


OFFSET_CENTRE = (1.0e4, -3.0e3, 7.0e2)


def plummer_offset():
    """Centre of the precision workload's sphere."""
    return OFFSET_CENTRE


def precision_offset(n: int = 1 << 20, seed: int = 3) -> Workload:
    """N=2^20 Plummer offset to (1e4,-3e3,7e2), log-uniform masses in [1e-3,1]
    renormalised to 1, eps=2^-9, dt=2^-9, 1 force evaluation + 4 steps, FP64
    positions."""
    p, v, m = plummer(n, seed, masses="loguniform", offset=OFFSET_CENTRE)
    m32 = _f32_exact(m)
    return Workload("plummer_n1048576_offset_mixed", n, p, v, m32, 2.0 ** -9, 2.0 ** -9, 4, "f64",
                    extra={"offset": OFFSET_CENTRE, "subsample": subsample(n, 4096, seed)})


def adjoint_case(n: int = 16384, seed: int = 5, target_seed: int = 6) -> Workload:
    """N=16384 Plummer, eps=2^-7, dt=2^-8, K=64 steps, FP64 positions; target
    y = x(0) + N(0, 0.05^2) offsets (seed 6)."""
    p, v, m = plummer(n, seed)
    y = p + gaussian((n, 3), target_seed, 0.05)
    return Workload("plummer_n16384_adjoint", n, p, v, _f32_exact(m), 2.0 ** -7, 2.0 ** -8, 64, "f64",
                    extra={"target": y, "ckpt_every": 8})


def ragged_batch(nsys: int = 4096, seed: int = 4, nmin: int = 64, nmax: int = 4096):
    """Ragged ensemble: sizes log-uniform in [nmin,nmax], each an equal-mass
    Plummer sphere with its own seed, eps_s = 4/sqrt(N_s), FP32 state.
    Returns (offsets (nsys+1,) i64, pos, vel, mass (concatenated), eps (nsys,))."""
    sizes = ragged_sizes(nsys, nmin, nmax, seed)
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    P, V, M = [], [], []
    for s, ns in enumerate(sizes):
        p, v, m = plummer(int(ns), seed * 1000003 + s + 1)
        P.append(p); V.append(v); M.append(m)
    pos = _f32_exact(np.concatenate(P))
    vel = _f32_exact(np.concatenate(V))
    mass = _f32_exact(np.concatenate(M))
    eps = _f32_exact(4.0 / np.sqrt(sizes.astype(np.float64)))
    return offsets, pos, vel, mass, eps
