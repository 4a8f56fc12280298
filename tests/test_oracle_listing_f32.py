"""Pins of the oracle's FP32 restatement of Listing 4 (Sec. III.A).

The restatement claims two things, each pinned here by something other than
itself:

- It performs the listing's FP32 operations, in the listing's order, each
  correctly rounded.  Checked bit for bit against a brute force in exact
  rational arithmetic (Python fractions), rounded to binary32 once per
  operation, on tiny systems: a reordered FMA chain, a missing rounding or a
  wrong association fails it.
- Its error against Eq. 1 is that of FP32 arithmetic.  Checked against the
  FP64 oracle with the a-priori bound of recursive summation: per body and
  component |a32 - a64| <= (n + 24) u sum_j |t_j| with u = 2^-24 and t_j the
  exact pair terms (each term carries at most about a dozen roundings, the
  running sum at most n - 1 more).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import nbody_inputs as ni

U = 2.0 ** -24


def _f32(x: Fraction) -> np.float32:
    """Round an exact rational to the nearest binary32 (ties to even); normal range only."""
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    ax = abs(x)
    e = math.floor(math.log2(ax))
    while Fraction(2) ** e > ax:
        e -= 1
    while Fraction(2) ** (e + 1) <= ax:
        e += 1
    assert -126 <= e <= 127, "outside the normal binary32 range"
    scale = Fraction(2) ** (e - 23)
    q = ax / scale
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return np.float32(sign * float(fl * scale))


def _fma(a, b, c) -> np.float32:
    return _f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def _listing_exact(pos, mass, eps):
    """Listing 4's per-pair sequence with one correct binary32 rounding per
    operation (numpy float32 add/mul/div/sqrt round correctly; the fused
    multiply-adds are rounded from exact rationals)."""
    pos = np.asarray(pos, np.float32)
    mass = np.asarray(mass, np.float32)
    e = np.float32(eps)
    eps2 = e * e
    n = pos.shape[0]
    acc = np.zeros((n, 3), np.float32)
    pot = np.zeros(n, np.float32)
    for i in range(n):
        ax = ay = az = p = np.float32(0.0)
        for j in range(n):
            if j == i:
                continue
            dx = pos[j, 0] - pos[i, 0]
            dy = pos[j, 1] - pos[i, 1]
            dz = pos[j, 2] - pos[i, 2]
            r2 = _fma(dz, dz, _fma(dy, dy, _fma(dx, dx, eps2)))
            w = np.float32(1.0) / np.sqrt(r2)
            w = w * (w * w)
            w = w * mass[j]
            ax = _fma(dx, w, ax)
            ay = _fma(dy, w, ay)
            az = _fma(dz, w, az)
            p = _fma(r2, w, p)
        acc[i] = (ax, ay, az)
        pot[i] = -p
    return acc, pot


def test_two_bodies_exact(oracle_mod):
    """Separation 2 along x, masses 1 and 3, eps = 0: every intermediate is a
    power of two times a small integer, so the results are exact."""
    a, p = oracle_mod.accel_listing_f32(np.array([[0.0, 0, 0], [2.0, 0, 0]]), np.array([1.0, 3.0]), 0.0)
    assert a.dtype == np.float32 and p.dtype == np.float32
    assert np.array_equal(a, np.array([[0.75, 0, 0], [-0.25, 0, 0]], np.float32))
    assert np.array_equal(p, np.array([-1.5, -0.5], np.float32))


@pytest.mark.parametrize("seed", range(8))
def test_bitwise_against_exact_rounding(oracle_mod, seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(2, 7))
    pos = rng.uniform(-3.0, 3.0, size=(n, 3))
    mass = rng.uniform(0.1, 2.0, size=n)
    eps = float(rng.uniform(0.01, 0.3))
    a, p = oracle_mod.accel_listing_f32(pos, mass, eps)
    ra, rp = _listing_exact(pos, mass, eps)
    assert np.array_equal(a, ra), (seed, a - ra)
    assert np.array_equal(p, rp), (seed, p - rp)


@pytest.mark.parametrize("n,eps,masses", [(512, 2.0 ** -7, "equal"), (777, 1e-3, "loguniform"),
                                          (300, 0.0, "loguniform")])
def test_within_fp32_bound_of_fp64_oracle(oracle_mod, n, eps, masses):
    p, _, m = ni.plummer(n, 900 + n, masses=masses)
    p = p.astype(np.float32).astype(np.float64)  # both sides see the same inputs
    m = m.astype(np.float32).astype(np.float64)
    eps = float(np.float32(eps))
    a64, p64 = oracle_mod.accel(p, m, eps)
    a32, p32 = oracle_mod.accel_listing_f32(p, m, eps)
    # exact pair terms, |t_j| per component, summed (numpy FP64, O(n^2))
    d = p[None, :, :] - p[:, None, :]
    s = np.sum(d * d, axis=2) + eps * eps
    np.fill_diagonal(s, np.inf)
    ta = np.abs(d) * (m[None, :] / s ** 1.5)[:, :, None]
    tp = m[None, :] / np.sqrt(s)
    gam = (n + 24) * U
    assert np.all(np.abs(a32 - a64) <= gam * ta.sum(axis=1))
    assert np.all(np.abs(p32 - p64) <= gam * tp.sum(axis=1))
    rel = np.linalg.norm(a32 - a64, axis=1) / np.linalg.norm(a64, axis=1)
    assert np.median(rel) <= 16 * U  # typical error: a few ulps, far below the worst case


def test_subset_matches_full(oracle_mod):
    p, _, m = ni.plummer(1000, 17, masses="loguniform")
    a, q = oracle_mod.accel_listing_f32(p, m, 0.01)
    idx = ni.subsample(1000, 64, 3)
    b, r = oracle_mod.accel_listing_f32(p, m, 0.01, idx=idx)
    assert np.array_equal(a[idx], b) and np.array_equal(q[idx], r)
