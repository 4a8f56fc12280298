"""Property tests of the FP64 oracle on random small systems (seeded loops).

Each law below holds exactly for Eq. 1 and the potential, so a slip in an
exponent, a sign or an index breaks it for almost every random system:

- similarity: positions and softening scaled by L, masses by M, give
  accelerations scaled by M/L^2 and potentials by M/L;
- Newton's third law: sum_i m_i a_i = 0;
- superposition: the field of a system is the sum of the fields its two halves
  exert (sink/source split against the self-excluding sum);
- the potential energy W = 1/2 sum m_i phi_i equals the sum over pairs.

The random systems come from numpy's seeded generator (2..12 bodies, uniform
positions in a cube of half-width 0.5..5, masses in [0.1, 2], softening in
[0.01, 0.5]), so every case runs on every machine with no extra package.
"""
import numpy as np
import pytest

CASES = 60


def system(seed, max_n=10):
    rng = np.random.default_rng(1_000_003 * seed + 17)
    n = int(rng.integers(2, max_n + 1))
    spread = rng.uniform(0.5, 5.0)
    pos = rng.uniform(-spread, spread, size=(n, 3))
    mass = rng.uniform(0.1, 2.0, size=n)
    eps = rng.uniform(0.01, 0.5)
    return pos, mass, eps, rng


@pytest.mark.parametrize("seed", range(CASES))
def test_similarity_law(oracle_mod, seed):
    pos, mass, eps, rng = system(seed)
    L, M = rng.uniform(0.25, 4.0, size=2)
    a0, p0 = oracle_mod.accel(pos, mass, eps)
    a1, p1 = oracle_mod.accel(pos * L, mass * M, eps * L)
    np.testing.assert_allclose(a1, a0 * (M / L**2), rtol=1e-12, atol=1e-14 * np.abs(a0).max() * M / L**2)
    np.testing.assert_allclose(p1, p0 * (M / L), rtol=1e-12)


@pytest.mark.parametrize("seed", range(CASES))
def test_third_law(oracle_mod, seed):
    pos, mass, eps, _ = system(seed)
    a, _ = oracle_mod.accel(pos, mass, eps)
    f = mass[:, None] * a
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("seed", range(40))
def test_superposition_of_halves(oracle_mod, seed):
    pos, mass, eps, _ = system(seed, max_n=12)
    n = pos.shape[0]
    k = n // 2
    a, p = oracle_mod.accel(pos, mass, eps)
    # field on the first half: from the other bodies of the first half (self
    # excluded) plus the second half as external sources
    a_in, p_in = oracle_mod.accel(pos[:k], mass[:k], eps) if k > 0 else (np.zeros((0, 3)), np.zeros(0))
    a_ex, p_ex = oracle_mod.accel_ij(pos[:k], pos[k:], mass[k:], eps)
    np.testing.assert_allclose(a_in + a_ex, a[:k], rtol=1e-11, atol=1e-13 * np.abs(a).max())
    np.testing.assert_allclose(p_in + p_ex, p[:k], rtol=1e-11)


@pytest.mark.parametrize("seed", range(40))
def test_potential_energy_is_pair_sum(oracle_mod, seed):
    pos, mass, eps, _ = system(seed)
    _, phi = oracle_mod.accel(pos, mass, eps)
    w = 0.0
    n = pos.shape[0]
    for i in range(n):
        for j in range(i + 1, n):
            w -= mass[i] * mass[j] / np.sqrt(np.sum((pos[j] - pos[i]) ** 2) + eps * eps)
    assert abs(0.5 * np.dot(mass, phi) - w) <= 1e-12 * abs(w)
