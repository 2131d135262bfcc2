"""Pins of the oracle's random streams against independent facts.

* The Philox round structure is checked against NumPy's own Philox4x64-10
  bit generator (an independent implementation of the same published family);
  the 32-bit instance the method uses runs through the very same round code.
* The without-repetition sampler is checked by brute force (bijectivity,
  prefix property) and by frequency tests; the Gaussians by moments and a
  Kolmogorov-Smirnov test.
"""

import numpy as np
import pytest
from scipy import stats

from oracle import rng


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((0x1234567890ABCDEF, 42), (5, 7, 9, 11)),
    ((2**64 - 1, 2**64 - 1), (2**64 - 2, 2**64 - 1, 2**64 - 1, 2**64 - 1)),
    ((0x243F6A8885A308D3, 0x13198A2E03707344), (0xA4093822299F31D0, 0x082EFA98EC4E6C89, 3, 0)),
])
def test_philox_round_structure_matches_numpy_philox4x64(key, ctr):
    # NumPy increments the 256-bit counter before each block: block 1 uses ctr + 1.
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    assert [int(v) for v in g.state['state']['counter']] == list(ctr)
    got = [int(v) for v in g.random_raw(4)]
    c = ctr[0] + (ctr[1] << 64) + (ctr[2] << 128) + (ctr[3] << 192) + 1
    words = tuple((c >> (64 * i)) & (2**64 - 1) for i in range(4))
    want = rng.philox4(words, key, rng.PHILOX4x64)
    assert got == list(want)


def test_philox4x32_vectorised_equals_scalar_words():
    rs = np.random.default_rng(7)
    ctr = rs.integers(0, 2**32, size=(4, 64), dtype=np.uint64)
    key = (0xDEADBEEF, 0x01234567)
    vec = rng.philox4(tuple(ctr), key)
    for i in range(64):
        sc = rng.philox4(tuple(int(ctr[w, i]) for w in range(4)), key, scalar=True)
        assert tuple(int(v[i]) for v in vec) == sc
    assert all(int(v.max()) < 2**32 for v in vec)


def test_philox4x32_is_a_bijection_sample():
    # distinct counters must give distinct outputs (Philox is a bijection per key)
    c0 = np.arange(50000, dtype=np.uint64)
    z = np.zeros_like(c0)
    out = rng.philox4((c0, z, z, z), (1, 2))
    packed = set(zip(*(v.tolist() for v in out)))
    assert len(packed) == len(c0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 16, 17, 255, 1000, 4096, 65537])
def test_fiber_indices_is_a_permutation_of_range(N):
    for seed, node in ((0, 0), (123456789, 3)):
        pi = rng.fiber_indices(N, N, seed, node)
        assert sorted(pi.tolist()) == list(range(N))


def test_fiber_indices_prefix_property_and_bounds():
    N = 2_097_152  # 128^3, the mode-k column count of a 128^4 tensor
    full = rng.fiber_indices(N, 5000, 1, 2)
    assert np.array_equal(rng.fiber_indices(N, 1280, 1, 2), full[:1280])
    assert full.min() >= 0 and full.max() < N
    assert len(np.unique(full)) == 5000


def test_fiber_indices_streams_differ_by_seed_and_node():
    a = rng.fiber_indices(10**6, 100, 5, 0)
    b = rng.fiber_indices(10**6, 100, 5, 1)
    c = rng.fiber_indices(10**6, 100, 6, 0)
    assert len(set(a) & set(b)) < 5 and len(set(a) & set(c)) < 5


def test_fiber_indices_uniform_inclusion_frequency():
    # each index of [0, N) is in the sample with probability s/N (uniform
    # sampling without repetition, Sec. 3.1); chi-square over 2000 seeds
    N, s, T = 40, 10, 2000
    counts = np.zeros(N)
    first = np.zeros(N)
    for seed in range(T):
        pi = rng.fiber_indices(N, s, seed, 0)
        counts[pi] += 1
        first[pi[0]] += 1
    exp = T * s / N
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2 * (N - s) / N, N - 1) > 1e-4  # finite-population correction
    chi2f = ((first - T / N) ** 2 / (T / N)).sum()
    assert stats.chi2.sf(chi2f, N - 1) > 1e-4


def test_gaussian_moments_and_ks():
    m = np.arange(200000, dtype=np.uint64) * np.uint64(2654435761) % np.uint64(2**40)
    g = rng.gaussian(m, np.uint64(3), seed=99, node=1)
    assert abs(g.mean()) < 5 * 1 / np.sqrt(g.size)
    assert abs(g.var() - 1) < 5 * np.sqrt(2 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-4


def test_gaussian_columns_uncorrelated_and_keyed_by_fiber_index():
    pi = rng.fiber_indices(10**7, 20000, 4, 2)
    Om = rng.sketch_matrix(pi, 6, 4, 2)
    C = np.corrcoef(Om.T)
    assert np.abs(C - np.eye(6)).max() < 0.05
    # the same fiber index gives the same row whatever its sample position
    Om2 = rng.sketch_matrix(pi[::-1], 6, 4, 2)
    assert np.array_equal(Om2, Om[::-1])
