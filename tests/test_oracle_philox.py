"""Pins of the oracle's counter-based generator and of the draws built on it.

Philox (Salmon et al., SC'11) is defined by its round structure and constants. The 4x64 member
is checked word for word against numpy's independent Philox4x64-10; the 4x32 member the
library uses shares the round code with it. Bootstrap multiplicities and mtry subsets are then
checked statistically against their exact distributions.
"""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("key", [[0, 0], [0x0123456789ABCDEF, 0xFEDCBA9876543210],
                                 [2 ** 64 - 1, 12345]])
def test_philox4x64_matches_numpy(key):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array([0, 0, 0, 0], dtype=np.uint64))
    raw = bg.random_raw(4 * 6)
    for block in range(6):
        # numpy advances the 256-bit counter before each block: block b uses counter b + 1
        ours = O.philox4x64([block + 1, 0, 0, 0], key)
        assert [int(v) for v in ours] == [int(v) for v in raw[4 * block:4 * block + 4]]


def test_philox4x64_counter_carry_matches_numpy():
    key = [7, 9]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array([2 ** 64 - 1, 5, 0, 0], dtype=np.uint64))
    raw = bg.random_raw(4)
    ours = O.philox4x64([0, 6, 0, 0], key)
    assert [int(v) for v in ours] == [int(v) for v in raw]


def test_philox4x32_is_a_bijection_sample_and_avalanche():
    """Distinct counters give distinct outputs, and one flipped counter bit flips about half
    of the 128 output bits (the mixing property the generator is designed for)."""
    key = [0xDEADBEEF, 0x12345678]
    seen = set()
    flips = []
    for c in range(3000):
        a = O.philox4x32([c, 0, 0, 0], key)
        seen.add(tuple(int(v) for v in a))
        b = O.philox4x32([c ^ (1 << (c % 32)), 0, 0, 0], key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert len(seen) == 3000
    assert abs(np.mean(flips) - 64.0) < 1.0


def test_philox4x32_uniform_words():
    key = [156, 0]
    words = np.array([O.philox4x32([c, 1, 2, 3], key) for c in range(4096)], dtype=np.uint64).ravel()
    hist = np.bincount((words >> 28).astype(np.int64), minlength=16)
    exp = words.size / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 37.7        # chi-square, 15 dof, p = 0.001


def test_bootstrap_multiplicities_binomial():
    """w[row] ~ Binomial(N, 1/N): chi-square on the multiplicity histogram pooled over trees."""
    N = 2000
    counts = np.concatenate([O.bootstrap_counts(156, t, N) for t in range(20)])
    assert all(O.bootstrap_counts(156, t, N).sum() == N for t in range(3))
    kmax = 5
    obs = np.array([np.sum(counts == k) for k in range(kmax)] + [np.sum(counts >= kmax)], float)
    p = np.array([math.comb(N, k) * (1 / N) ** k * (1 - 1 / N) ** (N - k) for k in range(kmax)])
    p = np.append(p, 1 - p.sum())
    exp = p * counts.size
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 20.5        # 5 dof, p = 0.001
    assert abs(np.mean(counts > 0) - (1 - (1 - 1 / N) ** N)) < 0.01


def test_mtry_draw_is_uniform_subset():
    F, m = 32, 10
    freq = np.zeros(F)
    for i in range(3000):
        s = O.mtry_draw(156, 3, 4, i, F, m)
        assert len(s) == m and len(set(s.tolist())) == m
        assert np.all(np.diff(s) > 0) and s.min() >= 0 and s.max() < F
        freq[s] += 1
    exp = 3000 * m / F
    chi2 = ((freq - exp) ** 2 / exp).sum()
    assert chi2 < 61.1        # 31 dof, p = 0.001


def test_mtry_draw_edge_cases():
    assert O.mtry_draw(1, 0, 0, 0, 5, 9).tolist() == [0, 1, 2, 3, 4]
    assert O.mtry_draw(1, 0, 0, 0, 1, 1).tolist() == [0]
    a = O.mtry_draw(1, 2, 3, 4, 40, 7)
    b = O.mtry_draw(1, 2, 3, 4, 40, 7)
    assert np.array_equal(a, b) and len(a) == 7
