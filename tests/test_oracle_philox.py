"""Pins of the oracle's counter-based generator and of the draws built on it.

Philox (Salmon et al., SC'11) is defined by its round structure and constants. The 4x64 member
is checked word for word against numpy's independent Philox4x64-10, and the 4x32 member the
method uses against Triton's independent Philox4x32-10 (its `tl.philox`, run by Triton's CPU
interpreter). Bootstrap multiplicities and mtry subsets are then checked statistically against
their exact distributions.
"""
import json
import math
import os
import subprocess
import sys

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


_TRITON_PHILOX = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def philox_kernel(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i), 10)
    tl.store(o0 + i, a)
    tl.store(o1 + i, b)
    tl.store(o2 + i, c)
    tl.store(o3 + i, d)

args = json.loads(sys.argv[1])
out = []
for seed, ctrs in args:
    n = len(ctrs)
    cols = [torch.from_numpy(np.array([c[w] for c in ctrs], dtype=np.uint32).view(np.int32)) for w in range(4)]
    res = [torch.empty(n, dtype=torch.int32) for _ in range(4)]
    philox_kernel[(1,)](seed, *cols, *res, N=n)
    words = [r.numpy().view(np.uint32) for r in res]
    out.append([[int(words[w][j]) for w in range(4)] for j in range(n)])
print(json.dumps(out))
"""


def test_philox4x32_matches_triton():
    """Word for word against Triton's Philox4x32-10 (key = the seed's low and high words)."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(2026)
    cases = []
    for seed in (0, 0x0123456789ABCDEF, 2 ** 64 - 1, 156):
        ctrs = [[0, 0, 0, 0], [2 ** 32 - 1] * 4] + \
            [[int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)] for _ in range(14)]
        cases.append([seed, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX, json.dumps(cases)], capture_output=True, text=True,
                       env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton's interpreter is not usable here: " + r.stderr.strip().splitlines()[-1][:200])
    theirs = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctrs), words in zip(cases, theirs):
        for ctr, w in zip(ctrs, words):
            ours = O.philox4x32(ctr, [seed & 0xFFFFFFFF, seed >> 32])
            assert [int(v) for v in ours] == w, (seed, ctr)
