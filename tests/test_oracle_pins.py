"""Pins of the CPU oracle against facts fixed by the mathematics, not by the oracle itself.

* hand-derived trees (tests/golden/cart_hand_cases.json);
* exact brute-force enumeration with Fractions on tiny inputs (tests/bruteforce.py);
* closed forms and special cases: leaf = rounded bootstrap mean, piecewise-constant recovery,
  interpolation, the textbook best stump, sklearn's DecisionTreeRegressor partition;
* invariants: shift of y, monotone maps of a column, forest = mean of its trees.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth
from tests import bruteforce as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cart_hand_cases.json")


def _tree_list(tr):
    out = []
    for j in range(tr.num_nodes):
        if tr.feature[j] < 0:
            out.append([-1, int(tr.value[j])])
        else:
            out.append([int(tr.feature[j]), float(tr.thr[j]), int(tr.left[j])])
    return out


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_derived_cases(case):
    X = np.array(case["X"], dtype=np.float32)
    y = np.array(case["y"], dtype=np.int64)
    F = X.shape[0]
    fr = O.fit(X, y, 1, F, case["min_node"], case["max_depth"], seed=1, bootstrap=False)
    got = _tree_list(fr.tree(0))
    assert got == case["tree"]
    tr = fr.tree(0)
    for j in range(tr.num_nodes):            # thresholds are stored as +0, never -0
        if tr.feature[j] >= 0:
            assert np.float32(tr.thr[j]).view(np.uint32) != 0x80000000


def _bf_compare(X, y, seed, t, mtry, min_node, max_depth, bootstrap):
    F, N = X.shape
    fr = O.fit(X, y, 1, mtry, min_node, max_depth, seed=seed, bootstrap=bootstrap, t0=t)
    tr = fr.tree(0)
    w = O.bootstrap_counts(seed, t, N).tolist() if bootstrap else [1] * N
    Xl = [X[f].astype(np.float64).tolist() for f in range(F)]
    yl = [int(v) for v in y]
    nodes = BF.grow(Xl, yl, w, lambda d, i: O.mtry_draw(seed, t, d, i, F, mtry).tolist(),
                    min_node, max_depth)
    assert tr.num_nodes == len(nodes)
    for j, nd in enumerate(nodes):
        assert tr.feature[j] == nd["feature"], j
        assert tr.left[j] == nd["left"], j
        assert tr.n[j] == nd["n"] and tr.S[j] == nd["S"], j
        if nd["feature"] >= 0:
            assert np.float32(tr.thr[j]) == np.float32(nd["thr"]), j
        else:
            assert tr.value[j] == nd["value"], j


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_tiny(seed):
    rng = np.random.default_rng(1000 + seed)
    N = int(rng.integers(1, 13))
    F = int(rng.integers(1, 4))
    card = int(rng.integers(1, 6)) if seed % 3 else None
    X = (rng.integers(0, card, size=(F, N)).astype(np.float32) if card
         else rng.normal(size=(F, N)).astype(np.float32))
    y = rng.integers(-20, 21, size=N).astype(np.int64) * (1 << int(rng.integers(0, 30)))
    mtry = int(rng.integers(1, F + 1))
    min_node = int(rng.integers(1, 4))
    max_depth = int(rng.integers(0, 4))
    _bf_compare(X, y, seed=77 + seed, t=seed % 5, mtry=mtry, min_node=min_node,
                max_depth=max_depth, bootstrap=bool(seed % 2))


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_large_targets(seed):
    """Targets near the library's limit |y| <= 2^40 exercise the full-width exact arithmetic."""
    rng = np.random.default_rng(5000 + seed)
    N, F = 10, 3
    X = rng.integers(0, 4, size=(F, N)).astype(np.float32)
    y = rng.integers(-(1 << 40), (1 << 40) + 1, size=N).astype(np.int64)
    _bf_compare(X, y, seed=seed, t=3, mtry=2, min_node=1, max_depth=0, bootstrap=True)


def test_gain_cmp_exact_vs_fractions():
    rng = np.random.default_rng(3)
    big = 1 << 62
    for _ in range(2000):
        n = int(rng.integers(2, 1 << 22))
        S = int(rng.integers(-big // 2, big // 2))
        a_nL = int(rng.integers(1, n))
        b_nL = int(rng.integers(1, n))
        a_SL = int(rng.integers(-big // 2, big // 2))
        b_SL = a_SL if rng.random() < 0.2 else int(rng.integers(-big // 2, big // 2))
        if rng.random() < 0.2:
            b_nL = a_nL
        a = (a_nL, a_SL, n - a_nL, S - a_SL)
        b = (b_nL, b_SL, n - b_nL, S - b_SL)
        Ga = Fraction(a[1] ** 2, a[0]) + Fraction(a[3] ** 2, a[2])
        Gb = Fraction(b[1] ** 2, b[0]) + Fraction(b[3] ** 2, b[2])
        assert O.gain_cmp(a, b) == (Ga > Gb) - (Ga < Gb)


def test_round_mean_half_up():
    rng = np.random.default_rng(4)
    for _ in range(3000):
        n = int(rng.integers(1, 1 << 22))
        S = int(rng.integers(-(1 << 62), 1 << 62))
        exp = Fraction(S, n) + Fraction(1, 2)
        assert O.round_mean(S, n) == exp.numerator // exp.denominator
    assert O.round_mean(3, 2) == 2 and O.round_mean(-3, 2) == -1 and O.round_mean(5, 2) == 3


def _leaf_rows(tr, X):
    F, N = X.shape
    out = np.zeros(N, np.int64)
    for r in range(N):
        j = 0
        while tr.feature[j] >= 0:
            j = tr.left[j] + (0 if X[tr.feature[j], r] <= tr.thr[j] else 1)
        out[r] = j
    return out


def test_leaf_is_rounded_bootstrap_mean():
    wl = synth.small_case(11, 300, 5, card=7)
    fr = O.fit(wl.X, wl.y, 6, 3, 4, seed=9, bootstrap=True)
    for k in range(6):
        tr = fr.tree(k)
        w = O.bootstrap_counts(9, k, wl.n_rows).astype(np.int64)
        leaf = _leaf_rows(tr, wl.X)
        for j in np.flatnonzero(tr.feature < 0):
            sel = (leaf == j) & (w > 0)
            n = int(w[sel].sum())
            S = sum(int(a) * int(b) for a, b in zip(w[sel], wl.y[sel]))
            assert n == tr.n[j] and S == tr.S[j]
            exp = Fraction(S, n) + Fraction(1, 2)
            assert tr.value[j] == exp.numerator // exp.denominator


def test_piecewise_constant_recovery():
    """Cells on a 4x3 grid of two columns, value 10*L0 + L1 (lexicographically increasing), so
    any node holding two cells has a boundary with different child means: growth ends with
    pure leaves and every training row is predicted exactly."""
    rng = np.random.default_rng(21)
    N = 400
    L0 = rng.integers(0, 4, N)
    L1 = rng.integers(0, 3, N)
    X = np.stack([L0 + rng.uniform(0, 0.9, N), L1 + rng.uniform(0, 0.9, N),
                  rng.normal(size=N), rng.normal(size=N)]).astype(np.float32)
    c = (10 * L0 + L1).astype(np.int64) << 32
    fr = O.fit(X, c, 1, 4, 1, seed=3, bootstrap=False)
    pred, _ = fr.predict(X)
    assert np.array_equal(pred, c)


def test_piecewise_constant_bootstrap_in_sample():
    """With bootstrap on, every tree still sees every cell (60 rows each), its leaves are pure,
    and each training row is routed to its own cell in every tree: exact in-sample recovery."""
    rng = np.random.default_rng(22)
    N = 300
    L0 = np.repeat(np.arange(5), 60)
    rng.shuffle(L0)
    X = np.stack([L0.astype(np.float32)])
    c = (L0 * 7).astype(np.int64) << 32
    fr = O.fit(X, c, 8, 1, 1, seed=5, bootstrap=True)
    pred, _ = fr.predict(X)
    assert np.array_equal(pred, c)


def test_interpolation_special_case():
    wl = synth.small_case(31, 150, 3)
    fr = O.fit(wl.X, wl.y, 1, 3, 1, seed=1, bootstrap=False)
    pred, _ = fr.predict(wl.X)
    assert np.array_equal(pred, wl.y)


def test_stump_is_textbook_best_split():
    """max_depth 1, all features, no bootstrap: the root split minimises the summed squared error
    of the two halves (enumerated here with the SSE form, exact Fractions)."""
    for seed in range(5):
        wl = synth.small_case(40 + seed, 40, 3, card=9, y_levels=5)
        X, y = wl.X, [int(v) for v in wl.y]
        fr = O.fit(X, wl.y, 1, 3, 1, max_depth=1, seed=1, bootstrap=False)
        tr = fr.tree(0)
        best = None
        for f in range(3):
            for v in sorted(set(X[f].tolist()))[:-1]:
                L = [y[r] for r in range(len(y)) if X[f, r] <= v]
                R = [y[r] for r in range(len(y)) if not X[f, r] <= v]
                sse = sum((Fraction(a) - Fraction(sum(L), len(L))) ** 2 for a in L) + \
                    sum((Fraction(a) - Fraction(sum(R), len(R))) ** 2 for a in R)
                if best is None or sse < best[0]:
                    best = (sse, f, v)
        tot = sum((Fraction(a) - Fraction(sum(y), len(y))) ** 2 for a in y)
        if best[0] < tot:
            assert tr.feature[0] == best[1] and np.float32(tr.thr[0]) == np.float32(best[2])
            assert tr.num_nodes == 3
        else:
            assert tr.num_nodes == 1


@pytest.mark.parametrize("min_node", [1, 4])
def test_sklearn_decision_tree_partition(min_node):
    """Independent library special case: bootstrap off, every feature tried, tie-free data."""
    sk_tree = pytest.importorskip("sklearn.tree")
    for seed in range(3):
        wl = synth.small_case(60 + seed, 200, 4)
        fr = O.fit(wl.X, wl.y, 1, 4, min_node, seed=1, bootstrap=False)
        tr = fr.tree(0)
        ours = _leaf_rows(tr, wl.X)
        yf = wl.y.astype(np.float64) / 2 ** 32
        sk = sk_tree.DecisionTreeRegressor(min_samples_split=min_node + 1, min_samples_leaf=1,
                                           random_state=0).fit(wl.X.T, yf)
        theirs = sk.apply(wl.X.T)
        pairs = set(zip(ours.tolist(), theirs.tolist()))
        assert len(pairs) == len(set(ours.tolist())) == len(set(theirs.tolist()))
        pred, _ = fr.predict(wl.X)
        np.testing.assert_allclose(pred / 2 ** 32, sk.predict(wl.X.T), atol=2e-9)


def test_shift_invariance():
    wl = synth.small_case(70, 400, 6, card=11)
    c = 123456789
    a = O.fit(wl.X, wl.y, 5, 3, 3, seed=2)
    b = O.fit(wl.X, wl.y + c, 5, 3, 3, seed=2)
    for k in range(5):
        ta, tb = a.tree(k), b.tree(k)
        assert np.array_equal(ta.feature, tb.feature) and np.array_equal(ta.thr, tb.thr)
        leaf = ta.feature < 0
        assert np.array_equal(ta.value[leaf] + c, tb.value[leaf])
    pa, _ = a.predict(wl.X)
    pb, _ = b.predict(wl.X)
    assert np.array_equal(pa + c, pb)


def test_monotone_transform_invariance():
    wl = synth.small_case(71, 400, 5)
    X2 = wl.X.copy()
    X2[2] = np.exp(wl.X[2]).astype(np.float32)          # strictly increasing map of column 2
    assert len(np.unique(X2[2])) == len(np.unique(wl.X[2]))
    a = O.fit(wl.X, wl.y, 4, 3, 2, seed=4)
    b = O.fit(X2, wl.y, 4, 3, 2, seed=4)
    for k in range(4):
        ta, tb = a.tree(k), b.tree(k)
        assert np.array_equal(ta.feature, tb.feature) and np.array_equal(ta.left, tb.left)
        assert np.array_equal(ta.value, tb.value)
        m = ta.feature == 2
        assert np.array_equal(np.exp(ta.thr[m]).astype(np.float32), tb.thr[m])
    assert np.array_equal(a.predict(wl.X)[0], b.predict(X2)[0])


def test_forest_is_rounded_mean_of_trees():
    wl = synth.small_case(72, 300, 6, card=13)
    T = 7
    fr = O.fit(wl.X, wl.y, T, 2, 3, seed=8)
    pred, P = fr.predict(wl.X)
    total = np.zeros(wl.n_rows, dtype=object)
    for t in range(T):
        single = O.fit(wl.X, wl.y, 1, 2, 3, seed=8, t0=t)
        _, s = single.predict(wl.X)
        total = total + s.astype(object)
    assert np.array_equal(P.astype(object), total)
    exp = [(2 * int(p) + T) // (2 * T) for p in total]
    assert pred.tolist() == exp


def test_variance_numerator():
    wl = synth.small_case(73, 100, 4, card=5)
    T = 5
    fr = O.fit(wl.X, wl.y, T, 2, 2, seed=8)
    _, P, V = fr.predict(wl.X, want_var=True)
    leaves = []
    for t in range(T):
        single = O.fit(wl.X, wl.y, 1, 2, 2, seed=8, t0=t)
        leaves.append(single.predict(wl.X)[1])
    for q in range(wl.n_rows):
        vs = [int(leaves[t][q]) for t in range(T)]
        assert V[q] == T * sum(v * v for v in vs) - sum(vs) ** 2


def test_select_device_is_argmin():
    wl = synth.plain_forest_workload()
    fr = O.fit(wl.X, wl.y, 8, 10, 5, seed=156)
    kfeat = wl.X[:30, ::60][:, :12]
    devs = list(range(15))
    best, pred = fr.select_device(kfeat, 2, devs)
    for k in range(kfeat.shape[1]):
        q = np.zeros((32, 15), np.float32)
        q[:30] = kfeat[:, k:k + 1]
        q[30] = np.arange(15)
        q[31] = 2
        p, _ = fr.predict(q)
        assert np.array_equal(pred[k], p)
        m = p.min()
        assert best[k] == min(d for d in devs if p[d] == m)


def test_oracle_trees_grown_on_threads_match_serial():
    """The benchmark's CPU baseline grows trees on several host threads: same trees."""
    import concurrent.futures as cf
    wl = synth.small_case(74, 600, 8, card=20)
    with cf.ThreadPoolExecutor(4) as ex:
        parts = list(ex.map(lambda t: O.fit(wl.X, wl.y, 12, 3, 2, seed=5, t0=t, t1=t + 1), range(12)))
    full = O.fit(wl.X, wl.y, 12, 3, 2, seed=5)
    for k in range(12):
        a, b = parts[k].tree(0), full.tree(k)
        assert np.array_equal(a.feature, b.feature) and np.array_equal(a.thr, b.thr)
        assert np.array_equal(a.value, b.value) and np.array_equal(a.left, b.left)


def test_oob_sums_are_the_out_of_bag_trees():
    """Out-of-bag sums equal the sum over exactly the trees whose bootstrap skipped the row,
    each tree evaluated as a single-tree forest; rows drawn by every tree have count 0."""
    wl = synth.small_case(75, 250, 5, card=9)
    T = 9
    fr = O.fit(wl.X, wl.y, T, 3, 2, seed=12)
    s, c = fr.oob(wl.X)
    exp_s = np.zeros(wl.n_rows, object)
    exp_c = np.zeros(wl.n_rows, np.int64)
    for t in range(T):
        w = O.bootstrap_counts(12, t, wl.n_rows)
        _, leaf = O.fit(wl.X, wl.y, 1, 3, 2, seed=12, t0=t).predict(wl.X)
        out = w == 0
        exp_s[out] += leaf[out].astype(object)
        exp_c[out] += 1
    assert np.array_equal(s.astype(object), exp_s) and np.array_equal(c, exp_c)
    assert 0.2 < (c > 0).mean() <= 1.0                       # about 1 - 0.632^9 of the rows
    nb = O.fit(wl.X, wl.y, 3, 3, 2, seed=12, bootstrap=False)
    assert not nb.oob(wl.X)[1].any()


def test_oob_error_is_the_mean_squared_out_of_bag_residual():
    """The oracle's out-of-bag error: each out-of-bag prediction is the round-half-up mean of
    the out-of-bag leaf sums, and the error their mean squared residual in the target's units
    (against a float64 evaluation of the same definition)."""
    wl = synth.small_case(76, 300, 6, card=11)
    fr = O.fit(wl.X, wl.y, 12, 3, 2, seed=5)
    s, c = fr.oob(wl.X)
    pred, mse, rows = fr.oob_error(wl.X, wl.y)
    m = c > 0
    assert rows == int(m.sum()) and 0 < rows < wl.n_rows and not pred[~m].any()
    exact = np.array([Fraction(int(a), int(b)) for a, b in zip(s[m], c[m])], object)
    # round half up: the prediction is within 1/2 of the exact mean, and ties go up
    assert all(abs(Fraction(int(p)) - e) <= Fraction(1, 2) and Fraction(int(p)) - e != Fraction(-1, 2)
               for p, e in zip(pred[m], exact))
    ref = np.mean(((pred[m].astype(np.float64) - wl.y[m].astype(np.float64)) / 2.0 ** 32) ** 2)
    assert abs(mse - ref) <= 1e-12 * ref
