"""GPU path vs the CPU oracle, bit for bit, through the C ABI.

Trees are compared node by node in the packed encoding (feature, threshold bits, child index,
leaf value); predictions, variance numerators and device choices element by element.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth
from tests.forest_util import assert_tree_equal, gpu_tree, walk_packed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1811_00156_gb300 import aiwcrf as A


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_fit(wl, T, mtry, min_node, max_depth=0, seed=156, bootstrap=True, first_tree=0):
    return A.aiwcrf_fit(A.params(T, mtry, min_node, max_depth, seed, bootstrap, first_tree), dev(wl.X), dev(wl.y))


def gpu_predict(forest, Xq, var=False):
    Q = Xq.shape[1]
    out = torch.empty(Q, dtype=torch.int64, device="cuda")
    ov = torch.empty(2 * Q, dtype=torch.int64, device="cuda") if var else None
    A.aiwcrf_predict(forest, dev(Xq), out, ov)
    torch.cuda.synchronize()
    if var:
        v = ov.cpu().numpy().view(np.uint64)
        return out.cpu().numpy(), [int(v[2 * q]) | (int(v[2 * q + 1]) << 64) for q in range(Q)]
    return out.cpu().numpy()


def compare_forest(forest, ref, T, tree_ids=None):
    dec = A.decode_forest(forest.serialize())
    assert dec["T"] == T
    for k in (range(T) if tree_ids is None else tree_ids):
        assert_tree_equal(gpu_tree(dec, k), ref.tree(k), where=f"tree {k}")
    return dec


def test_aiwc_2220_forest_bit_exact():
    """2,220 rows, 128 trees, mtry 10, min_node 5: every tree, prediction and variance."""
    wl = synth.plain_forest_workload()
    T = 128
    f = gpu_fit(wl, T, 10, 5)
    ref = O.fit(wl.X, wl.y, T, 10, 5, seed=156)
    compare_forest(f, ref, T)
    p, v = gpu_predict(f, wl.X, var=True)
    rp, _, rv = ref.predict(wl.X, want_var=True)
    assert np.array_equal(p, rp)
    assert v == rv
    st = f.stats()
    assert st["total_nodes"] == sum(ref.tree(k).num_nodes for k in range(T))
    assert st["groups"] == len({tuple(c) for c in wl.X.T.tolist()})
    assert st["nodes_evaluated"] == sum(int(ref.tree(k).evaluated.sum()) for k in range(T))


CASES = [
    # n, F, card, T, mtry, min_node, max_depth, bootstrap, y_levels
    (1, 4, None, 3, 2, 1, 0, True, None),
    (2, 3, None, 3, 3, 1, 0, False, None),
    (32, 5, None, 4, 3, 1, 0, False, None),
    (33, 5, None, 4, 3, 1, 0, False, None),
    (257, 7, 9, 6, 3, 2, 0, True, 3),
    (1000, 32, None, 8, 10, 5, 0, True, None),
    (1000, 32, 40, 8, 32, 1, 0, True, None),
    (1500, 1, None, 5, 1, 3, 0, True, None),
    (777, 3, 5, 5, 1, 2, 3, True, 2),
    (1200, 40, 30, 5, 17, 4, 0, True, None),
    (600, 128, 12, 3, 50, 5, 0, True, None),
    (900, 6, None, 4, 6, 1, 1, False, None),
    (900, 6, None, 4, 6, 1, 2, True, None),
    (5000, 12, None, 3, 12, 20, 0, True, None),       # > 3,072 bins: grouped histograms
    (3000, 4, 2, 6, 2, 1, 0, True, 1),                # binary features, many exact ties
    (400, 8, 6, 5, 4, 500, 0, True, None),            # min_node above n: every root is a leaf
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{}_F{}_c{}_T{}_m{}_mn{}_d{}_b{}_y{}".format(*c))
def test_small_cases_bit_exact(case):
    n, F, card, T, mtry, min_node, max_depth, boot, ylev = case
    wl = synth.small_case(100 + n + F, n, F, card=card, y_levels=ylev)
    f = gpu_fit(wl, T, mtry, min_node, max_depth, seed=11, bootstrap=boot)
    ref = O.fit(wl.X, wl.y, T, mtry, min_node, max_depth, seed=11, bootstrap=boot)
    compare_forest(f, ref, T)
    Xq = synth.small_case(5 + n, 300, F, card=card).X
    assert np.array_equal(gpu_predict(f, Xq), ref.predict(Xq)[0])


def test_degenerate_inputs():
    rng = np.random.default_rng(3)
    # constant features: no candidate anywhere, one leaf per tree
    X = np.ones((5, 300), np.float32)
    y = rng.integers(-1 << 40, 1 << 40, 300).astype(np.int64)
    wl = synth.Workload(X=X, y=y, name="const-x")
    f = gpu_fit(wl, 4, 3, 1)
    compare_forest(f, O.fit(X, y, 4, 3, 1, seed=156), 4)
    # constant target: pure root
    wl2 = synth.Workload(X=rng.normal(size=(5, 300)).astype(np.float32), y=np.full(300, 12345, np.int64), name="const-y")
    f2 = gpu_fit(wl2, 4, 3, 1)
    compare_forest(f2, O.fit(wl2.X, wl2.y, 4, 3, 1, seed=156), 4)
    # signed zeros and extreme targets
    X3 = rng.integers(-2, 3, (3, 500)).astype(np.float32)
    X3[X3 == 0] = np.where(rng.random((X3 == 0).sum()) < 0.5, -0.0, 0.0)
    y3 = np.where(rng.random(500) < 0.5, 1 << 40, -(1 << 40)).astype(np.int64)
    wl3 = synth.Workload(X=X3, y=y3, name="zeros")
    f3 = gpu_fit(wl3, 5, 2, 1)
    compare_forest(f3, O.fit(X3, y3, 5, 2, 1, seed=156), 5)


@pytest.mark.parametrize("Q", [1, 511, 512, 513, 10007])
def test_predict_ragged_query_counts(Q):
    wl = synth.plain_forest_workload()
    f = gpu_fit(wl, 20, 10, 5)
    ref = O.fit(wl.X, wl.y, 20, 10, 5, seed=156)
    Xq = synth.queries(Q, seed=Q)
    p, v = gpu_predict(f, Xq, var=True)
    rp, _, rv = ref.predict(Xq, want_var=True)
    assert np.array_equal(p, rp) and v == rv


def test_select_device_matches_oracle():
    wl = synth.plain_forest_workload()
    f = gpu_fit(wl, 32, 10, 5)
    ref = O.fit(wl.X, wl.y, 32, 10, 5, seed=156)
    kfeat = np.ascontiguousarray(synth.queries(64, seed=9)[:30])
    for size in range(4):
        best = torch.empty(64, dtype=torch.int32, device="cuda")
        pred = torch.empty(64 * 15, dtype=torch.int64, device="cuda")
        A.aiwcrf_select_device(f, dev(kfeat), size, list(range(15)), best, pred)
        rb, rp = ref.select_device(kfeat, size, list(range(15)))
        assert np.array_equal(best.cpu().numpy(), rb)
        assert np.array_equal(pred.cpu().numpy().reshape(64, 15), rp)
    # a device subset in a shuffled order, host outputs
    ids = [11, 3, 7, 0]
    hb = np.zeros(64, np.int32)
    A.aiwcrf_select_device(f, kfeat, 2, ids, hb)
    assert np.array_equal(hb, ref.select_device(kfeat, 2, ids)[0])


def test_host_buffers_and_serialization_roundtrip():
    wl = synth.small_case(5, 800, 9, card=20)
    f_dev = gpu_fit(wl, 6, 4, 2)
    f_host = A.aiwcrf_fit(A.params(6, 4, 2), wl.X, wl.y)        # numpy host arrays
    assert f_dev.serialize() == f_host.serialize()
    g = A.aiwcrf_forest_deserialize(f_dev.serialize())
    Xq = synth.small_case(6, 999, 9, card=20).X
    out = np.zeros(999, np.int64)
    A.aiwcrf_predict(g, Xq, out)                                 # host in, host out
    assert np.array_equal(out, gpu_predict(f_dev, Xq))


def test_page_locked_queries_are_read_in_place():
    """Page-locked host features are read by the device in place (no staging copy): the same
    predictions as device features, on the unsorted (small) and the sorted (large) walk, with
    host and device outputs."""
    wl = synth.scaled_forest_workload()
    f = gpu_fit(wl, 16, 10, 5)
    for Q in (1_000, 70_001):
        Xq = synth.queries(Q, seed=Q)
        ref = gpu_predict(f, Xq)
        pinned = torch.from_numpy(Xq).pin_memory()
        out = np.zeros(Q, np.int64)
        A.aiwcrf_predict(f, pinned.numpy(), out)                 # page-locked in, host out
        assert np.array_equal(out, ref)
        out_d = torch.empty(Q, dtype=torch.int64, device="cuda")
        A.aiwcrf_predict(f, pinned.numpy(), out_d)               # page-locked in, device out
        torch.cuda.synchronize()
        assert np.array_equal(out_d.cpu().numpy(), ref)


def test_fit_scratch_reuse_across_sizes_and_threads():
    """The fit's scratch arena (kept per host thread between fits) never leaks one fit's data
    into the next: fits of alternating sizes repeat their bytes, and fits on two host threads at
    once (two arenas, two streams) give the single-thread bytes."""
    import threading
    small = synth.small_case(7, 600, 9, card=20)
    big = synth.scaled_forest_workload()
    ref_small = gpu_fit(small, 8, 4, 2).serialize()
    ref_big = gpu_fit(big, 24, 10, 5).serialize()
    for _ in range(2):
        assert gpu_fit(small, 8, 4, 2).serialize() == ref_small
        assert gpu_fit(big, 24, 10, 5).serialize() == ref_big
    out, errs = {}, []

    def work(name, wl, T, m, mn):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                X, y = dev(wl.X), dev(wl.y)
                blobs = [A.aiwcrf_fit(A.params(T, m, mn), X, y, stream=st).serialize() for _ in range(3)]
            out[name] = blobs
        except Exception as e:                                   # reported below
            errs.append(repr(e))

    th = [threading.Thread(target=work, args=("small", small, 8, 4, 2)),
          threading.Thread(target=work, args=("big", big, 24, 10, 5))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    assert out["small"] == [ref_small] * 3 and out["big"] == [ref_big] * 3


def test_background_fit_grids_give_the_same_forest():
    # the level kernels' grid only decides which CTA takes which node: fewer CTAs per SM (a
    # background fit) must give the same bytes, on the big-node and the small-node paths
    wl = synth.scaled_forest_workload(replicates=4)
    full = A.aiwcrf_fit(A.params(24, 10, 5), dev(wl.X), dev(wl.y)).serialize()
    for cps in (1, 2, 3):
        assert A.aiwcrf_fit(A.params(24, 10, 5, ctas_per_sm=cps), dev(wl.X), dev(wl.y)).serialize() == full
    with pytest.raises(A.AiwcrfError):
        A.aiwcrf_fit(A.params(4, 10, 5, ctas_per_sm=4), dev(wl.X), dev(wl.y))


def test_tree_sharding_and_partial_sums():
    wl = synth.small_case(8, 1500, 32, card=50)
    T = 12
    full = gpu_fit(wl, T, 10, 5)
    a = gpu_fit(wl, 5, 10, 5, first_tree=0)
    b = gpu_fit(wl, T - 5, 10, 5, first_tree=5)
    da, db, df = (A.decode_forest(x.serialize()) for x in (a, b, full))
    for k in range(T):
        src, kk = (da, k) if k < 5 else (db, k - 5)
        assert np.array_equal(gpu_tree(src, kk), gpu_tree(df, k))
    Xq = synth.small_case(9, 4000, 32, card=50).X
    sa = torch.empty(4000, dtype=torch.int64, device="cuda")
    sb = torch.empty(4000, dtype=torch.int64, device="cuda")
    A.aiwcrf_predict_sum(a, dev(Xq), sa)
    A.aiwcrf_predict_sum(b, dev(Xq), sb)
    out = torch.empty(4000, dtype=torch.int64, device="cuda")
    A.aiwcrf_round_mean(sa + sb, T, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), gpu_predict(full, Xq))


def test_fit_subsets_equals_per_subset_fits():
    wl, folds = synth.loko_folds()
    folds = folds[:5]
    offs = np.cumsum([0] + [len(tr) for tr, _ in folds]).astype(np.int64)
    rows = np.concatenate([tr for tr, _ in folds]).astype(np.int32)
    T = 16
    forests = A.aiwcrf_fit_subsets(A.params(T, 10, 5), dev(wl.X), dev(wl.y), offs, dev(rows))
    for g, (tr, te) in enumerate(folds):
        Xs = np.ascontiguousarray(wl.X[:, tr])
        ref = O.fit(Xs, wl.y[tr], T, 10, 5, seed=156)
        compare_forest(forests[g], ref, T)
        Xt = np.ascontiguousarray(wl.X[:, te])
        assert np.array_equal(gpu_predict(forests[g], Xt), ref.predict(Xt)[0])


def test_error_codes():
    wl = synth.small_case(1, 100, 4)
    X = wl.X.copy()
    X[2, 7] = np.nan
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_fit(A.params(2, 2, 1), dev(X), dev(wl.y))
    assert e.value.code == -2
    y = wl.y.copy()
    y[3] = (1 << 40) + 1
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_fit(A.params(2, 2, 1), dev(wl.X), dev(y))
    assert e.value.code == -1
    # the library stays usable after errors
    f = gpu_fit(wl, 2, 2, 1)
    assert f.info()["num_trees"] == 2


@pytest.mark.parametrize("n,F,card", [(70_000, 3, None), (120_000, 2, 100_000)])
def test_columns_with_more_than_65536_values_bit_exact(n, F, card):
    """Columns with more distinct values than two-byte ranks hold (four-byte ranks): trees node
    by node, predictions and out-of-bag sums against the oracle."""
    wl = synth.small_case(200 + F, n, F, card=card)
    T = 3
    f = gpu_fit(wl, T, 2, 40, seed=21)
    ref = O.fit(wl.X, wl.y, T, 2, 40, seed=21)
    assert f.stats()["rank_bytes"] == 4
    compare_forest(f, ref, T)
    Xq = synth.small_case(9, 4000, F, card=card).X
    Xq[:, :3] = wl.X[:, :3]                         # training values: codes at the thresholds
    assert np.array_equal(gpu_predict(f, Xq), ref.predict(Xq)[0])
    s = torch.empty(n, dtype=torch.int64, device="cuda")
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    A.aiwcrf_oob(f, dev(wl.X), s, c)
    torch.cuda.synchronize()
    rs, rc = ref.oob(wl.X)
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)


def _oracle_trees_parallel(X, y, T, mtry, min_node, seed, workers=16):
    chunks = [(t0, min(T, t0 + 8)) for t0 in range(0, T, 8)]
    with cf.ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(lambda c: O.fit(X, y, T, mtry, min_node, seed=seed, t0=c[0], t1=c[1]), chunks))
    return parts


def test_aiwc_111000_full_size():
    """111,000 rows x 500 trees and 1,000,000 queries, the benchmark's launch configuration.
    Trees 0, 1, 255, 499 are grown alone by the oracle and compared node by node; the full
    forest's predictions are checked on a query sample by walking the packed trees, and the
    variance numerators of the sample by their definition."""
    wl = synth.scaled_forest_workload()
    T = 500
    f = gpu_fit(wl, T, 10, 5)
    dec = A.decode_forest(f.serialize())
    for t in (0, 1, 255, 499):
        ref = O.fit(wl.X, wl.y, T, 10, 5, seed=156, t0=t, t1=t + 1)
        assert_tree_equal(gpu_tree(dec, t), ref.tree(0), where=f"tree {t}")
    Q = 1_000_000
    Xq = synth.queries(Q)
    p, v = gpu_predict(f, Xq, var=True)
    rng = np.random.default_rng(0)
    for q in rng.choice(Q, 40, replace=False):
        leaves = [walk_packed(gpu_tree(dec, t), Xq[:, q]) for t in range(T)]
        P = sum(leaves)
        assert p[q] == (2 * P + T) // (2 * T)
        assert v[q] == T * sum(x * x for x in leaves) - P * P


def test_aiwc_111000_full_forest_predictions_vs_oracle():
    """The whole 500-tree oracle forest (grown tree-parallel on the host cores) against the GPU
    forest on a 20,000-query sample of the 1,000,000-query workload."""
    wl = synth.scaled_forest_workload()
    T = 500
    f = gpu_fit(wl, T, 10, 5)
    parts = _oracle_trees_parallel(wl.X, wl.y, T, 10, 5, 156)
    Xq = np.ascontiguousarray(synth.queries(1_000_000)[:, ::50])
    P = sum(part.predict(Xq, total_trees=T)[1].astype(object) for part in parts)
    exp = np.array([(2 * int(s) + T) // (2 * T) for s in P], np.int64)
    assert np.array_equal(gpu_predict(f, Xq), exp)


def test_predict_special_query_values():
    """Coded walks must take the float walk's path for NaN, signed zeros, infinities, training
    values themselves and values between or beyond them."""
    rng = np.random.default_rng(12)
    X = rng.integers(-3, 4, (4, 900)).astype(np.float32) * np.float32(0.5)
    X[X == 0] = np.where(rng.random((X == 0).sum()) < 0.5, -0.0, 0.0)
    y = rng.integers(-1 << 36, 1 << 36, 900).astype(np.int64)
    wl = synth.Workload(X=X, y=y, name="special")
    f = gpu_fit(wl, 9, 2, 1)
    ref = O.fit(X, y, 9, 2, 1, seed=156)
    specials = np.array([np.nan, -0.0, 0.0, np.inf, -np.inf, -1.5, -1.25, 1.5, 1.75, 99.0, -99.0, 0.25],
                        np.float32)
    Xq = rng.choice(specials, size=(4, 5000)).astype(np.float32)
    assert np.array_equal(gpu_predict(f, Xq), ref.predict(Xq)[0])
    g = A.aiwcrf_forest_deserialize(f.serialize())          # thresholds-only value tables
    out = torch.empty(5000, dtype=torch.int64, device="cuda")
    A.aiwcrf_predict(g, dev(Xq), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.predict(Xq)[0])


def test_oob_matches_oracle():
    wl = synth.plain_forest_workload()
    T = 64
    f = gpu_fit(wl, T, 10, 5)
    ref = O.fit(wl.X, wl.y, T, 10, 5, seed=156)
    s = torch.empty(wl.n_rows, dtype=torch.int64, device="cuda")
    c = torch.empty(wl.n_rows, dtype=torch.int32, device="cuda")
    A.aiwcrf_oob(f, dev(wl.X), s, c)
    torch.cuda.synchronize()
    rs, rc = ref.oob(wl.X)
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)
    # the error itself, on the device through the C ABI: predictions exact, the mean within
    # the rounding of its one double division and conversion (a few ulp)
    ref_pred, ref_mse, ref_rows = ref.oob_error(wl.X, wl.y)
    pred = torch.empty(wl.n_rows, dtype=torch.int64, device="cuda")
    mse, rows = A.aiwcrf_oob_error(f, dev(wl.X), dev(wl.y), pred)
    assert np.array_equal(pred.cpu().numpy(), ref_pred) and rows == ref_rows
    assert abs(mse - ref_mse) <= 4 * np.spacing(ref_mse) and 0.0 < mse < 1.0     # log10-seconds squared
    mse_h, rows_h = A.aiwcrf_oob_error(f, wl.X, wl.y)                            # host arrays
    assert mse_h == mse and rows_h == rows
    # subset forests keep no bitmaps
    fs = A.aiwcrf_fit_subsets(A.params(4, 10, 5), dev(wl.X), dev(wl.y), np.array([0, 100], np.int64),
                              dev(np.arange(100, dtype=np.int32)))
    with pytest.raises(A.AiwcrfError):
        A.aiwcrf_oob(fs[0], dev(wl.X), s, c)


def test_sorted_walk_of_large_batches_equals_unsorted_chunks():
    # batches of >= 65,536 queries on a compact forest are walked in the order of their leading
    # codes; the sums, predictions and variance numerators must not change
    wl = synth.scaled_forest_workload(replicates=2)
    f = gpu_fit(wl, 40, 10, 5)
    Xq = synth.queries(150_001, seed=77)
    Xq[:, 5] = np.nan
    big = gpu_predict(f, Xq, var=True)
    chunks = [gpu_predict(f, np.ascontiguousarray(Xq[:, a:a + 40_000]), var=True) for a in range(0, 150_001, 40_000)]
    np.testing.assert_array_equal(big[0], np.concatenate([c[0] for c in chunks]))
    np.testing.assert_array_equal(big[1], np.concatenate([c[1] for c in chunks]))
