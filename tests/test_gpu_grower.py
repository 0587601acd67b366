"""The growers give the same forest: the tree-resident kernel (one CTA per tree, every depth in
shared memory), the level-synchronous kernels (three launches per depth) with histogram search,
and the level-synchronous kernels with presorted lists, byte for byte in the serialized forest
and in every fit counter. The oracle comparisons of test_gpu_parity.py run with the automatic
choice, which takes the tree-resident kernel for every case whose trees fit and the lists for
columns of more than 4,096 values."""
import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth
from tests.forest_util import assert_tree_equal, gpu_tree

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
    yield
    A.aiwcrf_set_grower(A.GROWER_AUTO)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fit_with(grower, wl, prm):
    A.aiwcrf_set_grower(grower)
    try:
        return A.aiwcrf_fit(prm, dev(wl.X), dev(wl.y))
    finally:
        A.aiwcrf_set_grower(A.GROWER_AUTO)


def same_forest(a, b, ga=None, gb=None):
    ga = A.GROWER_TREE if ga is None else ga
    gb = A.GROWER_LEVEL if gb is None else gb
    assert a.serialize() == b.serialize()
    sa, sb = a.stats(), b.stats()
    assert sa.pop("grower") == ga and sb.pop("grower") == gb
    assert sa == sb


CASES = [
    # name, workload, params
    ("aiwc-2220", lambda: synth.plain_forest_workload(), dict(T=128, mtry=10, min_node=5)),
    ("aiwc-111000", lambda: synth.scaled_forest_workload(), dict(T=40, mtry=10, min_node=5)),
    ("depth3", lambda: synth.plain_forest_workload(), dict(T=16, mtry=10, min_node=5, max_depth=3)),
    ("mtry-all-no-bootstrap", lambda: synth.plain_forest_workload(), dict(T=8, mtry=32, min_node=1, bootstrap=False)),
    ("single-row", lambda: synth.small_case(9, 1, 4), dict(T=3, mtry=2, min_node=1)),
    ("binary-ties", lambda: synth.small_case(4, 3000, 4, card=2, y_levels=1), dict(T=6, mtry=2, min_node=1)),
    ("card-256", lambda: synth.small_case(5, 4000, 8, card=256), dict(T=6, mtry=5, min_node=2)),
    ("all-leaves", lambda: synth.small_case(6, 400, 8, card=6), dict(T=5, mtry=4, min_node=500)),
    ("F1", lambda: synth.small_case(7, 1500, 1, card=200), dict(T=5, mtry=1, min_node=3)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_growers_give_identical_forests(case):
    _, make, kw = case
    wl = make()
    prm = A.params(kw["T"], kw["mtry"], kw["min_node"], kw.get("max_depth", 0), 156, kw.get("bootstrap", True))
    same_forest(fit_with(A.GROWER_TREE, wl, prm), fit_with(A.GROWER_LEVEL, wl, prm))


def test_tree_grower_matches_the_oracle_on_the_benchmark_data():
    """A few trees of the 111,000-row benchmark forest, node by node against the oracle."""
    wl = synth.scaled_forest_workload()
    f = fit_with(A.GROWER_TREE, wl, A.params(3, 10, 5, first_tree=498))
    ref = O.fit(wl.X, wl.y, 3, 10, 5, seed=156, t0=498)
    dec = A.decode_forest(f.serialize())
    for k in range(3):
        assert_tree_equal(gpu_tree(dec, k), ref.tree(k), where=f"tree {k}")


def test_subset_fits_agree_between_growers():
    wl, folds = synth.loko_folds()
    folds = folds[:5]
    off = np.zeros(len(folds) + 1, np.int64)
    rows = []
    for i, (train, _) in enumerate(folds):
        rows.append(train.astype(np.int32))
        off[i + 1] = off[i] + len(train)
    rows = np.concatenate(rows)
    prm = A.params(32, 10, 5)
    out = {}
    for g in (A.GROWER_TREE, A.GROWER_LEVEL):
        A.aiwcrf_set_grower(g)
        try:
            out[g] = A.aiwcrf_fit_subsets(prm, dev(wl.X), dev(wl.y), off, dev(rows))
        finally:
            A.aiwcrf_set_grower(A.GROWER_AUTO)
    for a, b in zip(out[A.GROWER_TREE], out[A.GROWER_LEVEL]):
        same_forest(a, b)


def test_tree_grower_refuses_trees_that_do_not_fit_and_auto_falls_back():
    wl = synth.small_case(8, 2000, 6)                 # 2,000 distinct values: two-byte ranks
    prm = A.params(4, 3, 2)
    with pytest.raises(A.AiwcrfError) as e:
        fit_with(A.GROWER_TREE, wl, prm)
    assert e.value.code == -8
    f = A.aiwcrf_fit(prm, dev(wl.X), dev(wl.y))
    assert f.stats()["grower"] == A.GROWER_LEVEL
    with pytest.raises(A.AiwcrfError):
        A.aiwcrf_set_grower(7)


LIST_CASES = CASES + [
    ("card-5000", lambda: synth.small_case(11, 5000, 6), dict(T=6, mtry=3, min_node=2)),
    ("card-70000", lambda: synth.small_case(12, 70000, 3), dict(T=2, mtry=2, min_node=40)),
    ("card-3000-depth4", lambda: synth.small_case(13, 3000, 5, card=3000), dict(T=5, mtry=5, min_node=1, max_depth=4)),
    ("card-9000-no-bootstrap", lambda: synth.small_case(14, 9000, 4), dict(T=3, mtry=4, min_node=3, bootstrap=False)),
]


@pytest.mark.parametrize("case", LIST_CASES, ids=[c[0] for c in LIST_CASES])
def test_list_search_gives_identical_forests(case):
    """Presorted lists against the histogram search, on the growers' cases and on columns with
    thousands to tens of thousands of values (several histogram passes per node)."""
    _, make, kw = case
    wl = make()
    prm = A.params(kw["T"], kw["mtry"], kw["min_node"], kw.get("max_depth", 0), 156, kw.get("bootstrap", True))
    same_forest(fit_with(A.GROWER_LISTS, wl, prm), fit_with(A.GROWER_LEVEL, wl, prm), A.GROWER_LISTS, A.GROWER_LEVEL)


def test_subset_fits_agree_with_lists():
    wl, folds = synth.loko_folds()
    folds = folds[:4]
    off = np.zeros(len(folds) + 1, np.int64)
    rows = []
    for i, (train, _) in enumerate(folds):
        rows.append(train.astype(np.int32))
        off[i + 1] = off[i] + len(train)
    rows = np.concatenate(rows)
    prm = A.params(16, 10, 5)
    out = {}
    for g in (A.GROWER_LISTS, A.GROWER_LEVEL):
        A.aiwcrf_set_grower(g)
        try:
            out[g] = A.aiwcrf_fit_subsets(prm, dev(wl.X), dev(wl.y), off, dev(rows))
        finally:
            A.aiwcrf_set_grower(A.GROWER_AUTO)
    for a, b in zip(out[A.GROWER_LISTS], out[A.GROWER_LEVEL]):
        same_forest(a, b, A.GROWER_LISTS, A.GROWER_LEVEL)


def test_auto_takes_lists_for_many_values_and_matches_the_oracle():
    wl = synth.small_case(15, 6000, 5)                # about 6,000 values per column
    prm = A.params(4, 3, 3)
    f = A.aiwcrf_fit(prm, dev(wl.X), dev(wl.y))
    assert f.stats()["grower"] == A.GROWER_LISTS
    ref = O.fit(wl.X, wl.y, 4, 3, 3, seed=156)
    dec = A.decode_forest(f.serialize())
    for k in range(4):
        assert_tree_equal(gpu_tree(dec, k), ref.tree(k), where=f"tree {k}")


def test_per_row_benchmark_trees_with_lists_match_the_oracle():
    """A tree of the 111,000-row per-row workload (every row its own feature vector)."""
    wl = synth.per_row_forest_workload()
    f = A.aiwcrf_fit(A.params(1, 10, 5, first_tree=17), dev(wl.X), dev(wl.y))
    assert f.stats()["grower"] == A.GROWER_LISTS
    ref = O.fit(wl.X, wl.y, 1, 10, 5, seed=156, t0=17)
    dec = A.decode_forest(f.serialize())
    for k in range(1):
        assert_tree_equal(gpu_tree(dec, k), ref.tree(k), where=f"tree {k}")
