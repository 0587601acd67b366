"""Simulated-annealing tuning of num.trees, mtry and min.node.size against the out-of-bag error
(aiwcrf_tune_sa, Sec. III-C).

The annealer's own rules are checked from its trace: bounds, the start, the acceptance of every
candidate that is no worse than the current state, the best being the earliest lowest error, and
determinism in the seed. Each trace error is aiwcrf_oob_error of a fresh fit with those
parameters, and the best setting's error is pinned to the oracle's exact out-of-bag error.
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth

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


@pytest.fixture(scope="module")
def run():
    wl = synth.plain_forest_workload()
    tp = A.tune_params(steps=14, trees=(4, 48), mtry=(1, 32), node=(1, 12), t0=0.2, cooling=0.9, seed=3)
    start = A.params(64, 10, 5)                                  # num.trees clamped to 48
    best, mse, trace = A.aiwcrf_tune_sa(tp, start, dev(wl.X), dev(wl.y))
    return wl, tp, start, best, mse, trace


def test_trace_follows_the_annealer_rules(run):
    wl, tp, start, best, mse, trace = run
    assert len(trace) == tp.steps + 1
    assert (trace[0]["num_trees"], trace[0]["mtry"], trace[0]["min_node_size"]) == (48, 10, 5)
    assert trace[0]["accepted"] == 1
    e_cur = trace[0]["oob_mse"]
    for t in trace[1:]:
        assert tp.trees_min <= t["num_trees"] <= tp.trees_max and tp.mtry_min <= t["mtry"] <= tp.mtry_max
        assert tp.node_min <= t["min_node_size"] <= tp.node_max
        if t["oob_mse"] <= e_cur:
            assert t["accepted"] == 1                             # never refuse an improvement
        if t["accepted"]:
            e_cur = t["oob_mse"]
    errs = [t["oob_mse"] for t in trace]
    k = int(np.argmin(errs))                                      # the earliest lowest error
    assert mse == errs[k]
    assert (best.num_trees, best.mtry, best.min_node_size) == (trace[k]["num_trees"], trace[k]["mtry"],
                                                               trace[k]["min_node_size"])
    assert best.seed == start.seed and best.bootstrap == start.bootstrap and best.max_depth == start.max_depth


def test_trace_errors_are_the_fits_oob_errors_and_the_oracles(run):
    wl, tp, start, best, mse, trace = run
    for t in (trace[0], trace[len(trace) // 2], trace[-1]):
        f = A.aiwcrf_fit(A.params(t["num_trees"], t["mtry"], t["min_node_size"]), dev(wl.X), dev(wl.y))
        e, _ = A.aiwcrf_oob_error(f, dev(wl.X), dev(wl.y))
        assert e == t["oob_mse"]
    ref = O.fit(wl.X, wl.y, best.num_trees, best.mtry, best.min_node_size, seed=156)
    _, ref_mse, _ = ref.oob_error(wl.X, wl.y)
    assert abs(mse - ref_mse) <= 4 * np.spacing(ref_mse)


def test_same_seed_same_walk_and_argument_checks(run):
    wl, tp, start, best, mse, trace = run
    best2, mse2, trace2 = A.aiwcrf_tune_sa(tp, start, wl.X, wl.y)         # host arrays this time
    assert trace2 == trace and mse2 == mse
    for bad in (A.tune_params(trees=(0, 4)), A.tune_params(mtry=(5, 4)), A.tune_params(t0=0.0),
                A.tune_params(cooling=1.5), A.tune_params(steps=-1)):
        with pytest.raises(A.AiwcrfError):
            A.aiwcrf_tune_sa(bad, start, dev(wl.X), dev(wl.y))
