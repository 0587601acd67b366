"""Fit plans: the fit captured once as a CUDA graph (device-side loop over tree levels) and replayed.

Every plan forest must equal, byte for byte, the forest aiwcrf_fit / aiwcrf_fit_subsets grows
from the same data (those are pinned to the oracle in test_gpu_parity.py): on the first and later
runs, under every launch schedule the autotuner can choose, after the bound data change in
place, and a run on data that outgrows the plan's capacity must fail cleanly.
"""
import numpy as np
import pytest

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


def blobs(forests):
    return [f.serialize() for f in forests]


def test_plan_equals_fit_across_runs_and_schedules():
    wl = synth.scaled_forest_workload(replicates=4)
    X, y = dev(wl.X), dev(wl.y)
    params = A.params(48, 10, 5)
    ref = A.aiwcrf_fit(params, X, y).serialize()
    plan = A.FitPlan(params, X, y)
    assert blobs(plan.run()) == [ref]
    assert blobs(plan.run()) == [ref]                       # a replay
    for big, small in [(1, 1), (3, 4), (2, 3), (1, 4)]:
        plan.set_schedule(big, small)
        assert blobs(plan.run()) == [ref], (big, small)
    f = plan.run()[0]
    assert f.stats()["levels"] == A.aiwcrf_fit(params, X, y).stats()["levels"]
    plan.close()


def test_plan_with_depth_limit_and_no_bootstrap():
    wl = synth.small_case(31, 1500, 12, card=40)
    X, y = dev(wl.X), dev(wl.y)
    for params in (A.params(16, 5, 2, max_depth=4), A.params(8, 12, 1, bootstrap=False)):
        ref = A.aiwcrf_fit(params, X, y).serialize()
        assert blobs(A.FitPlan(params, X, y).run()) == [ref]


def test_plan_subsets_equal_fit_subsets():
    wl, folds = synth.loko_folds()
    folds = folds[:7]
    offs = np.cumsum([0] + [len(tr) for tr, _ in folds]).astype(np.int64)
    rows = dev(np.concatenate([tr for tr, _ in folds]).astype(np.int32))
    X, y = dev(wl.X), dev(wl.y)
    params = A.params(24, 10, 5)
    ref = blobs(A.aiwcrf_fit_subsets(params, X, y, offs, rows))
    plan = A.FitPlan(params, X, y, offs, rows)
    assert blobs(plan.run()) == ref
    chosen, tried = plan.tune(reps=1)
    assert len(tried) >= 12 and chosen["ms"] == min(t["ms"] for t in tried)
    assert (chosen["level_big_ctas_per_sm"], chosen["level_small_ctas_per_sm"]) in \
        {(t["level_big_ctas_per_sm"], t["level_small_ctas_per_sm"]) for t in tried}
    assert blobs(plan.run()) == ref


def test_plan_reads_the_bound_data_at_every_run():
    wl = synth.plain_forest_workload()
    X, y = dev(wl.X), dev(wl.y)
    params = A.params(32, 10, 5)
    plan = A.FitPlan(params, X, y)
    assert blobs(plan.run()) == [A.aiwcrf_fit(params, X, y).serialize()]
    y2 = synth.plain_forest_workload(seed=synth.DATA_SEED + 9).y     # new targets, same features
    y.copy_(torch.from_numpy(y2))
    assert blobs(plan.run()) == [A.aiwcrf_fit(params, X, y).serialize()]


def test_plan_capacity_overflow_fails_cleanly():
    rng = np.random.default_rng(3)
    base = rng.normal(size=(8, 10)).astype(np.float32)
    Xd = np.ascontiguousarray(base[:, rng.integers(0, 10, 1000)])      # 10 distinct rows
    y = dev(rng.integers(-2 ** 33, 2 ** 33, 1000).astype(np.int64))
    X = dev(Xd)
    params = A.params(6, 4, 2)
    plan = A.FitPlan(params, X, y)
    assert blobs(plan.run()) == [A.aiwcrf_fit(params, X, y).serialize()]
    X.copy_(torch.from_numpy(rng.normal(size=(8, 1000)).astype(np.float32)))   # 1000 distinct rows
    with pytest.raises(A.AiwcrfError) as e:
        plan.run()
    assert e.value.code == -8
    # the plan stays usable once the data fits again
    X.copy_(torch.from_numpy(Xd))
    assert blobs(plan.run()) == [A.aiwcrf_fit(params, X, y).serialize()]


def test_plan_needs_device_memory():
    wl = synth.small_case(5, 100, 4)
    with pytest.raises(A.AiwcrfError) as e:
        A.FitPlan(A.params(2, 2, 2), wl.X, wl.y)
    assert e.value.code == -3
