"""Surrogate device selection with the forest as fallback (aiwcrf_select_device_gated).

The gate's decisions are integer-exact and pinned to the oracle: the ensemble-variance numerators
of the forest's first trees come from the oracle's own forest of those trees, the out-of-range
test from the training matrix, and every kernel that falls back must get the oracle forest's
device and predictions. Kernels that pass the gate must get the argmin of the surrogate's own
predictions for the same queries.
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T, MTRY, MIN_NODE, VAR_TREES = 64, 10, 5, 16
DEV = np.arange(synth.N_DEVICES, dtype=np.int32)


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_00156_gb300 import aiwcrf
    return aiwcrf


@pytest.fixture(scope="module")
def models(A):
    wl = synth.plain_forest_workload()
    f = A.aiwcrf_fit(A.params(T, MTRY, MIN_NODE), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    Xs = torch.from_numpy(synth.queries(65536, seed=31)).cuda()
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=4, batch=1024), f, Xs)
    of = O.fit(wl.X, wl.y, T, MTRY, MIN_NODE)
    op = O.fit(wl.X, wl.y, VAR_TREES, MTRY, MIN_NODE)        # the first VAR_TREES trees
    return wl, f, sg, of, op


def kernels(K, seed):
    kf = synth.queries(K, seed=seed)[:synth.N_AIWC].copy()
    kf[4, 3] = 1e30                     # far above every training value
    kf[17, 5] = -1e30                   # far below
    kf[9, 7] = np.nan
    return np.ascontiguousarray(kf)


def expand(kf, size):
    K = kf.shape[1]
    D = DEV.size
    Xq = np.empty((synth.N_FEATURES, K * D), np.float32)
    Xq[:synth.N_AIWC] = np.repeat(kf, D, axis=1)
    Xq[synth.COL_DEVICE] = np.tile(DEV, K)
    Xq[synth.COL_SIZE] = size
    return Xq


def expected(A, models, kf, size, thr, ood):
    wl, f, sg, of, op = models
    K, D = kf.shape[1], DEV.size
    Xq = expand(kf, size)
    _, _, V = op.predict(Xq, want_var=True)
    V = np.array(V, dtype=object).reshape(K, D)
    q = int(np.floor(np.float64(np.float32(thr)) * 2.0 ** 64))
    var_fb = (V > q * VAR_TREES * VAR_TREES).any(axis=1)
    lo = wl.X.min(axis=1)[:, None]
    hi = wl.X.max(axis=1)[:, None]
    with np.errstate(invalid="ignore"):
        out = ~((Xq >= lo) & (Xq <= hi))
    ood_fb = out.any(axis=0).reshape(K, D).any(axis=1) if ood else np.zeros(K, bool)
    fb = var_fb | ood_fb
    s = torch.empty(K * D, dtype=torch.float32, device="cuda")
    sg.predict(torch.from_numpy(Xq).cuda(), s)
    s = s.cpu().numpy().reshape(K, D)
    best = DEV[np.argmin(s, axis=1)]
    pred = s.copy()
    obest, opred = of.select_device(kf, size, DEV)
    best[fb] = obest[fb]
    pred[fb] = (opred[fb].astype(np.float64) * 2.0 ** -32).astype(np.float32)
    return fb, ood_fb, var_fb, best, pred


def median_kernel_variance(models, kf, size):
    """Median over kernels of the largest prefix variance among the kernel's devices, (log10 s)^2."""
    wl, f, sg, of, op = models
    _, _, V = op.predict(expand(kf, size), want_var=True)
    v = np.array([float(x) for x in V]).reshape(kf.shape[1], -1) / (VAR_TREES ** 2 * 2.0 ** 64)
    return float(np.float32(np.median(v.max(axis=1))))


@pytest.mark.parametrize("thr,ood", [("median", True), (0.0, False), (1000.0, False), ("median", False)])
def test_gate_matches_oracle(A, models, thr, ood):
    wl, f, sg, of, op = models
    K, size = 300, 2
    kf = kernels(K, seed=41)
    if thr == "median":
        thr = median_kernel_variance(models, kf, size)
    fb, ood_fb, var_fb, best, pred = expected(A, models, kf, size, thr, ood)
    ob = torch.empty(K, dtype=torch.int32, device="cuda")
    opr = torch.empty(K * DEV.size, dtype=torch.float32, device="cuda")
    ofb = torch.empty(K, dtype=torch.uint8, device="cuda")
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(VAR_TREES, thr, ood), torch.from_numpy(kf).cuda(), size,
                                      DEV, ob, opr, ofb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ofb.cpu().numpy().astype(bool), fb)
    np.testing.assert_array_equal(ob.cpu().numpy(), best)
    np.testing.assert_array_equal(opr.cpu().numpy().reshape(K, -1), pred)
    assert st == {"kernels": K, "fallback": int(fb.sum()), "fallback_ood": int(ood_fb.sum()),
                  "fallback_var": int(var_fb.sum())}
    if thr == 1000.0:
        assert st["fallback"] == 0
    if ood:
        assert ood_fb[[3, 5, 7]].all()
    if thr not in (0.0, 1000.0):
        assert K // 4 < st["fallback"] < 3 * K // 4         # both paths taken


def test_gate_everything_falls_back_equals_select_device(A, models):
    wl, f, sg, of, op = models
    K = 97
    kf = np.ascontiguousarray(synth.queries(K, seed=43)[:synth.N_AIWC])
    ob = torch.empty(K, dtype=torch.int32, device="cuda")
    ofb = torch.empty(K, dtype=torch.uint8, device="cuda")
    # a threshold no prefix variance stays at or below: only identical trees pass
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(VAR_TREES, 0.0, True), torch.from_numpy(kf).cuda(), 1,
                                      DEV, ob, None, ofb)
    ref = torch.empty(K, dtype=torch.int32, device="cuda")
    A.aiwcrf_select_device(f, torch.from_numpy(kf).cuda(), 1, DEV, ref)
    torch.cuda.synchronize()
    m = ofb.cpu().numpy().astype(bool)
    assert st["fallback"] == int(m.sum()) and m.sum() > K // 2
    np.testing.assert_array_equal(ob.cpu().numpy()[m], ref.cpu().numpy()[m])


def test_gate_argument_checks(A, models):
    wl, f, sg, of, op = models
    kf = torch.from_numpy(kernels(8, seed=44)).cuda()
    ob = torch.empty(8, dtype=torch.int32, device="cuda")
    for g in (A.gate_params(0, 0.01), A.gate_params(T + 1, 0.01), A.gate_params(8, -1.0),
              A.gate_params(8, 2.0 ** 21), A.GateParams(8, 0.01, 2, 0), A.GateParams(8, 0.01, 1, 1)):
        with pytest.raises(A.AiwcrfError) as e:
            A.aiwcrf_select_device_gated(f, sg, g, kf, 0, DEV, ob)
        assert e.value.code == -1
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_select_device_gated(f, sg, A.gate_params(8, 0.01), kernels(8, seed=44), 0, DEV, ob)
    assert e.value.code == -3
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(8, 0.01), kf[:, :0].contiguous(), 0, DEV, ob)
    assert st["kernels"] == 0
