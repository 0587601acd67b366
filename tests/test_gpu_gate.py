"""Surrogate device selection with the forest as fallback (aiwcrf_select_device_gated).

The gate is pinned to the oracle: the exact ensemble-variance numerators of the forest's first
trees come from the oracle's own forest of those trees, the margin test is the header's double
arithmetic written out in Python (same operations, same order, so the decisions must agree bit
for bit), the out-of-range test comes from the training matrix, and every kernel that falls back
must get the oracle forest's device and predictions. Kernels that pass the gate must get the
argmin of the surrogate's own predictions for the same queries.
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


def surrogate_outputs(models, Xq):
    sg = models[2]
    s = torch.empty(Xq.shape[1], dtype=torch.float32, device="cuda")
    sg.predict(torch.from_numpy(Xq).cuda(), s)
    return s.cpu().numpy().reshape(-1, DEV.size)


def margin_terms(models, kf, size):
    """Per kernel: best and runner-up device indices, the margin m (double) and V_b + V_r (int)."""
    wl, f, sg, of, op = models
    K, D = kf.shape[1], DEV.size
    Xq = expand(kf, size)
    _, _, V = op.predict(Xq, want_var=True)
    V = np.array(V, dtype=object).reshape(K, D)
    s = surrogate_outputs(models, Xq)
    sv = np.where(np.isnan(s), np.float32(np.inf), s)
    b = np.argmin(sv, axis=1)                                   # ties: first = lower device id
    r = np.empty(K, np.int64)
    for k in range(K):
        rest = np.delete(np.arange(D), b[k])
        r[k] = rest[np.argmin(sv[k, rest])]
    m = [float(np.float64(sv[k, r[k]]) - np.float64(sv[k, b[k]])) for k in range(K)]
    Vs = [int(V[k, b[k]]) + int(V[k, r[k]]) for k in range(K)]
    return s, b, m, Vs


def expected(A, models, kf, size, z, ood, tau=0.0):
    """The gate written out from its definition in the header, in Python doubles."""
    wl, f, sg, of, op = models
    K = kf.shape[1]
    s, b, m, Vs = margin_terms(models, kf, size)
    zf = float(np.float32(z))
    z2 = zf * zf
    scale = float(VAR_TREES) * float(VAR_TREES) * 2.0 ** 64
    var_fb = np.zeros(K, bool)
    for k in range(K):
        vs = float(Vs[k] >> 64) * 2.0 ** 64 + float(Vs[k] & (2 ** 64 - 1))
        var_fb[k] = (m[k] * m[k]) * scale <= z2 * vs or m[k] < float(np.float32(tau))
    Xq = expand(kf, size)
    lo = wl.X.min(axis=1)[:, None]
    hi = wl.X.max(axis=1)[:, None]
    with np.errstate(invalid="ignore"):
        out = ~((Xq >= lo) & (Xq <= hi))
    ood_fb = out.any(axis=0).reshape(K, -1).any(axis=1) if ood else np.zeros(K, bool)
    fb = var_fb | ood_fb
    best = DEV[b].copy()
    pred = s.copy()
    obest, opred = of.select_device(kf, size, DEV)
    best[fb] = obest[fb]
    pred[fb] = (opred[fb].astype(np.float64) * 2.0 ** -32).astype(np.float32)
    return fb, ood_fb, var_fb, best, pred


def median_critical_z(models, kf, size):
    """Median over kernels of the z at which the margin test flips."""
    s, b, m, Vs = margin_terms(models, kf, size)
    zc = [abs(mk) * VAR_TREES * 2.0 ** 32 / np.sqrt(float(v)) if v > 0 else np.inf for mk, v in zip(m, Vs)]
    return float(np.float32(np.median(zc)))


def median_margin(models, kf, size):
    return float(np.float32(np.median(margin_terms(models, kf, size)[2])))


@pytest.mark.parametrize("z,ood,tau", [("median", True, 0.0), (0.0, False, 0.0), (1e5, False, 0.0),
                                       ("median", False, 0.0), (0.0, True, "median"), (0.0, False, "median")])
def test_gate_matches_oracle(A, models, z, ood, tau):
    wl, f, sg, of, op = models
    K, size = 300, 2
    kf = kernels(K, seed=41)
    if z == "median":
        z = median_critical_z(models, kf, size)
    if tau == "median":
        tau = median_margin(models, kf, size)
    fb, ood_fb, var_fb, best, pred = expected(A, models, kf, size, z, ood, tau)
    ob = torch.empty(K, dtype=torch.int32, device="cuda")
    opr = torch.empty(K * DEV.size, dtype=torch.float32, device="cuda")
    ofb = torch.empty(K, dtype=torch.uint8, device="cuda")
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(VAR_TREES, z, ood, tau), torch.from_numpy(kf).cuda(),
                                      size, DEV, ob, opr, ofb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ofb.cpu().numpy().astype(bool), fb)
    np.testing.assert_array_equal(ob.cpu().numpy(), best)
    np.testing.assert_array_equal(opr.cpu().numpy().reshape(K, -1), pred)
    assert st == {"kernels": K, "fallback": int(fb.sum()), "fallback_ood": int(ood_fb.sum()),
                  "fallback_var": int(var_fb.sum())}
    if z == 0.0 and tau == 0.0:     # only exact ties between the two best devices are uncertain at z = 0
        m = margin_terms(models, kf, size)[2]
        np.testing.assert_array_equal(var_fb, np.array(m) == 0.0)
    if z == 1e5:
        assert st["fallback_var"] > K * 9 // 10
    if ood:
        assert ood_fb[[3, 5, 7]].all()
    if not isinstance(z, float) or z not in (0.0, 1e5) or tau != 0.0:
        assert K // 4 < st["fallback_var"] < 3 * K // 4         # both paths taken


def test_gate_everything_falls_back_equals_select_device(A, models):
    wl, f, sg, of, op = models
    K = 97
    kf = np.ascontiguousarray(synth.queries(K, seed=43)[:synth.N_AIWC])
    ob = torch.empty(K, dtype=torch.int32, device="cuda")
    ofb = torch.empty(K, dtype=torch.uint8, device="cuda")
    # a margin no surrogate decision clears: (nearly) every kernel falls back
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(VAR_TREES, 1e5, True), torch.from_numpy(kf).cuda(), 1,
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
    for g in (A.gate_params(0, 1.0), A.gate_params(T + 1, 1.0), A.gate_params(8, -1.0),
              A.gate_params(8, 2.0 ** 21), A.GateParams(8, 1.0, 2, 0), A.GateParams(8, 1.0, 1, -1.0),
              A.GateParams(8, 1.0, 1, 2.0 ** 21), A.GateParams(8, 1.0, 1, float("nan"))):
        with pytest.raises(A.AiwcrfError) as e:
            A.aiwcrf_select_device_gated(f, sg, g, kf, 0, DEV, ob)
        assert e.value.code == -1
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_select_device_gated(f, sg, A.gate_params(8, 1.0), kernels(8, seed=44), 0, DEV, ob)
    assert e.value.code == -3
    st = A.aiwcrf_select_device_gated(f, sg, A.gate_params(8, 1.0), kf[:, :0].contiguous(), 0, DEV, ob)
    assert st["kernels"] == 0


def test_surrogate_selection_gains_throughput_over_forest(A):
    """What the trained network gains over forest-only selection: more kernels per second at a
    stated agreement with the forest's choice (a 500-tree forest of the 111,000-row workload)."""
    import time
    wl = synth.scaled_forest_workload()
    f = A.aiwcrf_fit(A.params(500, MTRY, MIN_NODE), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=4, batch=4096),
                                f, torch.from_numpy(synth.queries(262144, seed=32)).cuda())
    K = 65536
    kf = torch.from_numpy(np.ascontiguousarray(synth.queries(K, seed=45)[:synth.N_AIWC])).cuda()
    fb = torch.empty(K, dtype=torch.int32, device="cuda")
    sb = torch.empty(K, dtype=torch.int32, device="cuda")
    alone = A.gate_params(1, 0.0, ood=False)            # the surrogate's choice for every kernel

    def best_of(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    t_forest = best_of(lambda: A.aiwcrf_select_device(f, kf, 2, DEV, fb))
    t_sur = best_of(lambda: A.aiwcrf_select_device_gated(f, sg, alone, kf, 2, DEV, sb))
    agree = float((fb.cpu().numpy() == sb.cpu().numpy()).mean())
    assert t_forest / t_sur > 1.5, (t_forest, t_sur)
    assert agree > 0.6, agree
