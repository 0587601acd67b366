"""Gated requests in the device-selection server: the surrogate resident beside the forest.

Every gated answer (device, float predictions, fallback flag) is compared with
aiwcrf_select_device_gated, called alone on a forest fitted by aiwcrf_fit on the same rows with the
same surrogate and gate (that call is pinned to the oracle in test_gpu_gate.py), and every exact
answer with aiwcrf_select_device: requests alone, gated and exact requests forced into shared
batches, under Poisson load with a random mix, after a refit, and through the surrogate's life
cycle in the server (set, caller's copy freed, removed while requests wait).
"""
import numpy as np
import pytest

from paper_1811_00156_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1811_00156_gb300 import aiwcrf as A

T, MTRY, MIN_NODE, VAR_TREES, Z = 64, 10, 5, 16, 0.05
DEVICES = np.arange(synth.N_DEVICES, dtype=np.int32)
D = DEVICES.size


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def fitp():
    return A.params(T, MTRY, MIN_NODE)


_TAU = {}


def gate():
    """Out-of-range and variance tests (small z), and a margin threshold at the median surrogate
    margin of the pool, so that about half of the in-range kernels fall back."""
    return A.gate_params(VAR_TREES, Z, ood=True, tau=_TAU["tau"])


def median_margin(sg, pool):
    K = pool.shape[1]
    m = []
    for s in range(synth.N_SIZES):
        Xq = np.empty((synth.N_FEATURES, K * D), np.float32)
        Xq[:synth.N_AIWC] = np.repeat(pool, D, axis=1)
        Xq[synth.COL_DEVICE] = np.tile(DEVICES, K)
        Xq[synth.COL_SIZE] = s
        out = torch.empty(K * D, dtype=torch.float32, device="cuda")
        sg.predict(torch.from_numpy(Xq).cuda(), out)
        v = np.sort(out.cpu().numpy().reshape(K, D).astype(np.float64), axis=1)
        m.append(v[:, 1] - v[:, 0])
    m = np.concatenate(m)
    return float(np.median(m[np.isfinite(m)]))


@pytest.fixture(scope="module")
def base():
    return synth.plain_forest_workload()


@pytest.fixture(scope="module")
def pool():
    # the query distribution, with kernels outside the training range and NaNs (they fall back)
    P = synth.queries(512, seed=synth.QUERY_SEED + 5)[:synth.N_AIWC].copy()
    P[4, 3] = 1e30
    P[17, 40] = -1e30
    P[9, 77] = np.nan
    return np.ascontiguousarray(P)


@pytest.fixture(scope="module")
def surrogate(base, pool):
    f = A.aiwcrf_fit(fitp(), base.X, base.y)
    Xs = torch.from_numpy(synth.queries(32768, seed=31)).cuda()
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=2, batch=1024), f, Xs)
    _TAU["tau"] = median_margin(sg, pool)
    return sg


def gated_reference(X, y, sg, pool, sizes=range(synth.N_SIZES)):
    """size -> (best[P], pred[P, D] float, fallback[P]) from aiwcrf_select_device_gated."""
    f = A.aiwcrf_fit(fitp(), np.ascontiguousarray(X), np.ascontiguousarray(y))
    kf = torch.from_numpy(pool).cuda()
    P = pool.shape[1]
    out = {}
    for s in sizes:
        best = torch.empty(P, dtype=torch.int32, device="cuda")
        pred = torch.empty(P * D, dtype=torch.float32, device="cuda")
        fb = torch.empty(P, dtype=torch.uint8, device="cuda")
        A.aiwcrf_select_device_gated(f, sg, gate(), kf, s, DEVICES, best, pred, fb)
        out[s] = (best.cpu().numpy(), pred.view(P, D).cpu().numpy(), fb.cpu().numpy())
    return out


def exact_reference(X, y, pool, sizes=range(synth.N_SIZES)):
    f = A.aiwcrf_fit(fitp(), np.ascontiguousarray(X), np.ascontiguousarray(y))
    out = {}
    for s in sizes:
        best = np.zeros(pool.shape[1], np.int32)
        pred = np.zeros((pool.shape[1], D), np.int64)
        A.aiwcrf_select_device(f, pool, s, DEVICES, best, pred)
        out[s] = (best, pred)
    return out


def check_gated(got, ref, lo, hi, msg=""):
    best, pred, fb = got[:3]
    np.testing.assert_array_equal(best, ref[0][lo:hi], err_msg=msg)
    np.testing.assert_array_equal(pred, ref[1][lo:hi], err_msg=msg)      # bit for bit
    np.testing.assert_array_equal(fb, ref[2][lo:hi], err_msg=msg)


def test_gated_request_alone_matches_select_device_gated(base, pool, surrogate):
    ref = gated_reference(base.X, base.y, surrogate, pool)
    # both paths are exercised: the gate keeps some kernels and sends others to the forest
    fb_all = np.concatenate([ref[s][2] for s in ref])
    assert 0 < fb_all.sum() < fb_all.size
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        srv.set_surrogate(surrogate, gate())
        assert srv.stats()["surrogate_bytes"] > 0
        n_k = n_fb = 0
        for i, (lo, s) in enumerate([(0, 0), (64, 1), (100, 2), (448, 3), (37, 2)]):
            hi = lo + 64
            got = srv.wait_gated(srv.submit(np.ascontiguousarray(pool[:, lo:hi]), s, gated=True))
            assert got[3] == 0
            check_gated(got, ref[s], lo, hi, msg=f"request {i}")
            n_k += hi - lo
            n_fb += int(got[2].sum())
        st = srv.stats()
    assert st["gated_kernels"] == n_k and st["gated_fallback"] == n_fb
    assert st["gated_fallback_ood"] + st["gated_fallback_var"] >= n_fb


def test_gated_and_exact_requests_share_batches(base, pool, surrogate):
    gref = gated_reference(base.X, base.y, surrogate, pool)
    xref = exact_reference(base.X, base.y, pool)
    rng = np.random.default_rng(5)
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        srv.set_surrogate(surrogate, gate())
        for rnd in range(4):
            srv.pause(True)
            reqs = []
            for j in range(16):
                k = int(rng.integers(1, 65))
                lo = int(rng.integers(0, pool.shape[1] - k + 1))
                s = int(rng.integers(0, synth.N_SIZES))
                g = bool((j + rnd) % 3 != 0)
                reqs.append((srv.submit(np.ascontiguousarray(pool[:, lo:lo + k]), s, gated=g), g, lo, k, s))
            srv.pause(False)
            for t, g, lo, k, s in reqs:
                if g:
                    check_gated(srv.wait_gated(t), gref[s], lo, lo + k, msg=f"gated {lo}+{k} size {s}")
                else:
                    best, pred, _ = srv.wait(t)
                    np.testing.assert_array_equal(best, xref[s][0][lo:lo + k])
                    np.testing.assert_array_equal(pred, xref[s][1][lo:lo + k])
        batches, _ = srv.trace()
    mixed = batches[(batches["gated_kernels"] > 0) & (batches["gated_kernels"] < batches["kernels"])]
    assert mixed.size >= 1                          # gated and exact kernels in one batch


def test_poisson_load_with_gated_mix(base, pool, surrogate):
    gref = gated_reference(base.X, base.y, surrogate, pool)
    xref = exact_reference(base.X, base.y, pool)
    rng = np.random.default_rng(23)
    n = 1200
    k = rng.integers(1, 65, n).astype(np.int32)
    first = np.array([rng.integers(0, pool.shape[1] - kk + 1) for kk in k], np.int64)
    size = rng.integers(0, synth.N_SIZES, n).astype(np.int32)
    gated = (rng.random(n) < 0.5).astype(np.uint8)
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        srv.set_surrogate(surrogate, gate())
        rep, best, gen, lat = srv.run_load(pool, first, k, size, rate_per_s=20000.0, seed=3, gated=gated)
        st = srv.stats()
    assert rep["failed"] == 0 and rep["rejected"] == 0 and (lat >= 0).all() and (gen == 0).all()
    off = 0
    for i in range(n):
        s, lo, kk = int(size[i]), int(first[i]), int(k[i])
        want = (gref if gated[i] else xref)[s][0][lo:lo + kk]
        np.testing.assert_array_equal(best[off:off + kk], want, err_msg=f"request {i} gated {gated[i]}")
        off += kk
    assert st["gated_kernels"] == int(k[gated == 1].sum())


def test_gated_answers_follow_a_refit(base, pool, surrogate):
    extra = synth.plain_forest_workload(seed=synth.DATA_SEED + 1)
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        srv.set_surrogate(surrogate, gate())
        srv.append(extra.X, extra.y)
        srv.refit(wait=True)
        got = srv.wait_gated(srv.submit(np.ascontiguousarray(pool[:, :64]), 1, gated=True))
    assert got[3] == 1
    ref = gated_reference(np.concatenate([base.X, extra.X], axis=1), np.concatenate([base.y, extra.y]), surrogate,
                          pool, sizes=[1])
    check_gated(got, ref[1], 0, 64)


def test_surrogate_life_cycle_in_the_server(base, pool, surrogate):
    f = A.aiwcrf_fit(fitp(), base.X, base.y)
    Xs = torch.from_numpy(synth.queries(8192, seed=33)).cuda()
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=1, batch=1024), f, Xs)
    ref = gated_reference(base.X, base.y, sg, pool, sizes=[0])
    kf = np.ascontiguousarray(pool[:, :32])
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        with pytest.raises(RuntimeError):
            srv.submit(kf, 0, gated=True)                   # no surrogate yet
        with pytest.raises(RuntimeError):
            srv.set_surrogate(sg, A.gate_params(T + 1, Z))  # var_trees above the forest's trees
        with pytest.raises(RuntimeError):
            srv.set_surrogate(sg, A.gate_params(VAR_TREES, Z, tau=-1.0))
        with pytest.raises(RuntimeError):
            srv.set_surrogate(sg, None)
        srv.set_surrogate(sg, gate())
        del sg                                              # the server holds its own copy
        import gc
        gc.collect()
        t = srv.submit(kf, 0, gated=True)
        with pytest.raises(RuntimeError):
            srv.wait(t)                                     # wrong kind: refused, ticket kept
        check_gated(srv.wait_gated(t), ref[0], 0, 32)
        te = srv.submit(kf, 0)
        with pytest.raises(RuntimeError):
            srv.wait_gated(te)
        srv.wait(te)
        # removed while a gated request waits: it fails, an exact one is answered
        srv.pause(True)
        tg = srv.submit(kf, 0, gated=True)
        tx = srv.submit(kf, 0)
        srv.set_surrogate(None)
        srv.pause(False)
        with pytest.raises(RuntimeError):
            srv.wait_gated(tg)
        srv.wait(tx)
        assert srv.stats()["surrogate_bytes"] == 0
        with pytest.raises(RuntimeError):
            srv.submit(kf, 0, gated=True)
