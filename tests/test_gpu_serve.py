"""Device-selection server on the GPU.

Every answer the server gives is compared with aiwcrf_select_device on a forest fitted by
aiwcrf_fit on the same rows (itself pinned to the oracle in test_gpu_parity.py, and here once
more directly): for one request alone, for requests forced into shared batches, under a Poisson
load with many batches in flight, across refits, and when the arena limits admission.
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_00156_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1811_00156_gb300 import aiwcrf as A

T, MTRY, MIN_NODE = 128, 10, 5
DEVICES = np.arange(synth.N_DEVICES, dtype=np.int32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def base():
    return synth.plain_forest_workload()


@pytest.fixture(scope="module")
def pool():
    # kernel features of the query distribution; a few NaNs (they go right at every split)
    P = synth.queries(512, seed=synth.QUERY_SEED + 3)[:synth.N_AIWC].copy()
    P[3, 17] = np.nan
    P[11, 200] = np.nan
    return np.ascontiguousarray(P)


def fitp():
    return A.params(T, MTRY, MIN_NODE)


def reference(X, y, pool, sizes=range(synth.N_SIZES), fp=None):
    """best[size][p] and pred[size][p, D] from aiwcrf_select_device over the whole pool."""
    f = A.aiwcrf_fit(fp or fitp(), np.ascontiguousarray(X), np.ascontiguousarray(y))
    out = {}
    for s in sizes:
        best = np.zeros(pool.shape[1], np.int32)
        pred = np.zeros((pool.shape[1], DEVICES.size), np.int64)
        A.aiwcrf_select_device(f, pool, s, DEVICES, best, pred)
        out[s] = (best, pred)
    return out


def random_requests(rng, n, P, kmax=64):
    k = rng.integers(1, kmax + 1, n).astype(np.int32)
    first = np.array([rng.integers(0, P - kk + 1) for kk in k], np.int64)
    size = rng.integers(0, synth.N_SIZES, n).astype(np.int32)
    return first, k, size


def test_single_request_matches_select_device_and_oracle(base, pool):
    ref = reference(base.X, base.y, pool, sizes=[2])
    with A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES) as srv:
        kf = np.ascontiguousarray(pool[:, 100:164])
        best, pred, gen = srv.wait(srv.submit(kf, 2))
        assert gen == 0
        np.testing.assert_array_equal(best, ref[2][0][100:164])
        np.testing.assert_array_equal(pred, ref[2][1][100:164])
        st = srv.stats()
        assert st["completed"] == 1 and st["generation"] == 0 and st["training_rows"] == base.y.size
    # the oracle's own device choice for the first kernels (no NaN among them)
    of = O.fit(base.X, base.y, T, MTRY, MIN_NODE)
    obest, opred = of.select_device(np.ascontiguousarray(pool[:, 100:116]), 2, DEVICES)
    np.testing.assert_array_equal(best[:16], obest)
    np.testing.assert_array_equal(pred[:16], opred)


def test_wide_value_tables_use_the_eight_byte_walk():
    # continuous columns: more than 255 distinct values, so the forest has no compact copy
    wl = synth.small_case(seed=21, n=3000, f=synth.N_FEATURES)
    X = wl.X.copy()
    X[synth.COL_DEVICE] = np.arange(3000) % synth.N_DEVICES
    X[synth.COL_SIZE] = np.arange(3000) % synth.N_SIZES
    kf = synth.small_case(seed=22, n=40, f=synth.N_AIWC).X
    ref = reference(X, wl.y, kf, sizes=[1])
    with A.Server(A.server_params(), fitp(), X, wl.y, DEVICES) as srv:
        best, pred, _ = srv.wait(srv.submit(kf, 1))
    np.testing.assert_array_equal(best, ref[1][0])
    np.testing.assert_array_equal(pred, ref[1][1])


def test_requests_batched_together_match_alone(base, pool):
    rng = np.random.default_rng(5)
    first, k, size = random_requests(rng, 24, pool.shape[1])
    with A.Server(A.server_params(n_streams=2, batch_kernels=1024), fitp(), base.X, base.y, DEVICES) as srv:
        alone = []
        for i in range(first.size):
            kf = np.ascontiguousarray(pool[:, first[i]:first[i] + k[i]])
            alone.append(srv.wait(srv.submit(kf, int(size[i]))))
        b0 = srv.stats()["batches"]
        assert b0 == first.size
        srv.pause(True)
        tickets = [srv.submit(np.ascontiguousarray(pool[:, first[i]:first[i] + k[i]]), int(size[i]))
                   for i in range(first.size)]
        srv.pause(False)
        mixed = [srv.wait(t) for t in tickets]
        st = srv.stats()
    nb = st["batches"] - b0
    assert nb <= int(np.ceil(k.sum() / 1024)) + 1, nb      # the queue went out in shared batches
    assert st["batch_kernels_max"] > 64
    for (b1, p1, g1), (b2, p2, g2) in zip(alone, mixed):
        np.testing.assert_array_equal(b1, b2)
        np.testing.assert_array_equal(p1, p2)
        assert g1 == g2 == 0


def test_poisson_load_matches_reference(base, pool):
    ref = reference(base.X, base.y, pool)
    rng = np.random.default_rng(11)
    first, k, size = random_requests(rng, 3000, pool.shape[1])
    with A.Server(A.server_params(n_streams=4), fitp(), base.X, base.y, DEVICES) as srv:
        rep, best, gen, lat = srv.run_load(pool, first, k, size, rate_per_s=40000.0, seed=3)
        st = srv.stats()
    assert rep["n_requests"] == 3000 and rep["failed"] == 0 and rep["rejected"] == 0
    assert (gen == 0).all() and (lat > 0).all()
    assert 0 < rep["p50_us"] <= rep["p99_us"] <= rep["max_us"]
    assert rep["requests_per_s"] > 0 and rep["batches"] == st["batches"]
    off = 0
    for i in range(first.size):
        want = ref[int(size[i])][0][first[i]:first[i] + k[i]]
        np.testing.assert_array_equal(best[off:off + k[i]], want)
        off += k[i]


def test_refits_swap_in_forests_of_the_appended_rows(base, pool):
    extra = [synth.plain_forest_workload(seed=synth.DATA_SEED + 1 + r) for r in range(2)]
    rng = np.random.default_rng(17)
    first, k, size = random_requests(rng, 1500, pool.shape[1])
    sp = A.server_params(refit_every=400, refit_rows=base.y.size)
    with A.Server(sp, fitp(), base.X, base.y, DEVICES) as srv:
        for e in extra:
            srv.append(e.X, e.y)
        assert srv.stats()["appended_rows"] == 2 * base.y.size
        rep, best, gen, _ = srv.run_load(pool, first, k, size, rate_per_s=20000.0, seed=9)
        srv.refit(wait=True)            # no rows left: same rows, a new generation
        st = srv.stats()
        tb, tp, tg = srv.wait(srv.submit(np.ascontiguousarray(pool[:, :64]), 0))
    assert st["refits"] >= 3 and st["refit_failures"] == 0 and st["appended_rows"] == 0
    assert st["training_rows"] == 3 * base.y.size and tg == st["generation"]
    assert set(np.unique(gen)) <= {0, 1, 2, 3, 4} and gen.min() == 0
    Xs, ys = [base.X], [base.y]
    refs = {}
    for g in range(3):
        refs[g] = reference(np.concatenate(Xs, axis=1), np.concatenate(ys), pool)
        if g < 2:
            Xs.append(extra[g].X)
            ys.append(extra[g].y)
    off = 0
    for i in range(first.size):
        g = min(int(gen[i]), 2)         # later generations refit the same rows
        want = refs[g][int(size[i])][0][first[i]:first[i] + k[i]]
        np.testing.assert_array_equal(best[off:off + k[i]], want, err_msg=f"request {i} generation {gen[i]}")
        off += k[i]
    np.testing.assert_array_equal(tb, refs[2][0][0][:64])
    np.testing.assert_array_equal(tp, refs[2][0][1][:64])


def test_admission_by_arena_and_queue(base, pool):
    F, D = synth.N_FEATURES, DEVICES.size

    def req_bytes(K):
        up = lambda b: (b + 255) // 256 * 256
        return up(4 * F * K) + up(K * (8 * D + 4))

    sp = A.server_params(n_streams=4, max_request_kernels=64, batch_kernels=1024, max_pending=12,
                         arena_bytes=req_bytes(128))
    ref = reference(base.X, base.y, pool, sizes=[3])
    with A.Server(sp, fitp(), base.X, base.y, DEVICES) as srv:
        with pytest.raises(A.AiwcrfError) as e:
            srv.submit(np.ascontiguousarray(pool[:, :65]), 3)
        assert e.value.code == -8
        srv.pause(True)
        tickets = [srv.submit(np.ascontiguousarray(pool[:, 64 * i:64 * i + 64]), 3) for i in range(6)]
        tickets += [srv.submit(np.ascontiguousarray(pool[:, 400 + i:401 + i]), 3) for i in range(6)]
        with pytest.raises(A.AiwcrfError) as e:
            srv.submit(np.ascontiguousarray(pool[:, :4]), 3)
        assert e.value.code == -8
        srv.pause(False)
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["rejected"] == 2 and st["completed"] == 12
    assert st["arena_waits"] >= 1 and st["arena_peak_bytes"] <= req_bytes(128)
    assert st["batch_kernels_max"] <= 128
    for i in range(6):
        np.testing.assert_array_equal(res[i][0], ref[3][0][64 * i:64 * i + 64])
    for i in range(6):
        np.testing.assert_array_equal(res[6 + i][0], ref[3][0][400 + i:401 + i])


def test_shutdown_with_queued_requests(base, pool):
    srv = A.Server(A.server_params(), fitp(), base.X, base.y, DEVICES)
    srv.pause(True)
    for i in range(3):
        srv.submit(np.ascontiguousarray(pool[:, i:i + 8]), 0)
    srv.close()
