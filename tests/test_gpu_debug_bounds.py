"""The bounds-checking build (libaiwcrf_debug.so, -DAIWCRF_DEBUG_BOUNDS) on the small parity
cases: every gathered entry row or group id, node id, walk node, split feature, histogram bin and
output position of the fit, predict, out-of-bag and selection kernels is checked on the device,
and no check may fire, while the results stay bit-exact against the oracle. The checks run in a
child process that loads the debug library (AIWCRF_LIB=debug)."""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import numpy as np, torch
    import oracle as O
    from paper_1811_00156_gb300 import aiwcrf as A, synth
    from tests.forest_util import assert_tree_equal, gpu_tree
    assert A.LIB_PATH.endswith("libaiwcrf_debug.so")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    assert A.aiwcrf_debug_bounds() == 0
    cases = [
        ("tree", synth.plain_forest_workload(), 16, 10, 5),
        ("level-2B", synth.small_case(31, 1500, 6), 6, 4, 2),
        ("level-4B", synth.small_case(32, 70000, 2), 2, 2, 60),
        ("ties", synth.small_case(33, 3000, 4, card=2, y_levels=1), 6, 2, 1),
    ]
    for name, wl, T, mtry, mn in cases:
        f = A.aiwcrf_fit(A.params(T, mtry, mn, seed=9), dev(wl.X), dev(wl.y))
        ref = O.fit(wl.X, wl.y, T, mtry, mn, seed=9)
        dec = A.decode_forest(f.serialize())
        for k in range(T):
            assert_tree_equal(gpu_tree(dec, k), ref.tree(k), where=f"{name} tree {k}")
        Xq = synth.small_case(5, 3000, wl.X.shape[0]).X
        out = torch.empty(Xq.shape[1], dtype=torch.int64, device="cuda")
        A.aiwcrf_predict(f, dev(Xq), out)
        s = torch.empty(wl.n_rows, dtype=torch.int64, device="cuda")
        c = torch.empty(wl.n_rows, dtype=torch.int32, device="cuda")
        A.aiwcrf_oob(f, dev(wl.X), s, c)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref.predict(Xq)[0]), name
        rs, rc = ref.oob(wl.X)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc), name
        assert A.aiwcrf_debug_bounds() == 0, name
    # selection through the tree-parallel kernel and the query-parallel path
    wl = synth.plain_forest_workload()
    f = A.aiwcrf_fit(A.params(32, 10, 5), dev(wl.X), dev(wl.y))
    ref = O.fit(wl.X, wl.y, 32, 10, 5, seed=156)
    for K, D in ((40, 15), (5, 100)):
        kf = np.ascontiguousarray(synth.queries(K, seed=K)[:30])
        devs = list(range(D))
        best = torch.empty(K, dtype=torch.int32, device="cuda")
        A.aiwcrf_select_device(f, dev(kf), 1, devs, best)
        torch.cuda.synchronize()
        assert np.array_equal(best.cpu().numpy(), ref.select_device(kf, 1, devs)[0])
    assert A.aiwcrf_debug_bounds() == 0
    print("debug-bounds ok")
""")


def test_debug_build_checks_fire_on_nothing_and_results_stay_exact():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_00156_gb300 import aiwcrf as A
    assert A.aiwcrf_debug_bounds() == -1                  # the release library compiles them away
    env = dict(os.environ, AIWCRF_LIB="debug", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "debug-bounds ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
