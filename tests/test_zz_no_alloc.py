"""The allocation-free device selection (aiwcrf_select_device_noalloc) against the allocating
one (aiwcrf_select_device), through the C ABI.

Callers that cannot allocate device memory (for instance a scheduler hook inside another
application whose allocator owns the device memory) use the no-alloc entry point; its scratch is
one static device array shared by every call. The check runs two calls in a row with different
inputs, so a result left behind in the shared array by the first call cannot pass for the second.
Results are integers (device ids and Q32.32 predictions): they must match exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_00156_gb300 import aiwcrf
    return aiwcrf


def test_noalloc_matches_allocating_select_twice(A):
    from paper_1811_00156_gb300 import synth
    wl = synth.plain_forest_workload()
    forest = A.aiwcrf_fit(A.params(24, 10, 5), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    calls = [(64, 2, list(range(15)), 3), (17, 0, [9, 2, 14, 5, 0], 4)]
    for K, size, devices, seed in calls:
        kfeat = torch.from_numpy(np.ascontiguousarray(synth.queries(K, seed=seed)[:30])).cuda()
        best_a = torch.empty(K, dtype=torch.int32, device="cuda")
        pred_a = torch.empty(K * len(devices), dtype=torch.int64, device="cuda")
        A.aiwcrf_select_device(forest, kfeat, size, devices, best_a, pred_a)
        best_b = torch.full((K,), -7, dtype=torch.int32, device="cuda")
        pred_b = torch.full((K * len(devices),), -7, dtype=torch.int64, device="cuda")
        A.aiwcrf_select_device_noalloc(forest, kfeat, size, devices, best_b, pred_b)
        torch.cuda.synchronize()
        assert torch.equal(best_a, best_b)
        assert torch.equal(pred_a, pred_b)
        assert set(best_b.cpu().tolist()) <= set(devices)


class _DefaultPool:
    """The current device's default stream-ordered memory pool, read through the driver API:
    the library's stream-ordered allocations (cudaMallocAsync) come from it."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8          # CUmemPool_attribute values

    def __init__(self):
        import ctypes as C
        self.C = C
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int(0)
        assert self.cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = self.C.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, self.C.byref(v)) == 0
        return v.value

    def reset_high(self):
        """Reset the high-water mark of used pool memory to the current use."""
        zero = self.C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, self.C.byref(zero)) == 0


def test_noalloc_allocates_no_device_memory(A):
    """Across a warm call, neither the default pool's high-water mark of used memory nor the
    device's free memory moves; the same probe sees the allocating entry point allocate."""
    from paper_1811_00156_gb300 import synth
    wl = synth.plain_forest_workload()
    forest = A.aiwcrf_fit(A.params(16, 10, 5), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    K, devices = 48, list(range(15))
    kfeat = torch.from_numpy(np.ascontiguousarray(synth.queries(K, seed=21)[:30])).cuda()
    best = torch.empty(K, dtype=torch.int32, device="cuda")
    pred = torch.empty(K * len(devices), dtype=torch.int64, device="cuda")
    A.aiwcrf_select_device_noalloc(forest, kfeat, 1, devices, best, pred)       # warm: modules loaded
    A.aiwcrf_select_device(forest, kfeat, 1, devices, best, pred)
    torch.cuda.synchronize()
    pool = _DefaultPool()
    used0 = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    A.aiwcrf_select_device_noalloc(forest, kfeat, 1, devices, best, pred)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) == used0
    assert torch.cuda.mem_get_info()[0] == free0
    A.aiwcrf_select_device(forest, kfeat, 1, devices, best, pred)              # the probe's control
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > used0


def test_noalloc_rejects_requests_beyond_the_static_scratch(A):
    from paper_1811_00156_gb300 import synth
    wl = synth.small_case(3, 300, 32, card=20)
    forest = A.aiwcrf_fit(A.params(4, 10, 5), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    K = 20000                                        # 20,000 kernels x 15 devices: far above 1 MiB
    kfeat = torch.zeros((30, K), dtype=torch.float32, device="cuda")
    best = torch.empty(K, dtype=torch.int32, device="cuda")
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_select_device_noalloc(forest, kfeat, 1, list(range(15)), best)
    assert e.value.code == -8
    # host outputs would need staging, which allocates: rejected
    host_best = np.zeros(4, np.int32)
    with pytest.raises(A.AiwcrfError) as e:
        A.aiwcrf_select_device_noalloc(forest, kfeat[:, :4].contiguous(), 1, list(range(15)), host_best)
    assert e.value.code == -3
