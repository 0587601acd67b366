// noalloc.cu -- device selection for callers that must not allocate device memory.
//
// aiwcrf_select_device allocates its scratch (expanded queries, their rank codes, the
// predictions) on the stream. Some callers cannot allow that: a scheduler hook that runs inside
// another application's process, where device memory is owned by that application's allocator
// and a cudaMalloc/cudaFree would break its budget or force a device-wide synchronisation at a
// point where the hook must not block. This file gives them aiwcrf_select_device_noalloc, whose
// scratch is one file-scope __device__ array that every GPU loading the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace aiwcrf {

// The shared scratch. In host code this name is only a host-side stand-in for the symbol, not
// a device address: the address each device uses comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_select_scratch[AIWCRF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {};

// Once per device, with that device current: look up the array's device address.
int scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(AIWCRF_E_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(select scratch)");
        g_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_ptr[dev];
    return AIWCRF_OK;
}

bool is_device_ptr(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}
}  // namespace

}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" int aiwcrf_select_device_noalloc(const aiwcrf_forest *forest, const float *kfeat, int32_t n_kernels,
                                            int32_t size_class, const int32_t *device_ids, int32_t n_devices,
                                            int32_t *out_best, int64_t *out_pred, void *cuda_stream)
{
    clear_last_error();
    if (!forest || !kfeat || !device_ids || !out_best)
        return fail(AIWCRF_E_INVALID_ARG, "forest, kfeat, device_ids and out_best must not be NULL");
    if (n_kernels < 1 || n_devices < 1) return fail(AIWCRF_E_INVALID_ARG, "n_kernels and n_devices must be >= 1");
    if (forest->F < 3) return fail(AIWCRF_E_INVALID_ARG, "the forest needs >= 3 features (kernel, device, size)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
    if (dev != forest->device) return fail(AIWCRF_E_BAD_POINTER, "the forest lives on another device");
    if (!is_device_ptr(kfeat, dev) || !is_device_ptr(out_best, dev) || (out_pred && !is_device_ptr(out_pred, dev)))
        return fail(AIWCRF_E_BAD_POINTER, "kfeat, out_best and out_pred must be memory of the current device");
    const size_t need = select_noalloc_bytes(forest, n_kernels, n_devices);
    if (need > (size_t)AIWCRF_NOALLOC_SCRATCH_BYTES)
        return fail(AIWCRF_E_LIMIT, "request needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                                        std::to_string((size_t)AIWCRF_NOALLOC_SCRATCH_BYTES));
    unsigned char *scratch = nullptr;
    int rc = scratch_for_device(dev, &scratch);
    if (rc) return rc;
    return select_launch_noalloc(forest, kfeat, n_kernels, size_class, device_ids, n_devices, out_best, out_pred,
                                 scratch, (cudaStream_t)cuda_stream);
}
