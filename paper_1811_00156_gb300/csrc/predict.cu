// predict.cu -- forest queries (Sec. I, Sec. V) and device selection (Sec. VI).
//
// predict_kernel: one CTA owns 256 * QPT queries, whose features it stages once in shared
// memory ([query][F + 1] floats, conflict-free across queries). It then walks every tree of
// the forest for all its queries. Trees stream through two shared-memory slots with 1-D bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier): while the CTA walks
// tree t from one slot, tree t + 1 is landing in the other. A tree larger than a slot is
// walked straight from global memory. Per-query sums are exact int64 (plus an exact 128-bit
// sum of squares for the variance), so the result does not depend on any ordering.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.cuh"

namespace aiwcrf {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

constexpr int kPredThreads = 256;
constexpr uint32_t kWaitLimit = 1u << 24;     // try_wait polls before giving up

// stage tree t into slot (or just complete the phase if it does not fit)
__device__ __forceinline__ void issue_tree(const uint64_t *nodes, const int64_t *tree_off, int t,
                                           int tree_cap, uint64_t *slot, uint64_t *bar)
{
    const int64_t a = tree_off[t], nn = tree_off[t + 1] - a;
    if (nn <= tree_cap) {
        const uint32_t bytes = (uint32_t)nn * 8u;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(slot, nodes + a, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

__device__ __forceinline__ int64_t leaf_value(uint64_t nd)
{
    return ((int64_t)(nd << 1)) >> 1;
}

__device__ __forceinline__ uint32_t next_node(uint64_t nd, const float *x)
{
    const uint32_t f = (uint32_t)(nd >> 56) & 0x7Fu;
    const uint32_t lc = (uint32_t)(nd >> 32) & 0xFFFFFFu;
    return lc + (x[f] <= __uint_as_float((uint32_t)nd) ? 0u : 1u);
}

template <int QPT, bool VAR>
__global__ void __launch_bounds__(kPredThreads) predict_kernel(
    const uint64_t *__restrict__ nodes, const int64_t *__restrict__ tree_off, int T, const float *__restrict__ Xq,
    int64_t Q, int F, int64_t total_trees, int tree_cap, int64_t *out_sum, int64_t *out_pred, uint64_t *out_var,
    uint32_t *err)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    uint64_t *slot0 = reinterpret_cast<uint64_t *>(sm_raw);
    uint64_t *slot1 = slot0 + tree_cap;
    float *xs = reinterpret_cast<float *>(slot1 + tree_cap);
    const int tid = threadIdx.x;
    const int QT = kPredThreads * QPT, ld = F + 1;
    const int64_t q0 = (int64_t)blockIdx.x * QT;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int f = 0; f < F; ++f) {
        const float *col = Xq + (size_t)f * (size_t)Q;
        for (int k = tid; k < QT; k += kPredThreads) {
            const int64_t q = q0 + k;
            xs[k * ld + f] = q < Q ? col[q] : 0.0f;
        }
    }
    __syncthreads();
    if (tid == 0) {
        issue_tree(nodes, tree_off, 0, tree_cap, slot0, &bar[0]);
        if (T > 1) issue_tree(nodes, tree_off, 1, tree_cap, slot1, &bar[1]);
    }

    int64_t acc[QPT];
    u128_t sq[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) { acc[i] = 0; sq[i] = 0; }

    for (int t = 0; t < T; ++t) {
        const int s = t & 1;
        const uint32_t parity = (uint32_t)((t >> 1) & 1);
        uint64_t *slot = s ? slot1 : slot0;
        bool ok = false;
        for (uint32_t it = 0; it < kWaitLimit && !ok; ++it) ok = mbar_try_wait(&bar[s], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, kErrTimeout);
            // give the other slot's copy a bounded chance to land before the CTA exits
            for (uint32_t it = 0; it < kWaitLimit; ++it)
                if (mbar_try_wait(&bar[s ^ 1], parity ^ (uint32_t)(s == 1))) break;
            return;
        }
        const int64_t a = tree_off[t];
        const bool fits = tree_off[t + 1] - a <= tree_cap;
        const uint64_t *tn = fits ? slot : nodes + a;

        uint32_t j[QPT];
        bool done[QPT];
#pragma unroll
        for (int i = 0; i < QPT; ++i) { j[i] = 0u; done[i] = false; }
        bool all = false;
        while (!all) {
            all = true;
#pragma unroll
            for (int i = 0; i < QPT; ++i) {
                if (!done[i]) {
                    const uint64_t nd = tn[j[i]];
                    if ((int64_t)nd < 0) {
                        const int64_t v = leaf_value(nd);
                        acc[i] += v;
                        if (VAR) sq[i] += (u128_t)((i128_t)v * (i128_t)v);
                        done[i] = true;
                    } else {
                        j[i] = next_node(nd, xs + (tid + i * kPredThreads) * ld);
                        all = false;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < T) issue_tree(nodes, tree_off, t + 2, tree_cap, slot, &bar[s]);
    }

#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int64_t q = q0 + tid + i * kPredThreads;
        if (q >= Q) continue;
        if (out_sum) out_sum[q] = acc[i];
        if (out_pred) {
            const i128_t num = (i128_t)2 * acc[i] + total_trees, den = (i128_t)2 * total_trees;
            i128_t d = num / den;
            if (num % den != 0 && num < 0) d -= 1;
            out_pred[q] = (int64_t)d;
        }
        if (VAR) {
            const u128_t V = (u128_t)total_trees * sq[i] - (u128_t)((i128_t)acc[i] * (i128_t)acc[i]);
            out_var[2 * q] = (uint64_t)V;
            out_var[2 * q + 1] = (uint64_t)(V >> 64);
        }
    }
}

__global__ void round_mean_kernel(const int64_t *sums, int64_t n, int64_t T, int64_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const i128_t num = (i128_t)2 * sums[i] + T, den = (i128_t)2 * T;
    i128_t d = num / den;
    if (num % den != 0 && num < 0) d -= 1;
    out[i] = (int64_t)d;
}

// query (k, j) of device selection: kernel k's features, device_ids[j], size_class
__global__ void expand_queries_kernel(const float *kfeat, int32_t K, int32_t size_class, const int32_t *dev,
                                      int32_t D, int32_t F, float *q)
{
    const int64_t Qn = (int64_t)K * D;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Qn) return;
    const int32_t k = (int32_t)(i / D), jd = (int32_t)(i % D);
    for (int f = 0; f < F - 2; ++f) q[(size_t)f * (size_t)Qn + i] = kfeat[(size_t)f * (size_t)K + k];
    q[(size_t)(F - 2) * (size_t)Qn + i] = (float)dev[jd];
    q[(size_t)(F - 1) * (size_t)Qn + i] = (float)size_class;
}

// argmin over devices per kernel; ties to the lower device id
__global__ void argmin_kernel(const int64_t *pred, const int32_t *dev, int32_t K, int32_t D, int32_t *best,
                              int64_t *out_pred)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int64_t bp = 0;
    int32_t bd = -1;
    for (int32_t jd = 0; jd < D; ++jd) {
        const int64_t p = pred[(size_t)k * (size_t)D + jd];
        if (out_pred) out_pred[(size_t)k * (size_t)D + jd] = p;
        if (bd < 0 || p < bp || (p == bp && dev[jd] < bd)) { bp = p; bd = dev[jd]; }
    }
    best[k] = bd;
}

namespace {

template <int QPT, bool VAR>
int launch_predict(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                   uint64_t *d_var, int64_t total_trees, cudaStream_t s, uint32_t *d_err)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int xs_bytes = kPredThreads * QPT * (f->F + 1) * 4;
    int budget = optin - xs_bytes - 1024;
    // two slots, each a whole number of 16-byte units, capped at 48 KB
    int tree_cap = std::min<int>(budget / 16, 6144);
    tree_cap &= ~1;
    if ((int64_t)tree_cap > f->max_tree_nodes) tree_cap = (int)((f->max_tree_nodes + 1) & ~(int64_t)1);
    if (tree_cap < 2) tree_cap = 2;
    const int smem = 2 * tree_cap * 8 + xs_bytes;
    auto kern = predict_kernel<QPT, VAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(predict_kernel)");
    const int64_t grid = (Q + (int64_t)kPredThreads * QPT - 1) / ((int64_t)kPredThreads * QPT);
    kern<<<(unsigned)grid, kPredThreads, smem, s>>>(f->d_nodes, f->d_tree_off, (int)f->T, dXq, Q, f->F,
                                                    total_trees, tree_cap, d_sum, d_pred, d_var, d_err);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "predict_kernel launch");
    return AIWCRF_OK;
}

}  // namespace

int predict_launch(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                   uint64_t *d_var, int64_t total_trees, cudaStream_t s)
{
    if (Q == 0) return AIWCRF_OK;
    uint32_t *d_err = nullptr;
    cudaError_t e = cudaMallocAsync(&d_err, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "device allocation failed");
    cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    prof_begin(s, kProfPredict);
    int rc;
    if (f->F <= 48) {
        rc = d_var ? launch_predict<2, true>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err)
                   : launch_predict<2, false>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err);
    } else {
        rc = d_var ? launch_predict<1, true>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err)
                   : launch_predict<1, false>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err);
    }
    prof_end(s, kProfPredict);
    uint32_t h_err = 0;
    if (rc == AIWCRF_OK) {
        e = cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "predict");
    }
    cudaFreeAsync(d_err, s);
    if (rc == AIWCRF_OK && (h_err & kErrTimeout)) rc = fail(AIWCRF_E_TIMEOUT, "a bounded device wait gave up");
    return rc;
}

int round_mean_launch(const int64_t *d_sum, int64_t Q, int64_t total_trees, int64_t *d_out, cudaStream_t s)
{
    if (Q == 0) return AIWCRF_OK;
    round_mean_kernel<<<(unsigned)((Q + 255) / 256), 256, 0, s>>>(d_sum, Q, total_trees, d_out);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "round_mean_kernel launch");
    return AIWCRF_OK;
}

int select_launch(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                  const int32_t *d_dev, int32_t D, int32_t *d_best, int64_t *d_pred, float *d_q,
                  int64_t *d_p, cudaStream_t s)
{
    const int64_t Qn = (int64_t)K * D;
    prof_begin(s, kProfSelect);
    expand_queries_kernel<<<(unsigned)((Qn + 255) / 256), 256, 0, s>>>(d_kfeat, K, size_class, d_dev, D, f->F, d_q);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "expand_queries_kernel launch");
    prof_end(s, kProfSelect);
    int rc = predict_launch(f, d_q, Qn, nullptr, d_p, nullptr, f->T, s);
    if (rc != AIWCRF_OK) return rc;
    prof_begin(s, kProfSelect);
    argmin_kernel<<<(unsigned)((K + 127) / 128), 128, 0, s>>>(d_p, d_dev, K, D, d_best, d_pred);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "argmin_kernel launch");
    prof_end(s, kProfSelect);
    return AIWCRF_OK;
}

}  // namespace aiwcrf
