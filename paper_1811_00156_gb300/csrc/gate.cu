// gate.cu -- device selection through the learned surrogate, with the forest as fallback and as
// the arbiter of its uncertain answers (the selection of Sec. VI, made cheaper; the paper's
// model is the forest alone).
//
// Pipeline on the caller's stream:
//  1. expand the K kernels into K x D queries (kernel features, device id, size class);
//  2. surrogate inference (fused tcgen05 kernel) for every query;
//  3. exact ensemble-variance numerators over the forest's first var_trees trees;
//  4. gate_kernel, one warp per kernel: out-of-range test of every feature of its D queries
//     against the forest's value tables, the surrogate's best and runner-up devices, the test of
//     their margin against the two contenders' ensemble spread and against a fixed threshold,
//     and the kernels that fall back appended to a list;
//  5. the fallback kernels' queries gathered, predicted by the whole forest, and their device
//     chosen from the exact int64 predictions (fix_kernel).
// Which kernel lands where in the fallback list depends on the order of the atomics, but every
// kernel's result depends only on its own queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace aiwcrf {

// argmin step over (value, device id): smaller value, then lower id; id INT_MAX = empty
__device__ __forceinline__ void take_min(float &bs, int32_t &bd, float os, int32_t od)
{
    if (od != INT_MAX && (bd == INT_MAX || os < bs || (os == bs && od < bd))) { bs = os; bd = od; }
}

__device__ __forceinline__ void warp_min(float &bs, int32_t &bd)
{
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const float os = __shfl_xor_sync(0xFFFFFFFFu, bs, w);
        const int32_t od = __shfl_xor_sync(0xFFFFFFFFu, bd, w);
        take_min(bs, bd, os, od);
    }
}

// One warp per kernel: range test of every feature of its D queries, the surrogate's best and
// runner-up devices, and the margin tests: against the two contenders' prefix variances, and
// against the fixed threshold tau. With list
// set, flag[k] is 1 for a kernel that falls back and the kernel is appended to list (counts:
// fallbacks, out-of-range, margin); without, flag[k] holds the reasons as bits (kGateForest,
// kGateOod, kGateVar) and nothing is counted.
__global__ void gate_kernel(const float *__restrict__ q, int64_t Qn, int F, int D, const float *__restrict__ fvals,
                            int64_t fstride, const uint32_t *__restrict__ fcard, const uint64_t *__restrict__ var,
                            double z2, double scale, double tau, int ood, const float *__restrict__ sur,
                            const int32_t *__restrict__ dev, int K, uint8_t *flag, int32_t *best, float *pred,
                            int32_t *list, unsigned long long *counts)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= K) return;                        // warp-uniform
    bool o = false;
    float bs = INFINITY, rs = INFINITY;
    int32_t bd = INT_MAX, rd = INT_MAX;
    for (int j = lane; j < D; j += 32) {
        const int64_t i = k * D + j;
        if (ood) {
            for (int f = 0; f < F; ++f) {
                const float x = q[(size_t)f * (size_t)Qn + (size_t)i];
                const float *V = fvals + (size_t)f * (size_t)fstride;
                const uint32_t c = fcard[f];
                if (c == 0 || !(x >= V[0] && x <= V[c - 1])) o = true;
            }
        }
        float sv = sur[i];
        if (pred) pred[i] = sv;
        if (sv != sv) sv = INFINITY;
        take_min(bs, bd, sv, dev[j]);
    }
    warp_min(bs, bd);                          // every lane now holds the best (bs, bd)
    // runner-up: the best among the devices other than bd
    int jb = -1;
    for (int j = lane; j < D; j += 32) {
        float sv = sur[k * D + j];
        if (sv != sv) sv = INFINITY;
        if (dev[j] == bd) { jb = j; continue; }
        take_min(rs, rd, sv, dev[j]);
    }
    warp_min(rs, rd);
    int jr = -1;
    for (int j = lane; j < D; j += 32)
        if (rd != INT_MAX && dev[j] == rd) jr = j;
    // the lanes holding b and r publish their queries' index; max over lanes
    for (int w = 16; w; w >>= 1) {
        jb = max(jb, __shfl_xor_sync(0xFFFFFFFFu, jb, w));
        jr = max(jr, __shfl_xor_sync(0xFFFFFFFFu, jr, w));
    }
    const bool any_o = __any_sync(0xFFFFFFFFu, o);
    if (lane == 0) {
        bool v = false;
        if (jr >= 0) {
            const int64_t ib = k * D + jb, ir = k * D + jr;
            const u128_t Vb = ((u128_t)var[2 * ib + 1] << 64) | var[2 * ib];
            const u128_t Vr = ((u128_t)var[2 * ir + 1] << 64) | var[2 * ir];
            const u128_t Vs = Vb + Vr;
            const double vs = __dadd_rn(__dmul_rn(__ull2double_rn((unsigned long long)(Vs >> 64)), 0x1p64),
                                        __ull2double_rn((unsigned long long)Vs));
            const double m = __dsub_rn((double)rs, (double)bs);
            const double lhs = __dmul_rn(__dmul_rn(m, m), scale);
            const double rhs = __dmul_rn(z2, vs);
            v = lhs <= rhs || m < tau;
        }
        const bool fb = any_o || v;
        flag[k] = !list ? (uint8_t)((fb ? kGateForest : 0u) | (any_o ? kGateOod : 0u) | (v ? kGateVar : 0u))
                        : (uint8_t)(fb ? 1 : 0);
        best[k] = bd;
        if (fb && list) {
            const unsigned long long slot = atomicAdd(&counts[0], 1ull);
            list[slot] = (int32_t)k;
            if (any_o) atomicAdd(&counts[1], 1ull);
            if (v) atomicAdd(&counts[2], 1ull);
        }
    }
}

// fq (F x n*D): the queries of the listed kernels
__global__ void gather_kernel(const float *__restrict__ q, int64_t Qn, int F, int D, const int32_t *__restrict__ list,
                              int64_t n, float *__restrict__ fq)
{
    const int64_t Qf = n * D;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (i >= Qf || f >= F) return;
    const int64_t k = list[i / D];
    const int j = (int)(i % D);
    fq[(size_t)f * (size_t)Qf + (size_t)i] = q[(size_t)f * (size_t)Qn + (size_t)(k * D + j)];
}

// one warp per listed kernel: the forest's exact choice and predictions
__global__ void fix_kernel(const int64_t *__restrict__ fpred, const int32_t *__restrict__ list, int64_t n, int D,
                           const int32_t *__restrict__ dev, int32_t *best, float *pred)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int64_t k = list[i];
    int64_t bp = LLONG_MAX;
    int32_t bd = INT_MAX;
    for (int j = lane; j < D; j += 32) {
        const int64_t p = fpred[i * D + j];
        if (pred) pred[k * D + j] = (float)((double)p * 0x1p-32);
        const int32_t id = dev[j];
        if (p < bp || (p == bp && id < bd)) { bp = p; bd = id; }
    }
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const int64_t op = __shfl_xor_sync(0xFFFFFFFFu, bp, w);
        const int32_t od = __shfl_xor_sync(0xFFFFFFFFu, bd, w);
        if (op < bp || (op == bp && od < bd)) { bp = op; bd = od; }
    }
    if (lane == 0) best[k] = bd;
}

namespace {

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

}  // namespace

int gate_check(const aiwcrf_forest *forest, const aiwcrf_gate_params *gate)
{
    if (gate->var_trees < 1 || gate->var_trees > forest->T || !(gate->z >= 0.0f) || !(gate->z < 1048576.0f) ||
        (gate->ood != 0 && gate->ood != 1) || !(gate->tau >= 0.0f) || !(gate->tau < 1048576.0f))
        return fail(AIWCRF_E_INVALID_ARG, "gate parameters out of range");
    return AIWCRF_OK;
}

size_t gate_scratch_bytes(int32_t F, int64_t Qn)
{
    return a256(4 * (size_t)F * (size_t)Qn) + a256(4 * (size_t)Qn) + a256(16 * (size_t)Qn) +
           a256(predict_codes_bytes_max(F, Qn));
}

GateBuffers gate_scratch_split(void *scratch, int32_t F, int64_t Qn)
{
    GateBuffers b{};
    unsigned char *c = static_cast<unsigned char *>(scratch);
    b.q = reinterpret_cast<float *>(c);
    c += a256(4 * (size_t)F * (size_t)Qn);
    b.sur = reinterpret_cast<float *>(c);
    c += a256(4 * (size_t)Qn);
    b.var = reinterpret_cast<uint64_t *>(c);
    c += a256(16 * (size_t)Qn);
    b.codes = c;
    return b;
}

int gate_enqueue(const aiwcrf_forest *forest, const aiwcrf_surrogate *sg, const aiwcrf_gate_params &gate,
                 const float *d_kfeat, int32_t K, int64_t ld, int32_t size_class, const float *d_size_row,
                 const int32_t *d_dev, int32_t D, const GateBuffers &b, cudaStream_t s)
{
    if (K == 0) return AIWCRF_OK;
    const int F = forest->F;
    const int64_t Qn = (int64_t)K * D;
    // the margin test's constants: (z * z) and var_trees^2 * 2^64 (exact in double)
    const double z2 = (double)gate.z * (double)gate.z;
    const double scale = (double)gate.var_trees * (double)gate.var_trees * 0x1p64;
    int rc;
    if ((rc = expand_launch(d_kfeat, K, ld, size_class, d_size_row, d_dev, D, F, b.q, s))) return rc;
    if ((rc = surrogate_predict_enqueue(sg, b.q, Qn, b.sur, b.err, s))) return rc;
    if ((rc = predict_prefix_var_enqueue(forest, b.q, Qn, gate.var_trees, b.var, s, b.err, b.codes))) return rc;
    const unsigned gblocks = (unsigned)(((int64_t)K * 32 + 255) / 256);
    gate_kernel<<<gblocks, 256, 0, s>>>(b.q, Qn, F, D, forest->d_fvals, forest->fstride, forest->d_fcard, b.var, z2,
                                        scale, (double)gate.tau, gate.ood, b.sur, d_dev, K, b.flag, b.best, b.pred,
                                        b.list, b.counts);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gate_kernel launch");
    return AIWCRF_OK;
}

}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" int aiwcrf_select_device_gated(const aiwcrf_forest *forest, const aiwcrf_surrogate *surrogate,
                                          const aiwcrf_gate_params *gate, const float *kfeat, int32_t n_kernels,
                                          int32_t size_class, const int32_t *device_ids, int32_t n_devices,
                                          int32_t *out_best, float *out_pred, uint8_t *out_fallback,
                                          aiwcrf_gate_stats *stats, void *cuda_stream)
{
    aiwcrf::clear_last_error();
    if (!forest || !surrogate || !gate || !device_ids)
        return fail(AIWCRF_E_INVALID_ARG, "forest, surrogate, gate and device_ids must not be NULL");
    if (n_kernels < 0 || n_devices < 1) return fail(AIWCRF_E_INVALID_ARG, "n_kernels >= 0 and n_devices >= 1");
    int rc = gate_check(forest, gate);
    if (rc) return rc;
    if (stats) *stats = aiwcrf_gate_stats{n_kernels, 0, 0, 0};
    if (n_kernels == 0) return AIWCRF_OK;
    if (!kfeat || !out_best) return fail(AIWCRF_E_INVALID_ARG, "kfeat and out_best must not be NULL");
    if (!on_device(kfeat) || !on_device(out_best) || (out_pred && !on_device(out_pred)) ||
        (out_fallback && !on_device(out_fallback)))
        return fail(AIWCRF_E_BAD_POINTER, "kfeat and the outputs must be device memory");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int F = forest->F, D = n_devices, K = n_kernels;
    const int64_t Qn = (int64_t)K * D;
    keep_pool_memory(forest->device);

    // scratch: device ids, queries, surrogate outputs, variance numerators, query codes, flags,
    // list, counters, error flag; then the fallback's gathered queries and predictions
    const size_t b_dev = a256(4 * (size_t)D), b_q = a256(4 * (size_t)F * (size_t)Qn), b_sur = a256(4 * (size_t)Qn);
    const size_t b_var = a256(16 * (size_t)Qn), b_codes = a256(predict_codes_bytes(forest, Qn));
    const size_t b_flag = a256((size_t)K), b_list = a256(4 * (size_t)K), b_cnt = a256(8 * 4);
    const size_t b_fp = a256(8 * (size_t)Qn);
    const size_t total = b_dev + b_q + b_sur + b_var + b_codes + b_flag + b_list + b_cnt + b_q + b_fp;
    unsigned char *blk = nullptr;
    if (cudaMallocAsync(&blk, total, s) != cudaSuccess) return fail(AIWCRF_E_OOM, "gated selection scratch");
    struct Free { unsigned char *p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{blk, s};
    unsigned char *c = blk;
    int32_t *d_dev = reinterpret_cast<int32_t *>(c); c += b_dev;
    float *d_q = reinterpret_cast<float *>(c); c += b_q;
    float *d_sur = reinterpret_cast<float *>(c); c += b_sur;
    uint64_t *d_var = reinterpret_cast<uint64_t *>(c); c += b_var;
    void *d_codes = c; c += b_codes;
    uint8_t *d_flag = out_fallback ? out_fallback : reinterpret_cast<uint8_t *>(c); c += b_flag;
    int32_t *d_list = reinterpret_cast<int32_t *>(c); c += b_list;
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(c);
    uint32_t *d_err = reinterpret_cast<uint32_t *>(d_cnt + 3); c += b_cnt;
    float *d_fq = reinterpret_cast<float *>(c); c += b_q;
    int64_t *d_fpred = reinterpret_cast<int64_t *>(c);

    cudaError_t e = cudaMemcpyAsync(d_dev, device_ids, 4 * (size_t)D, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 32, s);
    if (e != cudaSuccess) return cuda_fail(e, "gated selection set-up");
    prof_begin(s, kProfSelect);
    const GateBuffers gb{d_q, d_sur, d_var, d_codes, d_flag, out_best, out_pred, d_list, d_cnt, d_err};
    if ((rc = gate_enqueue(forest, surrogate, *gate, kfeat, K, K, size_class, nullptr, d_dev, D, gb, s))) return rc;
    unsigned long long h_cnt[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(h_cnt, d_cnt, 32, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gated selection");
    const int64_t n = (int64_t)h_cnt[0];
    if (n > 0) {
        const int64_t Qf = n * D;
        gather_kernel<<<dim3((unsigned)((Qf + 255) / 256), (unsigned)F), 256, 0, s>>>(d_q, Qn, F, D, d_list, n, d_fq);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gather_kernel launch");
        if ((rc = predict_enqueue(forest, d_fq, Qf, nullptr, d_fpred, s, d_err, d_codes))) return rc;
        fix_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(d_fpred, d_list, n, D, d_dev, out_best, out_pred);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fix_kernel launch");
    }
    prof_end(s, kProfSelect);
    uint32_t h_err = 0;
    e = cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gated selection");
    if (h_err & kErrTimeout) return fail(AIWCRF_E_TIMEOUT, "a bounded device wait gave up");
    if (stats) *stats = aiwcrf_gate_stats{K, n, (int64_t)h_cnt[1], (int64_t)h_cnt[2]};
    return AIWCRF_OK;
}
