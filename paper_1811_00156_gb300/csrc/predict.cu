// predict.cu -- forest queries (Sec. I, Sec. V) and device selection (Sec. VI).
//
// code_queries_kernel turns every query feature into its rank code c(x) = #{training values of
// the feature < x}; the forest keeps a copy of its nodes whose thresholds are the ranks of the
// training values they are, and x <= threshold  <=>  c(x) <= rank, so the walk is exact.
// predict_kernel: one CTA owns 256 * QPT queries whose codes (one byte per feature when every
// column has at most 255 values) it stages once in shared memory. It then walks every tree for
// all its queries, QPT independent walks per thread. Trees stream through two shared-memory
// slots with 1-D bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier):
// while the CTA walks tree t from one slot, tree t + 1 is landing in the other. A tree larger
// than a slot is walked straight from global memory. Per-query sums are exact int64 (plus an
// exact 128-bit sum of squares for the variance), so the result does not depend on any order.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

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
// device selections with at most this many queries use the tree-parallel kernel
constexpr int64_t kTreeParallelMaxQueries = 1 << 18;
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

// Rank codes of queries: c(x) = #{table values < x}; NaN goes right of every threshold
// (c = table size). One thread per query codes all F features (a binary search of each value
// table) into the query's row in shared memory; the CTA then writes its rows, which are
// contiguous in global memory, with 16-byte stores, so that every byte of the code matrix is
// written once, whole sectors at a time. A row is row_words 4-byte words; its padding is zero.
constexpr int kCodeThreads = 128;

// The binary searches of kCodeGroup features run side by side (their table loads in flight
// together), each for a fixed steps = bit width of the largest table: the same lower bound as
// a search that stops early.
constexpr int kCodeGroup = 4;

template <typename CT>
__global__ void __launch_bounds__(kCodeThreads) code_queries_kernel(const float *__restrict__ Xq, int64_t Q, int F,
                                                                   const float *__restrict__ fvals, int64_t fstride,
                                                                   const uint32_t *__restrict__ fcard,
                                                                   CT *__restrict__ codes, int row_words, int steps)
{
    extern __shared__ __align__(16) uint32_t code_rows[];         // kCodeThreads * row_words words
    const int tid = threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.x * kCodeThreads, q = q0 + tid;
    uint32_t *row = code_rows + (size_t)tid * (size_t)row_words;   // odd row_words: distinct banks
    for (int w = 0; w < row_words; ++w) row[w] = 0u;
    if (q < Q) {
        CT *c = reinterpret_cast<CT *>(row);
        for (int f0 = 0; f0 < F; f0 += kCodeGroup) {
            float x[kCodeGroup];
            uint32_t lo[kCodeGroup], len[kCodeGroup];
#pragma unroll
            for (int u = 0; u < kCodeGroup; ++u) {
                const int f = f0 + u;
                // features are read once: streaming loads (evict first in L1 and L2) leave the
                // codes written here resident in L2 for the key and walk kernels that read them
                x[u] = f < F ? __ldcs(&Xq[(size_t)f * (size_t)Q + q]) : 0.0f;
                const uint32_t n = f < F ? __ldg(&fcard[f]) : 0u;
                lo[u] = x[u] != x[u] ? n : 0u;                      // NaN: past every value
                len[u] = x[u] != x[u] ? 0u : n;
            }
            for (int it = 0; it < steps; ++it) {
#pragma unroll
                for (int u = 0; u < kCodeGroup; ++u) {
                    if (len[u]) {
                        const uint32_t half = len[u] >> 1;
                        if (__ldg(&fvals[(size_t)(f0 + u) * (size_t)fstride + lo[u] + half]) < x[u]) {
                            lo[u] += half + 1u;
                            len[u] -= half + 1u;
                        } else {
                            len[u] = half;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kCodeGroup; ++u)
                if (f0 + u < F) c[f0 + u] = (CT)lo[u];
        }
    }
    __syncthreads();
    const int64_t n = min((int64_t)kCodeThreads, Q - q0);
    const int words = (int)n * row_words;
    uint32_t *dst = reinterpret_cast<uint32_t *>(codes) + (size_t)q0 * (size_t)row_words;
    const int vec = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 ? words >> 2 : 0;
    for (int i = tid; i < vec; i += kCodeThreads)
        reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(code_rows)[i];
    for (int i = 4 * vec + tid; i < words; i += kCodeThreads) dst[i] = code_rows[i];
}

// bytes of one feature's code for a forest: one when every value table has at most 255 values
__host__ __forceinline__ int code_bytes_of(const aiwcrf_forest *f)
{
    return f->max_card <= 255u ? 1 : (f->max_card <= 65535u ? 2 : 4);
}

// Words of one query's code row: F codes rounded up to whole words, made odd so that rows
// staged side by side in shared memory start on distinct banks.
__host__ __forceinline__ int code_row_words(int F, int code_bytes)
{
    int w = (F * code_bytes + 3) / 4;
    if ((w & 1) == 0) ++w;
    return w;
}

// codes of Q queries (row_words words per query) on the stream
template <typename CT>
cudaError_t launch_code_queries(const aiwcrf_forest *f, const float *dXq, int64_t Q, CT *d_codes, int row_words,
                                cudaStream_t s)
{
    if (Q == 0) return cudaSuccess;
    const size_t smem = (size_t)kCodeThreads * (size_t)row_words * 4;        // <= 66 KB (F <= 128)
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(code_queries_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int steps = 32 - __builtin_clz(f->max_card | 1u);               // bit width of the largest table
    code_queries_kernel<CT><<<(unsigned)((Q + kCodeThreads - 1) / kCodeThreads), kCodeThreads, smem, s>>>(
        dXq, Q, f->F, f->d_fvals, f->fstride, f->d_fcard, d_codes, row_words, steps);
    count_launches(1);
    return cudaGetLastError();
}

// One step of QPT independent walks through one tree (coded thresholds).
template <typename CT, int QPT, typename NodePtr>
__device__ __forceinline__ void walk_tree(NodePtr tn, const CT *const (&xr)[QPT], int64_t (&acc)[QPT],
                                          u128_t (&sq)[QPT], bool var, uint32_t nn)
{
    uint32_t j[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) j[i] = 0u;
    for (;;) {
        bool more = false;
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            const uint64_t nd = tn[j[i]];
            const uint32_t hi = (uint32_t)(nd >> 32);
            const bool leaf = (int32_t)hi < 0;
            const uint32_t f = leaf ? 0u : ((hi >> 24) & 0x7Fu);
            const uint32_t c = (uint32_t)xr[i][f];
            const uint32_t nxt = (hi & 0xFFFFFFu) + (c > ((uint32_t)nd & 0xFFFFFFu) ? 1u : 0u);
            j[i] = leaf ? j[i] : AIWCRF_IDX(nxt, nn, kBoundWalk);
            more |= !leaf;
        }
        if (!more) break;
    }
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int64_t v = leaf_value(tn[j[i]]);
        acc[i] += v;
        if (var) sq[i] += (u128_t)((i128_t)v * (i128_t)v);
    }
}

// Coded walk. The CTA's 256 * QPT query codes sit in shared memory as rows of ld_words
// 32-bit words (an odd count, so neighbouring queries hit different banks).
template <typename CT, int QPT, bool VAR>
__global__ void __launch_bounds__(kPredThreads) predict_kernel(
    const uint64_t *__restrict__ nodes, const int64_t *__restrict__ tree_off, int T, const CT *__restrict__ codes,
    int64_t Q, int ld_words, int64_t total_trees, int tree_cap, int64_t *out_sum, int64_t *out_pred,
    uint64_t *out_var, uint32_t *err)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    uint64_t *slot0 = reinterpret_cast<uint64_t *>(sm_raw);
    uint64_t *slot1 = slot0 + tree_cap;
    uint32_t *xw = reinterpret_cast<uint32_t *>(slot1 + tree_cap);
    const int tid = threadIdx.x;
    const int QT = kPredThreads * QPT;
    const int64_t q0 = (int64_t)blockIdx.x * QT;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    // stage the tile's codes: global rows of ld_words words -> shared rows of ld_words words
    {
        const uint32_t *gw = reinterpret_cast<const uint32_t *>(codes);
        const int64_t nq = min((int64_t)QT, Q - q0);
        const int64_t words = nq * ld_words;
        const uint32_t *src = gw + (size_t)q0 * (size_t)ld_words;
        for (int64_t k = tid; k < words; k += kPredThreads) xw[k] = src[k];
    }
    __syncthreads();
    if (tid == 0) {
        issue_tree(nodes, tree_off, 0, tree_cap, slot0, &bar[0]);
        if (T > 1) issue_tree(nodes, tree_off, 1, tree_cap, slot1, &bar[1]);
    }

    const CT *xr[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i)
        xr[i] = reinterpret_cast<const CT *>(xw + (size_t)(tid + i * kPredThreads) * (size_t)ld_words);
    int64_t acc[QPT];
    u128_t sq[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) { acc[i] = 0; sq[i] = 0; }

    for (int t = 0; t < T; ++t) {
        const int s = t & 1;
        const uint32_t parity = (uint32_t)((t >> 1) & 1);
        bool ok = false;
        for (uint32_t it = 0; it < kWaitLimit && !ok; ++it) ok = mbar_try_wait(&bar[s], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, kErrTimeout);
            // give the other slot's copy (tree t + 1) a bounded chance to land before exiting
            if (t + 1 < T)
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(&bar[s ^ 1], (uint32_t)(((t + 1) >> 1) & 1))) break;
            return;
        }
        const int64_t a = tree_off[t];
        const uint32_t nn = (uint32_t)(tree_off[t + 1] - a);
        if (nn <= (uint32_t)tree_cap) {
            if (s) walk_tree<CT, QPT>(slot1, xr, acc, sq, VAR, nn);
            else walk_tree<CT, QPT>(slot0, xr, acc, sq, VAR, nn);
        } else {
            walk_tree<CT, QPT>(nodes + a, xr, acc, sq, VAR, nn);
        }
        __syncthreads();
        if (tid == 0 && t + 2 < T) issue_tree(nodes, tree_off, t + 2, tree_cap, s ? slot1 : slot0, &bar[s]);
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

// ------------------------------------------------------------------------------------------
// compact 4-byte coded nodes (one CTA per tree)
// ------------------------------------------------------------------------------------------
__global__ void compact_nodes_kernel(const uint64_t *__restrict__ cnodes, const int64_t *__restrict__ tree_off,
                                     const int64_t *__restrict__ tree_off4, uint32_t *__restrict__ c32)
{
    const int t = blockIdx.x;
    const int64_t a = tree_off[t], m = tree_off[t + 1] - a;
    const int64_t a4 = tree_off4[t], m4 = tree_off4[t + 1] - a4;
    for (int64_t j = threadIdx.x; j < m4; j += blockDim.x) {
        // a leaf (and a pad) is its own child: left = j, threshold 255 (no code exceeds it),
        // feature field 255 with the top bit as the leaf flag
        uint32_t v = 0xFFFF0000u | (uint32_t)j;
        if (j < m) {
            const uint64_t nd = cnodes[a + j];
            if (!(nd >> 63)) {
                const uint32_t f = (uint32_t)(nd >> 56) & 0x7Fu;
                const uint32_t lc = (uint32_t)(nd >> 32) & 0xFFFFFFu;
                const uint32_t code = (uint32_t)nd & 0xFFFFFFu;
                v = (f << 24) | (code << 16) | lc;
            }
        }
        c32[a4 + j] = v;
    }
}

__device__ __forceinline__ void issue_tree4(const uint32_t *c32, const int64_t *tree_off4, int t, int tree_cap,
                                            uint32_t *slot, uint64_t *bar)
{
    const int64_t a = tree_off4[t], nn = tree_off4[t + 1] - a;
    if (nn <= tree_cap) {
        const uint32_t bytes = (uint32_t)nn * 4u;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(slot, c32 + a, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

// Walk of compact nodes; returns each chain's leaf index within the tree. A leaf is its own
// child, so a step past it stays on it: chains step kWalkSteps nodes at a time with no per-step
// leaf test, and the warp stops once the last node of every chain was a leaf. (A leaf's feature
// field is 255: its code read lands in the padding after the query rows and is never above the
// leaf's threshold 255.)
constexpr int kWalkSteps = 2;
template <int QPT, typename NodePtr>
__device__ __forceinline__ void walk_tree4(NodePtr tn, const uint8_t *const (&xr)[QPT], uint32_t (&j)[QPT], uint32_t nn)
{
    uint32_t nd[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) j[i] = 0u;
    for (;;) {
#pragma unroll
        for (int u = 0; u < kWalkSteps; ++u) {
#pragma unroll
            for (int i = 0; i < QPT; ++i) {
                nd[i] = tn[j[i]];
                const uint32_t c = (uint32_t)xr[i][nd[i] >> 24];
                j[i] = AIWCRF_IDX((nd[i] & 0xFFFFu) + (c > ((nd[i] >> 16) & 0xFFu) ? 1u : 0u), nn, kBoundWalk);
            }
        }
        bool done = true;
#pragma unroll
        for (int i = 0; i < QPT; ++i) done = done && (int32_t)nd[i] < 0;
        if (__all_sync(kFull, done)) break;
    }
}

// The byte-code walk over compact trees. Leaf values are loaded from the 8-byte node array
// (L2-resident) and added one tree later, so their latency overlaps the next walk.
template <int QPT, bool VAR, bool PERM>
__global__ void __launch_bounds__(kPredThreads) predict4_kernel(
    const uint32_t *__restrict__ c32, const int64_t *__restrict__ tree_off4, const uint64_t *__restrict__ nodes,
    const int64_t *__restrict__ tree_off, int T, const uint8_t *__restrict__ codes, int64_t Q, int ld_words,
    int64_t total_trees, int tree_cap, int64_t *out_sum, int64_t *out_pred, uint64_t *out_var, uint32_t *err,
    const uint32_t *__restrict__ perm)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    uint32_t *slot0 = reinterpret_cast<uint32_t *>(sm_raw);
    uint32_t *slot1 = slot0 + tree_cap;
    uint32_t *xw = slot1 + tree_cap;
    const int tid = threadIdx.x;
    const int QT = kPredThreads * QPT;
    const int64_t q0 = (int64_t)blockIdx.x * QT;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    {
        // the tile's query codes; with PERM, tile position i holds query perm[q0 + i]
        const uint32_t *gw = reinterpret_cast<const uint32_t *>(codes);
        const int64_t nq = min((int64_t)QT, Q - q0);
        const int64_t words = nq * ld_words;
        if (PERM) {
            for (int64_t k = tid; k < words; k += kPredThreads) {
                const int64_t r = k / ld_words, w = k - r * ld_words;
                xw[k] = gw[(size_t)perm[q0 + r] * (size_t)ld_words + (size_t)w];
            }
        } else {
            const uint32_t *src = gw + (size_t)q0 * (size_t)ld_words;
            for (int64_t k = tid; k < words; k += kPredThreads) xw[k] = src[k];
        }
    }
    __syncthreads();
    if (tid == 0) {
        issue_tree4(c32, tree_off4, 0, tree_cap, slot0, &bar[0]);
        if (T > 1) issue_tree4(c32, tree_off4, 1, tree_cap, slot1, &bar[1]);
    }

    const uint8_t *xr[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i)
        xr[i] = reinterpret_cast<const uint8_t *>(xw + (size_t)(tid + i * kPredThreads) * (size_t)ld_words);
    int64_t acc[QPT], pend[QPT];
    u128_t sq[QPT];
#pragma unroll
    for (int i = 0; i < QPT; ++i) { acc[i] = 0; pend[i] = 0; sq[i] = 0; }

    // the tree's offsets are loaded one tree ahead, so their latency overlaps a walk
    int64_t a4 = tree_off4[0], b4 = T > 0 ? tree_off4[1] : 0, ta = tree_off[0];
    for (int t = 0; t < T; ++t) {
        const int s = t & 1;
        const uint32_t parity = (uint32_t)((t >> 1) & 1);
        const int tn1 = t + 1 < T ? t + 1 : t;
        const int64_t b4n = tree_off4[tn1 + 1], tan = tree_off[tn1];
        bool ok = false;
        for (uint32_t it = 0; it < kWaitLimit && !ok; ++it) ok = mbar_try_wait(&bar[s], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, kErrTimeout);
            if (t + 1 < T)
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(&bar[s ^ 1], (uint32_t)(((t + 1) >> 1) & 1))) break;
            return;
        }
        uint32_t j[QPT];
        const uint32_t nn4 = (uint32_t)(b4 - a4);
        if (b4 - a4 <= tree_cap) {
            if (s) walk_tree4<QPT>(slot1, xr, j, nn4);
            else walk_tree4<QPT>(slot0, xr, j, nn4);
        } else {
            walk_tree4<QPT>(c32 + a4, xr, j, nn4);
        }
        // add the previous tree's leaves, then start loading this tree's
        const uint64_t *tn = nodes + ta;
        a4 = b4;
        b4 = b4n;
        ta = tan;
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            acc[i] += pend[i];
            if (VAR) sq[i] += (u128_t)((i128_t)pend[i] * (i128_t)pend[i]);
            pend[i] = leaf_value(__ldg(&tn[j[i]]));
        }
        __syncthreads();
        if (tid == 0 && t + 2 < T) issue_tree4(c32, tree_off4, t + 2, tree_cap, s ? slot1 : slot0, &bar[s]);
    }
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        acc[i] += pend[i];
        if (VAR) sq[i] += (u128_t)((i128_t)pend[i] * (i128_t)pend[i]);
    }

#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int64_t qs = q0 + tid + i * kPredThreads;
        if (qs >= Q) continue;
        const int64_t q = PERM ? (int64_t)perm[qs] : qs;
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

// Split features of every tree's first kTopNodes nodes (breadth-first: the top levels).
constexpr int kTopNodes = 7;
__global__ void top_features_kernel(const uint64_t *__restrict__ cnodes, const int64_t *__restrict__ tree_off, int T,
                                    uint32_t *counts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int64_t a = tree_off[t], m = min((int64_t)kTopNodes, tree_off[t + 1] - a);
    for (int64_t j = 0; j < m; ++j) {
        const uint64_t nd = cnodes[a + j];
        if (!(nd >> 63)) atomicAdd(&counts[(nd >> 56) & 0x7Fu], 1u);
    }
}

// 32-bit sort key of a coded query: the one-byte codes of four features, most significant first
__global__ void query_key_kernel(const uint8_t *__restrict__ codes, int ld_bytes, int64_t Q, int4 kf,
                                 uint32_t *__restrict__ keys, uint32_t *__restrict__ idx)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const uint8_t *c = codes + (size_t)q * (size_t)ld_bytes;
    uint32_t k = 0;
    k |= kf.x >= 0 ? (uint32_t)c[kf.x] << 24 : 0u;
    k |= kf.y >= 0 ? (uint32_t)c[kf.y] << 16 : 0u;
    k |= kf.z >= 0 ? (uint32_t)c[kf.z] << 8 : 0u;
    k |= kf.w >= 0 ? (uint32_t)c[kf.w] : 0u;
    keys[q] = k;
    idx[q] = (uint32_t)q;
}

// ------------------------------------------------------------------------------------------
// out-of-bag evaluation (the tuning objective of Sec. III-B): per training row, the exact sum of
// the leaf values of the trees whose bootstrap did not draw it, and their number
// ------------------------------------------------------------------------------------------
template <typename CT>
__global__ void oob_kernel(const uint64_t *__restrict__ cnodes, const int64_t *__restrict__ tree_off, int T,
                           const CT *__restrict__ codes, int ld, int64_t N, const uint32_t *__restrict__ inbag,
                           int64_t words, int64_t *__restrict__ out_sum, int32_t *__restrict__ out_count)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const CT *x = codes + (size_t)row * (size_t)ld;
    int64_t sum = 0;
    int32_t cnt = 0;
    for (int t = 0; t < T; ++t) {
        if ((__ldg(&inbag[(size_t)t * (size_t)words + (size_t)(row >> 5)]) >> (row & 31)) & 1u) continue;
        const uint64_t *tn = cnodes + tree_off[t];
        const uint32_t nn = (uint32_t)(tree_off[t + 1] - tree_off[t]);
        uint32_t j = 0;
        for (;;) {
            const uint64_t nd = __ldg(&tn[j]);
            if (nd >> 63) { sum += leaf_value(nd); break; }
            const uint32_t f = AIWCRF_IDX((uint32_t)(nd >> 56) & 0x7Fu, (uint32_t)ld, kBoundFeature);
            j = AIWCRF_IDX(((uint32_t)(nd >> 32) & 0xFFFFFFu) + ((uint32_t)x[f] > ((uint32_t)nd & 0xFFFFFFu) ? 1u : 0u), nn,
                           kBoundWalk);
        }
        ++cnt;
    }
    out_sum[row] = sum;
    out_count[row] = cnt;
}

// Out-of-bag error (Sec. III-B): per row with c > 0 out-of-bag trees its out-of-bag prediction
// p = floor((2 s + c) / (2 c)) and the squared error (p - y)^2, exact in 128 bits; each CTA
// writes the sum of its rows' squared errors and their number, oob_error_finish_kernel adds the
// CTA sums in CTA order and divides once.
constexpr int kOobErrThreads = 256;

__global__ void __launch_bounds__(kOobErrThreads) oob_error_kernel(const int64_t *__restrict__ sum,
                                                                   const int32_t *__restrict__ cnt,
                                                                   const int64_t *__restrict__ y, int64_t N,
                                                                   int64_t *__restrict__ pred, OobPart *part,
                                                                   uint32_t *err)
{
    __shared__ OobPart red[kOobErrThreads / 32];
    const int64_t row = (int64_t)blockIdx.x * kOobErrThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long lo = 0ull, hi = 0ull, rows = 0ull;
    if (row < N) {
        const int32_t c = cnt[row];
        int64_t p = 0;
        if (c > 0) {
            const long long yr = y[row];
            if (yr > AIWCRF_MAX_ABS_Y || yr < -AIWCRF_MAX_ABS_Y) atomicOr(err, kErrY);
            p = round_mean(sum[row], (uint32_t)c);
            const i128_t d = (i128_t)p - (i128_t)yr;                 // |d| < 2^42
            const u128_t a = d < 0 ? (u128_t)(-d) : (u128_t)d;
            const u128_t sq = a * a;
            lo = (unsigned long long)sq;
            hi = (unsigned long long)(sq >> 64);
            rows = 1ull;
        }
        if (pred) pred[row] = p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long olo = __shfl_xor_sync(kFull, lo, o), ohi = __shfl_xor_sync(kFull, hi, o);
        const unsigned long long nlo = lo + olo;
        hi += ohi + (nlo < lo ? 1ull : 0ull);
        lo = nlo;
        rows += __shfl_xor_sync(kFull, rows, o);
    }
    if (lane == 0) { red[warp].lo = lo; red[warp].hi = hi; red[warp].rows = rows; }
    __syncthreads();
    if (threadIdx.x == 0) {
        OobPart t = red[0];
        for (int w = 1; w < kOobErrThreads / 32; ++w) {
            const unsigned long long nlo = t.lo + red[w].lo;
            t.hi += red[w].hi + (nlo < t.lo ? 1ull : 0ull);
            t.lo = nlo;
            t.rows += red[w].rows;
        }
        part[blockIdx.x] = t;
    }
}

__global__ void oob_error_finish_kernel(const OobPart *part, int nparts, OobResult *res)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long lo = 0ull, hi = 0ull, rows = 0ull;
    for (int i = 0; i < nparts; ++i) {
        const unsigned long long nlo = lo + part[i].lo;
        hi += part[i].hi + (nlo < lo ? 1ull : 0ull);
        lo = nlo;
        rows += part[i].rows;
    }
    res->sq_lo = lo;
    res->sq_hi = hi;
    res->rows = (long long)rows;
    // sum < 2^106: hi converts exactly, lo once rounded; mean in units of the target squared
    const double sq = __dadd_rn(__dmul_rn((double)hi, 18446744073709551616.0), (double)lo);
    res->mse = rows ? __dmul_rn(__ddiv_rn(sq, (double)rows), 5.42101086242752217e-20) : 0.0;   // 2^-64
}

int oob_error_launch(const int64_t *d_sum, const int32_t *d_count, const int64_t *d_y, int64_t N, int64_t *d_pred,
                     OobPart *d_parts, OobResult *d_res, uint32_t *d_err, cudaStream_t s)
{
    const int nparts = (int)std::max<int64_t>(1, (N + kOobErrThreads - 1) / kOobErrThreads);
    oob_error_kernel<<<(unsigned)nparts, kOobErrThreads, 0, s>>>(d_sum, d_count, d_y, N, d_pred, d_parts, d_err);
    oob_error_finish_kernel<<<1, 32, 0, s>>>(d_parts, nparts, d_res);
    count_launches(2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "oob_error launch");
    return AIWCRF_OK;
}

size_t oob_error_parts(int64_t N)
{
    return (size_t)std::max<int64_t>(1, (N + kOobErrThreads - 1) / kOobErrThreads);
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

// query (k, j) of device selection: kernel k's features (kfeat, leading dimension ld),
// device_ids[j], and size_class, or size_row[k] where size_row is given
__global__ void expand_queries_kernel(const float *kfeat, int32_t K, int64_t ld, int32_t size_class,
                                      const float *size_row, const int32_t *dev, int32_t D, int32_t F, float *q)
{
    const int64_t Qn = (int64_t)K * D;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Qn) return;
    const int32_t k = (int32_t)(i / D), jd = (int32_t)(i % D);
    for (int f = 0; f < F - 2; ++f) q[(size_t)f * (size_t)Qn + i] = kfeat[(size_t)f * (size_t)ld + k];
    q[(size_t)(F - 2) * (size_t)Qn + i] = (float)dev[jd];
    q[(size_t)(F - 1) * (size_t)Qn + i] =
        size_row ? size_row[k] : (float)size_class;
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

constexpr int kQPT = 2;
// compact-forest batches of at least this many queries are walked in sorted order
constexpr int64_t kSortMinQueries = 1 << 16;

// Shared memory of the 8-byte node walk (predict_kernel): kQPT code rows per thread, 256 bytes
// after them, and two tree slots sized to the forest's largest tree up to 48 KB each.
struct WalkSmem {
    int tree_cap;
    int bytes;
};

WalkSmem walk8_smem(const aiwcrf_forest *f, int row_words)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int xs_bytes = kPredThreads * kQPT * row_words * 4 + 256;
    int tree_cap = std::min<int>((optin - xs_bytes - 1024) / 16, 6144);
    if ((int64_t)tree_cap > f->max_tree_nodes) tree_cap = (int)f->max_tree_nodes;
    tree_cap &= ~1;
    if (tree_cap < 2) tree_cap = 2;
    return WalkSmem{tree_cap, 2 * tree_cap * 8 + xs_bytes};
}

template <typename CT, bool VAR>
int launch_predict(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                   uint64_t *d_var, int64_t total_trees, cudaStream_t s, uint32_t *d_err, void *codes_scratch,
                   int64_t walk_T)
{
    const int ld_words = code_row_words(f->F, (int)sizeof(CT));
    CT *d_codes = static_cast<CT *>(codes_scratch);
    cudaError_t e = cudaSuccess;
    if (!d_codes && cudaMallocAsync(&d_codes, (size_t)Q * (size_t)ld_words * 4, s) != cudaSuccess)
        return fail(AIWCRF_E_OOM, "device allocation of the query codes failed");
    struct Free { CT *p; cudaStream_t s; ~Free() { if (p) cudaFreeAsync(p, s); } } fr{codes_scratch ? nullptr : d_codes, s};
    if ((e = launch_code_queries<CT>(f, dXq, Q, d_codes, ld_words, s)) != cudaSuccess)
        return cuda_fail(e, "code_queries_kernel launch");
    const WalkSmem ws = walk8_smem(f, ld_words);
    const int tree_cap = ws.tree_cap, smem = ws.bytes;
    auto kern = predict_kernel<CT, kQPT, VAR>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(predict_kernel)");
    const int64_t grid = (Q + (int64_t)kPredThreads * kQPT - 1) / ((int64_t)kPredThreads * kQPT);
    prof_begin(s, kProfWalk);
    kern<<<(unsigned)grid, kPredThreads, smem, s>>>(f->d_cnodes, f->d_tree_off, (int)walk_T, d_codes, Q, ld_words,
                                                    total_trees, tree_cap, d_sum, d_pred, d_var, d_err);
    prof_end(s, kProfWalk);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "predict_kernel launch");
    return AIWCRF_OK;
}

template <bool VAR>
int launch_predict4(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                    uint64_t *d_var, int64_t total_trees, cudaStream_t s, uint32_t *d_err, void *codes_scratch,
                    int64_t walk_T)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int ld_words = code_row_words(f->F, 1);
    uint8_t *d_codes = static_cast<uint8_t *>(codes_scratch);
    cudaError_t e = cudaSuccess;
    if (!d_codes && cudaMallocAsync(&d_codes, (size_t)Q * (size_t)ld_words * 4, s) != cudaSuccess)
        return fail(AIWCRF_E_OOM, "device allocation of the query codes failed");
    struct Free { uint8_t *p; cudaStream_t s; ~Free() { if (p) cudaFreeAsync(p, s); } } fr{codes_scratch ? nullptr : d_codes, s};
    if ((e = launch_code_queries<uint8_t>(f, dXq, Q, d_codes, ld_words, s)) != cudaSuccess)
        return cuda_fail(e, "code_queries_kernel launch");
    // query code rows, then 256 bytes that a leaf's code read (feature field 255) may touch
    const int xs_bytes = kPredThreads * kQPT * ld_words * 4 + 256;
    // two tree slots of 4-byte nodes, sized to the largest tree up to 48 KB each
    int tree_cap = std::min<int>((optin - xs_bytes - 1024) / 8, 12288);
    if ((int64_t)tree_cap > f->max_tree4) tree_cap = (int)f->max_tree4;
    tree_cap &= ~3;
    if (tree_cap < 4) tree_cap = 4;
    const int smem = 2 * tree_cap * 4 + xs_bytes;
    // large batches walk in the order of their leading codes (own scratch only)
    const bool sorted = !codes_scratch && Q >= kSortMinQueries && Q < ((int64_t)1 << 32) && f->key_feats[0] >= 0;
    uint32_t *perm = nullptr;
    struct FreeSort { uint32_t *p; cudaStream_t s; ~FreeSort() { if (p) cudaFreeAsync(p, s); } } fs{nullptr, s};
    if (sorted) {
        const size_t nq = (size_t)Q + 1, hw = radix_sort_hist_words(Q, 1);
        uint32_t *buf = nullptr;
        if (cudaMallocAsync(&buf, sizeof(uint32_t) * (4 * nq + hw), s) != cudaSuccess)
            return fail(AIWCRF_E_OOM, "device allocation of the query order failed");
        fs.p = buf;
        uint32_t *kA = buf, *vA = buf + nq, *kB = buf + 2 * nq, *vB = buf + 3 * nq, *hist = buf + 4 * nq;
        const int4 kf = make_int4(f->key_feats[0], f->key_feats[1], f->key_feats[2], f->key_feats[3]);
        query_key_kernel<<<(unsigned)((Q + 255) / 256), 256, 0, s>>>(d_codes, ld_words * 4, Q, kf, kA, vA);
        count_launches(1);
        int rc = radix_sort_segments(kA, vA, kB, vB, Q, 1, Q, hist, s);
        if (rc != AIWCRF_OK) return rc;
        perm = vA;
    }
    auto kern = sorted ? predict4_kernel<kQPT, VAR, true> : predict4_kernel<kQPT, VAR, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(predict4_kernel)");
    const int64_t grid = (Q + (int64_t)kPredThreads * kQPT - 1) / ((int64_t)kPredThreads * kQPT);
    prof_begin(s, kProfWalk);
    kern<<<(unsigned)grid, kPredThreads, smem, s>>>(f->d_c32, f->d_tree_off4, f->d_nodes, f->d_tree_off, (int)walk_T,
                                                    d_codes, Q, ld_words, total_trees, tree_cap, d_sum, d_pred, d_var,
                                                    d_err, perm);
    prof_end(s, kProfWalk);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "predict4_kernel launch");
    return AIWCRF_OK;
}

template <typename CT>
int launch_predict_ct(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                      uint64_t *d_var, int64_t total_trees, cudaStream_t s, uint32_t *d_err, void *scratch = nullptr,
                      int64_t walk_T = -1)
{
    if (walk_T < 0) walk_T = f->T;
    if (f->compact)
        return d_var ? launch_predict4<true>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err, scratch, walk_T)
                     : launch_predict4<false>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err, scratch, walk_T);
    return d_var ? launch_predict<CT, true>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err, scratch, walk_T)
                 : launch_predict<CT, false>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err, scratch, walk_T);
}

}  // namespace

size_t predict_codes_bytes(const aiwcrf_forest *f, int64_t Q)
{
    return (size_t)Q * (size_t)code_row_words(f->F, code_bytes_of(f)) * 4;
}

size_t predict_codes_bytes_max(int32_t F, int64_t Q)
{
    return (size_t)Q * (size_t)code_row_words(F, 4) * 4;
}

int predict_enqueue(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                    cudaStream_t s, uint32_t *d_err, void *codes_scratch)
{
    if (Q == 0) return AIWCRF_OK;
    if (f->max_card <= 255u) return launch_predict_ct<uint8_t>(f, dXq, Q, d_sum, d_pred, nullptr, f->T, s, d_err, codes_scratch);
    if (f->max_card <= 65535u) return launch_predict_ct<uint16_t>(f, dXq, Q, d_sum, d_pred, nullptr, f->T, s, d_err, codes_scratch);
    return launch_predict_ct<uint32_t>(f, dXq, Q, d_sum, d_pred, nullptr, f->T, s, d_err, codes_scratch);
}

int predict_prefix_var_enqueue(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t n_trees,
                               uint64_t *d_var, cudaStream_t s, uint32_t *d_err, void *codes_scratch)
{
    if (Q == 0) return AIWCRF_OK;
    if (f->max_card <= 255u)
        return launch_predict_ct<uint8_t>(f, dXq, Q, nullptr, nullptr, d_var, n_trees, s, d_err, codes_scratch, n_trees);
    if (f->max_card <= 65535u)
        return launch_predict_ct<uint16_t>(f, dXq, Q, nullptr, nullptr, d_var, n_trees, s, d_err, codes_scratch, n_trees);
    return launch_predict_ct<uint32_t>(f, dXq, Q, nullptr, nullptr, d_var, n_trees, s, d_err, codes_scratch, n_trees);
}

int expand_launch(const float *d_kfeat, int32_t K, int64_t ld, int32_t size_class, const float *d_size_row,
                  const int32_t *d_dev, int32_t D, int32_t F, float *d_q, cudaStream_t s)
{
    const int64_t Qn = (int64_t)K * D;
    if (Qn == 0) return AIWCRF_OK;
    expand_queries_kernel<<<(unsigned)((Qn + 255) / 256), 256, 0, s>>>(d_kfeat, K, ld, size_class, d_size_row, d_dev,
                                                                        D, F, d_q);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "expand_queries_kernel launch");
    return AIWCRF_OK;
}

int predict_launch(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                   uint64_t *d_var, int64_t total_trees, cudaStream_t s)
{
    if (Q == 0) return AIWCRF_OK;
    keep_pool_memory(f->device);
    uint32_t *d_err = nullptr;
    cudaError_t e = cudaMallocAsync(&d_err, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "device allocation failed");
    cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    prof_begin(s, kProfPredict);
    int rc;
    if (f->max_card <= 255u) rc = launch_predict_ct<uint8_t>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err);
    else if (f->max_card <= 65535u) rc = launch_predict_ct<uint16_t>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err);
    else rc = launch_predict_ct<uint32_t>(f, dXq, Q, d_sum, d_pred, d_var, total_trees, s, d_err);
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

namespace {
template <typename CT>
int oob_ct(const aiwcrf_forest *f, const float *dX, int64_t N, int64_t *d_sum, int32_t *d_count, cudaStream_t s)
{
    const int ld_words = code_row_words(f->F, (int)sizeof(CT));
    const int ld = ld_words * 4 / (int)sizeof(CT);
    CT *d_codes = nullptr;
    cudaError_t e = cudaMallocAsync(&d_codes, (size_t)N * (size_t)ld_words * 4, s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "device allocation of the row codes failed");
    struct Free { CT *p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{d_codes, s};
    if ((e = launch_code_queries<CT>(f, dX, N, d_codes, ld_words, s)) != cudaSuccess)
        return cuda_fail(e, "code_queries_kernel launch");
    oob_kernel<CT><<<(unsigned)((N + 127) / 128), 128, 0, s>>>(f->d_cnodes, f->d_tree_off, (int)f->T, d_codes, ld, N,
                                                              f->d_inbag, f->inbag_words, d_sum, d_count);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "oob launch");
    return AIWCRF_OK;
}
}  // namespace

int oob_launch(const aiwcrf_forest *f, const float *dX, int64_t N, int64_t *d_sum, int32_t *d_count, cudaStream_t s)
{
    if (N == 0) return AIWCRF_OK;
    keep_pool_memory(f->device);
    if (f->max_card <= 255u) return oob_ct<uint8_t>(f, dX, N, d_sum, d_count, s);
    if (f->max_card <= 65535u) return oob_ct<uint16_t>(f, dX, N, d_sum, d_count, s);
    return oob_ct<uint32_t>(f, dX, N, d_sum, d_count, s);
}

int forest_build_compact(aiwcrf_forest *f, cudaStream_t s)
{
    if (!f->compact) return AIWCRF_OK;
    compact_nodes_kernel<<<(unsigned)f->T, 256, 0, s>>>(f->d_cnodes, f->d_tree_off, f->d_tree_off4, f->d_c32);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "compact_nodes_kernel launch");
    // the features the trees split on first, for the order of large query batches
    uint32_t *d_cnt = nullptr;
    if (cudaMallocAsync(&d_cnt, 4 * (size_t)f->F, s) != cudaSuccess) return fail(AIWCRF_E_OOM, "feature counts");
    e = cudaMemsetAsync(d_cnt, 0, 4 * (size_t)f->F, s);
    if (e == cudaSuccess) {
        top_features_kernel<<<(unsigned)((f->T + 127) / 128), 128, 0, s>>>(f->d_cnodes, f->d_tree_off, (int)f->T, d_cnt);
        count_launches(1);
        e = cudaGetLastError();
    }
    std::vector<uint32_t> h((size_t)f->F, 0u);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_cnt, 4 * (size_t)f->F, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_cnt, s);
    if (e != cudaSuccess) return cuda_fail(e, "top split features");
    std::vector<int> order((size_t)f->F);
    for (int i = 0; i < f->F; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return h[(size_t)x] > h[(size_t)y]; });
    for (int k = 0; k < 4; ++k)
        f->key_feats[k] = (k < f->F && h[(size_t)order[(size_t)k]] > 0) ? order[(size_t)k] : -1;
    return AIWCRF_OK;
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
    if (D <= 64 && Qn <= kTreeParallelMaxQueries && size_class >= 0) {
        // few queries: spread the trees over CTAs instead of the queries; the query scratch
        // (F * Qn floats) holds the kernel's zeroed sums and counters
        unsigned long long *d_sum = reinterpret_cast<unsigned long long *>(d_q);
        uint32_t *d_cnt = reinterpret_cast<uint32_t *>(d_sum + Qn);
        const cudaError_t e = cudaMemsetAsync(d_sum, 0, 8 * (size_t)Qn + 4 * (size_t)K, s);
        if (e != cudaSuccess) return cuda_fail(e, "select scratch");
        prof_begin(s, kProfSelect);
        const int rc = select_small_launch(f, d_kfeat, K, size_class, d_dev, D, d_best, d_pred ? d_pred : d_p, d_sum,
                                           d_cnt, s);
        prof_end(s, kProfSelect);
        return rc;
    }
    prof_begin(s, kProfSelect);
    expand_queries_kernel<<<(unsigned)((Qn + 255) / 256), 256, 0, s>>>(d_kfeat, K, (int64_t)K, size_class, nullptr, d_dev, D,
                                                                        f->F,
                                                                        d_q);
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

// ------------------------------------------------------------------------------------------
// Device selection inside caller-provided scratch (no allocation). Scratch layout, each part
// 256-byte aligned: device ids (D int32), expanded queries (F x K*D float), query codes
// (K*D rows of ld_words words), predictions (K*D int64), error flag (u32).
// ------------------------------------------------------------------------------------------
namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int code_ld_words(const aiwcrf_forest *f)
{
    return code_row_words(f->F, code_bytes_of(f));
}

template <typename CT>
int select_noalloc_ct(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class, int32_t D,
                      int32_t *d_best, int64_t *d_pred, const int32_t *d_dev, float *d_q, uint32_t *d_codes,
                      int64_t *d_p, uint32_t *d_err, cudaStream_t s)
{
    const int64_t Qn = (int64_t)K * D;
    const int ld_words = code_ld_words(f);
    expand_queries_kernel<<<(unsigned)((Qn + 255) / 256), 256, 0, s>>>(d_kfeat, K, (int64_t)K, size_class, nullptr, d_dev, D,
                                                                        f->F,
                                                                        d_q);
    count_launches(1);
    cudaError_t e = launch_code_queries<CT>(f, d_q, Qn, reinterpret_cast<CT *>(d_codes), ld_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "code_queries_kernel launch");
    const WalkSmem ws = walk8_smem(f, ld_words);
    const int tree_cap = ws.tree_cap, smem = ws.bytes;
    auto kern = predict_kernel<CT, kQPT, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(predict_kernel)");
    const int64_t grid = (Qn + (int64_t)kPredThreads * kQPT - 1) / ((int64_t)kPredThreads * kQPT);
    kern<<<(unsigned)grid, kPredThreads, smem, s>>>(f->d_cnodes, f->d_tree_off, (int)f->T,
                                                    reinterpret_cast<const CT *>(d_codes), Qn, ld_words, f->T,
                                                    tree_cap, nullptr, d_p, nullptr, d_err);
    argmin_kernel<<<(unsigned)((K + 127) / 128), 128, 0, s>>>(d_p, d_dev, K, D, d_best, d_pred);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "select_device launch");
    return AIWCRF_OK;
}

}  // namespace

size_t select_noalloc_bytes(const aiwcrf_forest *f, int32_t K, int32_t D)
{
    const size_t Qn = (size_t)K * (size_t)D;
    return align256(sizeof(int32_t) * (size_t)D) + align256(sizeof(float) * (size_t)f->F * Qn) +
           align256(Qn * (size_t)code_ld_words(f) * 4) + align256(sizeof(int64_t) * Qn) + align256(sizeof(uint32_t));
}

int select_launch_noalloc(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                          const int32_t *h_dev, int32_t D, int32_t *d_best, int64_t *d_pred, unsigned char *scratch,
                          cudaStream_t s)
{
    const size_t Qn = (size_t)K * (size_t)D;
    unsigned char *p = scratch;
    int32_t *d_dev = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * (size_t)D);
    float *d_q = reinterpret_cast<float *>(p);
    p += align256(sizeof(float) * (size_t)f->F * Qn);
    uint32_t *d_codes = reinterpret_cast<uint32_t *>(p);
    p += align256(Qn * (size_t)code_ld_words(f) * 4);
    int64_t *d_p = reinterpret_cast<int64_t *>(p);
    p += align256(sizeof(int64_t) * Qn);
    uint32_t *d_err = reinterpret_cast<uint32_t *>(p);
    // device_ids may be host or device memory (unified addressing: no staging buffer needed)
    cudaError_t e = cudaMemcpyAsync(d_dev, h_dev, sizeof(int32_t) * (size_t)D, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);    // the flag must start at 0
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);     // nothing this call enqueued may still use the shared array
        return cuda_fail(e, "select_device scratch set-up");
    }
    prof_begin(s, kProfSelect);
    int rc;
    if (f->max_card <= 255u)
        rc = select_noalloc_ct<uint8_t>(f, d_kfeat, K, size_class, D, d_best, d_pred, d_dev, d_q, d_codes, d_p, d_err, s);
    else if (f->max_card <= 65535u)
        rc = select_noalloc_ct<uint16_t>(f, d_kfeat, K, size_class, D, d_best, d_pred, d_dev, d_q, d_codes, d_p, d_err, s);
    else
        rc = select_noalloc_ct<uint32_t>(f, d_kfeat, K, size_class, D, d_best, d_pred, d_dev, d_q, d_codes, d_p, d_err, s);
    prof_end(s, kProfSelect);
    if (rc != AIWCRF_OK) {
        cudaStreamSynchronize(s);     // kernels enqueued before the failure finish with the array
        return rc;
    }
    uint32_t h_err = 0;
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "select_device");
    if (h_err & kErrTimeout) return fail(AIWCRF_E_TIMEOUT, "a bounded device wait gave up");
    return AIWCRF_OK;
}

}  // namespace aiwcrf

namespace aiwcrf {
AIWCRF_BOUNDS_READER(bounds_flags_predict)
}  // namespace aiwcrf
