// sort.cu -- stable LSD radix sort of (key, value) u32 pairs in S independent segments, on many
// CTAs: per 8-bit pass, (1) every 4,096-element tile counts its digits, (2) one CTA per segment
// scans the (digit, tile) counts, (3) every tile scatters its elements in a stable order (warp
// match on the digit, then per-digit prefix over the tile's warps).
#include <cuda_runtime.h>

#include <string>

#include "internal.cuh"

namespace aiwcrf {

constexpr int kSortThreads = 256;
constexpr int kSortSub = 16;
constexpr int kSortTile = kSortThreads * kSortSub;

__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                                 int64_t stride, int shift, int nb,
                                                                 uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    const int b = blockIdx.x, seg = blockIdx.y, tid = threadIdx.x;
    h[tid] = 0u;
    __syncthreads();
    const uint32_t *k = keys + (size_t)seg * (size_t)stride;
    const int64_t end = min(n, (int64_t)(b + 1) * kSortTile);
    for (int64_t i = (int64_t)b * kSortTile + tid; i < end; i += kSortThreads) atomicAdd(&h[(k[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[((size_t)seg * 256 + tid) * (size_t)nb + b] = h[tid];
}

// exclusive scan of one segment's 256 * nb counts, digit-major: every thread sums a contiguous
// run of 16-byte words (independent loads), one block scan of the run sums, then every thread
// rewrites its run from its own prefix. (A segment starts 1,024 * nb bytes after the 16-byte
// aligned base, and 256 * nb counts are whole words.)
__global__ void __launch_bounds__(1024) sort_scan_kernel(uint32_t *hist, int nb)
{
    __shared__ uint32_t warp_tmp[32];
    uint4 *h4 = reinterpret_cast<uint4 *>(hist + (size_t)blockIdx.x * 256 * (size_t)nb);
    const int64_t total4 = 64 * (int64_t)nb;
    const int64_t per = (total4 + 1023) / 1024;
    const int64_t lo = min(total4, (int64_t)threadIdx.x * per), hi = min(total4, lo + per);
    uint32_t sum = 0;
#pragma unroll 4
    for (int64_t i = lo; i < hi; ++i) {
        const uint4 v = h4[i];
        sum += v.x + v.y + v.z + v.w;
    }
    uint32_t tot;
    uint32_t run = block_incl_scan(sum, warp_tmp, tot) - sum;
#pragma unroll 4
    for (int64_t i = lo; i < hi; ++i) {
        const uint4 v = h4[i];
        uint4 o;
        o.x = run; run += v.x;
        o.y = run; run += v.y;
        o.z = run; run += v.z;
        o.w = run; run += v.w;
        h4[i] = o;
    }
}

__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const uint32_t *__restrict__ kin,
                                                                    const uint32_t *__restrict__ vin,
                                                                    uint32_t *__restrict__ kout,
                                                                    uint32_t *__restrict__ vout, int64_t n,
                                                                    int64_t stride, int shift, int nb,
                                                                    const uint32_t *__restrict__ hist)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t tile_tot[256];
    const int b = blockIdx.x, seg = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t off = (size_t)seg * (size_t)stride;
    base[tid] = hist[((size_t)seg * 256 + tid) * (size_t)nb + b];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0u;
    __syncthreads();
    for (int sub = 0; sub < kSortSub; ++sub) {
        const int64_t i = (int64_t)b * kSortTile + (int64_t)sub * kSortThreads + tid;
        if ((int64_t)b * kSortTile + (int64_t)sub * kSortThreads >= n) break;    // block-uniform
        const bool valid = i < n;
        const uint32_t k = valid ? kin[off + i] : 0u;
        const uint32_t v = valid ? vin[off + i] : 0u;
        const uint32_t d = (k >> shift) & 255u;
        const uint32_t peers = __match_any_sync(kFull, valid ? d : (256u + lane));
        const uint32_t rk = __popc(peers & lanemask_lt());
        if (valid && rk == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            tile_tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = base[d] + wcnt[warp][d] + rk;
            kout[off + pos] = k;
            vout[off + pos] = v;
        }
        __syncthreads();
        base[tid] += tile_tot[tid];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0u;
        __syncthreads();
    }
}

size_t radix_sort_hist_words(int64_t n, int S)
{
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)S * 256 * (size_t)(nb > 0 ? nb : 1) + 1;
}

int radix_sort_segments(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, int64_t n,
                        int S, int64_t stride, uint32_t *hist, cudaStream_t s)
{
    if (n <= 0 || S <= 0) return AIWCRF_OK;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    const dim3 grid((unsigned)nb, (unsigned)S);
    uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        sort_hist_kernel<<<grid, kSortThreads, 0, s>>>(ki, n, stride, shift, nb, hist);
        sort_scan_kernel<<<(unsigned)S, 1024, 0, s>>>(hist, nb);
        sort_scatter_kernel<<<grid, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, stride, shift, nb, hist);
        count_launches(3);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "radix sort launch");
        uint32_t *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    return AIWCRF_OK;   // four passes: the result is back in (keys_a, vals_a)
}

}  // namespace aiwcrf
