// mlp.cu -- tensor-core (tcgen05) BF16 GEMM with FP32 accumulation in TMEM, the building block
// of the learned surrogate's training and inference kernels.
//
// tc_gemm_kernel: C = A * B^T with A (M x K) and B (N x K) in BF16; one CTA owns 128 rows of C
// and a range of K. Every 64-wide K chunk of A and B is staged into shared memory in the
// K-major core-matrix layout (transposing on the way when an operand is stored K x M), one
// thread issues four 128 x N x 16 MMAs into the TMEM accumulator and commits them to an
// mbarrier; four warps then read the accumulator rows with tcgen05.ld. K ranges of several
// CTAs (split K) are summed afterwards in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.cuh"
#include "tc.cuh"

namespace aiwcrf {

using bf16 = __nv_bfloat16;

constexpr int kGemmThreads = 128;

// Stage rows [r0, r0 + rows) x K-elements [k0, k0 + 64) of an operand into a core-matrix tile.
// Element (r, k) of the operand is G[r * ld + k] (stored row by row) or G[k * ld + r] (stored
// K x rows, TRANS). Outside [0, rmax) x [0, K) the tile holds zeros. ld is a multiple of 8 and
// G 16-byte aligned.
template <bool TRANS>
__device__ __forceinline__ void stage_tile(unsigned char *tile, const bf16 *__restrict__ G, int ld, int r0, int rows,
                                           int rmax, int k0, int K)
{
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    if (!TRANS) {
        for (int p = threadIdx.x; p < rows * 8; p += blockDim.x) {
            const int r = p >> 3, kk = (p & 7) * 8;
            const int gr = r0 + r, gk = k0 + kk;
            uint4 v = zero;
            if (gr < rmax) {
                if (gk + 8 <= K) {
                    v = __ldg(reinterpret_cast<const uint4 *>(G + (size_t)gr * (size_t)ld + gk));
                } else if (gk < K) {
                    uint16_t h[8];
                    for (int i = 0; i < 8; ++i)
                        h[i] = gk + i < K ? __bfloat16_as_ushort(G[(size_t)gr * (size_t)ld + gk + i]) : (uint16_t)0;
                    v = make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                                   h[6] | (uint32_t)h[7] << 16);
                }
            }
            *reinterpret_cast<uint4 *>(tile + tc::core_offset((uint32_t)r, (uint32_t)kk)) = v;
        }
    } else {
        const int rgroups = rows >> 3;
        for (int p = threadIdx.x; p < rgroups * 64; p += blockDim.x) {
            const int k = p / rgroups, rg = p % rgroups;
            const int gk = k0 + k, gr = r0 + rg * 8;
            uint16_t h[8];
            if (gk < K && gr + 8 <= rmax) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(G + (size_t)gk * (size_t)ld + gr));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                for (int i = 0; i < 4; ++i) { h[2 * i] = (uint16_t)w[i]; h[2 * i + 1] = (uint16_t)(w[i] >> 16); }
            } else {
                for (int i = 0; i < 8; ++i)
                    h[i] = (gk < K && gr + i < rmax) ? __bfloat16_as_ushort(G[(size_t)gk * (size_t)ld + gr + i])
                                                     : (uint16_t)0;
            }
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<uint16_t *>(tile + tc::core_offset((uint32_t)(rg * 8 + i), (uint32_t)k)) = h[i];
        }
    }
}

__host__ __device__ constexpr uint32_t tmem_cols_for(int N)
{
    return N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
}

// part[kz][m][n] = sum over CTA column kz's K chunks of A(m, k) B(n, k), for the columns
// [n0, n0 + NT) of CTA layer blockIdx.z (n0 = blockIdx.z * NT); N and NT multiples of 16, <= 256
template <bool AT, bool BT>
__global__ void __launch_bounds__(kGemmThreads) tc_gemm_kernel(const bf16 *__restrict__ A, int lda,
                                                               const bf16 *__restrict__ B, int ldb, float *part, int M,
                                                               int N, int K, int chunks_per_cta, int NT, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm;                    // 128 x 64 BF16 = 16 KB
    unsigned char *sB = sm + 16384;            // NT x 64 BF16 <= 32 KB
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, kz = blockIdx.y, n0 = blockIdx.z * NT;
    const int nchunks = (K + 63) / 64;
    const int kc0 = kz * chunks_per_cta, kc1 = min(kc0 + chunks_per_cta, nchunks);
    const uint32_t ncols = tmem_cols_for(NT);

    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = tc::make_idesc_bf16(128, (uint32_t)NT);

    bool ok = true;
    uint32_t phase = 0;
    for (int kc = kc0; kc < kc1; ++kc) {
        stage_tile<AT>(sA, A, lda, m0, 128, M, kc * 64, K);
        stage_tile<BT>(sB, B, ldb, n0, NT, N, kc * 64, K);
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                tc::mma_bf16(tbase, tc::make_desc(a0 + 256u * s, tc::kLbo, tc::kSbo),
                             tc::make_desc(b0 + 256u * s, tc::kLbo, tc::kSbo), idesc, (kc > kc0 || s > 0) ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        const bool done = tc::mbar_wait(&bar, phase);          // the tiles may be overwritten after this
        phase ^= 1u;
        if (!__syncthreads_and(done)) { ok = false; break; }
        tc::fence_after_sync();
    }

    if (ok) {
        const int m = m0 + 32 * warp + lane;
        float *dst = part + ((size_t)kz * (size_t)M + (size_t)m) * (size_t)N + n0;
        for (int c = 0; c < NT; c += 32) {
            float v[32];
            if (kc1 > kc0) tc::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            else
                for (int i = 0; i < 32; ++i) v[i] = 0.0f;
            if (m < M)
                for (int i = 0; i < 32 && c + i < NT; i += 4)
                    *reinterpret_cast<float4 *>(dst + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    } else if (tid == 0) {
        atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, ncols);
    }
}

// C[m][n] = sum_kz part[kz][m][n], in kz order
__global__ void sum_parts_kernel(const float *__restrict__ part, int splits, int64_t MN, float *__restrict__ C)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * (size_t)MN + i];
    C[i] = s;
}

// host: C (M x N, FP32) = A * B^T; part needs splits * M * N floats (splits from ksplit)
int tc_gemm(const bf16 *A, int lda, bool a_trans, const bf16 *B, int ldb, bool b_trans, float *C, int M, int N, int K,
            int ksplit, float *part, uint32_t *d_err, cudaStream_t s)
{
    if (M < 1 || K < 1 || N < 16 || N > 256 || (N % 16) || (lda % 8) || (ldb % 8))
        return fail(AIWCRF_E_INVALID_ARG, "tc_gemm: N must be a multiple of 16 in [16, 256], lda and ldb multiples of 8");
    const int nchunks = (K + 63) / 64;
    const int splits = std::max(1, std::min(ksplit, nchunks));
    const int per = (nchunks + splits - 1) / splits;
    // columns per CTA: halved (in multiples of 16) until the grid has at least 128 CTAs
    const int mtiles = (M + 127) / 128;
    int NT = N;
    while ((int64_t)mtiles * splits * (N / NT) < 128 && NT % 32 == 0 && N % (NT / 2) == 0) NT /= 2;
    const int smem = 16384 + NT * 128;
    // enough shared memory per CTA that no more CTAs fit an SM than its 512 TMEM columns hold
    const int per_sm = 512 / (int)tmem_cols_for(NT);
    const int smem_launch = std::max(smem, 233472 / (per_sm + 1));
    const dim3 grid((unsigned)mtiles, (unsigned)splits, (unsigned)(N / NT));
    cudaError_t e;
#define AIWCRF_TC_LAUNCH(AT, BT)                                                                                   \
    e = cudaFuncSetAttribute(tc_gemm_kernel<AT, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_launch);    \
    if (e == cudaSuccess) {                                                                                        \
        tc_gemm_kernel<AT, BT><<<grid, kGemmThreads, smem_launch, s>>>(A, lda, B, ldb, splits > 1 ? part : C, M,  \
                                                                      N, K, per, NT, d_err);                       \
    }
    if (!a_trans && !b_trans) { AIWCRF_TC_LAUNCH(false, false) }
    else if (!a_trans && b_trans) { AIWCRF_TC_LAUNCH(false, true) }
    else if (a_trans && !b_trans) { AIWCRF_TC_LAUNCH(true, false) }
    else { AIWCRF_TC_LAUNCH(true, true) }
#undef AIWCRF_TC_LAUNCH
    count_launches(1);
    if (e != cudaSuccess) return cuda_fail(e, "tc_gemm attribute");
    if (splits > 1) {
        const int64_t MN = (int64_t)M * N;
        sum_parts_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, s>>>(part, splits, MN, C);
        count_launches(1);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tc_gemm launch");
    return AIWCRF_OK;
}

}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" int aiwcrf_tc_gemm_bf16(const void *A, int32_t lda, int32_t a_trans, const void *B, int32_t ldb,
                                   int32_t b_trans, float *C, int32_t M, int32_t N, int32_t K, int32_t ksplit,
                                   void *cuda_stream)
{
    aiwcrf::clear_last_error();
    if (!A || !B || !C) return fail(AIWCRF_E_INVALID_ARG, "A, B and C must not be NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nchunks = (K + 63) / 64;
    const int splits = std::max(1, std::min((int)ksplit, nchunks));
    float *part = nullptr;
    uint32_t *d_err = nullptr;
    cudaError_t e = cudaMallocAsync(&d_err, sizeof(uint32_t), s);
    if (e == cudaSuccess && splits > 1) e = cudaMallocAsync(&part, sizeof(float) * (size_t)splits * M * N, s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "tc_gemm scratch");
    cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    int rc = tc_gemm((const bf16 *)A, lda, a_trans != 0, (const bf16 *)B, ldb, b_trans != 0, C, M, N, K, ksplit, part,
                     d_err, s);
    uint32_t h_err = 0;
    if (rc == AIWCRF_OK) {
        e = cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tc_gemm");
    }
    if (part) cudaFreeAsync(part, s);
    cudaFreeAsync(d_err, s);
    if (rc == AIWCRF_OK && (h_err & kErrTimeout)) rc = fail(AIWCRF_E_TIMEOUT, "tc_gemm: an MMA wait gave up");
    return rc;
}
