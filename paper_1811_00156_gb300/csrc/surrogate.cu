// surrogate.cu -- a small MLP distilled from the forest's own predictions (not in the paper; the
// paper's model is the forest, Sec. III-B). Inputs: the AIWC columns standardised (log2 first
// for columns spanning orders of magnitude), one-hot device and size class, padded to 64;
// layers 64 -> 256 -> 256 -> 1 with GELU; BF16 weights and activations, FP32 accumulation.
//
// Training (Adam, MSE on the forest's log10-time predictions) runs as a stream of kernels per
// batch: encode, two tensor-core GEMMs forward, three backward (weight gradients with the batch
// as K, split over CTAs), fixed-order column sums for the biases, Adam, and BF16 weight copies.
// Inference is one persistent fused kernel: both weight matrices stay in shared memory; for
// every 128 queries the encoded tile is written straight into the MMA operand layout, layer 1
// accumulates into TMEM columns 0..255 and layer 2 into 256..511, and the epilogues apply bias
// and GELU (and the final dot product) from tcgen05.ld registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace aiwcrf {

using bf16 = __nv_bfloat16;

constexpr int kIn = 64;
constexpr int kHid = 256;
constexpr int oW1 = 0;
constexpr int ob1 = oW1 + kHid * kIn;
constexpr int oW2 = ob1 + kHid;
constexpr int ob2 = oW2 + kHid * kHid;
constexpr int ow3 = ob2 + kHid;
constexpr int ob3 = ow3 + kHid;
constexpr int kParams = ob3 + 1;

__device__ __forceinline__ float gelu(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

#ifndef AIWCRF_SUR_GELU_AS
#define AIWCRF_SUR_GELU_AS 1    // inference epilogues: erf by Abramowitz & Stegun 7.1.26
#endif
#ifndef AIWCRF_SUR_SMEM_BIAS
#define AIWCRF_SUR_SMEM_BIAS 1  // inference: b1 and b2 staged in shared memory
#endif

// erf(x) by the rational-exponential approximation of Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (absolute error at most 1.5e-7 for x >= 0, extended as
// an odd function): 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2), t = 1 / (1 + p x).
// Evaluated with the approximate reciprocal and exponential: the absolute error of the result
// stays below 1e-6 (the FP32 evaluation adds a few units of 2^-24 to the formula's 1.5e-7).
__device__ __forceinline__ float erf_as(float x)
{
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    const float poly =
        fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t, 0.254829592f) * t;
    return copysignf(fmaf(-poly, __expf(-ax * ax), 1.0f), x);
}

// GELU of the inference epilogues
__device__ __forceinline__ float gelu_infer(float x)
{
#if AIWCRF_SUR_GELU_AS
    return 0.5f * x * (1.0f + erf_as(x * 0.70710678118654752f));
#else
    return gelu(x);
#endif
}

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct Encoder {
    const float *mu, *sd;
    const uint8_t *logf;
    int n_aiwc, n_dev, n_size;
};

// input vector of one row: standardised AIWC columns, one-hot device, one-hot size, zeros
__device__ __forceinline__ float encode_value(const Encoder &e, const float *X, int64_t ld, int64_t row, int k)
{
    if (k < e.n_aiwc) {
        float x = X[(size_t)k * (size_t)ld + row];
        if (e.logf[k]) x = log2f(fmaxf(x, 1.0f));
        return (x - e.mu[k]) / e.sd[k];
    }
    if (k < e.n_aiwc + e.n_dev) {
        const float d = X[(size_t)e.n_aiwc * (size_t)ld + row];
        return (d == (float)(k - e.n_aiwc)) ? 1.0f : 0.0f;
    }
    if (k < e.n_aiwc + e.n_dev + e.n_size) {
        const float s = X[(size_t)(e.n_aiwc + 1) * (size_t)ld + row];
        return (s == (float)(k - e.n_aiwc - e.n_dev)) ? 1.0f : 0.0f;
    }
    return 0.0f;
}

// ------------------------------------------------------------------------------------------
// training kernels
// ------------------------------------------------------------------------------------------
// step: when set, the batch starts at row (*step mod spe) * B of the permutation instead of r0
// (a replayed training step reads its place in the epoch from the device step counter)
__global__ void encode_batch_kernel(Encoder e, const float *__restrict__ X, int64_t ld, const uint32_t *__restrict__ perm,
                                    int64_t r0, int B, const float *__restrict__ yall, bf16 *__restrict__ xin,
                                    float *__restrict__ yb, const int64_t *step, int64_t spe)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * kIn) return;
    if (step) r0 = (*step % spe) * (int64_t)B;
    const int b = i / kIn, k = i % kIn;
    const int64_t row = perm ? (int64_t)perm[r0 + b] : r0 + b;
    xin[i] = __float2bfloat16_rn(encode_value(e, X, ld, row, k));
    if (k == 0 && yb) yb[b] = yall[row];
}

// z1 += b1 (kept for the backward pass); h1 = BF16(GELU(z1))
__global__ void act1_kernel(float *__restrict__ z1, const float *__restrict__ b1, bf16 *__restrict__ h1, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = z1[i] + b1[i % kHid];
    z1[i] = z;
    h1[i] = __float2bfloat16_rn(gelu(z));
}

// one warp per row: z2 += b2, h2 = GELU(z2), out = h2 . w3 + b3, dout = (out - y) / B
__global__ void act2_out_kernel(float *__restrict__ z2, const float *__restrict__ b2, const float *__restrict__ w3,
                                const float *__restrict__ b3, float *__restrict__ h2, const float *__restrict__ y, int B,
                                float *__restrict__ out, float *__restrict__ dout, float *__restrict__ loss_rows)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= B) return;
    float dot = 0.0f;
    for (int j = lane; j < kHid; j += 32) {
        const float z = z2[(size_t)b * kHid + j] + b2[j];
        z2[(size_t)b * kHid + j] = z;
        const float h = gelu(z);
        h2[(size_t)b * kHid + j] = h;
        dot += h * w3[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(kFull, dot, o);
    if (lane == 0) {
        const float o = dot + b3[0];
        if (out) out[b] = o;
        if (y) {
            const float d = o - y[b];
            dout[b] = d / (float)B;
            loss_rows[b] = 0.5f * d * d;
        }
    }
}

// dz2 = dout * w3 * GELU'(z2)
__global__ void back2_kernel(const float *__restrict__ z2, const float *__restrict__ w3, const float *__restrict__ dout,
                             bf16 *__restrict__ dz2b, float *__restrict__ dz2f, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = i / kHid, j = i % kHid;
    const float d = dout[b] * w3[j] * gelu_grad(z2[i]);
    dz2f[i] = d;
    dz2b[i] = __float2bfloat16_rn(d);
}

// dz1 = dh1 * GELU'(z1)
__global__ void back1_kernel(const float *__restrict__ dh1, const float *__restrict__ z1, bf16 *__restrict__ dz1b,
                             float *__restrict__ dz1f, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d = dh1[i] * gelu_grad(z1[i]);
    dz1f[i] = d;
    dz1b[i] = __float2bfloat16_rn(d);
}

// dst[j] = sum_b v[b][j] (* w[b]) for the kHid columns of v (leading dimension kHid), in two
// fixed-order passes with coalesced reads: block (g, c) sums columns [32 g, 32 g + 32) over the
// c-th of kColChunks row ranges (eight row lanes, then the lanes in order) into part; then
// colsum_finish_kernel adds the kColChunks partial sums of each column in order.
constexpr int kColChunks = 16;

__global__ void __launch_bounds__(256) colsum_part_kernel(const float *__restrict__ v, int rows,
                                                          const float *__restrict__ w, float *__restrict__ part)
{
    __shared__ float red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int per = (rows + kColChunks - 1) / kColChunks;
    const int r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
    float s = 0.0f;
    for (int b = r0 + ty; b < r1; b += 8) s += v[(size_t)b * kHid + c] * (w ? w[b] : 1.0f);
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][tx];
        part[blockIdx.y * kHid + c] = t;
    }
}

__global__ void colsum_finish_kernel(const float *__restrict__ part, float *__restrict__ dst)
{
    const int j = threadIdx.x;
    float s = 0.0f;
    for (int y = 0; y < kColChunks; ++y) s += part[y * kHid + j];
    dst[j] = s;
}

// c12: when set, the bias corrections of step *step are c12[2 * step] and c12[2 * step + 1]
// (computed on the host for every step, as c1 and c2 are otherwise)
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float beta1, float beta2, float eps, float c1, float c2,
                            const float *__restrict__ c12, const int64_t *step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c12) { c1 = c12[2 * *step]; c2 = c12[2 * *step + 1]; }
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void step_advance_kernel(int64_t *step) { *step += 1; }

__global__ void to_bf16_kernel(const float *__restrict__ src, bf16 *__restrict__ dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void sum_kernel(const float *__restrict__ v, int n, float *__restrict__ dst)
{
    __shared__ float red[256];
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) dst[0] = red[0];
}

// ------------------------------------------------------------------------------------------
// fused inference
// ------------------------------------------------------------------------------------------
// two floats as BF16 (round to nearest even) in one word, the first in the low half
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

constexpr int kInferThreads = 512;
constexpr int kInferColGroups = kInferThreads / 128;          // warps sharing one TMEM lane quarter
constexpr int kInferCols = 256 / kInferColGroups;              // accumulator columns per warp
constexpr int kInferSmem = 32768 + 4 * 32768 + 4 * 16384;     // W1, W2 (4 K-chunks), H1 (4 K-chunks)

__global__ void __launch_bounds__(kInferThreads, 1) surrogate_infer_kernel(
    Encoder e, const float *__restrict__ Xq, int64_t Q, const bf16 *__restrict__ W1b, const bf16 *__restrict__ W2b,
    const float *__restrict__ b1, const float *__restrict__ b2, const float *__restrict__ w3, const float *__restrict__ b3,
    float *__restrict__ out, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sW1 = sm;                    // 256 x 64
    unsigned char *sW2 = sm + 32768;            // 4 chunks of 256 x 64
    unsigned char *sH = sm + 32768 + 4 * 32768; // 4 chunks of 128 x 64; chunk 0 holds the input tile first
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
#if AIWCRF_SUR_SMEM_BIAS
    __shared__ float b1s[kHid], b2s[kHid];
    // the output dot's partial sums sit in the last activation chunk: free once layer 2's MMAs
    // are done, and the next tile's encoding writes chunk 0 only
    float(*part)[128] = reinterpret_cast<float(*)[128]>(sH + 3 * 16384);
#define AIWCRF_B1(j) b1s[j]
#define AIWCRF_B2(j) b2s[j]
#else
    __shared__ float part[kInferColGroups][128];
#define AIWCRF_B1(j) __ldg(&b1[j])
#define AIWCRF_B2(j) __ldg(&b2[j])
#endif
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, half = warp >> 2;          // TMEM lane quarter, column group

    // weights, once per CTA, in the operand layout
    for (int p = tid; p < 256 * 8; p += kInferThreads) {
        const int r = p >> 3, kk = (p & 7) * 8;
        *reinterpret_cast<uint4 *>(sW1 + tc::core_offset(r, kk)) =
            __ldg(reinterpret_cast<const uint4 *>(W1b + (size_t)r * kIn + kk));
    }
    for (int p = tid; p < 4 * 256 * 8; p += kInferThreads) {
        const int kc = p / (256 * 8), rr = p % (256 * 8);
        const int r = rr >> 3, kk = (rr & 7) * 8;
        *reinterpret_cast<uint4 *>(sW2 + kc * 32768 + tc::core_offset(r, kk)) =
            __ldg(reinterpret_cast<const uint4 *>(W2b + (size_t)r * kHid + kc * 64 + kk));
    }
#if AIWCRF_SUR_SMEM_BIAS
    for (int j = tid; j < kHid; j += kInferThreads) { b1s[j] = __ldg(&b1[j]); b2s[j] = __ldg(&b2[j]); }
#endif
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = tc::make_idesc_bf16(128, 256);
    const int64_t ntiles = (Q + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;

    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t q0 = tile * 128;
        {   // encode the query tile: thread (row, part) encodes inputs [part * kIn / G, ...) of one row
            const int row = tid & 127, kpart = tid >> 7;
            const int64_t q = q0 + row;
            constexpr int kPer = kIn / kInferColGroups;
            for (int kk = kpart * kPer; kk < (kpart + 1) * kPer; kk += 8) {
                uint32_t w[4];
                for (int i = 0; i < 4; ++i) {
                    const float v0 = q < Q ? encode_value(e, Xq, Q, q, kk + 2 * i) : 0.0f;
                    const float v1 = q < Q ? encode_value(e, Xq, Q, q, kk + 2 * i + 1) : 0.0f;
                    w[i] = pack_bf16x2(v0, v1);
                }
                *reinterpret_cast<uint4 *>(sH + tc::core_offset(row, kk)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sH), w0 = tc::smem_addr(sW1);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                tc::mma_bf16(tbase, tc::make_desc(a0 + 256u * s, tc::kLbo, tc::kSbo),
                             tc::make_desc(w0 + 256u * s, tc::kLbo, tc::kSbo), idesc, s > 0 ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&bar, phase));
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after_sync();
        {   // epilogue 1: bias, GELU, BF16 into the layer-2 operand tile
            const int r = 32 * q4 + lane;
            for (int c = 0; c < kInferCols / 32; ++c) {
                const int col0 = kInferCols * half + 32 * c;
                float v[32];
                tc::tmem_ld32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)col0, v);
                for (int g8 = 0; g8 < 32; g8 += 8) {
                    uint32_t w[4];
                    for (int i = 0; i < 4; ++i) {
                        const int j0 = col0 + g8 + 2 * i;
                        const float h0 = gelu_infer(v[g8 + 2 * i] + AIWCRF_B1(j0));
                        const float h1 = gelu_infer(v[g8 + 2 * i + 1] + AIWCRF_B1(j0 + 1));
                        w[i] = pack_bf16x2(h0, h1);
                    }
                    const int k = col0 + g8;
                    *reinterpret_cast<uint4 *>(sH + (k >> 6) * 16384 + tc::core_offset(r, k & 63)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        tc::fence_before_sync();
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sH), w0 = tc::smem_addr(sW2);
            for (int kc = 0; kc < 4; ++kc)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    tc::mma_bf16(tbase + 256u, tc::make_desc(a0 + 16384u * kc + 256u * s, tc::kLbo, tc::kSbo),
                                 tc::make_desc(w0 + 32768u * kc + 256u * s, tc::kLbo, tc::kSbo), idesc,
                                 (kc > 0 || s > 0) ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&bar, phase));
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after_sync();
        {   // epilogue 2: bias, GELU, dot with w3
            const int r = 32 * q4 + lane;
            float dot = 0.0f;
            for (int c = 0; c < kInferCols / 32; ++c) {
                const int col0 = kInferCols * half + 32 * c;
                float v[32];
                tc::tmem_ld32(tbase + ((uint32_t)(32 * q4) << 16) + 256u + (uint32_t)col0, v);
                for (int i = 0; i < 32; ++i) dot += gelu_infer(v[i] + AIWCRF_B2(col0 + i)) * __ldg(&w3[col0 + i]);
            }
            part[half][r] = dot;
        }
        tc::fence_before_sync();
        __syncthreads();
        if (tid < 128 && q0 + tid < Q) {
            float o = __ldg(&b3[0]);
#pragma unroll
            for (int g = 0; g < kInferColGroups; ++g) o += part[g][tid];
            out[q0 + tid] = o;
        }
    }
    if (!ok && tid == 0) atomicOr(err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

}  // namespace aiwcrf

// ------------------------------------------------------------------------------------------
// the surrogate object and the C ABI
// ------------------------------------------------------------------------------------------
struct aiwcrf_surrogate {
    int device = 0;
    int32_t F = 0, n_aiwc = 0, n_dev = 0, n_size = 0;
    void *d_block = nullptr;
    float *d_param = nullptr, *d_mu = nullptr, *d_sd = nullptr;
    uint8_t *d_logf = nullptr;
    aiwcrf::bf16 *d_W1b = nullptr, *d_W2b = nullptr;
    std::vector<float> mu, sd;
    std::vector<uint8_t> logf;
    aiwcrf_surrogate_fit_stats stats = {};
};

namespace aiwcrf {
namespace {

// work reading the network may still be in flight on any stream: wait for it, then give the
// block back to the pool (stream-ordered, no device-wide wait inside the free)
void surrogate_release(aiwcrf_surrogate *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    if (s->d_block) cudaFreeAsync(s->d_block, cudaStreamPerThread);
    cudaStreamSynchronize(cudaStreamPerThread);
    delete s;
}

size_t surrogate_block_bytes(int32_t n_aiwc)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(4 * (size_t)kParams) + 2 * up(4 * (size_t)n_aiwc) + up((size_t)n_aiwc) + up(2 * (size_t)kHid * kIn) +
           up(2 * (size_t)kHid * kHid);
}

int surrogate_alloc(aiwcrf_surrogate *s)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bp = up(4 * (size_t)kParams), bf = up(4 * (size_t)s->n_aiwc), bl = up((size_t)s->n_aiwc);
    const size_t bw1 = up(2 * (size_t)kHid * kIn);
    // from the stream-ordered pool, whose frees never wait for the whole device (a
    // selection server may be busy on other streams)
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, surrogate_block_bytes(s->n_aiwc), cudaStreamPerThread);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "surrogate allocation");
    unsigned char *c = static_cast<unsigned char *>(p);
    s->d_block = p;
    s->d_param = reinterpret_cast<float *>(c);
    s->d_mu = reinterpret_cast<float *>(c + bp);
    s->d_sd = reinterpret_cast<float *>(c + bp + bf);
    s->d_logf = c + bp + 2 * bf;
    s->d_W1b = reinterpret_cast<bf16 *>(c + bp + 2 * bf + bl);
    s->d_W2b = reinterpret_cast<bf16 *>(c + bp + 2 * bf + bl + bw1);
    return AIWCRF_OK;
}

Encoder encoder_of(const aiwcrf_surrogate *s)
{
    Encoder e;
    e.mu = s->d_mu; e.sd = s->d_sd; e.logf = s->d_logf;
    e.n_aiwc = s->n_aiwc; e.n_dev = s->n_dev; e.n_size = s->n_size;
    return e;
}

int refresh_bf16(aiwcrf_surrogate *s, cudaStream_t st)
{
    to_bf16_kernel<<<(kHid * kIn + 255) / 256, 256, 0, st>>>(s->d_param + oW1, s->d_W1b, kHid * kIn);
    to_bf16_kernel<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(s->d_param + oW2, s->d_W2b, kHid * kHid);
    count_launches(2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AIWCRF_OK : cuda_fail(e, "bf16 weight copies");
}

// scratch of one training batch
struct Batch {
    int B = 0;
    bf16 *xin = nullptr, *h1 = nullptr, *dz2b = nullptr, *dz1b = nullptr;
    float *yb = nullptr, *z1 = nullptr, *z2 = nullptr, *h2 = nullptr, *out = nullptr, *dout = nullptr;
    float *loss_rows = nullptr, *dz2f = nullptr, *dh1 = nullptr, *dz1f = nullptr, *grad = nullptr, *part = nullptr;
    float *m = nullptr, *v = nullptr, *loss = nullptr;
    uint32_t *err = nullptr;
    void *block = nullptr;
    cudaStream_t s = nullptr;
    ~Batch() { if (block) cudaFreeAsync(block, s); }
    int alloc(int B_, cudaStream_t st)
    {
        B = B_;
        s = st;
        auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t BH = (size_t)B * kHid;
        const size_t sizes[] = {up(2 * (size_t)B * kIn), up(2 * BH), up(2 * BH), up(2 * BH),     // xin h1 dz2b dz1b
                                up(4 * (size_t)B), up(4 * BH), up(4 * BH), up(4 * BH), up(4 * (size_t)B),
                                up(4 * (size_t)B), up(4 * (size_t)B), up(4 * BH), up(4 * BH), up(4 * BH),
                                up(4 * (size_t)kParams), up(4 * (size_t)16 * kHid * kHid), up(4 * (size_t)kParams),
                                up(4 * (size_t)kParams), up(4), up(4)};
        size_t tot = 0;
        for (size_t b : sizes) tot += b;
        if (cudaMallocAsync(&block, tot, st) != cudaSuccess) return fail(AIWCRF_E_OOM, "surrogate batch scratch");
        unsigned char *c = static_cast<unsigned char *>(block);
        void **dst[] = {(void **)&xin, (void **)&h1, (void **)&dz2b, (void **)&dz1b, (void **)&yb, (void **)&z1,
                        (void **)&z2, (void **)&h2, (void **)&out, (void **)&dout, (void **)&loss_rows,
                        (void **)&dz2f, (void **)&dh1, (void **)&dz1f, (void **)&grad, (void **)&part, (void **)&m,
                        (void **)&v, (void **)&loss, (void **)&err};
        for (int i = 0; i < 20; ++i) { *dst[i] = c; c += sizes[i]; }
        cudaMemsetAsync(m, 0, 4 * (size_t)kParams, st);
        cudaMemsetAsync(v, 0, 4 * (size_t)kParams, st);
        cudaMemsetAsync(err, 0, 4, st);
        return AIWCRF_OK;
    }
};

#define SG_LAUNCH_CHECK(what)                                            \
    do {                                                                 \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);               \
    } while (0)

// forward + backward of one batch; gradients land in bt.grad (parameter layout)
int forward_backward(const aiwcrf_surrogate *sg, Batch &bt, const float *X, int64_t ld, const uint32_t *perm,
                     int64_t r0, const float *y, cudaStream_t s, const int64_t *step = nullptr, int64_t spe = 1)
{
    const int B = bt.B, BH = B * kHid, ks = 16;
    const Encoder e = encoder_of(sg);
    const float *P = sg->d_param;
    int rc;
    encode_batch_kernel<<<(B * kIn + 255) / 256, 256, 0, s>>>(e, X, ld, perm, r0, B, y, bt.xin, bt.yb, step, spe);
    if ((rc = tc_gemm(bt.xin, kIn, false, sg->d_W1b, kIn, false, bt.z1, B, kHid, kIn, 1, bt.part, bt.err, s))) return rc;
    act1_kernel<<<(BH + 255) / 256, 256, 0, s>>>(bt.z1, P + ob1, bt.h1, BH);
    if ((rc = tc_gemm(bt.h1, kHid, false, sg->d_W2b, kHid, false, bt.z2, B, kHid, kHid, 1, bt.part, bt.err, s))) return rc;
    act2_out_kernel<<<(B + 7) / 8, 256, 0, s>>>(bt.z2, P + ob2, P + ow3, P + ob3, bt.h2, bt.yb, B, bt.out, bt.dout,
                                                bt.loss_rows);
    back2_kernel<<<(BH + 255) / 256, 256, 0, s>>>(bt.z2, P + ow3, bt.dout, bt.dz2b, bt.dz2f, BH);
    colsum_part_kernel<<<dim3(kHid / 32, kColChunks), 256, 0, s>>>(bt.h2, B, bt.dout, bt.part);    // dw3
    colsum_finish_kernel<<<1, kHid, 0, s>>>(bt.part, bt.grad + ow3);
    sum_kernel<<<1, 256, 0, s>>>(bt.dout, B, bt.grad + ob3);                            // db3
    colsum_part_kernel<<<dim3(kHid / 32, kColChunks), 256, 0, s>>>(bt.dz2f, B, nullptr, bt.part);  // db2
    colsum_finish_kernel<<<1, kHid, 0, s>>>(bt.part, bt.grad + ob2);
    sum_kernel<<<1, 256, 0, s>>>(bt.loss_rows, B, bt.loss);
    count_launches(10);
    SG_LAUNCH_CHECK("surrogate forward");
    // dW2 = dz2^T h1 ; dh1 = dz2 W2 ; dz1 = dh1 GELU'(z1) ; dW1 = dz1^T xin
    if ((rc = tc_gemm(bt.dz2b, kHid, true, bt.h1, kHid, true, bt.grad + oW2, kHid, kHid, B, ks, bt.part, bt.err, s))) return rc;
    if ((rc = tc_gemm(bt.dz2b, kHid, false, sg->d_W2b, kHid, true, bt.dh1, B, kHid, kHid, 1, bt.part, bt.err, s))) return rc;
    back1_kernel<<<(BH + 255) / 256, 256, 0, s>>>(bt.dh1, bt.z1, bt.dz1b, bt.dz1f, BH);
    colsum_part_kernel<<<dim3(kHid / 32, kColChunks), 256, 0, s>>>(bt.dz1f, B, nullptr, bt.part);  // db1
    colsum_finish_kernel<<<1, kHid, 0, s>>>(bt.part, bt.grad + ob1);
    count_launches(3);
    if ((rc = tc_gemm(bt.dz1b, kHid, true, bt.xin, kIn, true, bt.grad + oW1, kHid, kIn, B, ks, bt.part, bt.err, s))) return rc;
    SG_LAUNCH_CHECK("surrogate backward");
    return AIWCRF_OK;
}

// A training step captured as a CUDA graph on its own stream (so that a caller's legacy default
// stream is never captured), instantiated once and replayed.
struct TrainGraph {
    cudaStream_t ts = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    size_t nodes = 0;
    ~TrainGraph()
    {
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        if (ts) cudaStreamDestroy(ts);
    }
    template <class F>
    int capture(F &&body)
    {
        cudaError_t e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate step capture");
        const int rc = body(ts);
        e = cudaStreamEndCapture(ts, &g);
        if (rc) return rc;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nodes);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate step graph");
        return AIWCRF_OK;
    }
    int replay()
    {
        const cudaError_t e = cudaGraphLaunch(x, ts);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate step replay");
        count_launches((int64_t)nodes);
        return AIWCRF_OK;
    }
};

int check_err(const Batch &bt, cudaStream_t s)
{
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, bt.err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate");
    if (h & kErrTimeout) return fail(AIWCRF_E_TIMEOUT, "a tensor-core wait gave up");
    return AIWCRF_OK;
}

// feature transform from a sample: log2 for columns that are >= 1 and span three orders of
// magnitude; mean and standard deviation of the (transformed) column
void fit_encoder(aiwcrf_surrogate *sg, const std::vector<float> &sample, int64_t n)
{
    sg->mu.assign((size_t)sg->n_aiwc, 0.0f);
    sg->sd.assign((size_t)sg->n_aiwc, 1.0f);
    sg->logf.assign((size_t)sg->n_aiwc, 0);
    for (int f = 0; f < sg->n_aiwc; ++f) {
        const float *c = sample.data() + (size_t)f * (size_t)n;
        float lo = c[0], hi = c[0];
        for (int64_t i = 0; i < n; ++i) { lo = std::min(lo, c[i]); hi = std::max(hi, c[i]); }
        const bool lg = lo >= 1.0f && hi >= 1000.0f * lo;
        double s1 = 0, s2 = 0;
        for (int64_t i = 0; i < n; ++i) {
            const double x = lg ? std::log2(std::max((double)c[i], 1.0)) : (double)c[i];
            s1 += x;
            s2 += x * x;
        }
        const double m = s1 / (double)n, var = std::max(s2 / (double)n - m * m, 1e-12);
        sg->logf[(size_t)f] = lg ? 1 : 0;
        sg->mu[(size_t)f] = (float)m;
        sg->sd[(size_t)f] = (float)std::sqrt(var);
    }
}

void init_params(std::vector<float> &P, uint64_t seed, int in_dim)
{
    std::mt19937_64 rng(seed);
    P.assign((size_t)kParams, 0.0f);
    std::uniform_real_distribution<float> u(-1.0f, 1.0f);
    const float a1 = std::sqrt(6.0f / (float)in_dim), a2 = std::sqrt(6.0f / (float)kHid);
    for (int r = 0; r < kHid; ++r)
        for (int k = 0; k < in_dim; ++k) P[(size_t)(oW1 + r * kIn + k)] = a1 * u(rng);
    for (int i = 0; i < kHid * kHid; ++i) P[(size_t)(oW2 + i)] = a2 * u(rng);
    for (int i = 0; i < kHid; ++i) P[(size_t)(ow3 + i)] = a2 * u(rng) * 0.5f;
}

int upload_encoder(aiwcrf_surrogate *sg)
{
    cudaError_t e = cudaMemcpy(sg->d_mu, sg->mu.data(), 4 * sg->mu.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sg->d_sd, sg->sd.data(), 4 * sg->sd.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sg->d_logf, sg->logf.data(), sg->logf.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? AIWCRF_OK : cuda_fail(e, "surrogate encoder upload");
}

int new_surrogate(int32_t F, int32_t n_dev, int32_t n_size, aiwcrf_surrogate **out)
{
    if (F < 3 || n_dev < 1 || n_size < 1 || (F - 2) + n_dev + n_size > kIn)
        return fail(AIWCRF_E_INVALID_ARG, "surrogate inputs: (F - 2) + n_devices + n_sizes must be <= 64");
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
    aiwcrf_surrogate *sg = new aiwcrf_surrogate();
    sg->device = dev;
    sg->F = F; sg->n_aiwc = F - 2; sg->n_dev = n_dev; sg->n_size = n_size;
    int rc = surrogate_alloc(sg);
    if (rc) { delete sg; return rc; }
    *out = sg;
    return AIWCRF_OK;
}

}  // namespace

int surrogate_clone(const aiwcrf_surrogate *src, aiwcrf_surrogate **out)
{
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != src->device) cudaSetDevice(src->device);
    aiwcrf_surrogate *sg = nullptr;
    int rc = new_surrogate(src->F, src->n_dev, src->n_size, &sg);
    if (!rc) {
        sg->mu = src->mu;
        sg->sd = src->sd;
        sg->logf = src->logf;
        sg->stats = src->stats;
        // the same sizes give the same block layout: one device-to-device copy
        cudaError_t e = cudaMemcpyAsync(sg->d_block, src->d_block, surrogate_block_bytes(src->n_aiwc),
                                        cudaMemcpyDeviceToDevice, cudaStreamPerThread);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "surrogate copy");
            surrogate_release(sg);
            sg = nullptr;
        }
    }
    if (cur != src->device) cudaSetDevice(cur);
    if (rc) return rc;
    *out = sg;
    return AIWCRF_OK;
}

SurrogateInfo surrogate_info(const aiwcrf_surrogate *sg)
{
    return SurrogateInfo{sg->device, sg->F, (int64_t)surrogate_block_bytes(sg->n_aiwc)};
}

void surrogate_release_async(aiwcrf_surrogate *sg, cudaStream_t s)
{
    if (!sg) return;
    if (sg->d_block) cudaFreeAsync(sg->d_block, s);
    delete sg;
}

int surrogate_predict_enqueue(const aiwcrf_surrogate *sg, const float *dXq, int64_t Q, float *d_out, uint32_t *d_err,
                              cudaStream_t s)
{
    if (Q == 0) return AIWCRF_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaFuncSetAttribute(surrogate_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate kernel attribute");
    const int64_t tiles = (Q + 127) / 128;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    surrogate_infer_kernel<<<grid, kInferThreads, kInferSmem, s>>>(encoder_of(sg), dXq, Q, sg->d_W1b, sg->d_W2b,
                                                                     sg->d_param + ob1, sg->d_param + ob2,
                                                                     sg->d_param + ow3, sg->d_param + ob3, d_out, d_err);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "surrogate_infer_kernel launch");
    return AIWCRF_OK;
}

int surrogate_predict_launch(const aiwcrf_surrogate *sg, const float *dXq, int64_t Q, float *d_out, cudaStream_t s)
{
    if (Q == 0) return AIWCRF_OK;
    uint32_t *d_err = nullptr;
    if (cudaMallocAsync(&d_err, 4, s) != cudaSuccess) return fail(AIWCRF_E_OOM, "surrogate error flag");
    cudaMemsetAsync(d_err, 0, 4, s);
    int rc = surrogate_predict_enqueue(sg, dXq, Q, d_out, d_err, s);
    if (rc) { cudaFreeAsync(d_err, s); return rc; }
    cudaError_t e = cudaSuccess;
    uint32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_err, s);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate predict");
    if (h & kErrTimeout) return fail(AIWCRF_E_TIMEOUT, "a tensor-core wait gave up");
    return AIWCRF_OK;
}

}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" {

int aiwcrf_surrogate_fit(const aiwcrf_surrogate_params *p, const aiwcrf_forest *teacher, const float *X, int64_t n,
                         int32_t n_features, void *cuda_stream, aiwcrf_surrogate **out)
{
    aiwcrf::clear_last_error();
    if (!p || !teacher || !X || !out) return fail(AIWCRF_E_INVALID_ARG, "params, teacher, X and out must not be NULL");
    if (n_features != teacher->F) return fail(AIWCRF_E_INVALID_ARG, "X must have the teacher's features");
    if (p->batch < 128 || p->batch % 128 || p->batch > 65536 || p->epochs < 1 || !(p->lr > 0.0f) || n < p->batch)
        return fail(AIWCRF_E_INVALID_ARG, "batch must be a multiple of 128 in [128, 65536], epochs >= 1, lr > 0, n >= batch");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, X) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(AIWCRF_E_BAD_POINTER, "X must be device memory");
    }
    keep_pool_memory(dev);
    aiwcrf_surrogate *sg = nullptr;
    int rc = new_surrogate(n_features, p->n_devices, p->n_sizes, &sg);
    if (rc) return rc;
    struct Guard { aiwcrf_surrogate *g; bool keep = false; ~Guard() { if (!keep && g) surrogate_release(g); } } guard{sg};

    // labels: the teacher forest's predictions (log10 seconds)
    float *d_y = nullptr;
    int64_t *d_pred = nullptr;
    if (cudaMallocAsync(&d_y, 4 * (size_t)n, s) != cudaSuccess || cudaMallocAsync(&d_pred, 8 * (size_t)n, s) != cudaSuccess)
        return fail(AIWCRF_E_OOM, "surrogate labels");
    struct FreeY { float *a; int64_t *b; cudaStream_t s; ~FreeY() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); } } fy{d_y, d_pred, s};
    if ((rc = predict_launch(teacher, X, n, nullptr, d_pred, nullptr, teacher->T, s))) return rc;
    {
        std::vector<int64_t> h((size_t)n);
        e = cudaMemcpyAsync(h.data(), d_pred, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate labels");
        std::vector<float> hy((size_t)n);
        for (int64_t i = 0; i < n; ++i) hy[(size_t)i] = (float)((double)h[(size_t)i] / 4294967296.0);
        e = cudaMemcpy(d_y, hy.data(), 4 * (size_t)n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate labels");
    }
    // encoder from a sample of the inputs
    {
        const int64_t m = std::min<int64_t>(n, 65536);
        std::vector<float> sample((size_t)sg->n_aiwc * (size_t)m);
        for (int f = 0; f < sg->n_aiwc; ++f) {
            e = cudaMemcpy(sample.data() + (size_t)f * (size_t)m, X + (size_t)f * (size_t)n, 4 * (size_t)m,
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "surrogate sample");
        }
        fit_encoder(sg, sample, m);
        if ((rc = upload_encoder(sg))) return rc;
    }
    std::vector<float> P;
    init_params(P, p->seed, sg->n_aiwc + sg->n_dev + sg->n_size);
    e = cudaMemcpy(sg->d_param, P.data(), 4 * (size_t)kParams, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate parameters");
    if ((rc = refresh_bf16(sg, s))) return rc;

    Batch bt;
    if ((rc = bt.alloc(p->batch, s))) return rc;
    const int64_t steps_per_epoch = n / p->batch;
    uint32_t *d_perm = nullptr;
    if (cudaMallocAsync(&d_perm, 4 * (size_t)n, s) != cudaSuccess) return fail(AIWCRF_E_OOM, "surrogate permutation");
    struct FreeP { uint32_t *a; cudaStream_t s; ~FreeP() { cudaFreeAsync(a, s); } } fp{d_perm, s};
    std::vector<uint32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (uint32_t)i;
    std::mt19937_64 rng(p->seed ^ 0x5DEECE66Dull);
    float first_loss = -1.0f, last_loss = -1.0f;
    const int64_t total_steps = (int64_t)p->epochs * steps_per_epoch;
    // Adam's bias corrections of every step, as the step-by-step loop computes them
    std::vector<float> c12((size_t)(2 * total_steps));
    for (int64_t t1 = 1; t1 <= total_steps; ++t1) {
        c12[(size_t)(2 * (t1 - 1))] = 1.0f - std::pow(p->beta1, (float)t1);
        c12[(size_t)(2 * (t1 - 1) + 1)] = 1.0f - std::pow(p->beta2, (float)t1);
    }
    // One training step (forward, backward, Adam, BF16 weight copies, step counter) is captured
    // once as a CUDA graph on a private stream and replayed: it reads its batch offset and bias
    // corrections through the device step counter, so the replays are the step-by-step loop's
    // launches without their host cost.
    TrainGraph tg;
    float *d_c12 = nullptr;
    int64_t *d_step = nullptr;
    if (cudaMallocAsync(&d_c12, 4 * c12.size(), s) != cudaSuccess || cudaMallocAsync(&d_step, 8, s) != cudaSuccess)
        return fail(AIWCRF_E_OOM, "surrogate step tables");
    struct FreeC { float *a; int64_t *b; cudaStream_t s; ~FreeC() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); } } fc{d_c12, d_step, s};
    e = cudaMemcpyAsync(d_c12, c12.data(), 4 * c12.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_step, 0, 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate step tables");
    if ((rc = tg.capture([&](cudaStream_t ts) {
             int r = forward_backward(sg, bt, X, n, d_perm, 0, d_y, ts, d_step, steps_per_epoch);
             if (r) return r;
             adam_kernel<<<(kParams + 255) / 256, 256, 0, ts>>>(sg->d_param, bt.grad, bt.m, bt.v, kParams, p->lr,
                                                                p->beta1, p->beta2, p->eps, 1.0f, 1.0f, d_c12, d_step);
             if ((r = refresh_bf16(sg, ts))) return r;
             step_advance_kernel<<<1, 1, 0, ts>>>(d_step);
             const cudaError_t e2 = cudaGetLastError();
             return e2 == cudaSuccess ? AIWCRF_OK : cuda_fail(e2, "surrogate step launches");
         })))
        return rc;
    int64_t t = 0;
    for (int ep = 0; ep < p->epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(d_perm, perm.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, tg.ts);
        if (e == cudaSuccess) e = cudaStreamSynchronize(tg.ts);      // the host array is reshuffled next epoch
        if (e != cudaSuccess) return cuda_fail(e, "surrogate permutation");
        for (int64_t k = 0; k < steps_per_epoch; ++k) {
            if ((rc = tg.replay())) return rc;
            ++t;
            if (k == 0 || k == steps_per_epoch - 1) {
                float hl = 0.0f;
                e = cudaMemcpyAsync(&hl, bt.loss, 4, cudaMemcpyDeviceToHost, tg.ts);
                if (e == cudaSuccess) e = cudaStreamSynchronize(tg.ts);
                if (e != cudaSuccess) return cuda_fail(e, "surrogate loss");
                if (first_loss < 0.0f) first_loss = hl / (float)p->batch;
                last_loss = hl / (float)p->batch;
            }
        }
    }
    e = cudaStreamSynchronize(tg.ts);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate training");
    if ((rc = check_err(bt, s))) return rc;
    sg->stats.steps = t;
    sg->stats.first_batch_loss = first_loss;
    sg->stats.last_batch_loss = last_loss;
    guard.keep = true;
    *out = sg;
    return AIWCRF_OK;
}

int aiwcrf_surrogate_predict(const aiwcrf_surrogate *sg, const float *Xq, int64_t n, float *out, void *cuda_stream)
{
    aiwcrf::clear_last_error();
    if (!sg || !Xq || !out) return fail(AIWCRF_E_INVALID_ARG, "surrogate, Xq and out must not be NULL");
    if (n < 0) return fail(AIWCRF_E_INVALID_ARG, "n must be >= 0");
    cudaPointerAttributes a1, a2;
    if (cudaPointerGetAttributes(&a1, Xq) != cudaSuccess || cudaPointerGetAttributes(&a2, out) != cudaSuccess ||
        a1.type != cudaMemoryTypeDevice || a2.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(AIWCRF_E_BAD_POINTER, "Xq and out must be device memory");
    }
    return surrogate_predict_launch(sg, Xq, n, out, (cudaStream_t)cuda_stream);
}

int aiwcrf_surrogate_grad(const aiwcrf_surrogate *sg, const float *X, const float *y, int32_t n, float *grad,
                          float *loss, void *cuda_stream)
{
    aiwcrf::clear_last_error();
    if (!sg || !X || !y || !grad || !loss || n < 128 || n % 128)
        return fail(AIWCRF_E_INVALID_ARG, "arguments must not be NULL; n a positive multiple of 128");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Batch bt;
    int rc;
    if ((rc = bt.alloc(n, s))) return rc;
    if ((rc = forward_backward(sg, bt, X, n, nullptr, 0, y, s))) return rc;
    cudaError_t e = cudaMemcpyAsync(grad, bt.grad, 4 * (size_t)kParams, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, bt.loss, 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate gradients");
    return check_err(bt, s);
}

int aiwcrf_surrogate_create(int32_t n_features, int32_t n_devices, int32_t n_sizes, const float *params,
                            const float *mu, const float *sd, const uint8_t *log2_cols, aiwcrf_surrogate **out)
{
    aiwcrf::clear_last_error();
    if (!params || !mu || !sd || !log2_cols || !out) return fail(AIWCRF_E_INVALID_ARG, "arguments must not be NULL");
    aiwcrf_surrogate *sg = nullptr;
    int rc = new_surrogate(n_features, n_devices, n_sizes, &sg);
    if (rc) return rc;
    sg->mu.assign(mu, mu + sg->n_aiwc);
    sg->sd.assign(sd, sd + sg->n_aiwc);
    sg->logf.assign(log2_cols, log2_cols + sg->n_aiwc);
    if (!(rc = upload_encoder(sg))) {
        cudaError_t e = cudaMemcpy(sg->d_param, params, 4 * (size_t)kParams, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "surrogate parameters");
    }
    if (!rc) rc = refresh_bf16(sg, nullptr);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "surrogate create");
    if (rc) { surrogate_release(sg); return rc; }
    *out = sg;
    return AIWCRF_OK;
}

int aiwcrf_surrogate_export(const aiwcrf_surrogate *sg, float *params, float *mu, float *sd, uint8_t *log2_cols)
{
    aiwcrf::clear_last_error();
    if (!sg) return fail(AIWCRF_E_INVALID_ARG, "surrogate is NULL");
    if (params && cudaMemcpy(params, sg->d_param, 4 * (size_t)kParams, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "surrogate export");
    if (mu) std::memcpy(mu, sg->mu.data(), 4 * sg->mu.size());
    if (sd) std::memcpy(sd, sg->sd.data(), 4 * sg->sd.size());
    if (log2_cols) std::memcpy(log2_cols, sg->logf.data(), sg->logf.size());
    return AIWCRF_OK;
}

int aiwcrf_surrogate_stats(const aiwcrf_surrogate *sg, aiwcrf_surrogate_fit_stats *out)
{
    aiwcrf::clear_last_error();
    if (!sg || !out) return fail(AIWCRF_E_INVALID_ARG, "arguments must not be NULL");
    *out = sg->stats;
    return AIWCRF_OK;
}

int32_t aiwcrf_surrogate_num_params(void) { return kParams; }

int aiwcrf_surrogate_free(aiwcrf_surrogate *sg)
{
    aiwcrf::clear_last_error();
    if (!sg) return AIWCRF_OK;
    surrogate_release(sg);
    return AIWCRF_OK;
}

}  // extern "C"
