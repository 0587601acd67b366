// internal.cuh -- types and device helpers shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/aiwcrf.h"

namespace aiwcrf {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kSmallNodeRows = 32;          // nodes with <= 32 distinct rows are searched by a warp
constexpr uint32_t kRankSentinel = 1u << 22;  // larger than any rank (ranks are < rows < 2^22)
constexpr uint32_t kRowBits = 24;           // row entry = row | (w << 24)
constexpr uint32_t kRowMask = (1u << kRowBits) - 1;
constexpr uint32_t kDomBoot = 0xB007u;      // Philox counter domain of bootstrap draws
constexpr uint32_t kDomMtry = 0x3779u;      // Philox counter domain of mtry keys

// device error flag bits (aggregated with atomicOr)
constexpr uint32_t kErrNaN = 1u;
constexpr uint32_t kErrCard = 2u;           // (unused: every column's ranks fit 32 bits)
constexpr uint32_t kErrBootOverflow = 4u;   // a bootstrap multiplicity above 255
constexpr uint32_t kErrTimeout = 8u;        // a bounded mbarrier wait gave up
constexpr uint32_t kErrY = 16u;             // |y| > 2^40
constexpr uint32_t kErrCapacity = 32u;      // a fit plan's capacity (groups, ranks, levels) was exceeded
constexpr uint32_t kErrTree = 32u;          // malformed tree met during a walk

// ------------------------------------------------------------------------------------------
// Debug builds (-DAIWCRF_DEBUG_BOUNDS) check every gathered index and node id of the hot paths
// against its array's extent. A violation sets the site's bit in the translation unit's device
// flag and the access goes to index 0 instead (every checked array is non-empty), so a bug shows
// as a flag, read by aiwcrf_debug_bounds(), rather than as an out-of-bounds access. Release
// builds compile the checks away.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kBoundRow = 1u;       // entry row or group id gathered for its ranks
constexpr uint32_t kBoundNode = 2u;      // node id of a level's node table or work list
constexpr uint32_t kBoundWalk = 4u;      // node id reached in a tree walk
constexpr uint32_t kBoundFeature = 8u;   // feature index of a split
constexpr uint32_t kBoundBin = 16u;      // histogram bin (rank) of a feature
constexpr uint32_t kBoundOut = 32u;      // output position (entries, children, packed nodes)

#ifdef AIWCRF_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_flag;

template <typename T>
__device__ __forceinline__ T checked_index(T i, uint64_t n, uint32_t site)
{
    if ((uint64_t)i < n) return i;
    atomicOr(&g_bounds_flag, site);
    return T(0);
}
#define AIWCRF_IDX(i, n, site) ::aiwcrf::checked_index((i), (uint64_t)(n), (site))
// host: this translation unit's flag, cleared by the read
#define AIWCRF_BOUNDS_READER(fn)                                                                   \
    uint32_t fn()                                                                                   \
    {                                                                                               \
        unsigned int v = 0, z = 0;                                                                  \
        if (cudaMemcpyFromSymbol(&v, g_bounds_flag, sizeof(v)) != cudaSuccess) return 0x80000000u;  \
        cudaMemcpyToSymbol(g_bounds_flag, &z, sizeof(z));                                           \
        return v;                                                                                   \
    }
#else
#define AIWCRF_IDX(i, n, site) (i)
#define AIWCRF_BOUNDS_READER(fn) \
    uint32_t fn() { return 0u; }
#endif

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds; each round multiplies counter
// words 0 and 2 by the two round multipliers, XORs the high halves into words 1 and 3 with
// the round key and swaps; the key advances by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c.x, b = c.z;
        const uint32_t hx = __umulhi(0xD2511F53u, a), lx = 0xD2511F53u * a;
        const uint32_t hz = __umulhi(0xCD9E8D57u, b), lz = 0xCD9E8D57u * b;
        c = make_uint4(hz ^ c.y ^ k0, lz, hx ^ c.w ^ k1, lx);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t uint4_word(uint4 v, int w)
{
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// ------------------------------------------------------------------------------------------
// small device utilities
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t float_key(float x)
{
    uint32_t b = __float_as_uint(x);
    if (b == 0x80000000u) b = 0u;                      // -0 and +0 are one value
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // order-preserving unsigned key
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// inclusive block scan of one u32 per thread (blockDim multiple of 32, <= 1024)
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *warp_tmp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) warp_tmp[lane] = w;             // inclusive warp prefix
    }
    __syncthreads();
    const uint32_t off = warp > 0 ? warp_tmp[warp - 1] : 0u;
    total = warp_tmp[nw - 1];
    __syncthreads();
    return x + off;
}

// ------------------------------------------------------------------------------------------
// Split candidates. Within a node (n = sum w, S = sum w*y) the CART gain of "left = ranks <= r"
// is G = S_L^2/n_L + S_R^2/n_R = S^2/n + delta^2 / (n n_L n_R), delta = n S_L - n_L S.
// So the search maximises D = delta^2 / (n_L n_R), exactly: a float estimate h = |delta| /
// sqrt(n_L n_R) (relative error < 2^-20) decides whenever two candidates differ by more than
// 2^-16, and 256-bit integer cross products decide the rest. Ties: lower feature, then lower
// rank. A split needs delta != 0 (strict gain over the parent).
// ------------------------------------------------------------------------------------------
struct Cand {
    float h;          // < 0: no candidate
    int32_t f;
    uint32_t r;
    uint32_t nL;      // sum w on the left
    int64_t SL;       // sum w*y on the left
};

__device__ __forceinline__ Cand cand_none()
{
    Cand c;
    c.h = -1.0f; c.f = 0x7FFFFFFF; c.r = 0xFFFFFFFFu; c.nL = 0; c.SL = 0;
    return c;
}

typedef unsigned __int128 u128_t;
typedef __int128 i128_t;

__device__ __forceinline__ i128_t cand_delta(uint32_t n, int64_t S, uint32_t nL, int64_t SL)
{
    return (i128_t)n * (i128_t)SL - (i128_t)nL * (i128_t)S;
}

__device__ __forceinline__ float cand_h(i128_t delta, uint32_t n, uint32_t nL)
{
    // |delta| < 2^96 and den < 2^64 are converted from 32-bit limbs (32-bit conversions stay off
    // the FP64 pipe): three limb conversions and two roundings for |delta|, two and one for den,
    // rsqrtf (at most 2 ulp) and the product keep the relative error of h below 2^-20
    const u128_t a = delta < 0 ? (u128_t)(-delta) : (u128_t)delta;
    const float fa = __fadd_rn(__fmaf_rn(__uint2float_rn((uint32_t)(a >> 64)), 18446744073709551616.0f,
                                         __fmul_rn(__uint2float_rn((uint32_t)(a >> 32)), 4294967296.0f)),
                               __uint2float_rn((uint32_t)a));
    const uint64_t den = (uint64_t)nL * (uint64_t)(n - nL);
    const float fd = __fmaf_rn(__uint2float_rn((uint32_t)(den >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)den));
    return __fmul_rn(fa, rsqrtf(fd));
}

// 256-bit value as four 64-bit limbs, least significant first
struct U256 { uint64_t w[4]; };

__device__ __forceinline__ U256 mul_128x128(u128_t a, u128_t b)
{
    const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    const uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    const u128_t p00 = (u128_t)a0 * b0, p01 = (u128_t)a0 * b1;
    const u128_t p10 = (u128_t)a1 * b0, p11 = (u128_t)a1 * b1;
    U256 r;
    r.w[0] = (uint64_t)p00;
    u128_t mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;          // < 3 * 2^64
    r.w[1] = (uint64_t)mid;
    u128_t hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
    r.w[2] = (uint64_t)hi;
    r.w[3] = (uint64_t)(hi >> 64) + (uint64_t)(p11 >> 64);
    return r;
}

__device__ __forceinline__ U256 mul_256x64(U256 a, uint64_t b)
{
    U256 r;
    u128_t carry = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const u128_t cur = (u128_t)a.w[i] * b + carry;
        r.w[i] = (uint64_t)cur;
        carry = cur >> 64;
    }
    return r;    // the callers' products are below 2^220
}

__device__ __forceinline__ int cmp_256(const U256 &a, const U256 &b)
{
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    }
    return 0;
}

// true if candidate a is better than b: larger D, then lower feature, then lower rank (plain
// scalar arguments: nothing of the caller's candidates needs an address)
static __device__ __noinline__ bool cand_better_exact_s(uint32_t a_nL, int64_t a_SL, int32_t a_f, uint32_t a_r,
                                                        uint32_t b_nL, int64_t b_SL, int32_t b_f, uint32_t b_r,
                                                        uint32_t n, int64_t S)
{
    if (!(a_nL == b_nL && a_SL == b_SL)) {
        const i128_t da = cand_delta(n, S, a_nL, a_SL), db = cand_delta(n, S, b_nL, b_SL);
        const u128_t ua = da < 0 ? (u128_t)(-da) : (u128_t)da;
        const u128_t ub = db < 0 ? (u128_t)(-db) : (u128_t)db;
        const uint64_t den_a = (uint64_t)a_nL * (uint64_t)(n - a_nL);
        const uint64_t den_b = (uint64_t)b_nL * (uint64_t)(n - b_nL);
        const int c = cmp_256(mul_256x64(mul_128x128(ua, ua), den_b), mul_256x64(mul_128x128(ub, ub), den_a));
        if (c != 0) return c > 0;
    }
    if (a_f != b_f) return a_f < b_f;
    return a_r < b_r;
}

// Two candidates with the same left sums, or with mirrored ones (nL' = n - nL, SL' = S - SL:
// delta' = -delta, the same n_L n_R), have equal gains: their order is the tie-break alone.
// Many tried features induce the same partition of a node's entries, so this case is settled
// inline and the exact 256-bit comparison (an out-of-line call) runs only for distinct gains.
__device__ __forceinline__ bool cand_better_exact(const Cand &a, const Cand &b, uint32_t n, int64_t S)
{
    if ((a.nL == b.nL && a.SL == b.SL) || (a.nL == n - b.nL && a.SL == S - b.SL))
        return a.f != b.f ? a.f < b.f : a.r < b.r;
    return cand_better_exact_s(a.nL, a.SL, a.f, a.r, b.nL, b.SL, b.f, b.r, n, S);
}

constexpr float kFilterHi = 1.0f + 1.0f / 65536.0f;
constexpr float kFilterLo = 1.0f - 1.0f / 65536.0f;

__device__ __forceinline__ bool cand_better(const Cand &a, const Cand &b, uint32_t n, int64_t S)
{
    if (a.h < 0.0f) return false;
    if (b.h < 0.0f) return true;
    if (a.h > b.h * kFilterHi) return true;
    if (a.h < b.h * kFilterLo) return false;
    return cand_better_exact(a, b, n, S);
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int src)
{
    Cand o;
    o.h = __shfl_sync(kFull, c.h, src);
    o.f = __shfl_sync(kFull, c.f, src);
    o.r = __shfl_sync(kFull, c.r, src);
    o.nL = __shfl_sync(kFull, c.nL, src);
    o.SL = (int64_t)__shfl_sync(kFull, (long long)c.SL, src);
    return o;
}

// Warp argmax under cand_better, the same result in every lane. Float max first; every lane
// whose estimate is within the filter margin of it is a contender (the true best always is);
// contenders are then compared exactly, in lane order.
__device__ __forceinline__ Cand warp_best(const Cand &mine, uint32_t n, int64_t S)
{
    float hm = mine.h;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) hm = fmaxf(hm, __shfl_xor_sync(kFull, hm, off));
    if (hm < 0.0f) return cand_none();
    const uint32_t cont = __ballot_sync(kFull, mine.h >= 0.0f && mine.h >= hm * kFilterLo);
    int src = __ffs(cont) - 1;
    Cand best = shfl_cand(mine, src);
    uint32_t rest = cont & (cont - 1);
    while (rest) {
        src = __ffs(rest) - 1;
        rest &= rest - 1;
        const Cand o = shfl_cand(mine, src);
        if (cand_better_exact(o, best, n, S)) best = o;
    }
    return best;
}

// Leaf value round(S/n), half up: floor((2S + n) / (2n)). 64-bit when 2S + n cannot overflow
// (|S| <= 2^61, always so for the targets' 2^40 bound and up to 2^21 rows of weight), else 128-bit.
__device__ __forceinline__ int64_t round_mean(int64_t S, uint32_t n)
{
    if (S <= ((int64_t)1 << 61) && S >= -((int64_t)1 << 61)) {
        const int64_t a = 2 * S + (int64_t)n, b = 2 * (int64_t)n;
        int64_t q = a / b;
        if (q * b != a && a < 0) q -= 1;
        return q;
    }
    const i128_t a = (i128_t)2 * S + n, b = (i128_t)2 * n;
    i128_t q = a / b;
    if (a % b != 0 && a < 0) q -= 1;
    return (int64_t)q;
}

// ------------------------------------------------------------------------------------------
// Level-synchronous growth state
// ------------------------------------------------------------------------------------------
struct NodeRec {          // an active node of the current depth
    uint32_t tree;        // forest-batch tree index
    uint32_t idx;         // BFS index within the depth, within its tree
    uint32_t start;       // segment start in the tree's row buffer
    uint32_t len;         // distinct in-bag rows
    uint32_t n;           // sum of multiplicities
    uint32_t pad;
    int64_t S;            // sum of w*y
};

struct SplitRes {         // outcome of one active node
    int32_t feature;      // >= 0 split; -1 leaf after a search; -2 leaf without a search
    uint32_t rank;
    uint32_t thr_bits;
    uint32_t nL;
    uint32_t lenL;
    uint32_t pad;
    int64_t v;            // S_L for a split (a leaf's value is computed where the node is encoded)
};

struct PackedRec {        // a finished node waiting for the final packing
    uint64_t node;        // encoded node (see aiwcrf.h), child index relative to its tree
    uint64_t cnode;       // the same node with its threshold replaced by its rank code
    uint32_t tree;
    uint32_t pos;         // BFS position within the tree
};

// Rank-coded copy of a split used by predict: bits 0..23 the threshold's index in the
// feature's sorted value table, bits 32..55 left child, bits 56..62 feature; leaves unchanged.
// A query value x is coded as c(x) = #{table values < x} (NaN: the table size), and
// x <= table[r]  <=>  c(x) <= r, so the coded walk takes exactly the float walk's path.
__device__ __forceinline__ uint64_t encode_split_coded(int f, uint32_t left, uint32_t code)
{
    return ((uint64_t)(uint32_t)f << 56) | ((uint64_t)left << 32) | (uint64_t)code;
}

__device__ __forceinline__ uint64_t encode_split(int f, uint32_t left, uint32_t thr_bits)
{
    return ((uint64_t)(uint32_t)f << 56) | ((uint64_t)left << 32) | (uint64_t)thr_bits;
}

__device__ __forceinline__ uint64_t encode_leaf(int64_t v)
{
    return (1ull << 63) | ((uint64_t)v & 0x7FFFFFFFFFFFFFFFull);
}

struct GrowStats {        // device counters of one fit (field order is used by finalize_kernel)
    unsigned long long entries_evaluated;
    unsigned long long entries_partitioned;
    unsigned long long nodes_evaluated;
    unsigned long long nodes_small;
    unsigned long long entries_evaluated_small;
    unsigned long long entries_partitioned_small;
};

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
// Stable LSD radix sort (four 8-bit passes) of S segments of n (key, value) u32 pairs, segment s
// at offset s * stride. The result ends in (keys_a, vals_a); (keys_b, vals_b) is scratch.
// hist needs S * 256 * ceil(n / 4096) + 1 words.
int radix_sort_segments(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, int64_t n,
                        int S, int64_t stride, uint32_t *hist, cudaStream_t s);
size_t radix_sort_hist_words(int64_t n, int S);

enum ProfClass {
    kProfRank = 0, kProfBoot, kProfLevelBig, kProfLevelSmall, kProfFinalize,
    kProfPack, kProfPredict, kProfSelect, kProfServe, kProfTree, kProfWalk, kProfListPart, kProfNum
};

void prof_begin(cudaStream_t s, int cls);
void count_launches(int n);      // kernels launched (for aiwcrf_launch_count)
void prof_end(cudaStream_t s, int cls);

struct Error {
    int code;
    std::string msg;
};

void set_error(int code, const std::string &msg);
void clear_last_error();         // every C entry point starts with an empty message
// bounds flags of the translation units that check (debug builds; cleared by the read)
uint32_t bounds_flags_fit();
uint32_t bounds_flags_predict();
uint32_t bounds_flags_serve();
// the grower of the next fits (AIWCRF_GROWER_*), process-wide
int set_grower_mode(int mode);
int grower_mode();
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

}  // namespace aiwcrf

struct aiwcrf_forest {
    int32_t F = 0;
    int64_t T = 0;
    int64_t num_nodes = 0;
    int64_t max_tree_nodes = 0;
    int device = 0;
    void *d_block = nullptr;              // one device allocation holding every array below
    uint64_t *d_nodes = nullptr;          // packed nodes
    uint64_t *d_cnodes = nullptr;         // the same nodes, thresholds as rank codes
    int64_t *d_tree_off = nullptr;        // T + 1 offsets (in nodes)
    float *d_fvals = nullptr;             // per feature sorted value table [F][fstride]
    uint32_t *d_fcard = nullptr;          // per feature table size
    int64_t fstride = 0;
    uint32_t max_card = 0;
    // 4-byte coded nodes for the shared-memory walk, when every code fits a byte and every tree
    // 65,536 nodes: bit 31 leaf; else bits 24..30 feature, 16..23 code, 0..15 left child.
    // Trees padded to a multiple of four nodes (16-byte aligned copies); leaf values are read
    // from d_nodes at the same tree-relative index.
    // out-of-bag evaluation: per tree ceil(oob_rows / 32) words, bit r = training row r in-bag
    int64_t oob_rows = 0;                 // 0: not available (deserialized or subset forests)
    int64_t inbag_words = 0;
    uint32_t *d_inbag = nullptr;
    bool compact = false;
    uint32_t *d_c32 = nullptr;
    int64_t *d_tree_off4 = nullptr;       // T + 1 offsets into d_c32
    int64_t num_c32 = 0;
    int64_t max_tree4 = 0;
    // features whose codes order large query batches before a compact walk (most used in the
    // trees' top levels first; -1: none), so that a warp's queries take similar paths
    int32_t key_feats[4] = {-1, -1, -1, -1};
    std::vector<int64_t> tree_off;        // host copy
    aiwcrf_fit_stats stats = {};
};

namespace aiwcrf {
// fit plans (fit.cu): the fit captured once as a CUDA graph and replayed
struct FitPlan;
int fit_plan_create(const aiwcrf_fit_params &p, const float *dX, const int64_t *dy, int64_t N, int32_t F,
                    const std::vector<int64_t> &sub_off, const int32_t *d_sub_rows, int32_t G, cudaStream_t s,
                    FitPlan **out);
int fit_plan_run(FitPlan *P, cudaStream_t s, std::vector<aiwcrf_forest *> &out);
int fit_plan_set_schedule(FitPlan *P, int cps_big, int cps_small);
void fit_plan_schedule(const FitPlan *P, int *cps_big, int *cps_small);
void fit_plan_free(FitPlan *P);
// the largest CTAs per SM each level kernel is built for
void fit_plan_limits(int *cps_big, int *cps_small);

// frees a forest once every stream of the device is idle
void forest_release(aiwcrf_forest *f);
// frees a forest in stream order on s; the caller has seen all work reading it complete
void forest_release_async(aiwcrf_forest *f, cudaStream_t s);
// one stream-ordered device allocation on s for the forest's arrays (nodes, coded nodes, tree
// offsets, value tables, compact nodes); sets the compact layout's host fields from tree_off
// and max_card
cudaError_t forest_alloc(aiwcrf_forest *f, cudaStream_t s);
// fills the compact 4-byte node array from d_cnodes (after d_cnodes and d_tree_off are written)
int forest_build_compact(aiwcrf_forest *f, cudaStream_t s);
// keep freed stream-ordered allocations cached in the device's default pool (once per device)
void keep_pool_memory(int device);
// a small pinned host buffer reused by the calling thread (at least 64 bytes)
// a page-locked host buffer of kPinnedScratchBytes per host thread (null if it cannot be had)
constexpr size_t kPinnedScratchBytes = 64 * 1024;
void *pinned_scratch();
}

namespace aiwcrf {
// implemented in fit.cu / predict.cu
int fit_batch(const aiwcrf_fit_params &p, const float *dX, const int64_t *dy, int64_t N, int32_t F,
              const std::vector<int64_t> &sub_off, const int32_t *d_sub_rows, int32_t G,
              cudaStream_t s, std::vector<aiwcrf_forest *> &out);
int tc_gemm(const __nv_bfloat16 *A, int lda, bool a_trans, const __nv_bfloat16 *B, int ldb, bool b_trans, float *C,
            int M, int N, int K, int ksplit, float *part, uint32_t *d_err, cudaStream_t s);
// predict without allocating or synchronising: codes_scratch holds predict_codes_bytes(f, Q)
size_t predict_codes_bytes(const aiwcrf_forest *f, int64_t Q);
// the most predict_codes_bytes can be for any forest of F features
size_t predict_codes_bytes_max(int32_t F, int64_t Q);
int predict_enqueue(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum, int64_t *d_pred,
                    cudaStream_t s, uint32_t *d_err, void *codes_scratch);
// fused surrogate inference on the stream, timeouts flagged in d_err (no allocation, no sync)
int surrogate_predict_enqueue(const aiwcrf_surrogate *sg, const float *dXq, int64_t Q, float *d_out, uint32_t *d_err,
                              cudaStream_t s);
// Device selection by the tree-parallel kernel (one CTA per kernel and 32 trees): d_kfeat is
// (F-2) x K, d_sum (K * D) and d_cnt (K) zero on entry and left zero, d_pred K x D; needs
// D <= 64 and size_class >= 0. Same integer results as predict + argmin.
int select_small_launch(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                        const int32_t *d_dev, int32_t D, int32_t *d_best, int64_t *d_pred, unsigned long long *d_sum,
                        uint32_t *d_cnt, cudaStream_t s);
// exact ensemble variance numerators of the first n_trees trees (2 u64 words per query)
int predict_prefix_var_enqueue(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t n_trees,
                               uint64_t *d_var, cudaStream_t s, uint32_t *d_err, void *codes_scratch);
// F x (K * D) queries: kernel k's F-2 features, device d_dev[j], size class (query k * D + j);
// d_kfeat has leading dimension ld; the size class is size_class, or d_size_row[k] if given
int expand_launch(const float *d_kfeat, int32_t K, int64_t ld, int32_t size_class, const float *d_size_row,
                  const int32_t *d_dev, int32_t D, int32_t F, float *d_q, cudaStream_t s);
int oob_launch(const aiwcrf_forest *f, const float *dX, int64_t N, int64_t *d_sum, int32_t *d_count, cudaStream_t s);

// Gated selection (gate.cu). A kernel's gate flag, when the reasons are kept: the forest answers
// it (kGateForest), a feature lay outside the training range (kGateOod), the surrogate's margin
// was within z deviations (kGateVar).
constexpr uint8_t kGateForest = 1u, kGateOod = 2u, kGateVar = 4u;
struct GateBuffers {
    float *q;                      // F x (K * D) queries
    float *sur;                    // K * D surrogate outputs
    uint64_t *var;                 // 2 words per query: prefix variance numerators
    void *codes;                   // predict_codes_bytes(forest, K * D)
    uint8_t *flag;                 // K
    int32_t *best;                 // K: the surrogate's device (the forest's is the caller's to write)
    float *pred;                   // K x D surrogate predictions, or null
    int32_t *list;                 // K fallback list with flag 0/1, or null for reason bits
    unsigned long long *counts;    // 3 counters with list, else unused
    uint32_t *err;                 // bounded-wait error flags
};
int gate_check(const aiwcrf_forest *forest, const aiwcrf_gate_params *gate);
// bytes of q, sur, var and codes for Qn queries of any forest of F features (256-byte aligned parts)
size_t gate_scratch_bytes(int32_t F, int64_t Qn);
// steps 1-4 of the gated selection for K kernels (d_kfeat leading dimension ld; size class
// size_class, or d_size_row[k] if given) on s, without allocating or synchronising
int gate_enqueue(const aiwcrf_forest *forest, const aiwcrf_surrogate *sg, const aiwcrf_gate_params &gate,
                 const float *d_kfeat, int32_t K, int64_t ld, int32_t size_class, const float *d_size_row,
                 const int32_t *d_dev, int32_t D, const GateBuffers &b, cudaStream_t s);
// a device copy of a surrogate on its device (parameters, transform, BF16 weights, statistics)
int surrogate_clone(const aiwcrf_surrogate *src, aiwcrf_surrogate **out);
// frees a surrogate in stream order on s; the caller has seen all work reading it complete
void surrogate_release_async(aiwcrf_surrogate *sg, cudaStream_t s);
struct SurrogateInfo {
    int device;
    int32_t F;
    int64_t bytes;     // device bytes it holds
};
SurrogateInfo surrogate_info(const aiwcrf_surrogate *sg);
// q, sur, var and codes of GateBuffers carved from gate_scratch_bytes(F, Qn) bytes at scratch
GateBuffers gate_scratch_split(void *scratch, int32_t F, int64_t Qn);
// out-of-bag error from aiwcrf_oob's sums and counts (d_y: the training targets): d_pred (or
// null) gets the out-of-bag predictions, d_res the exact sum of squared errors and the mean
struct OobPart { unsigned long long lo, hi, rows; };
struct OobResult { unsigned long long sq_lo, sq_hi; long long rows; double mse; };
size_t oob_error_parts(int64_t N);
int oob_error_launch(const int64_t *d_sum, const int32_t *d_count, const int64_t *d_y, int64_t N, int64_t *d_pred,
                     OobPart *d_parts, OobResult *d_res, uint32_t *d_err, cudaStream_t s);
int predict_launch(const aiwcrf_forest *f, const float *dXq, int64_t Q, int64_t *d_sum,
                   int64_t *d_pred, uint64_t *d_var, int64_t total_trees, cudaStream_t s);
int round_mean_launch(const int64_t *d_sum, int64_t Q, int64_t total_trees, int64_t *d_out,
                      cudaStream_t s);
int select_launch(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                  const int32_t *d_dev, int32_t D, int32_t *d_best, int64_t *d_pred,
                  float *d_scratch_q, int64_t *d_scratch_p, cudaStream_t s);
size_t select_noalloc_bytes(const aiwcrf_forest *f, int32_t K, int32_t D);
int select_launch_noalloc(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                          const int32_t *h_dev, int32_t D, int32_t *d_best, int64_t *d_pred, unsigned char *scratch,
                          cudaStream_t s);
}  // namespace aiwcrf
