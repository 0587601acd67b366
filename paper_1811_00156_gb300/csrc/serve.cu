// serve.cu -- the device-selection server: the scheduler of Sec. VI (pick the fastest device
// for each kernel about to run) as a resident service, with the retraining of Sec. I (refit
// when the training data changes) running beside it.
//
// Runtime (host C++):
//  - a dispatcher thread owns n_streams stream slots. It forms a batch from the pending
//    requests in arrival order whenever a slot is free (continuous batching: whatever arrived
//    while the other slots were busy goes into the next batch), stages the batch's features in
//    the slot's pinned buffer, and enqueues copy in, one selection kernel, copy out and an
//    event. It polls the events and completes the requests of finished batches;
//  - every batch's device inputs and outputs come from a first-fit arena carved out of one
//    allocation: a request is admitted into a batch only while its bytes fit the arena's free
//    space, so the server's device footprint is fixed at creation;
//  - gated requests (a surrogate resident beside the forest) share the batches: their kernels
//    come first, go through the gate's steps (query expansion, surrogate, prefix variances,
//    gate_kernel; gate.cu) and only those the gate sends back reach the selection kernel, whose
//    CTAs for the others return at once; no host synchronisation inside a batch;
//  - a refit thread fits new forests from the training rows plus appended rows on its own
//    low-priority stream, as a background fit (one level-kernel CTA per SM, so that selection
//    CTAs always find registers on every SM), and swaps them in; each batch holds a reference to the forest it was formed with,
//    and a forest is freed (stream-ordered) only after the last batch using it completed.
//
// Selection kernel (serve_select_kernel): one CTA per (kernel, chunk of 32 trees). It codes the
// kernel's features once as ranks in the forest's value tables (c(x) = #{training values < x};
// NaN past every value) plus one code per device, then its threads walk (tree, device) pairs,
// the threads of one tree side by side so that their paths, identical until a split on the
// device column, read the same nodes. Exact int64 sums per (kernel, device) are added
// atomically; the CTA that completes a kernel's last chunk (a per-kernel counter) rounds the
// sums to predictions, takes the argmin over devices (ties to the lower device id) and resets
// the sums and the counter for the slot's next batch. Integer sums make the result independent
// of the order in which CTAs finish: a request gets the same answer alone or batched with any
// others.
#include <cuda_runtime.h>
#include <sys/resource.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace aiwcrf {

struct ServeForest {
    const uint32_t *c32;
    const int64_t *tree_off4;
    const uint64_t *nodes;
    const uint64_t *cnodes;
    const int64_t *tree_off;
    const float *fvals;
    const uint32_t *fcard;
    int64_t fstride;
    int T;
    int F;
};

constexpr int kServeThreads = 256;
constexpr int kDevSlots = 16;                             // threads of one tree slot: devices
constexpr int kTreeSlots = kServeThreads / kDevSlots;    // 16 tree slots
constexpr int kTreesPerBlock = 2 * kTreeSlots;            // each thread walks two trees
constexpr int kServeMaxDevices = 64;

__device__ __forceinline__ int64_t serve_leaf(uint64_t nd)
{
    return ((int64_t)(nd << 1)) >> 1;
}

// The rank code of feature f for this thread's query: the kernel's codes are shared by the
// block, the device column's code is the thread's own.
__device__ __forceinline__ uint32_t serve_code(const uint32_t *kcode, uint32_t f, uint32_t fd, uint32_t dc)
{
    return f == fd ? dc : kcode[f];
}

// Two independent walks (trees t0, t1; -1 = none).
template <bool COMPACT>
__device__ __forceinline__ int64_t serve_walk2(const ServeForest &sf, int t0, int t1, const uint32_t *kcode,
                                               uint32_t fd, uint32_t dc)
{
    int64_t v = 0;
    if (COMPACT) {
        const uint32_t *n0 = sf.c32 + (t0 >= 0 ? sf.tree_off4[t0] : 0);
        const uint32_t *n1 = sf.c32 + (t1 >= 0 ? sf.tree_off4[t1] : 0);
#ifdef AIWCRF_DEBUG_BOUNDS
        const uint32_t m0 = t0 >= 0 ? (uint32_t)(sf.tree_off4[t0 + 1] - sf.tree_off4[t0]) : 1u;
        const uint32_t m1 = t1 >= 0 ? (uint32_t)(sf.tree_off4[t1 + 1] - sf.tree_off4[t1]) : 1u;
#endif
        uint32_t j0 = 0, j1 = 0;
        bool l0 = t0 < 0, l1 = t1 < 0;
        while (!(l0 && l1)) {
            const uint32_t a = __ldg(n0 + j0), b = __ldg(n1 + j1);
            const bool la = l0 || (int32_t)a < 0, lb = l1 || (int32_t)b < 0;
            const uint32_t ca = serve_code(kcode, la ? 0u : (a >> 24), fd, dc);
            const uint32_t cb = serve_code(kcode, lb ? 0u : (b >> 24), fd, dc);
            j0 = la ? j0 : AIWCRF_IDX((a & 0xFFFFu) + (ca > ((a >> 16) & 0xFFu) ? 1u : 0u), m0, kBoundWalk);
            j1 = lb ? j1 : AIWCRF_IDX((b & 0xFFFFu) + (cb > ((b >> 16) & 0xFFu) ? 1u : 0u), m1, kBoundWalk);
            l0 = la;
            l1 = lb;
        }
        if (t0 >= 0) v += serve_leaf(__ldg(sf.nodes + sf.tree_off[t0] + j0));
        if (t1 >= 0) v += serve_leaf(__ldg(sf.nodes + sf.tree_off[t1] + j1));
    } else {
        const uint64_t *n0 = sf.cnodes + (t0 >= 0 ? sf.tree_off[t0] : 0);
        const uint64_t *n1 = sf.cnodes + (t1 >= 0 ? sf.tree_off[t1] : 0);
#ifdef AIWCRF_DEBUG_BOUNDS
        const uint32_t m0 = t0 >= 0 ? (uint32_t)(sf.tree_off[t0 + 1] - sf.tree_off[t0]) : 1u;
        const uint32_t m1 = t1 >= 0 ? (uint32_t)(sf.tree_off[t1 + 1] - sf.tree_off[t1]) : 1u;
#endif
        uint32_t j0 = 0, j1 = 0;
        bool l0 = t0 < 0, l1 = t1 < 0;
        while (!(l0 && l1)) {
            const uint64_t a = __ldg(n0 + j0), b = __ldg(n1 + j1);
            const bool la = l0 || (a >> 63), lb = l1 || (b >> 63);
            const uint32_t ca = serve_code(kcode, la ? 0u : (uint32_t)(a >> 56) & 0x7Fu, fd, dc);
            const uint32_t cb = serve_code(kcode, lb ? 0u : (uint32_t)(b >> 56) & 0x7Fu, fd, dc);
            j0 = la ? j0 : AIWCRF_IDX(((uint32_t)(a >> 32) & 0xFFFFFFu) + (ca > ((uint32_t)a & 0xFFFFFFu) ? 1u : 0u), m0, kBoundWalk);
            j1 = lb ? j1 : AIWCRF_IDX(((uint32_t)(b >> 32) & 0xFFFFFFu) + (cb > ((uint32_t)b & 0xFFFFFFu) ? 1u : 0u), m1, kBoundWalk);
            l0 = la;
            l1 = lb;
        }
        if (t0 >= 0) v += serve_leaf(__ldg(n0 + j0));
        if (t1 >= 0) v += serve_leaf(__ldg(n1 + j1));
    }
    return v;
}

__device__ __forceinline__ uint32_t rank_code(const float *V, uint32_t card, float x)
{
    if (x != x) return card;
    uint32_t lo = 0, hi = card;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&V[mid]) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Block (kernel k, chunk g of 32 trees). Thread (tree slot ts, device slot jl) walks trees
// 32g + ts and 32g + ts + 16 for device jb + jl, for each pass jb = 0, 16, .. < D: the threads of
// one tree follow the same path until a split on the device column, so their node loads
// coincide. kq: F x Kb column-major batch features (row F-2 unused: the device id comes from
// dev[]; row F-1 the size class, unless size_override >= 0 gives it for every kernel, and then kq
// may have only F-2 rows). sums (Kb * D) and cnt (Kb) are zero on entry and left zero.
// pred: Kb x D row-major predictions; best: Kb device ids. Kernels k < n_gated went through the
// gate first: only those whose gate flag has kGateForest are answered here, and their
// predictions are also written to fpred as float log10 seconds.
template <bool COMPACT>
__global__ void __launch_bounds__(kServeThreads) serve_select_kernel(ServeForest sf, const float *__restrict__ kq,
                                                                     int Kb, const int32_t *__restrict__ dev, int D,
                                                                     int size_override, unsigned long long *sums,
                                                                     uint32_t *cnt, int64_t *pred, int32_t *best,
                                                                     const uint8_t *__restrict__ only, int n_gated,
                                                                     float *fpred)
{
    __shared__ uint32_t kcode[AIWCRF_MAX_FEATURES];
    __shared__ uint32_t dcode[kServeMaxDevices];
    __shared__ int64_t red[kServeThreads / 32][kDevSlots];
    __shared__ int last;
    const int k = blockIdx.x, g = blockIdx.y;
    if (k < n_gated && !(only[k] & kGateForest)) return;      // the surrogate's answer stands
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ts = tid / kDevSlots, jl = tid % kDevSlots;
    const uint32_t fd = (uint32_t)sf.F - 2u;
    for (int f = tid; f < sf.F; f += kServeThreads)
        if (f != (int)fd)
            kcode[f] = rank_code(sf.fvals + (size_t)f * (size_t)sf.fstride, sf.fcard[f],
                                 (f == sf.F - 1 && size_override >= 0) ? (float)size_override
                                                                       : kq[(size_t)f * (size_t)Kb + (size_t)k]);
    for (int j = tid; j < D; j += kServeThreads)
        dcode[j] = rank_code(sf.fvals + (size_t)fd * (size_t)sf.fstride, sf.fcard[fd], (float)dev[j]);
    __syncthreads();
    const int t0 = g * kTreesPerBlock + ts, t1 = t0 + kTreeSlots;
    for (int jb = 0; jb < D; jb += kDevSlots) {
        const int j = jb + jl;
        int64_t v = 0;
        if (j < D) v = serve_walk2<COMPACT>(sf, t0 < sf.T ? t0 : -1, t1 < sf.T ? t1 : -1, kcode, fd, dcode[j]);
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);             // the warp's two tree slots
        if (lane < kDevSlots) red[warp][lane] = v;
        __syncthreads();
        if (tid < kDevSlots && j < D) {
            int64_t sum = 0;
#pragma unroll
            for (int w = 0; w < kServeThreads / 32; ++w) sum += red[w][tid];
            atomicAdd(&sums[(size_t)k * (size_t)D + (size_t)j], (unsigned long long)sum);
            __threadfence();
        }
        __syncthreads();
    }
    if (tid == 0) last = atomicAdd(&cnt[k], 1u) == gridDim.y - 1u;
    __syncthreads();
    if (!last || warp != 0) return;
    // the last chunk of kernel k: every tree has been added for every device
    __threadfence();
    int64_t bp = LLONG_MAX;
    int32_t bd = INT_MAX;
    for (int j = lane; j < D; j += 32) {
        const int64_t s = (int64_t)atomicExch(&sums[(size_t)k * (size_t)D + (size_t)j], 0ull);
        const i128_t num = (i128_t)2 * s + sf.T, den = (i128_t)2 * sf.T;
        i128_t d = num / den;
        if (num % den != 0 && num < 0) d -= 1;
        const int64_t p = (int64_t)d;
        pred[(size_t)k * (size_t)D + (size_t)j] = p;
        if (k < n_gated) fpred[(size_t)k * (size_t)D + (size_t)j] = (float)((double)p * 0x1p-32);
        const int32_t id = dev[j];
        if (p < bp || (p == bp && id < bd)) { bp = p; bd = id; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const int64_t op = __shfl_xor_sync(0xFFFFFFFFu, bp, o);
        const int32_t od = __shfl_xor_sync(0xFFFFFFFFu, bd, o);
        if (op < bp || (op == bp && od < bd)) { bp = op; bd = od; }
    }
    if (lane == 0) {
        best[k] = bd;
        cnt[k] = 0u;
    }
}

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

// CPU time and context switches of the calling thread (where a stalled dispatcher's time went)
struct ThreadUsage {
    int64_t cpu_ns = 0;
    long vol = 0, invol = 0;
};

ThreadUsage thread_usage()
{
    ThreadUsage u;
    timespec ts;
    if (clock_gettime(CLOCK_THREAD_CPUTIME_ID, &ts) == 0) u.cpu_ns = (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
    rusage ru;
    if (getrusage(RUSAGE_THREAD, &ru) == 0) {
        u.vol = ru.ru_nvcsw;
        u.invol = ru.ru_nivcsw;
    }
    return u;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int64_t kIdlePollNs = 200000;   // the dispatcher polls this long before sleeping

int serve_launch(const aiwcrf_forest *f, const float *d_kq, int Kb, const int32_t *d_dev, int D, int size_override,
                 unsigned long long *d_sum, uint32_t *d_cnt, int64_t *d_pred, int32_t *d_best, cudaStream_t s,
                 const uint8_t *d_only = nullptr, int n_gated = 0, float *d_fpred = nullptr)
{
    ServeForest sf;
    sf.c32 = f->d_c32;
    sf.tree_off4 = f->d_tree_off4;
    sf.nodes = f->d_nodes;
    sf.cnodes = f->d_cnodes;
    sf.tree_off = f->d_tree_off;
    sf.fvals = f->d_fvals;
    sf.fcard = f->d_fcard;
    sf.fstride = f->fstride;
    sf.T = (int)f->T;
    sf.F = f->F;
    const dim3 grid((unsigned)Kb, (unsigned)((f->T + kTreesPerBlock - 1) / kTreesPerBlock));
    prof_begin(s, kProfServe);
    if (f->compact)
        serve_select_kernel<true><<<grid, kServeThreads, 0, s>>>(sf, d_kq, Kb, d_dev, D, size_override, d_sum, d_cnt,
                                                                 d_pred, d_best, d_only, n_gated, d_fpred);
    else
        serve_select_kernel<false><<<grid, kServeThreads, 0, s>>>(sf, d_kq, Kb, d_dev, D, size_override, d_sum, d_cnt,
                                                                  d_pred, d_best, d_only, n_gated, d_fpred);
    prof_end(s, kProfServe);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "serve_select_kernel launch");
    return AIWCRF_OK;
}

}  // namespace

int select_small_launch(const aiwcrf_forest *f, const float *d_kfeat, int32_t K, int32_t size_class,
                        const int32_t *d_dev, int32_t D, int32_t *d_best, int64_t *d_pred, unsigned long long *d_sum,
                        uint32_t *d_cnt, cudaStream_t s)
{
    if (D > kServeMaxDevices || f->F > AIWCRF_MAX_FEATURES || size_class < 0)
        return fail(AIWCRF_E_INVALID_ARG, "select_small_launch: unsupported shape");
    return serve_launch(f, d_kfeat, K, d_dev, D, size_class, d_sum, d_cnt, d_pred, d_best, s);
}

namespace {

// First-fit allocator over [0, cap) in 256-byte granules; free neighbours merge.
struct Arena {
    int64_t cap = 0, used = 0, peak = 0;
    std::map<int64_t, int64_t> free_;    // offset -> bytes

    void init(int64_t c)
    {
        cap = c;
        used = peak = 0;
        free_.clear();
        if (c > 0) free_[0] = c;
    }
    int64_t largest() const
    {
        int64_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    int64_t alloc(int64_t bytes)
    {
        bytes = (int64_t)up256((size_t)bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used += bytes;
            peak = std::max(peak, used);
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = (int64_t)up256((size_t)bytes);
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct LoadRun {
    std::mutex mu;
    std::condition_variable cv;
    bool abandoned = false;
    int64_t remaining = 0;
    int first_error = AIWCRF_OK;
    int32_t *best = nullptr;              // caller's, may be null
    int64_t *gen = nullptr;               // caller's, may be null
    std::vector<int64_t> lat;             // -1: not served
};

struct Request {
    int64_t ticket = -1;
    int32_t K = 0, size = 0;
    const float *src = nullptr;           // feature (f, k) at src[f * ld + k]
    int64_t ld = 0;
    std::vector<float> own;
    int64_t t_arrive = 0;
    // completion of a submitted request
    bool done = false;
    int32_t status = AIWCRF_OK;
    std::string msg;
    int64_t generation = -1;
    std::vector<int32_t> best;
    std::vector<int64_t> pred;
    // gated request: the surrogate answers unless the gate sends the kernel to the forest
    bool gated = false;
    std::vector<float> fpred;
    std::vector<uint8_t> fallback;
    // load-generator request
    std::shared_ptr<LoadRun> run;
    int64_t run_index = 0, run_best_off = 0;
};

struct Model {
    aiwcrf_forest *f = nullptr;
    int64_t gen = 0;
    int64_t rows = 0;
    int64_t bytes = 0;
};

// the server's own copy of a surrogate and the gate that decides when the forest answers instead
struct SurModel {
    aiwcrf_surrogate *sg = nullptr;
    aiwcrf_gate_params gate{};
    int64_t bytes = 0;
};

// Device bytes of one batch of Kb kernels, Kg of them gated (placed first): features, then the
// results copied back in one piece (exact predictions, devices, and for the gated kernels their
// float predictions, gate flags and the error word), then the gate's scratch.
struct BatchLayout {
    size_t out = 0;                                   // results, from the batch's start
    size_t pred = 0, best = 0, fpred = 0, flag = 0, err = 0, out_bytes = 0;   // within the results
    size_t scratch = 0, total = 0;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    float *h_in = nullptr;                // pinned F x batch_kernels
    unsigned char *h_out = nullptr;       // pinned batch_kernels x (8 D + 4)
    unsigned long long *d_sum = nullptr;  // batch_kernels x D, kept zero between batches
    uint32_t *d_cnt = nullptr;            // batch_kernels, kept zero between batches
    bool busy = false;
    int64_t off = -1, bytes = 0;
    int32_t Kb = 0, Kg = 0;               // kernels, of which the first Kg gated
    std::shared_ptr<SurModel> sur;        // the surrogate of the gated kernels
    std::vector<int64_t> offs;            // each request's first kernel in the batch
    int64_t t_formed = 0, t_enqueued = 0;
    int64_t enq_cpu = 0, last_poll = 0, poll_gap_max = 0;
    int32_t enq_vol = 0, enq_invol = 0;
    std::shared_ptr<Model> model;
    std::vector<std::shared_ptr<Request>> reqs;
};

struct SplitMix64 {
    uint64_t x;
    uint64_t next()
    {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

}  // namespace
}  // namespace aiwcrf

using namespace aiwcrf;

struct aiwcrf_server {
    aiwcrf_server_params sp{};
    aiwcrf_fit_params fp{};
    int32_t F = 0, D = 0;
    int device = 0;
    std::vector<int32_t> dev_ids;
    int32_t *d_dev = nullptr;
    unsigned char *d_arena = nullptr;
    Arena arena;
    std::vector<Slot> slots;

    std::mutex mu;                        // queue, tickets, arena, current model, counters
    std::condition_variable cv_disp, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::atomic<int64_t> n_pending{0};    // pending.size(), readable without the lock
    std::unordered_map<int64_t, std::shared_ptr<Request>> tickets;
    int64_t next_ticket = 1;
    bool stop = false, paused = false;
    std::shared_ptr<Model> current;
    std::shared_ptr<SurModel> cur_sur;    // null: gated requests are refused
    aiwcrf_server_counters st{};
    int64_t refit_mark = 0;

    std::mutex rmu;                       // training rows and refit requests
    std::condition_variable rcv, rcv_done;
    bool refit_req = false, refit_stop = false, refit_running = false;
    std::string last_refit_msg;
    int64_t refits_finished = 0;
    int last_refit_status = AIWCRF_OK;
    std::vector<std::vector<float>> xcols, acols;   // training / appended rows, per feature
    std::vector<int64_t> ytrain, yapp;
    cudaStream_t refit_stream = nullptr;

    std::mutex gmu;                       // forests and surrogates waiting to be freed (on the refit stream)
    std::vector<aiwcrf_forest *> graveyard;
    std::vector<aiwcrf_surrogate *> sgraveyard;

    std::thread disp, refitter;

    // traces (under mu)
    static constexpr int64_t kBatchRing = 65536, kRefitRing = 256;
    std::vector<aiwcrf_batch_trace> btrace = std::vector<aiwcrf_batch_trace>((size_t)kBatchRing);
    std::vector<aiwcrf_refit_trace> rtrace = std::vector<aiwcrf_refit_trace>((size_t)kRefitRing);
    int64_t n_btrace = 0, n_rtrace = 0;

    BatchLayout layout(int64_t Kb, int64_t Kg) const
    {
        auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
        BatchLayout L;
        L.out = up256(sizeof(float) * (size_t)F * (size_t)Kb);
        L.pred = 0;
        L.best = 8 * (size_t)Kb * (size_t)D;
        size_t o = L.best + 4 * (size_t)Kb;
        if (Kg > 0) {
            L.fpred = up16(o);
            L.flag = L.fpred + 4 * (size_t)Kg * (size_t)D;
            L.err = up16(L.flag + (size_t)Kg);
            o = L.err + 4;
        }
        L.out_bytes = o;
        L.scratch = L.out + up256(o);
        L.total = L.scratch + (Kg > 0 ? gate_scratch_bytes(F, Kg * (int64_t)D) : 0);
        return L;
    }

    int64_t req_bytes(int64_t K) const { return (int64_t)layout(K, 0).total; }

    std::shared_ptr<Model> wrap(aiwcrf_forest *f, int64_t gen, int64_t rows)
    {
        Model *m = new Model();
        m->f = f;
        m->gen = gen;
        m->rows = rows;
        m->bytes = 16 * f->num_nodes + 4 * f->num_c32 + 16 * (f->T + 1) + 4 * (int64_t)f->F * f->fstride +
                   4 * f->T * f->inbag_words;
        return std::shared_ptr<Model>(m, [this](Model *p) {
            {
                std::lock_guard<std::mutex> lk(gmu);
                graveyard.push_back(p->f);
            }
            delete p;
        });
    }

    std::shared_ptr<SurModel> wrap_surrogate(aiwcrf_surrogate *sg, const aiwcrf_gate_params &gate)
    {
        SurModel *m = new SurModel();
        m->sg = sg;
        m->gate = gate;
        m->bytes = surrogate_info(sg).bytes;
        return std::shared_ptr<SurModel>(m, [this](SurModel *p) {
            {
                std::lock_guard<std::mutex> lk(gmu);
                sgraveyard.push_back(p->sg);
            }
            delete p;
        });
    }

    void drain_graveyard()
    {
        std::vector<aiwcrf_forest *> g;
        std::vector<aiwcrf_surrogate *> sgs;
        {
            std::lock_guard<std::mutex> lk(gmu);
            g.swap(graveyard);
            sgs.swap(sgraveyard);
        }
        for (auto f : g) forest_release_async(f, refit_stream);
        for (auto sg : sgs) surrogate_release_async(sg, refit_stream);
    }

    // fit a forest on the current training rows (refit thread or creation)
    int fit_training(aiwcrf_forest **out, int64_t *rows, bool background, int64_t *t_staged = nullptr)
    {
        aiwcrf_fit_params fp_bg = fp;
        fp_bg.ctas_per_sm = 1;            // refits leave every SM room for selection batches
        const int64_t N = (int64_t)ytrain.size();
        std::vector<float> X((size_t)F * (size_t)N);
        for (int32_t f = 0; f < F; ++f) std::copy(xcols[(size_t)f].begin(), xcols[(size_t)f].end(), X.begin() + (size_t)f * (size_t)N);
        float *dX = nullptr;
        int64_t *dy = nullptr;
        cudaError_t e = cudaMallocAsync(&dX, sizeof(float) * X.size(), refit_stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&dy, sizeof(int64_t) * (size_t)N, refit_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, refit_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy, ytrain.data(), sizeof(int64_t) * (size_t)N, cudaMemcpyHostToDevice, refit_stream);
        int rc = e == cudaSuccess ? AIWCRF_OK : cuda_fail(e, "staging the training rows");
        if (t_staged) {
            cudaStreamSynchronize(refit_stream);
            *t_staged = now_ns();
        }
        if (rc == AIWCRF_OK) rc = aiwcrf_fit(background ? &fp_bg : &fp, dX, dy, N, F, refit_stream, out);
        if (dX) cudaFreeAsync(dX, refit_stream);
        if (dy) cudaFreeAsync(dy, refit_stream);
        cudaStreamSynchronize(refit_stream);
        *rows = N;
        return rc;
    }

    void finish(const std::shared_ptr<Request> &r, int status, const std::string &msg, int64_t gen,
                const int32_t *best, const int64_t *pred, int64_t t_done, const float *fpred = nullptr,
                const uint8_t *flags = nullptr)
    {
        if (r->run) {
            LoadRun &run = *r->run;
            std::lock_guard<std::mutex> lk(run.mu);
            if (!run.abandoned) {
                if (status == AIWCRF_OK) {
                    if (run.best && best) std::memcpy(run.best + r->run_best_off, best, sizeof(int32_t) * (size_t)r->K);
                    if (run.gen) run.gen[r->run_index] = gen;
                    run.lat[(size_t)r->run_index] = t_done - r->t_arrive;
                } else if (run.first_error == AIWCRF_OK) {
                    run.first_error = status;
                }
            }
            --run.remaining;
            run.cv.notify_all();
            return;
        }
        std::lock_guard<std::mutex> lk(mu);
        r->status = status;
        r->msg = msg;
        r->generation = gen;
        if (status == AIWCRF_OK) {
            r->best.assign(best, best + r->K);
            if (r->gated) {
                r->fpred.assign(fpred, fpred + (size_t)r->K * (size_t)D);
                r->fallback.resize((size_t)r->K);
                for (int32_t k = 0; k < r->K; ++k) r->fallback[(size_t)k] = (flags[k] & kGateForest) ? 1 : 0;
            } else {
                r->pred.assign(pred, pred + (size_t)r->K * (size_t)D);
            }
        }
        r->done = true;
        cv_done.notify_all();
    }

    void complete(Slot &sl, cudaError_t e)
    {
        const int64_t t = now_ns();
        const BatchLayout L = layout(sl.Kb, sl.Kg);
        int status = e == cudaSuccess ? AIWCRF_OK : AIWCRF_E_CUDA;
        std::string msg = e == cudaSuccess ? std::string() : std::string("selection batch: ") + cudaGetErrorString(e);
        const int64_t *hp = reinterpret_cast<const int64_t *>(sl.h_out + L.pred);
        const int32_t *hb = reinterpret_cast<const int32_t *>(sl.h_out + L.best);
        const float *hf = sl.Kg ? reinterpret_cast<const float *>(sl.h_out + L.fpred) : nullptr;
        const uint8_t *hfl = sl.Kg ? sl.h_out + L.flag : nullptr;
        if (status == AIWCRF_OK && sl.Kg && (*reinterpret_cast<const uint32_t *>(sl.h_out + L.err) & kErrTimeout)) {
            status = AIWCRF_E_TIMEOUT;
            msg = "selection batch: a bounded device wait gave up";
        }
        const int64_t gen = sl.model ? sl.model->gen : -1;
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            const int64_t off = sl.offs[i];
            finish(sl.reqs[i], status, msg, gen, hb + off, hp + off * D, t, hf ? hf + off * D : nullptr,
                   hfl ? hfl + off : nullptr);
        }
        int64_t n_fb = 0, n_ood = 0, n_var = 0;
        if (status == AIWCRF_OK)
            for (int32_t k = 0; k < sl.Kg; ++k) {
                n_fb += (hfl[k] & kGateForest) ? 1 : 0;
                n_ood += (hfl[k] & kGateOod) ? 1 : 0;
                n_var += (hfl[k] & kGateVar) ? 1 : 0;
            }
        bool want_refit = false;
        {
            std::lock_guard<std::mutex> lk(mu);
            aiwcrf_batch_trace &tr = btrace[(size_t)(n_btrace++ % kBatchRing)];
            tr.t_formed_ns = sl.t_formed;
            tr.t_enqueued_ns = sl.t_enqueued;
            tr.t_done_ns = t;
            tr.kernels = sl.Kb;
            tr.generation = (int32_t)gen;
            tr.enqueue_cpu_ns = sl.enq_cpu;
            tr.enqueue_voluntary_switches = sl.enq_vol;
            tr.enqueue_involuntary_switches = sl.enq_invol;
            tr.poll_gap_max_ns = std::max(sl.poll_gap_max, t - sl.last_poll);
            tr.gated_kernels = sl.Kg;
            tr.fallback_kernels = (int32_t)n_fb;
            st.gated_kernels += sl.Kg;
            st.gated_fallback += n_fb;
            st.gated_fallback_ood += n_ood;
            st.gated_fallback_var += n_var;
            arena.release(sl.off, sl.bytes);
            st.completed += (int64_t)sl.reqs.size();
            if (status != AIWCRF_OK) st.failed += (int64_t)sl.reqs.size();
            if (sp.refit_every > 0 && st.completed - refit_mark >= sp.refit_every) {
                refit_mark = st.completed;
                want_refit = true;
            }
        }
        sl.busy = false;
        sl.off = -1;
        sl.reqs.clear();
        sl.offs.clear();
        sl.model.reset();
        sl.sur.reset();
        if (want_refit) {
            std::lock_guard<std::mutex> lk(rmu);
            refit_req = true;
            rcv.notify_all();
        }
    }

    // Takes the batch (popped under mu, features staged in sl.h_in) to the GPU.
    // Gated kernels (the first Kg): expand, surrogate, prefix variances and gate (gate.cu); then
    // the selection kernel answers the exact kernels and the gated kernels the gate sent to the
    // forest. No host synchronisation inside a batch.
    void launch(Slot &sl)
    {
        const BatchLayout L = layout(sl.Kb, sl.Kg);
        const size_t in_bytes = sizeof(float) * (size_t)F * (size_t)sl.Kb;
        unsigned char *base = d_arena + sl.off;
        float *d_in = reinterpret_cast<float *>(base);
        unsigned char *d_out = base + L.out;
        int64_t *d_pred = reinterpret_cast<int64_t *>(d_out + L.pred);
        int32_t *d_best = reinterpret_cast<int32_t *>(d_out + L.best);
        float *d_fpred = sl.Kg ? reinterpret_cast<float *>(d_out + L.fpred) : nullptr;
        uint8_t *d_flag = sl.Kg ? d_out + L.flag : nullptr;
        uint32_t *d_err = sl.Kg ? reinterpret_cast<uint32_t *>(d_out + L.err) : nullptr;
        const ThreadUsage u0 = thread_usage();
        cudaError_t e = cudaMemcpyAsync(d_in, sl.h_in, in_bytes, cudaMemcpyHostToDevice, sl.s);
        if (e == cudaSuccess && sl.Kg) {
            e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), sl.s);
            GateBuffers gb = gate_scratch_split(base + L.scratch, F, (int64_t)sl.Kg * D);
            gb.flag = d_flag;
            gb.best = d_best;
            gb.pred = d_fpred;
            gb.err = d_err;
            if (e == cudaSuccess && gate_enqueue(sl.model->f, sl.sur->sg, sl.sur->gate, d_in, sl.Kg, sl.Kb, 0,
                                                 d_in + (size_t)(F - 1) * (size_t)sl.Kb, d_dev, D, gb,
                                                 sl.s) != AIWCRF_OK)
                e = cudaErrorLaunchFailure;
        }
        if (e == cudaSuccess && serve_launch(sl.model->f, d_in, sl.Kb, d_dev, D, -1, sl.d_sum, sl.d_cnt, d_pred, d_best,
                                             sl.s, d_flag, sl.Kg, d_fpred) != AIWCRF_OK)
            e = cudaErrorLaunchFailure;
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_out, d_out, L.out_bytes, cudaMemcpyDeviceToHost, sl.s);
        if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.s);
        sl.t_enqueued = now_ns();
        const ThreadUsage u1 = thread_usage();
        sl.enq_cpu = u1.cpu_ns - u0.cpu_ns;
        sl.enq_vol = (int32_t)(u1.vol - u0.vol);
        sl.enq_invol = (int32_t)(u1.invol - u0.invol);
        sl.last_poll = sl.t_enqueued;
        sl.poll_gap_max = 0;
        sl.busy = true;
        if (e != cudaSuccess) {
            cudaStreamSynchronize(sl.s);
            complete(sl, e);
        }
    }

    void dispatcher()
    {
        cudaSetDevice(device);
        for (;;) {
            bool progressed = false;
            bool any_busy = false;
            for (auto &sl : slots) {
                if (!sl.busy) continue;
                const cudaError_t e = cudaEventQuery(sl.ev);
                if (e == cudaErrorNotReady) {
                    const int64_t t = now_ns();
                    sl.poll_gap_max = std::max(sl.poll_gap_max, t - sl.last_poll);
                    sl.last_poll = t;
                    any_busy = true;
                    continue;
                }
                complete(sl, e);
                progressed = true;
            }
            drain_graveyard();
            Slot *free_slot = nullptr;
            for (auto &sl : slots)
                if (!sl.busy) { free_slot = &sl; break; }

            std::unique_lock<std::mutex> lk(mu);
            if (stop) {
                std::deque<std::shared_ptr<Request>> drop;
                drop.swap(pending);
                n_pending.store(0);
                lk.unlock();
                for (auto &r : drop) finish(r, AIWCRF_E_INVALID_ARG, "server shut down", -1, nullptr, nullptr, now_ns());
                if (!any_busy) {
                    bool busy = false;
                    for (auto &sl : slots) busy |= sl.busy;
                    if (!busy) break;
                }
                std::this_thread::yield();
                continue;
            }
            if (free_slot && !paused && !pending.empty()) {
                // form a batch: arrival order, within the batch size and the arena's free space
                const int64_t room = arena.largest();
                int64_t Kb = 0, Kg = 0;
                size_t n = 0;
                bool cut = false;
                while (n < pending.size()) {
                    const int64_t K2 = Kb + pending[n]->K, G2 = Kg + (pending[n]->gated ? pending[n]->K : 0);
                    if (K2 > sp.batch_kernels) break;
                    if ((int64_t)layout(K2, G2).total > room) { cut = true; break; }
                    Kb = K2;
                    Kg = G2;
                    ++n;
                }
                if (n > 0) {
                    if (cut) ++st.arena_waits;
                    Slot &sl = *free_slot;
                    sl.t_formed = now_ns();
                    sl.Kb = (int32_t)Kb;
                    sl.Kg = (int32_t)Kg;
                    sl.bytes = (int64_t)layout(Kb, Kg).total;
                    sl.off = arena.alloc(sl.bytes);
                    sl.reqs.assign(pending.begin(), pending.begin() + (std::ptrdiff_t)n);
                    pending.erase(pending.begin(), pending.begin() + (std::ptrdiff_t)n);
                    n_pending.store((int64_t)pending.size());
                    sl.model = current;
                    sl.sur = Kg ? cur_sur : nullptr;
                    ++st.batches;
                    st.batch_kernels_total += Kb;
                    st.batch_kernels_max = std::max(st.batch_kernels_max, Kb);
                    st.arena_peak_bytes = std::max(st.arena_peak_bytes, arena.peak);
                    // stage features while the requests' sources are guaranteed alive: the gated
                    // requests' kernels first, then the others, each request's kernels together
                    sl.offs.assign(sl.reqs.size(), 0);
                    int64_t kg = 0, kx = Kg;
                    for (size_t i = 0; i < sl.reqs.size(); ++i) {
                        const Request &r = *sl.reqs[i];
                        int64_t &k0 = r.gated ? kg : kx;
                        sl.offs[i] = k0;
                        for (int32_t f = 0; f < F; ++f) {
                            float *dst = sl.h_in + (size_t)f * (size_t)Kb + (size_t)k0;
                            if (f < F - 2) {
                                const float *src = r.src + (size_t)f * (size_t)r.ld;
                                std::memcpy(dst, src, sizeof(float) * (size_t)r.K);
                            } else {
                                const float val = f == F - 2 ? 0.0f : (float)r.size;
                                std::fill(dst, dst + r.K, val);
                            }
                        }
                        k0 += r.K;
                    }
                    lk.unlock();
                    launch(sl);
                    continue;
                }
            }
            if (!progressed) {
                if (any_busy) {
                    lk.unlock();
                    std::this_thread::yield();
                } else if (paused || pending.empty()) {
                    // idle: poll for a new request a little while before sleeping on the queue
                    if (!paused) {
                        lk.unlock();
                        const int64_t t_end = now_ns() + kIdlePollNs;
                        while (n_pending.load(std::memory_order_relaxed) == 0 && now_ns() < t_end)
                            std::this_thread::yield();
                        lk.lock();
                    }
                    if (!stop && (paused || pending.empty())) cv_disp.wait_for(lk, std::chrono::milliseconds(2));
                }
            }
        }
    }

    void refit_loop()
    {
        cudaSetDevice(device);
        for (;;) {
            std::unique_lock<std::mutex> lk(rmu);
            rcv.wait(lk, [&] { return refit_stop || refit_req; });
            if (refit_stop) break;
            refit_req = false;
            refit_running = true;
            const int64_t avail = (int64_t)yapp.size();
            const int64_t take = sp.refit_rows > 0 ? std::min<int64_t>(sp.refit_rows, avail) : avail;
            for (int32_t f = 0; f < F; ++f) {
                auto &a = acols[(size_t)f];
                xcols[(size_t)f].insert(xcols[(size_t)f].end(), a.begin(), a.begin() + take);
                a.erase(a.begin(), a.begin() + take);
            }
            ytrain.insert(ytrain.end(), yapp.begin(), yapp.begin() + take);
            yapp.erase(yapp.begin(), yapp.begin() + take);
            lk.unlock();

            aiwcrf_forest *f = nullptr;
            int64_t rows = 0;
            const int64_t t_fit = now_ns();
            int64_t t_staged = 0;
            const int rc = fit_training(&f, &rows, true, &t_staged);
            const int64_t t_fitted = now_ns();
            const int64_t us = (t_fitted - t_fit) / 1000;
            {
                std::lock_guard<std::mutex> g(mu);
                st.refit_us_total += us;
                st.refit_us_max = std::max(st.refit_us_max, us);
            }
            if (rc == AIWCRF_OK) {
                std::shared_ptr<Model> old;
                {
                    std::lock_guard<std::mutex> g(mu);
                    const int64_t gen = current ? current->gen + 1 : 0;
                    old = current;
                    current = wrap(f, gen, rows);
                    st.generation = gen;
                    st.training_rows = rows;
                    st.forest_bytes = current->bytes;
                    ++st.refits;
                    aiwcrf_refit_trace &tr = rtrace[(size_t)(n_rtrace++ % kRefitRing)];
                    tr.t_start_ns = t_fit;
                    tr.t_staged_ns = t_staged;
                    tr.t_fitted_ns = t_fitted;
                    tr.t_swapped_ns = now_ns();
                    tr.rows = rows;
                    tr.generation = gen;
                }
                old.reset();
            } else {
                std::lock_guard<std::mutex> g(mu);
                ++st.refit_failures;
            }
            const std::string msg = rc == AIWCRF_OK ? std::string() : std::string(aiwcrf_last_error());
            lk.lock();
            last_refit_status = rc;
            last_refit_msg = msg;
            refit_running = false;
            ++refits_finished;
            rcv_done.notify_all();
        }
    }

    int enqueue(const std::shared_ptr<Request> &r)
    {
        std::lock_guard<std::mutex> lk(mu);
        if (stop) return fail(AIWCRF_E_INVALID_ARG, "server is shutting down");
        if (r->gated && !cur_sur) return fail(AIWCRF_E_INVALID_ARG, "gated request: the server holds no surrogate");
        if ((int64_t)pending.size() >= sp.max_pending) {
            ++st.rejected;
            return fail(AIWCRF_E_LIMIT, "request refused: max_pending requests are waiting");
        }
        if (r->run == nullptr) {
            r->ticket = next_ticket++;
            tickets[r->ticket] = r;
        }
        pending.push_back(r);
        n_pending.store((int64_t)pending.size());
        ++st.submitted;
        cv_disp.notify_one();
        return AIWCRF_OK;
    }

    void shutdown()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
            cv_disp.notify_all();
        }
        if (disp.joinable()) disp.join();
        {
            std::lock_guard<std::mutex> lk(rmu);
            refit_stop = true;
            rcv.notify_all();
        }
        if (refitter.joinable()) refitter.join();
        current.reset();
        cur_sur.reset();
        drain_graveyard();
        if (refit_stream) cudaStreamSynchronize(refit_stream);
        for (auto &sl : slots) {
            if (sl.s) cudaStreamDestroy(sl.s);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.h_in) cudaFreeHost(sl.h_in);
            if (sl.h_out) cudaFreeHost(sl.h_out);
            if (sl.d_sum) cudaFree(sl.d_sum);
            if (sl.d_cnt) cudaFree(sl.d_cnt);
        }
        if (d_arena) cudaFree(d_arena);
        if (d_dev) cudaFree(d_dev);
        if (refit_stream) cudaStreamDestroy(refit_stream);
    }
};

namespace {

int check_rows(const float *X, const int64_t *y, int64_t n, int32_t F)
{
    for (int64_t i = 0; i < (int64_t)F * n; ++i)
        if (X[i] != X[i]) return fail(AIWCRF_E_NAN_INPUT, "NaN in the training features");
    for (int64_t i = 0; i < n; ++i)
        if (y[i] > AIWCRF_MAX_ABS_Y || y[i] < -AIWCRF_MAX_ABS_Y) return fail(AIWCRF_E_LIMIT, "|y| above 2^40");
    return AIWCRF_OK;
}

}  // namespace

extern "C" {

int aiwcrf_server_create(const aiwcrf_server_params *params, const aiwcrf_fit_params *fit, const float *X,
                         const int64_t *y, int64_t n_rows, int32_t n_features, const int32_t *device_ids,
                         int32_t n_devices, aiwcrf_server **out)
{
    aiwcrf::clear_last_error();
    if (!params || !fit || !X || !y || !device_ids || !out) return fail(AIWCRF_E_INVALID_ARG, "null argument");
    *out = nullptr;
    const aiwcrf_server_params &p = *params;
    if (n_features < 3 || n_features > AIWCRF_MAX_FEATURES || n_rows < 1 || n_rows > AIWCRF_MAX_ROWS)
        return fail(AIWCRF_E_INVALID_ARG, "n_features must be 3..128 and n_rows 1..2^22-1");
    if (n_devices < 1 || n_devices > kServeMaxDevices) return fail(AIWCRF_E_INVALID_ARG, "n_devices must be 1..64");
    if (p.n_streams < 1 || p.n_streams > 16 || p.max_request_kernels < 1 || p.max_request_kernels > 4096 ||
        p.batch_kernels < p.max_request_kernels || p.batch_kernels > 65536 || p.max_pending < 1 ||
        p.arena_bytes < 1 || p.refit_every < 0 || p.refit_rows < 0)
        return fail(AIWCRF_E_INVALID_ARG, "server parameters out of range");
    const int64_t one_request = (int64_t)(up256(sizeof(float) * (size_t)n_features * (size_t)p.max_request_kernels) +
                                          up256((size_t)p.max_request_kernels * ((size_t)n_devices * 8 + 4)));
    if (one_request > p.arena_bytes)
        return fail(AIWCRF_E_INVALID_ARG, "arena_bytes cannot hold one request of max_request_kernels kernels");
    int rc = check_rows(X, y, n_rows, n_features);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");

    auto *s = new aiwcrf_server();
    s->sp = p;
    s->fp = *fit;
    s->F = n_features;
    s->D = n_devices;
    s->device = dev;
    s->dev_ids.assign(device_ids, device_ids + n_devices);
    s->xcols.resize((size_t)n_features);
    s->acols.resize((size_t)n_features);
    for (int32_t f = 0; f < n_features; ++f)
        s->xcols[(size_t)f].assign(X + (size_t)f * (size_t)n_rows, X + (size_t)(f + 1) * (size_t)n_rows);
    s->ytrain.assign(y, y + n_rows);

    auto bail = [&](int code) {
        s->shutdown();
        delete s;
        return code;
    };
    const size_t KB = (size_t)p.batch_kernels, D = (size_t)n_devices;
    // selection batches go first: a refit's many small launches yield the SMs to them
    int prio_low = 0, prio_high = 0;
    e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->refit_stream, cudaStreamNonBlocking, prio_low);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_dev, sizeof(int32_t) * D);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_dev, device_ids, sizeof(int32_t) * D, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, (size_t)p.arena_bytes);
    s->slots.resize((size_t)p.n_streams);
    for (auto &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.s, cudaStreamNonBlocking, prio_high);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_in, sizeof(float) * (size_t)n_features * KB);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, s->layout((int64_t)KB, (int64_t)KB).out_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_sum, sizeof(unsigned long long) * KB * D);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_cnt, sizeof(uint32_t) * KB);
        if (e == cudaSuccess) e = cudaMemset(sl.d_sum, 0, sizeof(unsigned long long) * KB * D);
        if (e == cudaSuccess) e = cudaMemset(sl.d_cnt, 0, sizeof(uint32_t) * KB);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cuda_fail(e, "server set-up");
        return bail(e == cudaErrorMemoryAllocation ? AIWCRF_E_OOM : AIWCRF_E_CUDA);
    }
    s->arena.init(p.arena_bytes);
    s->st.arena_bytes = p.arena_bytes;
    // load both walk variants now: a refit can switch between them, and a kernel's first
    // launch would otherwise load its code in the middle of serving
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, serve_select_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, serve_select_kernel<false>);
    if (e != cudaSuccess) {
        cuda_fail(e, "loading the selection kernels");
        return bail(AIWCRF_E_CUDA);
    }

    aiwcrf_forest *f = nullptr;
    int64_t rows = 0;
    rc = s->fit_training(&f, &rows, false);
    if (rc) return bail(rc);
    s->current = s->wrap(f, 0, rows);
    s->st.generation = 0;
    s->st.training_rows = rows;
    s->st.forest_bytes = s->current->bytes;
    s->disp = std::thread([s] { s->dispatcher(); });
    s->refitter = std::thread([s] { s->refit_loop(); });
    *out = s;
    return AIWCRF_OK;
}

}  // extern "C"

namespace {

int submit_request(aiwcrf_server *server, const float *kfeat, int32_t n_kernels, int32_t size_class, bool gated,
                   int64_t *ticket)
{
    if (!server || !kfeat || !ticket) return fail(AIWCRF_E_INVALID_ARG, "null argument");
    if (n_kernels < 1) return fail(AIWCRF_E_INVALID_ARG, "n_kernels must be >= 1");
    if (n_kernels > server->sp.max_request_kernels ||
        (gated && (int64_t)server->layout(n_kernels, n_kernels).total > server->sp.arena_bytes)) {
        std::lock_guard<std::mutex> lk(server->mu);
        ++server->st.rejected;
        return fail(AIWCRF_E_LIMIT, n_kernels > server->sp.max_request_kernels
                                        ? "request has more than max_request_kernels kernels"
                                        : "a gated request of this size cannot fit the arena");
    }
    auto r = std::make_shared<Request>();
    r->K = n_kernels;
    r->size = size_class;
    r->gated = gated;
    r->own.assign(kfeat, kfeat + (size_t)(server->F - 2) * (size_t)n_kernels);
    r->src = r->own.data();
    r->ld = n_kernels;
    r->t_arrive = now_ns();
    const int rc = server->enqueue(r);
    if (rc == AIWCRF_OK) *ticket = r->ticket;
    return rc;
}

// waits for a ticket of the given kind; on completion retires it and returns the request
int wait_request(aiwcrf_server *server, int64_t ticket, int32_t timeout_ms, bool gated, std::shared_ptr<Request> *out)
{
    if (!server) return fail(AIWCRF_E_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(server->mu);
    auto it = server->tickets.find(ticket);
    if (it == server->tickets.end()) return fail(AIWCRF_E_INVALID_ARG, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (r->gated != gated)
        return fail(AIWCRF_E_INVALID_ARG, gated ? "not a gated request: use aiwcrf_server_wait"
                                                : "a gated request: use aiwcrf_server_wait_gated");
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) server->cv_done.wait(lk, ready);
    else if (!server->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(AIWCRF_E_TIMEOUT, "request still running");
    server->tickets.erase(ticket);
    if (r->status != AIWCRF_OK) return fail(r->status, r->msg);
    *out = r;
    return AIWCRF_OK;
}

}  // namespace

extern "C" {

int aiwcrf_server_submit(aiwcrf_server *server, const float *kfeat, int32_t n_kernels, int32_t size_class,
                         int64_t *ticket)
{
    aiwcrf::clear_last_error();
    return submit_request(server, kfeat, n_kernels, size_class, false, ticket);
}

int aiwcrf_server_submit_gated(aiwcrf_server *server, const float *kfeat, int32_t n_kernels, int32_t size_class,
                               int64_t *ticket)
{
    aiwcrf::clear_last_error();
    return submit_request(server, kfeat, n_kernels, size_class, true, ticket);
}

int aiwcrf_server_wait(aiwcrf_server *server, int64_t ticket, int32_t timeout_ms, int32_t *best, int64_t *pred,
                       int64_t *generation)
{
    aiwcrf::clear_last_error();
    std::shared_ptr<Request> r;
    const int rc = wait_request(server, ticket, timeout_ms, false, &r);
    if (rc) return rc;
    if (best) std::copy(r->best.begin(), r->best.end(), best);
    if (pred) std::copy(r->pred.begin(), r->pred.end(), pred);
    if (generation) *generation = r->generation;
    return AIWCRF_OK;
}

int aiwcrf_server_wait_gated(aiwcrf_server *server, int64_t ticket, int32_t timeout_ms, int32_t *best, float *pred,
                             uint8_t *fallback, int64_t *generation)
{
    aiwcrf::clear_last_error();
    std::shared_ptr<Request> r;
    const int rc = wait_request(server, ticket, timeout_ms, true, &r);
    if (rc) return rc;
    if (best) std::copy(r->best.begin(), r->best.end(), best);
    if (pred) std::copy(r->fpred.begin(), r->fpred.end(), pred);
    if (fallback) std::copy(r->fallback.begin(), r->fallback.end(), fallback);
    if (generation) *generation = r->generation;
    return AIWCRF_OK;
}

int aiwcrf_server_set_surrogate(aiwcrf_server *server, const aiwcrf_surrogate *surrogate,
                                const aiwcrf_gate_params *gate)
{
    aiwcrf::clear_last_error();
    if (!server) return fail(AIWCRF_E_INVALID_ARG, "null server");
    std::shared_ptr<SurModel> sm;
    if (surrogate) {
        if (!gate) return fail(AIWCRF_E_INVALID_ARG, "gate must not be NULL with a surrogate");
        std::shared_ptr<Model> cur;
        {
            std::lock_guard<std::mutex> lk(server->mu);
            cur = server->current;
        }
        int rc = gate_check(cur->f, gate);
        if (rc) return rc;
        const SurrogateInfo si = surrogate_info(surrogate);
        if (si.F != server->F) return fail(AIWCRF_E_INVALID_ARG, "the surrogate's n_features differs from the server's");
        if (si.device != server->device) return fail(AIWCRF_E_INVALID_ARG, "the surrogate is on another device");
        aiwcrf_surrogate *copy = nullptr;
        if ((rc = surrogate_clone(surrogate, &copy))) return rc;
        sm = server->wrap_surrogate(copy, *gate);
    }
    std::shared_ptr<SurModel> old;
    std::vector<std::shared_ptr<Request>> drop;
    {
        std::lock_guard<std::mutex> lk(server->mu);
        old = server->cur_sur;
        server->cur_sur = sm;
        server->st.surrogate_bytes = sm ? sm->bytes : 0;
        if (!sm) {
            // queued gated requests can no longer be answered
            std::deque<std::shared_ptr<Request>> keep;
            for (auto &r : server->pending) {
                if (r->gated) drop.push_back(r);
                else keep.push_back(r);
            }
            if (!drop.empty()) {
                server->pending.swap(keep);
                server->n_pending.store((int64_t)server->pending.size());
            }
        }
    }
    old.reset();
    for (auto &r : drop)
        server->finish(r, AIWCRF_E_INVALID_ARG, "gated request: the server's surrogate was removed", -1, nullptr,
                       nullptr, now_ns());
    return AIWCRF_OK;
}

int aiwcrf_server_append(aiwcrf_server *server, const float *X, const int64_t *y, int64_t n_rows)
{
    aiwcrf::clear_last_error();
    if (!server || !X || !y) return fail(AIWCRF_E_INVALID_ARG, "null argument");
    if (n_rows < 0) return fail(AIWCRF_E_INVALID_ARG, "n_rows < 0");
    int rc = check_rows(X, y, n_rows, server->F);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(server->rmu);
    if ((int64_t)server->ytrain.size() + (int64_t)server->yapp.size() + n_rows > AIWCRF_MAX_ROWS)
        return fail(AIWCRF_E_LIMIT, "training rows would exceed 2^22-1");
    for (int32_t f = 0; f < server->F; ++f)
        server->acols[(size_t)f].insert(server->acols[(size_t)f].end(), X + (size_t)f * (size_t)n_rows,
                                        X + (size_t)(f + 1) * (size_t)n_rows);
    server->yapp.insert(server->yapp.end(), y, y + n_rows);
    return AIWCRF_OK;
}

int aiwcrf_server_refit(aiwcrf_server *server, int32_t wait)
{
    aiwcrf::clear_last_error();
    if (!server) return fail(AIWCRF_E_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(server->rmu);
    // a refit already running read its rows before this call: wait for the one after it
    const int64_t target = server->refits_finished + 1 + (server->refit_running ? 1 : 0);
    server->refit_req = true;
    server->rcv.notify_all();
    if (!wait) return AIWCRF_OK;
    server->rcv_done.wait(lk, [&] { return server->refits_finished >= target || server->refit_stop; });
    if (server->last_refit_status != AIWCRF_OK) return fail(server->last_refit_status, "refit failed: " + server->last_refit_msg);
    return AIWCRF_OK;
}

int aiwcrf_server_pause(aiwcrf_server *server, int32_t paused)
{
    aiwcrf::clear_last_error();
    if (!server) return fail(AIWCRF_E_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(server->mu);
    server->paused = paused != 0;
    server->cv_disp.notify_all();
    return AIWCRF_OK;
}

int aiwcrf_server_stats(aiwcrf_server *server, aiwcrf_server_counters *out)
{
    aiwcrf::clear_last_error();
    if (!server || !out) return fail(AIWCRF_E_INVALID_ARG, "null argument");
    {
        std::lock_guard<std::mutex> lk(server->mu);
        *out = server->st;
        out->arena_peak_bytes = server->arena.peak;
    }
    std::lock_guard<std::mutex> lk(server->rmu);
    out->appended_rows = (int64_t)server->yapp.size();
    return AIWCRF_OK;
}

}  // extern "C"

namespace {

int run_load(aiwcrf_server *server, const float *pool, int64_t pool_kernels, const int64_t *first,
             const int32_t *n_kernels, const int32_t *size_class, const uint8_t *gated, int64_t n_requests,
             double rate_per_s, uint64_t seed, int32_t timeout_ms, int32_t *best, int64_t *generation,
             int64_t *latency_ns, aiwcrf_load_report *report)
{
    if (!server || !pool || !first || !n_kernels || !size_class || !report)
        return fail(AIWCRF_E_INVALID_ARG, "null argument");
    if (n_requests < 1 || !(rate_per_s > 0.0) || pool_kernels < 1)
        return fail(AIWCRF_E_INVALID_ARG, "n_requests, rate and pool size must be positive");
    std::vector<int64_t> best_off((size_t)n_requests);
    int64_t total_k = 0;
    for (int64_t i = 0; i < n_requests; ++i) {
        if (n_kernels[i] < 1 || first[i] < 0 || first[i] + n_kernels[i] > pool_kernels)
            return fail(AIWCRF_E_INVALID_ARG, "request outside the kernel pool");
        best_off[(size_t)i] = total_k;
        total_k += n_kernels[i];
    }
    auto run = std::make_shared<LoadRun>();
    run->remaining = n_requests;
    run->best = best;
    run->gen = generation;
    run->lat.assign((size_t)n_requests, -1);
    aiwcrf_server_counters s0;
    aiwcrf_server_stats(server, &s0);

    // arrival times of a Poisson process: exponential gaps by inversion of SplitMix64 uniforms
    SplitMix64 rng{seed};
    std::vector<int64_t> arrive((size_t)n_requests);
    const int64_t t0 = now_ns() + 1000000;
    double t = 0.0;
    for (int64_t i = 0; i < n_requests; ++i) {
        const double u = (double)(rng.next() >> 11) * 0x1.0p-53;
        t += -std::log1p(-u) / rate_per_s;
        arrive[(size_t)i] = t0 + (int64_t)(t * 1e9);
    }
    int64_t rejected = 0;
    for (int64_t i = 0; i < n_requests; ++i) {
        for (;;) {
            const int64_t d = arrive[(size_t)i] - now_ns();
            if (d <= 0) break;
            if (d > 300000) std::this_thread::sleep_for(std::chrono::nanoseconds(d - 200000));
            else std::this_thread::yield();
        }
        auto r = std::make_shared<Request>();
        r->K = n_kernels[i];
        r->size = size_class[i];
        r->src = pool + first[i];
        r->ld = pool_kernels;
        r->t_arrive = arrive[(size_t)i];
        r->run = run;
        r->run_index = i;
        r->run_best_off = best_off[(size_t)i];
        r->gated = gated && gated[i];
        const bool too_big = r->K > server->sp.max_request_kernels ||
                             (r->gated && (int64_t)server->layout(r->K, r->K).total > server->sp.arena_bytes);
        int rc = too_big ? AIWCRF_E_LIMIT : server->enqueue(r);
        if (rc != AIWCRF_OK) {
            std::lock_guard<std::mutex> lk(run->mu);
            --run->remaining;
            ++rejected;
        }
    }
    bool timed_out = false;
    {
        std::unique_lock<std::mutex> lk(run->mu);
        auto done = [&] { return run->remaining == 0; };
        if (timeout_ms < 0) run->cv.wait(lk, done);
        else timed_out = !run->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    }
    if (timed_out) {
        // stop reading the caller's pool and writing its outputs
        {
            std::lock_guard<std::mutex> lk(server->mu);
            std::deque<std::shared_ptr<Request>> keep;
            for (auto &r : server->pending)
                if (r->run != run) keep.push_back(r);
            server->pending.swap(keep);
            server->n_pending.store((int64_t)server->pending.size());
        }
        std::lock_guard<std::mutex> lk(run->mu);
        run->abandoned = true;
    }
    aiwcrf_server_counters s1;
    aiwcrf_server_stats(server, &s1);

    std::vector<int64_t> lat;
    int64_t t_last = 0;
    for (int64_t i = 0; i < n_requests; ++i) {
        const int64_t l = run->lat[(size_t)i];
        if (latency_ns) latency_ns[i] = l;
        if (l >= 0) {
            lat.push_back(l);
            t_last = std::max(t_last, arrive[(size_t)i] + l);
        }
    }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        size_t r = (size_t)std::ceil(p * (double)lat.size());
        r = std::min(std::max<size_t>(r, 1), lat.size());
        return (double)lat[r - 1] * 1e-3;
    };
    std::memset(report, 0, sizeof(*report));
    report->n_requests = (int64_t)lat.size();
    report->n_kernels = total_k;
    report->offered_rate = rate_per_s;
    report->wall_s = lat.empty() ? 0.0 : (double)(t_last - arrive[0]) * 1e-9;
    report->requests_per_s = report->wall_s > 0 ? (double)lat.size() / report->wall_s : 0.0;
    report->kernels_per_s = report->wall_s > 0 ? (double)total_k / report->wall_s : 0.0;
    report->p50_us = pct(0.50);
    report->p99_us = pct(0.99);
    double sum = 0.0;
    for (auto l : lat) sum += (double)l;
    report->mean_us = lat.empty() ? 0.0 : sum / (double)lat.size() * 1e-3;
    report->max_us = lat.empty() ? 0.0 : (double)lat.back() * 1e-3;
    report->batches = s1.batches - s0.batches;
    report->mean_batch_kernels =
        report->batches ? (double)(s1.batch_kernels_total - s0.batch_kernels_total) / (double)report->batches : 0.0;
    report->refits = s1.refits - s0.refits;
    report->failed = n_requests - (int64_t)lat.size() - rejected;
    report->rejected = rejected;
    if (timed_out) return fail(AIWCRF_E_TIMEOUT, "requests still running at the time limit");
    if (run->first_error != AIWCRF_OK) return fail(run->first_error, "a request failed");
    return AIWCRF_OK;
}

}  // namespace

extern "C" {

int aiwcrf_server_run_load(aiwcrf_server *server, const float *pool, int64_t pool_kernels, const int64_t *first,
                           const int32_t *n_kernels, const int32_t *size_class, int64_t n_requests, double rate_per_s,
                           uint64_t seed, int32_t timeout_ms, int32_t *best, int64_t *generation, int64_t *latency_ns,
                           aiwcrf_load_report *report)
{
    aiwcrf::clear_last_error();
    return run_load(server, pool, pool_kernels, first, n_kernels, size_class, nullptr, n_requests, rate_per_s, seed,
                    timeout_ms, best, generation, latency_ns, report);
}

int aiwcrf_server_run_load_gated(aiwcrf_server *server, const float *pool, int64_t pool_kernels, const int64_t *first,
                                 const int32_t *n_kernels, const int32_t *size_class, const uint8_t *gated,
                                 int64_t n_requests, double rate_per_s, uint64_t seed, int32_t timeout_ms,
                                 int32_t *best, int64_t *generation, int64_t *latency_ns, aiwcrf_load_report *report)
{
    aiwcrf::clear_last_error();
    return run_load(server, pool, pool_kernels, first, n_kernels, size_class, gated, n_requests, rate_per_s, seed,
                    timeout_ms, best, generation, latency_ns, report);
}

int aiwcrf_server_trace(aiwcrf_server *server, aiwcrf_batch_trace *batches, int64_t cap, int64_t *n,
                        aiwcrf_refit_trace *refits, int64_t rcap, int64_t *rn)
{
    aiwcrf::clear_last_error();
    if (!server || !n || !rn || cap < 0 || rcap < 0 || (cap && !batches) || (rcap && !refits))
        return fail(AIWCRF_E_INVALID_ARG, "bad trace arguments");
    std::lock_guard<std::mutex> lk(server->mu);
    auto copy = [](const auto &ring, int64_t total, int64_t ring_n, auto *dst, int64_t want) {
        const int64_t have = std::min(total, ring_n);
        const int64_t m = std::min(have, want);
        for (int64_t i = 0; i < m; ++i) dst[i] = ring[(size_t)((total - m + i) % ring_n)];
        return m;
    };
    *n = copy(server->btrace, server->n_btrace, aiwcrf_server::kBatchRing, batches, cap);
    *rn = copy(server->rtrace, server->n_rtrace, aiwcrf_server::kRefitRing, refits, rcap);
    return AIWCRF_OK;
}

int aiwcrf_server_destroy(aiwcrf_server *server)
{
    aiwcrf::clear_last_error();
    if (!server) return AIWCRF_OK;
    server->shutdown();
    delete server;
    return AIWCRF_OK;
}

}  // extern "C"

namespace aiwcrf {
AIWCRF_BOUNDS_READER(bounds_flags_serve)
}  // namespace aiwcrf
