// api.cu -- the extern "C" boundary declared in include/aiwcrf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace aiwcrf {

static thread_local std::string g_last_error;

void clear_last_error() { g_last_error.clear(); }

void set_error(int code, const std::string &msg)
{
    g_last_error = "aiwcrf error " + std::to_string(code) + ": " + msg;
}

int fail(int code, const std::string &msg)
{
    set_error(code, msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // clear a sticky launch error where possible
    return fail(AIWCRF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void forest_release(aiwcrf_forest *f)
{
    if (!f) return;
    // callers may still have work reading the forest in flight on any stream
    cudaDeviceSynchronize();
    if (f->d_block) cudaFreeAsync(f->d_block, cudaStreamPerThread);
    cudaStreamSynchronize(cudaStreamPerThread);
    delete f;
}

void forest_release_async(aiwcrf_forest *f, cudaStream_t s)
{
    if (!f) return;
    if (f->d_block) cudaFreeAsync(f->d_block, s);
    delete f;
}

cudaError_t forest_alloc(aiwcrf_forest *f, cudaStream_t s)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // compact layout: trees padded to a multiple of four nodes
    std::vector<int64_t> off4((size_t)f->T + 1, 0);
    f->max_tree4 = 0;
    for (int64_t t = 0; t < f->T; ++t) {
        const int64_t m = f->tree_off[(size_t)t + 1] - f->tree_off[(size_t)t];
        const int64_t m4 = (m + 3) & ~(int64_t)3;
        off4[(size_t)t + 1] = off4[(size_t)t] + m4;
        f->max_tree4 = std::max(f->max_tree4, m4);
    }
    f->compact = f->max_card <= 255u && f->max_tree_nodes <= 65536 && f->F <= 128;
    f->num_c32 = f->compact ? off4[(size_t)f->T] : 0;
    const size_t nn = (size_t)std::max<int64_t>(f->num_nodes, 2);
    const size_t b_nodes = up(8 * nn), b_off = up(8 * (size_t)(f->T + 1));
    const size_t b_vals = up(sizeof(float) * (size_t)f->F * (size_t)f->fstride), b_card = up(4 * (size_t)f->F);
    const size_t b_c32 = f->compact ? up(4 * (size_t)f->num_c32) + b_off : 0;
    const size_t b_inbag = up(4 * (size_t)f->T * (size_t)f->inbag_words);
    void *p = nullptr;
    keep_pool_memory(f->device);
    // stream-ordered, so that freeing a forest never waits for the whole device
    cudaError_t e = cudaMallocAsync(&p, 2 * b_nodes + b_off + b_vals + b_card + b_c32 + b_inbag, s);
    if (e != cudaSuccess) return e;
    unsigned char *c = static_cast<unsigned char *>(p);
    f->d_block = p;
    f->d_nodes = reinterpret_cast<uint64_t *>(c);
    f->d_cnodes = reinterpret_cast<uint64_t *>(c + b_nodes);
    f->d_tree_off = reinterpret_cast<int64_t *>(c + 2 * b_nodes);
    f->d_fvals = reinterpret_cast<float *>(c + 2 * b_nodes + b_off);
    f->d_fcard = reinterpret_cast<uint32_t *>(c + 2 * b_nodes + b_off + b_vals);
    if (f->inbag_words) f->d_inbag = reinterpret_cast<uint32_t *>(c + 2 * b_nodes + b_off + b_vals + b_card + b_c32);
    if (f->compact) {
        unsigned char *q = c + 2 * b_nodes + b_off + b_vals + b_card;
        f->d_tree_off4 = reinterpret_cast<int64_t *>(q);
        f->d_c32 = reinterpret_cast<uint32_t *>(q + b_off);
        e = cudaMemcpyAsync(f->d_tree_off4, off4.data(), 8 * (size_t)(f->T + 1), cudaMemcpyHostToDevice, s);
    }
    return e;
}

void keep_pool_memory(int device)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[device] = true;
}

void *pinned_scratch()
{
    struct Buf {
        void *p = nullptr;
        ~Buf() { if (p) cudaFreeHost(p); }
    };
    static thread_local Buf b;
    if (!b.p && cudaMallocHost(&b.p, kPinnedScratchBytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
    }
    return b.p;
}

static std::atomic<long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- profiling (CUDA events)
namespace {
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
uint32_t g_prof_mask = ~0u;       // kernel classes that record events while profiling is on
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;
thread_local std::vector<std::pair<int, cudaEvent_t>> t_open;

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

const char *kProfNames[kProfNum] = {"rank",    "bootstrap", "level_big", "level_small", "finalize",
                                    "pack",    "predict",   "select",    "serve",       "tree",
                                    "walk",    "list_partition"};
}  // namespace

// Every kernel class bracket is also an NVTX range on the launching host thread (a profiler's
// timeline groups each pass's launches under its name); profiling by events is separate.
void prof_begin(cudaStream_t s, int cls)
{
    nvtxRangePushA(kProfNames[cls]);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || !((g_prof_mask >> cls) & 1u)) return;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    t_open.push_back({cls, e});
}

void prof_end(cudaStream_t s, int cls)
{
    nvtxRangePop();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || !((g_prof_mask >> cls) & 1u)) return;
    for (size_t i = t_open.size(); i-- > 0;) {
        if (t_open[i].first == cls) {
            cudaEvent_t b = take_event();
            cudaEventRecord(b, s);
            g_prof.push_back({cls, t_open[i].second, b});
            t_open.erase(t_open.begin() + (long)i);
            return;
        }
    }
}

// ---------------------------------------------------------------- pointer staging
namespace {

enum PtrKind { kPtrHost, kPtrDevice, kPtrBad };

PtrKind classify(const void *p, int device)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return kPtrHost;
    }
    switch (at.type) {
    case cudaMemoryTypeUnregistered:
    case cudaMemoryTypeHost:
        return kPtrHost;
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
        return at.device == device ? kPtrDevice : kPtrBad;
    default:
        return kPtrBad;
    }
}

// An input array: device pointers pass through; host arrays are copied to a stream-ordered
// device buffer.
struct InArg {
    const void *dev = nullptr;
    void *owned = nullptr;
    cudaStream_t s = nullptr;
    ~InArg() { if (owned) cudaFreeAsync(owned, s); }
};

// The device address of page-locked host memory the device can read in place, or null.
const void *mapped_host(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// read_in_place: an input that one kernel streams through once may be read by the device
// straight from page-locked host memory (no staging buffer, no separate copy)
int stage_in(InArg &a, const void *p, size_t bytes, int device, cudaStream_t s, const char *name,
             bool read_in_place = false)
{
    a.s = s;
    const PtrKind k = classify(p, device);
    if (k == kPtrBad) return fail(AIWCRF_E_BAD_POINTER, std::string(name) + " is memory of another device");
    if (k == kPtrDevice) { a.dev = p; return AIWCRF_OK; }
    if (read_in_place && bytes) {
        if (const void *dp = mapped_host(p)) { a.dev = dp; return AIWCRF_OK; }
    }
    cudaError_t e = cudaMallocAsync(&a.owned, bytes ? bytes : 1, s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, std::string("staging ") + name + ": " + cudaGetErrorString(e));
    if (bytes) {
        e = cudaMemcpyAsync(a.owned, p, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, name);
    }
    a.dev = a.owned;
    return AIWCRF_OK;
}

// An output array: device pointers pass through; host arrays get a device buffer that is
// copied back by finish().
struct OutArg {
    void *dev = nullptr;
    void *owned = nullptr;
    void *host = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    ~OutArg() { if (owned) cudaFreeAsync(owned, s); }
};

int stage_out(OutArg &a, void *p, size_t bytes, int device, cudaStream_t s, const char *name)
{
    a.s = s;
    if (!p) return AIWCRF_OK;
    const PtrKind k = classify(p, device);
    if (k == kPtrBad) return fail(AIWCRF_E_BAD_POINTER, std::string(name) + " is memory of another device");
    if (k == kPtrDevice) { a.dev = p; return AIWCRF_OK; }
    cudaError_t e = cudaMallocAsync(&a.owned, bytes ? bytes : 1, s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, std::string("staging ") + name + ": " + cudaGetErrorString(e));
    a.dev = a.owned;
    a.host = p;
    a.bytes = bytes;
    return AIWCRF_OK;
}

int finish_out(OutArg &a)
{
    if (!a.host || !a.bytes) return AIWCRF_OK;
    cudaError_t e = cudaMemcpyAsync(a.host, a.dev, a.bytes, cudaMemcpyDeviceToHost, a.s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of an output to the host");
    return AIWCRF_OK;
}

int sync_if(bool any_host, cudaStream_t s)
{
    if (!any_host) return AIWCRF_OK;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return AIWCRF_OK;
}

int current_device(int *dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
    return AIWCRF_OK;
}

int check_params(const aiwcrf_fit_params *p, int64_t n_rows, int32_t n_features)
{
    if (!p) return fail(AIWCRF_E_INVALID_ARG, "params is NULL");
    if (p->num_trees < 1 || p->num_trees > AIWCRF_MAX_TREES)
        return fail(AIWCRF_E_INVALID_ARG, "num_trees must be in [1, 2^20]");
    if (p->mtry < 1) return fail(AIWCRF_E_INVALID_ARG, "mtry must be >= 1");
    if (p->min_node_size < 1) return fail(AIWCRF_E_INVALID_ARG, "min_node_size must be >= 1");
    if (p->max_depth < 0) return fail(AIWCRF_E_INVALID_ARG, "max_depth must be >= 0");
    if (p->bootstrap != 0 && p->bootstrap != 1) return fail(AIWCRF_E_INVALID_ARG, "bootstrap must be 0 or 1");
    if (p->ctas_per_sm < 0 || p->ctas_per_sm > 3) return fail(AIWCRF_E_INVALID_ARG, "ctas_per_sm must be 0..3");
    if (p->first_tree < 0 || p->first_tree + p->num_trees > 0xFFFFFFFFll)
        return fail(AIWCRF_E_INVALID_ARG, "first_tree out of range");
    if (n_rows < 1) return fail(AIWCRF_E_INVALID_ARG, "n_rows must be >= 1");
    if (n_rows > AIWCRF_MAX_ROWS) return fail(AIWCRF_E_LIMIT, "n_rows exceeds 2^22 - 1");
    if (n_features < 1 || n_features > AIWCRF_MAX_FEATURES)
        return fail(AIWCRF_E_INVALID_ARG, "n_features must be in [1, 128]");
    return AIWCRF_OK;
}

}  // namespace
}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" {

const char *aiwcrf_last_error(void) { return g_last_error.c_str(); }

int aiwcrf_fit(const aiwcrf_fit_params *params, const float *X, const int64_t *y, int64_t n_rows,
               int32_t n_features, void *cuda_stream, aiwcrf_forest **out)
{
    g_last_error.clear();
    int rc = check_params(params, n_rows, n_features);
    if (rc) return rc;
    if (!X || !y || !out) return fail(AIWCRF_E_INVALID_ARG, "X, y and out must not be NULL");
    int dev;
    if ((rc = current_device(&dev))) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InArg ax, ay;
    if ((rc = stage_in(ax, X, sizeof(float) * (size_t)n_features * (size_t)n_rows, dev, s, "X"))) return rc;
    if ((rc = stage_in(ay, y, sizeof(int64_t) * (size_t)n_rows, dev, s, "y"))) return rc;
    std::vector<aiwcrf_forest *> fs;
    rc = fit_batch(*params, (const float *)ax.dev, (const int64_t *)ay.dev, n_rows, n_features, {}, nullptr, 1, s, fs);
    if (rc) return rc;
    *out = fs[0];
    return AIWCRF_OK;
}

int aiwcrf_fit_subsets(const aiwcrf_fit_params *params, const float *X, const int64_t *y, int64_t n_rows,
                       int32_t n_features, const int64_t *subset_offsets, const int32_t *subset_rows,
                       int32_t n_subsets, void *cuda_stream, aiwcrf_forest **out)
{
    g_last_error.clear();
    int rc = check_params(params, n_rows, n_features);
    if (rc) return rc;
    if (!X || !y || !out || !subset_offsets || !subset_rows || n_subsets < 1)
        return fail(AIWCRF_E_INVALID_ARG, "X, y, subsets and out must be given, n_subsets >= 1");
    if ((int64_t)n_subsets * params->num_trees > (int64_t)AIWCRF_MAX_TREES * 16)
        return fail(AIWCRF_E_LIMIT, "too many trees in one batch");
    int dev;
    if ((rc = current_device(&dev))) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int64_t> off(subset_offsets, subset_offsets + n_subsets + 1);
    if (off[0] != 0) return fail(AIWCRF_E_INVALID_ARG, "subset_offsets[0] must be 0");
    for (int32_t g = 0; g < n_subsets; ++g)
        if (off[(size_t)g + 1] <= off[(size_t)g]) return fail(AIWCRF_E_INVALID_ARG, "every subset needs >= 1 row");
    const int64_t total = off[(size_t)n_subsets];
    // row validity (increasing, within range) is checked on the host copy
    std::vector<int32_t> rows((size_t)total);
    if (classify(subset_rows, dev) == kPtrDevice) {
        cudaError_t e = cudaMemcpyAsync(rows.data(), subset_rows, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading subset_rows");
    } else {
        std::memcpy(rows.data(), subset_rows, sizeof(int32_t) * (size_t)total);
    }
    for (int32_t g = 0; g < n_subsets; ++g)
        for (int64_t k = off[(size_t)g]; k < off[(size_t)g + 1]; ++k) {
            if (rows[(size_t)k] < 0 || rows[(size_t)k] >= n_rows || (k > off[(size_t)g] && rows[(size_t)k] <= rows[(size_t)k - 1]))
                return fail(AIWCRF_E_INVALID_ARG, "subset rows must be strictly increasing row indices");
        }
    InArg ax, ay, ar;
    if ((rc = stage_in(ax, X, sizeof(float) * (size_t)n_features * (size_t)n_rows, dev, s, "X"))) return rc;
    if ((rc = stage_in(ay, y, sizeof(int64_t) * (size_t)n_rows, dev, s, "y"))) return rc;
    if ((rc = stage_in(ar, rows.data(), sizeof(int32_t) * (size_t)total, dev, s, "subset_rows"))) return rc;
    std::vector<aiwcrf_forest *> fs;
    rc = fit_batch(*params, (const float *)ax.dev, (const int64_t *)ay.dev, n_rows, n_features, off,
                   (const int32_t *)ar.dev, n_subsets, s, fs);
    if (rc) return rc;
    for (int32_t g = 0; g < n_subsets; ++g) out[g] = fs[(size_t)g];
    cudaStreamSynchronize(s);   // the staged host copy of the rows must outlive its transfer
    return AIWCRF_OK;
}

struct aiwcrf_fit_plan {
    aiwcrf::FitPlan *impl = nullptr;
    int32_t n_forests = 1;
};

int aiwcrf_fit_plan_create(const aiwcrf_fit_params *params, const float *X, const int64_t *y, int64_t n_rows,
                           int32_t n_features, const int64_t *subset_offsets, const int32_t *subset_rows,
                           int32_t n_subsets, void *cuda_stream, aiwcrf_fit_plan **out)
{
    g_last_error.clear();
    int rc = check_params(params, n_rows, n_features);
    if (rc) return rc;
    if (!X || !y || !out) return fail(AIWCRF_E_INVALID_ARG, "X, y and out must not be NULL");
    *out = nullptr;
    int dev;
    if ((rc = current_device(&dev))) return rc;
    if (classify(X, dev) != kPtrDevice || classify(y, dev) != kPtrDevice ||
        (subset_rows && classify(subset_rows, dev) != kPtrDevice))
        return fail(AIWCRF_E_BAD_POINTER, "a fit plan binds device memory: X, y and subset_rows must be on the device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int64_t> off;
    int32_t G = 1;
    if (subset_rows) {
        if (!subset_offsets || n_subsets < 1) return fail(AIWCRF_E_INVALID_ARG, "subset_offsets and n_subsets >= 1 needed");
        if ((int64_t)n_subsets * params->num_trees > (int64_t)AIWCRF_MAX_TREES * 16)
            return fail(AIWCRF_E_LIMIT, "too many trees in one batch");
        off.assign(subset_offsets, subset_offsets + n_subsets + 1);
        if (off[0] != 0) return fail(AIWCRF_E_INVALID_ARG, "subset_offsets[0] must be 0");
        for (int32_t g = 0; g < n_subsets; ++g)
            if (off[(size_t)g + 1] <= off[(size_t)g]) return fail(AIWCRF_E_INVALID_ARG, "every subset needs >= 1 row");
        const int64_t total = off[(size_t)n_subsets];
        std::vector<int32_t> rows((size_t)total);
        cudaError_t e = cudaMemcpyAsync(rows.data(), subset_rows, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading subset_rows");
        for (int32_t g = 0; g < n_subsets; ++g)
            for (int64_t k = off[(size_t)g]; k < off[(size_t)g + 1]; ++k)
                if (rows[(size_t)k] < 0 || rows[(size_t)k] >= n_rows ||
                    (k > off[(size_t)g] && rows[(size_t)k] <= rows[(size_t)k - 1]))
                    return fail(AIWCRF_E_INVALID_ARG, "subset rows must be strictly increasing row indices");
        G = n_subsets;
    }
    aiwcrf::FitPlan *impl = nullptr;
    if ((rc = aiwcrf::fit_plan_create(*params, X, y, n_rows, n_features, off, subset_rows, G, s, &impl))) return rc;
    auto *pl = new aiwcrf_fit_plan();
    pl->impl = impl;
    pl->n_forests = G;
    *out = pl;
    return AIWCRF_OK;
}

int aiwcrf_fit_plan_run(aiwcrf_fit_plan *plan, void *cuda_stream, aiwcrf_forest **out)
{
    g_last_error.clear();
    if (!plan || !out) return fail(AIWCRF_E_INVALID_ARG, "plan and out must not be NULL");
    std::vector<aiwcrf_forest *> fs;
    const int rc = aiwcrf::fit_plan_run(plan->impl, (cudaStream_t)cuda_stream, fs);
    if (rc) return rc;
    for (size_t g = 0; g < fs.size(); ++g) out[g] = fs[g];
    return AIWCRF_OK;
}

int aiwcrf_fit_plan_set_schedule(aiwcrf_fit_plan *plan, const aiwcrf_fit_schedule *schedule)
{
    g_last_error.clear();
    if (!plan || !schedule) return fail(AIWCRF_E_INVALID_ARG, "plan and schedule must not be NULL");
    return aiwcrf::fit_plan_set_schedule(plan->impl, schedule->level_big_ctas_per_sm, schedule->level_small_ctas_per_sm);
}

int aiwcrf_fit_plan_tune(aiwcrf_fit_plan *plan, int32_t reps, void *cuda_stream, aiwcrf_fit_schedule *tried,
                         int32_t cap, int32_t *n_tried, aiwcrf_fit_schedule *chosen)
{
    g_last_error.clear();
    if (!plan || reps < 1 || cap < 0 || (cap > 0 && !tried))
        return fail(AIWCRF_E_INVALID_ARG, "plan, reps >= 1 and a tried array of cap entries are needed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<aiwcrf_fit_schedule> all;
    int max_big = 3, max_small = 4;
    aiwcrf::fit_plan_limits(&max_big, &max_small);
    for (int big = 1; big <= max_big; ++big)
        for (int small = 1; small <= max_small; ++small) {
            int rc = aiwcrf::fit_plan_set_schedule(plan->impl, big, small);
            if (rc) return rc;
            std::vector<double> ts;
            for (int r = 0; r <= reps; ++r) {              // one warm-up run
                std::vector<aiwcrf_forest *> fs;
                const auto t0 = std::chrono::steady_clock::now();
                rc = aiwcrf::fit_plan_run(plan->impl, s, fs);
                const auto t1 = std::chrono::steady_clock::now();
                for (auto f : fs) forest_release(f);
                if (rc) return rc;
                if (r > 0) ts.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            std::sort(ts.begin(), ts.end());
            aiwcrf_fit_schedule sc;
            sc.level_big_ctas_per_sm = big;
            sc.level_small_ctas_per_sm = small;
            sc.ms = (float)ts[ts.size() / 2];
            sc.reserved = 0;
            all.push_back(sc);
        }
    size_t bi = 0;
    for (size_t i = 1; i < all.size(); ++i)
        if (all[i].ms < all[bi].ms) bi = i;
    int rc = aiwcrf::fit_plan_set_schedule(plan->impl, all[bi].level_big_ctas_per_sm, all[bi].level_small_ctas_per_sm);
    if (rc) return rc;
    for (int32_t i = 0; i < cap && (size_t)i < all.size(); ++i) tried[i] = all[(size_t)i];
    if (n_tried) *n_tried = (int32_t)all.size();
    if (chosen) *chosen = all[bi];
    return AIWCRF_OK;
}

int aiwcrf_fit_plan_free(aiwcrf_fit_plan *plan)
{
    g_last_error.clear();
    if (!plan) return AIWCRF_OK;
    cudaDeviceSynchronize();
    aiwcrf::fit_plan_free(plan->impl);
    delete plan;
    return AIWCRF_OK;
}

static int predict_common(const aiwcrf_forest *f, const float *Xq, int64_t Q, int64_t *out_sum, int64_t *out_pred,
                          uint64_t *out_var, void *cuda_stream)
{
    if (!f) return fail(AIWCRF_E_INVALID_ARG, "forest is NULL");
    if (Q < 0 || Q > ((int64_t)1 << 36)) return fail(AIWCRF_E_INVALID_ARG, "n_queries out of range");
    if (Q > 0 && !Xq) return fail(AIWCRF_E_INVALID_ARG, "Xq is NULL");
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    if (dev != f->device) return fail(AIWCRF_E_BAD_POINTER, "the forest lives on another device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InArg aq;
    OutArg os, op, ov;
    if (Q == 0) return AIWCRF_OK;
    // the query features are read once, by the coding kernel: page-locked host memory in place
    if ((rc = stage_in(aq, Xq, sizeof(float) * (size_t)f->F * (size_t)Q, dev, s, "Xq", true))) return rc;
    if ((rc = stage_out(os, out_sum, sizeof(int64_t) * (size_t)Q, dev, s, "out_sum"))) return rc;
    if ((rc = stage_out(op, out_pred, sizeof(int64_t) * (size_t)Q, dev, s, "out_pred"))) return rc;
    if ((rc = stage_out(ov, out_var, 2 * sizeof(uint64_t) * (size_t)Q, dev, s, "out_var"))) return rc;
    rc = predict_launch(f, (const float *)aq.dev, Q, (int64_t *)os.dev, (int64_t *)op.dev, (uint64_t *)ov.dev,
                        f->T, s);
    if (rc) return rc;
    if ((rc = finish_out(os)) || (rc = finish_out(op)) || (rc = finish_out(ov))) return rc;
    return sync_if(os.host || op.host || ov.host, s);
}

int aiwcrf_predict(const aiwcrf_forest *forest, const float *Xq, int64_t n_queries, int64_t *out_pred,
                   uint64_t *out_var, void *cuda_stream)
{
    g_last_error.clear();
    if (!out_pred) return fail(AIWCRF_E_INVALID_ARG, "out_pred is NULL");
    return predict_common(forest, Xq, n_queries, nullptr, out_pred, out_var, cuda_stream);
}

int aiwcrf_predict_sum(const aiwcrf_forest *forest, const float *Xq, int64_t n_queries, int64_t *out_sum,
                       void *cuda_stream)
{
    g_last_error.clear();
    if (!out_sum) return fail(AIWCRF_E_INVALID_ARG, "out_sum is NULL");
    return predict_common(forest, Xq, n_queries, out_sum, nullptr, nullptr, cuda_stream);
}

int aiwcrf_oob(const aiwcrf_forest *forest, const float *X, int64_t n_rows, int64_t *out_sum, int32_t *out_count,
               void *cuda_stream)
{
    g_last_error.clear();
    if (!forest || !X || !out_sum || !out_count) return fail(AIWCRF_E_INVALID_ARG, "arguments must not be NULL");
    if (forest->oob_rows == 0)
        return fail(AIWCRF_E_INVALID_ARG, "out-of-bag evaluation needs a forest fitted by aiwcrf_fit in this process");
    if (n_rows != forest->oob_rows) return fail(AIWCRF_E_INVALID_ARG, "n_rows differs from the training matrix");
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    if (dev != forest->device) return fail(AIWCRF_E_BAD_POINTER, "the forest lives on another device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InArg ax;
    OutArg os, oc;
    if ((rc = stage_in(ax, X, sizeof(float) * (size_t)forest->F * (size_t)n_rows, dev, s, "X"))) return rc;
    if ((rc = stage_out(os, out_sum, sizeof(int64_t) * (size_t)n_rows, dev, s, "out_sum"))) return rc;
    if ((rc = stage_out(oc, out_count, sizeof(int32_t) * (size_t)n_rows, dev, s, "out_count"))) return rc;
    if ((rc = oob_launch(forest, (const float *)ax.dev, n_rows, (int64_t *)os.dev, (int32_t *)oc.dev, s))) return rc;
    if ((rc = finish_out(os)) || (rc = finish_out(oc))) return rc;
    return sync_if(os.host || oc.host, s);
}

int aiwcrf_oob_error(const aiwcrf_forest *forest, const float *X, const int64_t *y, int64_t n_rows, int64_t *out_pred,
                     double *out_mse, int64_t *out_rows, void *cuda_stream)
{
    g_last_error.clear();
    if (!forest || !X || !y || !out_mse) return fail(AIWCRF_E_INVALID_ARG, "forest, X, y and out_mse must not be NULL");
    if (forest->oob_rows == 0)
        return fail(AIWCRF_E_INVALID_ARG, "out-of-bag evaluation needs a forest fitted by aiwcrf_fit in this process");
    if (n_rows != forest->oob_rows) return fail(AIWCRF_E_INVALID_ARG, "n_rows differs from the training matrix");
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    if (dev != forest->device) return fail(AIWCRF_E_BAD_POINTER, "the forest lives on another device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InArg ax, ay;
    OutArg op;
    if ((rc = stage_in(ax, X, sizeof(float) * (size_t)forest->F * (size_t)n_rows, dev, s, "X"))) return rc;
    if ((rc = stage_in(ay, y, sizeof(int64_t) * (size_t)n_rows, dev, s, "y"))) return rc;
    if ((rc = stage_out(op, out_pred, sizeof(int64_t) * (size_t)n_rows, dev, s, "out_pred"))) return rc;
    // one scratch block: sums, counts, per-CTA partial sums, the result and an error flag
    const size_t parts = oob_error_parts(n_rows);
    const size_t b_sum = 8 * (size_t)n_rows, b_cnt = (4 * (size_t)n_rows + 15) & ~(size_t)15;
    const size_t bytes = b_sum + b_cnt + sizeof(OobPart) * parts + sizeof(OobResult) + 16;
    unsigned char *blk = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&blk), bytes, s);
    if (e != cudaSuccess) return fail(AIWCRF_E_OOM, "out-of-bag error scratch");
    struct Free { void *p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{blk, s};
    int64_t *d_sum = reinterpret_cast<int64_t *>(blk);
    int32_t *d_cnt = reinterpret_cast<int32_t *>(blk + b_sum);
    OobPart *d_parts = reinterpret_cast<OobPart *>(blk + b_sum + b_cnt);
    OobResult *d_res = reinterpret_cast<OobResult *>(d_parts + parts);
    uint32_t *d_err = reinterpret_cast<uint32_t *>(d_res + 1);
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s)) != cudaSuccess) return cuda_fail(e, "oob_error");
    if ((rc = oob_launch(forest, (const float *)ax.dev, n_rows, d_sum, d_cnt, s))) return rc;
    if ((rc = oob_error_launch(d_sum, d_cnt, (const int64_t *)ay.dev, n_rows, (int64_t *)op.dev, d_parts, d_res, d_err, s)))
        return rc;
    if ((rc = finish_out(op))) return rc;
    OobResult res;
    uint32_t h_err = 0;
    if ((e = cudaMemcpyAsync(&res, d_res, sizeof(OobResult), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "oob_error");
    if (h_err & kErrY) return fail(AIWCRF_E_INVALID_ARG, "a target value exceeds |y| <= 2^40");
    *out_mse = res.mse;
    if (out_rows) *out_rows = res.rows;
    return AIWCRF_OK;
}

int aiwcrf_round_mean(const int64_t *sums, int64_t n, int64_t total_trees, int64_t *out, void *cuda_stream)
{
    g_last_error.clear();
    if (n < 0 || total_trees < 1) return fail(AIWCRF_E_INVALID_ARG, "n must be >= 0 and total_trees >= 1");
    if (n > 0 && (!sums || !out)) return fail(AIWCRF_E_INVALID_ARG, "sums and out must not be NULL");
    if (n == 0) return AIWCRF_OK;
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InArg a;
    OutArg o;
    if ((rc = stage_in(a, sums, sizeof(int64_t) * (size_t)n, dev, s, "sums"))) return rc;
    if ((rc = stage_out(o, out, sizeof(int64_t) * (size_t)n, dev, s, "out"))) return rc;
    if ((rc = round_mean_launch((const int64_t *)a.dev, n, total_trees, (int64_t *)o.dev, s))) return rc;
    if ((rc = finish_out(o))) return rc;
    return sync_if(o.host != nullptr, s);
}

int aiwcrf_select_device(const aiwcrf_forest *forest, const float *kfeat, int32_t n_kernels, int32_t size_class,
                         const int32_t *device_ids, int32_t n_devices, int32_t *out_best, int64_t *out_pred,
                         void *cuda_stream)
{
    g_last_error.clear();
    if (!forest || !kfeat || !device_ids || !out_best)
        return fail(AIWCRF_E_INVALID_ARG, "forest, kfeat, device_ids and out_best must not be NULL");
    if (n_kernels < 1 || n_devices < 1 || (int64_t)n_kernels * n_devices > ((int64_t)1 << 31))
        return fail(AIWCRF_E_INVALID_ARG, "n_kernels and n_devices must be >= 1");
    if (forest->F < 3) return fail(AIWCRF_E_INVALID_ARG, "the forest needs >= 3 features (kernel, device, size)");
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    if (dev != forest->device) return fail(AIWCRF_E_BAD_POINTER, "the forest lives on another device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t Qn = (int64_t)n_kernels * n_devices;
    InArg ak, ad;
    OutArg ob, op;
    if ((rc = stage_in(ak, kfeat, sizeof(float) * (size_t)(forest->F - 2) * (size_t)n_kernels, dev, s, "kfeat"))) return rc;
    if ((rc = stage_in(ad, device_ids, sizeof(int32_t) * (size_t)n_devices, dev, s, "device_ids"))) return rc;
    if ((rc = stage_out(ob, out_best, sizeof(int32_t) * (size_t)n_kernels, dev, s, "out_best"))) return rc;
    if ((rc = stage_out(op, out_pred, sizeof(int64_t) * (size_t)Qn, dev, s, "out_pred"))) return rc;
    float *d_q = nullptr;
    int64_t *d_p = nullptr;
    cudaError_t e = cudaMallocAsync(&d_q, sizeof(float) * (size_t)forest->F * (size_t)Qn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_p, sizeof(int64_t) * (size_t)Qn, s);
    if (e != cudaSuccess) {
        if (d_q) cudaFreeAsync(d_q, s);
        return fail(AIWCRF_E_OOM, "select_device scratch");
    }
    rc = select_launch(forest, (const float *)ak.dev, n_kernels, size_class, (const int32_t *)ad.dev, n_devices,
                       (int32_t *)ob.dev, (int64_t *)op.dev, d_q, d_p, s);
    cudaFreeAsync(d_q, s);
    cudaFreeAsync(d_p, s);
    if (rc) return rc;
    if ((rc = finish_out(ob)) || (rc = finish_out(op))) return rc;
    // device_ids is usually a host array: its staged copy must be consumed before returning
    return sync_if(true, s);
}

int aiwcrf_forest_stats(const aiwcrf_forest *forest, aiwcrf_fit_stats *out)
{
    g_last_error.clear();
    if (!forest || !out) return fail(AIWCRF_E_INVALID_ARG, "forest and out must not be NULL");
    *out = forest->stats;
    return AIWCRF_OK;
}

int aiwcrf_forest_info(const aiwcrf_forest *forest, int64_t *num_trees, int64_t *num_nodes, int32_t *n_features)
{
    g_last_error.clear();
    if (!forest) return fail(AIWCRF_E_INVALID_ARG, "forest is NULL");
    if (num_trees) *num_trees = forest->T;
    if (num_nodes) *num_nodes = forest->num_nodes;
    if (n_features) *n_features = forest->F;
    return AIWCRF_OK;
}

static const char kMagic[8] = {'A', 'I', 'W', 'C', 'R', 'F', '0', '1'};

int aiwcrf_forest_serialize(const aiwcrf_forest *forest, void *buf, size_t cap, size_t *needed)
{
    g_last_error.clear();
    if (!forest || !needed) return fail(AIWCRF_E_INVALID_ARG, "forest and needed must not be NULL");
    const size_t bytes = 8 + 4 + 4 + 8 + 8 + 8 * (size_t)(forest->T + 1) + 8 * (size_t)forest->num_nodes;
    *needed = bytes;
    if (!buf) return AIWCRF_OK;
    if (cap < bytes) return fail(AIWCRF_E_INVALID_ARG, "buffer too small");
    unsigned char *p = (unsigned char *)buf;
    const uint32_t version = 1, F = (uint32_t)forest->F;
    std::memcpy(p, kMagic, 8); p += 8;
    std::memcpy(p, &version, 4); p += 4;
    std::memcpy(p, &F, 4); p += 4;
    std::memcpy(p, &forest->T, 8); p += 8;
    std::memcpy(p, &forest->num_nodes, 8); p += 8;
    std::memcpy(p, forest->tree_off.data(), 8 * (size_t)(forest->T + 1)); p += 8 * (size_t)(forest->T + 1);
    cudaError_t e = cudaMemcpy(p, forest->d_nodes, 8 * (size_t)forest->num_nodes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading forest nodes");
    return AIWCRF_OK;
}

int aiwcrf_forest_deserialize(const void *buf, size_t len, aiwcrf_forest **out)
{
    g_last_error.clear();
    if (!buf || !out) return fail(AIWCRF_E_INVALID_ARG, "buf and out must not be NULL");
    const unsigned char *p = (const unsigned char *)buf;
    if (len < 32 || std::memcmp(p, kMagic, 8) != 0) return fail(AIWCRF_E_CORRUPT, "bad magic");
    uint32_t version, F;
    int64_t T, nn;
    std::memcpy(&version, p + 8, 4);
    std::memcpy(&F, p + 12, 4);
    std::memcpy(&T, p + 16, 8);
    std::memcpy(&nn, p + 24, 8);
    if (version != 1 || F < 1 || F > AIWCRF_MAX_FEATURES || T < 1 || T > AIWCRF_MAX_TREES * 16ll || nn < 2 ||
        nn > ((int64_t)1 << 40))
        return fail(AIWCRF_E_CORRUPT, "bad header");
    if (len != 32 + 8 * (size_t)(T + 1) + 8 * (size_t)nn) return fail(AIWCRF_E_CORRUPT, "bad length");
    std::vector<int64_t> off((size_t)T + 1);
    std::memcpy(off.data(), p + 32, 8 * (size_t)(T + 1));
    const uint64_t *nodes = (const uint64_t *)(p + 32 + 8 * (size_t)(T + 1));
    if (off[0] != 0 || off[(size_t)T] != nn) return fail(AIWCRF_E_CORRUPT, "bad tree offsets");
    int64_t max_tree = 0;
    for (int64_t t = 0; t < T; ++t) {
        const int64_t a = off[(size_t)t], b = off[(size_t)t + 1], m = b - a;
        if (m < 2 || (m & 1) || (a & 1) || m > (1ll << 24)) return fail(AIWCRF_E_CORRUPT, "bad tree size");
        max_tree = m > max_tree ? m : max_tree;
        // every split points strictly forward, inside its tree, at a real feature
        for (int64_t j = 0; j < m; ++j) {
            uint64_t nd;
            std::memcpy(&nd, nodes + a + j, 8);
            if (nd >> 63) continue;
            const uint32_t fe = (uint32_t)(nd >> 56) & 0x7F, lc = (uint32_t)(nd >> 32) & 0xFFFFFF;
            if (fe >= F || (int64_t)lc <= j || (int64_t)lc + 1 >= m) return fail(AIWCRF_E_CORRUPT, "bad node");
        }
    }
    // value tables: per feature the sorted distinct thresholds (-0 read as +0); coded copy of
    // every split holds its threshold's index in that table
    std::vector<std::vector<float>> tab((size_t)F);
    std::vector<uint64_t> cnodes((size_t)nn);
    for (int64_t j = 0; j < nn; ++j) {
        uint64_t nd;
        std::memcpy(&nd, nodes + j, 8);
        if (nd >> 63) continue;
        uint32_t b = (uint32_t)nd;
        if (b == 0x80000000u) b = 0u;
        float x;
        std::memcpy(&x, &b, 4);
        if (x != x) return fail(AIWCRF_E_CORRUPT, "NaN threshold");
        tab[(size_t)((nd >> 56) & 0x7F)].push_back(x);
    }
    uint32_t max_card = 0;
    for (auto &v : tab) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        if (v.size() >= (1u << 24)) return fail(AIWCRF_E_LIMIT, "more than 2^24 - 1 thresholds for one feature");
        max_card = std::max<uint32_t>(max_card, (uint32_t)v.size());
    }
    for (int64_t j = 0; j < nn; ++j) {
        uint64_t nd;
        std::memcpy(&nd, nodes + j, 8);
        if (nd >> 63) { cnodes[(size_t)j] = nd; continue; }
        uint32_t b = (uint32_t)nd;
        if (b == 0x80000000u) b = 0u;
        float x;
        std::memcpy(&x, &b, 4);
        const auto &v = tab[(size_t)((nd >> 56) & 0x7F)];
        const uint32_t code = (uint32_t)(std::lower_bound(v.begin(), v.end(), x) - v.begin());
        cnodes[(size_t)j] = (nd & 0xFFFFFFFF00000000ull) | code;
    }
    const int64_t fstride = std::max<uint32_t>(max_card, 1u);
    std::vector<float> fv((size_t)F * (size_t)fstride, 0.0f);
    std::vector<uint32_t> fc((size_t)F);
    for (uint32_t f = 0; f < F; ++f) {
        fc[f] = (uint32_t)tab[f].size();
        std::copy(tab[f].begin(), tab[f].end(), fv.begin() + (size_t)f * (size_t)fstride);
    }
    int dev, rc;
    if ((rc = current_device(&dev))) return rc;
    aiwcrf_forest *f = new aiwcrf_forest();
    f->F = (int32_t)F; f->T = T; f->num_nodes = nn; f->max_tree_nodes = max_tree; f->device = dev;
    f->tree_off = off;
    f->max_card = max_card;
    f->fstride = fstride;
    const cudaStream_t st = cudaStreamPerThread;
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    cudaError_t e = forest_alloc(f, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_nodes, nodes, 8 * (size_t)nn, h2d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_cnodes, cnodes.data(), 8 * (size_t)nn, h2d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_tree_off, off.data(), 8 * (size_t)(T + 1), h2d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_fvals, fv.data(), sizeof(float) * fv.size(), h2d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_fcard, fc.data(), sizeof(uint32_t) * fc.size(), h2d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        forest_release(f);
        return cuda_fail(e, "uploading forest");
    }
    if ((rc = forest_build_compact(f, st)) != AIWCRF_OK || (rc = (cudaStreamSynchronize(st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "compact nodes"))) != AIWCRF_OK) {
        forest_release(f);
        return rc;
    }
    *out = f;
    return AIWCRF_OK;
}

int aiwcrf_forest_free(aiwcrf_forest *forest)
{
    g_last_error.clear();
    forest_release(forest);
    return AIWCRF_OK;
}

int aiwcrf_profile_enable(int32_t on)
{
    aiwcrf::clear_last_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return AIWCRF_OK;
}

int aiwcrf_profile_classes(uint32_t mask)
{
    aiwcrf::clear_last_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_mask = mask;
    return AIWCRF_OK;
}

int aiwcrf_profile_read(int32_t n, int64_t *launches, double *total_ms)
{
    aiwcrf::clear_last_error();
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof);
    }
    for (int32_t k = 0; k < n; ++k) { if (launches) launches[k] = 0; if (total_ms) total_ms[k] = 0.0; }
    int rc = AIWCRF_OK;
    for (auto &r : recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "reading profile events");
        if (r.cls < n) {
            if (launches) launches[r.cls] += 1;
            if (total_ms) total_ms[r.cls] += ms;
        }
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : recs) { g_event_pool.push_back(r.a); g_event_pool.push_back(r.b); }
    return rc;
}

const char *aiwcrf_profile_name(int32_t k)
{
    return (k >= 0 && k < kProfNum) ? kProfNames[k] : "";
}

int32_t aiwcrf_profile_num_classes(void) { return kProfNum; }

int64_t aiwcrf_debug_bounds(void)
{
    aiwcrf::clear_last_error();
#ifdef AIWCRF_DEBUG_BOUNDS
    return (int64_t)(aiwcrf::bounds_flags_fit() | aiwcrf::bounds_flags_predict() | aiwcrf::bounds_flags_serve());
#else
    return -1;
#endif
}

int aiwcrf_set_grower(int32_t grower)
{
    aiwcrf::clear_last_error();
    return aiwcrf::set_grower_mode(grower);
}

int64_t aiwcrf_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
