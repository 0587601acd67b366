// tune.cu -- simulated-annealing search of the forest's three tuning parameters against the
// out-of-bag prediction error (Sec. III-C: num.trees, mtry and min.node.size tuned at once,
// minimising the out-of-bag error). The paper runs the simulated annealing of an R package; this
// annealer is our own (the proposal, temperature and acceptance rules are stated in the header),
// and every step is a GPU fit followed by the exact out-of-bag error on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "internal.cuh"

namespace aiwcrf {
namespace {

struct Rng {                    // SplitMix64
    uint64_t x;
    uint64_t next()
    {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }           // [0, 1)
    int64_t below(int64_t n) { return (int64_t)(uniform() * (double)n); }    // [0, n)
};

// out-of-bag MSE of a fit with these parameters (on the training rows)
int evaluate(const aiwcrf_fit_params &p, const float *X, const int64_t *y, int64_t n, int32_t F, void *stream,
             double *mse)
{
    aiwcrf_forest *f = nullptr;
    int rc = aiwcrf_fit(&p, X, y, n, F, stream, &f);
    if (rc) return rc;
    rc = aiwcrf_oob_error(f, X, y, n, nullptr, mse, nullptr, stream);
    aiwcrf_forest_free(f);
    return rc;
}

}  // namespace
}  // namespace aiwcrf

using namespace aiwcrf;

extern "C" int aiwcrf_tune_sa(const aiwcrf_tune_params *tp, const aiwcrf_fit_params *start, const float *X,
                              const int64_t *y, int64_t n_rows, int32_t n_features, void *cuda_stream,
                              aiwcrf_tune_step *trace, aiwcrf_fit_params *best, double *best_mse)
{
    clear_last_error();
    if (!tp || !start || !X || !y || !best || !best_mse)
        return fail(AIWCRF_E_INVALID_ARG, "tp, start, X, y, best and best_mse must not be NULL");
    if (tp->steps < 0 || tp->trees_min < 1 || tp->trees_max < tp->trees_min || tp->mtry_min < 1 ||
        tp->mtry_max < tp->mtry_min || tp->node_min < 1 || tp->node_max < tp->node_min || !(tp->t0 > 0.0) ||
        !(tp->cooling > 0.0) || !(tp->cooling <= 1.0) || tp->reserved != 0)
        return fail(AIWCRF_E_INVALID_ARG, "tuning parameters out of range");
    const int32_t lo[3] = {tp->trees_min, tp->mtry_min, tp->node_min};
    const int32_t hi[3] = {tp->trees_max, tp->mtry_max, tp->node_max};
    auto get = [](const aiwcrf_fit_params &p, int k) {
        return k == 0 ? p.num_trees : k == 1 ? p.mtry : p.min_node_size;
    };
    auto set = [](aiwcrf_fit_params &p, int k, int32_t v) {
        if (k == 0) p.num_trees = v;
        else if (k == 1) p.mtry = v;
        else p.min_node_size = v;
    };
    aiwcrf_fit_params cur = *start;
    for (int k = 0; k < 3; ++k) set(cur, k, std::min(hi[k], std::max(lo[k], get(cur, k))));

    // fits are deterministic in their parameters: each distinct setting is evaluated once
    std::map<std::tuple<int32_t, int32_t, int32_t>, double> seen;
    auto eval = [&](const aiwcrf_fit_params &p, double *mse) -> int {
        const auto key = std::make_tuple(p.num_trees, p.mtry, p.min_node_size);
        auto it = seen.find(key);
        if (it != seen.end()) { *mse = it->second; return AIWCRF_OK; }
        const int rc = evaluate(p, X, y, n_rows, n_features, cuda_stream, mse);
        if (rc == AIWCRF_OK) seen[key] = *mse;
        return rc;
    };
    double e_cur = 0.0;
    int rc = eval(cur, &e_cur);
    if (rc) return rc;
    if (trace) trace[0] = aiwcrf_tune_step{cur.num_trees, cur.mtry, cur.min_node_size, 1, e_cur};
    aiwcrf_fit_params b = cur;
    double e_best = e_cur;
    const double temp0 = tp->t0 * std::max(e_cur, 1e-300);
    double temp = temp0;
    Rng rng{tp->seed};
    for (int32_t i = 1; i <= tp->steps; ++i) {
        // proposal: one parameter, uniform within a radius that shrinks with the temperature
        aiwcrf_fit_params cand = cur;
        const int k = (int)rng.below(3);
        const int32_t span = hi[k] - lo[k];
        const int32_t r = std::max<int32_t>(1, (int32_t)std::ceil(0.25 * (double)span * temp / temp0));
        const int32_t v0 = get(cur, k);
        int32_t v = v0 + (int32_t)rng.below(2 * (int64_t)r + 1) - r;
        v = std::min(hi[k], std::max(lo[k], v));
        if (v == v0 && span > 0) v = v0 < hi[k] ? v0 + 1 : v0 - 1;        // always move when it can
        set(cand, k, v);
        double e = 0.0;
        if ((rc = eval(cand, &e))) return rc;
        const double u = rng.uniform();
        const bool accept = e <= e_cur || u < std::exp(-(e - e_cur) / temp);
        if (accept) { cur = cand; e_cur = e; }
        if (e < e_best) { b = cand; e_best = e; }
        if (trace) trace[i] = aiwcrf_tune_step{cand.num_trees, cand.mtry, cand.min_node_size, accept ? 1 : 0, e};
        temp *= tp->cooling;
    }
    *best = b;
    *best_mse = e_best;
    return AIWCRF_OK;
}
