/*
 * aiwcrf.h -- C ABI of the GB300 random-forest library for AIWC performance prediction.
 *
 * The method (arXiv 1811.00156): architecture-independent AIWC features of an OpenCL kernel,
 * plus a device id and a problem-size class, are the predictors of a random-forest regression
 * (Sec. III-B: ranger, num.trees / mtry / min.node.size) whose response is the kernel's
 * execution time, here log10 seconds in Q32.32 fixed point. The fitted model is queried to
 * predict times (Sec. I notes that a query of the fitted model is cheap; Sec. V) and to
 * pick the fastest device for a kernel (Sec. VI).
 *
 * Conventions for every call:
 *  - Return 0 (AIWCRF_OK) on success, a negative AIWCRF_E_* code on failure; the failing call's
 *    message is available from aiwcrf_last_error() on the same host thread.
 *  - Array arguments may be host or device pointers; the library checks each one. Host inputs
 *    are copied to the device on the given stream; host outputs are written back and the call
 *    synchronises the stream before returning. With device outputs the call is stream-ordered
 *    and the results are valid once the stream reaches that point.
 *  - The caller owns every array it passes. The library owns each aiwcrf_forest until
 *    aiwcrf_forest_free(). A host thread that has fitted keeps up to 512 MiB of device scratch
 *    for its next fits (released when the thread exits).
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream). The device is the
 *    current CUDA device of the calling thread.
 *  - Matrices are column-major float32: element (feature f, row r) of an F x N matrix is at
 *    [f * N + r].
 *  - Targets, leaf values and predictions are int64 Q32.32 (value * 2^32).
 *  - There is no CPU fallback: without a usable CUDA device every call fails with
 *    AIWCRF_E_CUDA.
 */
#ifndef AIWCRF_H
#define AIWCRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AIWCRF_OK               0
#define AIWCRF_E_INVALID_ARG   -1   /* null pointer, size or parameter out of range */
#define AIWCRF_E_NAN_INPUT     -2   /* NaN in the training features */
#define AIWCRF_E_BAD_POINTER   -3   /* pointer is neither host memory nor memory of this device */
#define AIWCRF_E_OOM           -4   /* device allocation failed */
#define AIWCRF_E_CUDA          -5   /* a CUDA runtime call or kernel launch failed */
#define AIWCRF_E_TIMEOUT       -6   /* a bounded device-side wait gave up */
#define AIWCRF_E_CORRUPT       -7   /* serialized forest failed validation */
#define AIWCRF_E_LIMIT         -8   /* a documented size limit was exceeded (see below) */

/* Size limits (checked; AIWCRF_E_LIMIT or AIWCRF_E_INVALID_ARG when exceeded):
 *   n_rows <= 4,194,303 (2^22 - 1); |y| <= 2^40 (|log10 t| < 256);
 *   n_features <= 128 (a column may hold as many distinct values as rows: ranks are stored in
 *   1, 2 or 4 bytes as the columns need);
 *   num_trees <= 1,048,576; where a fit counts its draws per row in bytes (the groups' sums do
 *   not fit shared memory), a bootstrap multiplicity above 255 (probability ~ 1e-500) fails;
 *   where it sums them per group, any multiplicity is exact. */
#define AIWCRF_MAX_ROWS       ((1 << 22) - 1)
#define AIWCRF_MAX_FEATURES   128
#define AIWCRF_MAX_ABS_Y      (1LL << 40)
#define AIWCRF_MAX_TREES      (1 << 20)

typedef struct aiwcrf_forest aiwcrf_forest;   /* opaque, owned by the library */

/* Fit parameters: the three ranger parameters the paper tunes (Sec. III-B: num.trees, mtry,
 * min.node.size) plus depth limit, seed and bootstrap switch. */
typedef struct {
    int32_t num_trees;      /* >= 1 */
    int32_t mtry;           /* features tried per node, >= 1 (values above n_features try all) */
    int32_t min_node_size;  /* >= 1; a node with sum of multiplicities <= this is a leaf */
    int32_t max_depth;      /* 0 = unlimited; else nodes at this depth are leaves */
    uint64_t seed;          /* Philox4x32-10 key */
    int32_t bootstrap;      /* 1: n_rows draws with replacement per tree; 0: every row once */
    int32_t ctas_per_sm;    /* 0: the level kernels may fill every SM (3 CTAs each); 1..3: at most
                               that many of their CTAs per SM, leaving registers on every SM for
                               concurrent work (a background fit). The forest does not depend on
                               it. */
    int64_t first_tree;     /* global index of this forest's tree 0 (for tree-sharded fits;
                               tree t uses random counters of tree first_tree + t). >= 0 */
} aiwcrf_fit_params;

/* Per-fit counters, for byte accounting and tests. Rows with identical feature vectors form
 * one group; a tree carries one entry per group that holds in-bag rows (its summed
 * multiplicity and summed w*y), since such rows fall on the same side of every split. */
typedef struct {
    int64_t num_trees;
    int64_t total_nodes;
    int64_t levels;                     /* depth of the deepest tree + 1 */
    int64_t groups;                     /* distinct feature vectors among the rows */
    int64_t entries_evaluated;          /* sum over searched nodes of their entries */
    int64_t entries_partitioned;        /* sum over split nodes of their entries */
    int64_t nodes_evaluated;            /* nodes whose split was searched */
    int64_t nodes_small;                /* of those, searched by one warp (<= 32 entries) */
    int64_t entries_evaluated_small;    /* entries_evaluated of the warp-searched nodes */
    int64_t entries_partitioned_small;  /* entries_partitioned of the warp-searched nodes */
    int32_t n_features;
    int32_t mtry;
    int32_t rank_bytes;          /* bytes per stored rank: 1 if every column has <= 256 values */
    int32_t grower;              /* 1: level-synchronous kernels, 2: tree-resident kernel,
                                    3: level-synchronous with presorted lists */
} aiwcrf_fit_stats;

/* Fit a forest (Sec. III-B). X: F x N column-major float32 (no NaN); y: N int64 Q32.32.
 * Presorts and ranks every column once, draws each tree's bootstrap and per-node mtry
 * features with Philox4x32-10, grows all trees breadth first with an exact integer split
 * search (maximise S_L^2/n_L + S_R^2/n_R; ties: lowest feature, then lowest threshold; split
 * only with a strict gain), and packs the trees. On success *out receives a new forest. */
int aiwcrf_fit(const aiwcrf_fit_params *params, const float *X, const int64_t *y,
               int64_t n_rows, int32_t n_features, void *cuda_stream, aiwcrf_forest **out);

/* Batched fit of n_subsets forests on row subsets of one matrix, grown together (the
 * leave-one-kernel-out experiment of Alg. 1 / Table III trains one forest per omitted kernel).
 * Subset g is subset_rows[subset_offsets[g] .. subset_offsets[g+1]) (host int64 offsets,
 * n_subsets + 1 of them; rows strictly increasing, host or device int32). Forest g equals
 * aiwcrf_fit with the same params on the matrix of those rows. out: n_subsets handles. */
int aiwcrf_fit_subsets(const aiwcrf_fit_params *params, const float *X, const int64_t *y,
                       int64_t n_rows, int32_t n_features, const int64_t *subset_offsets,
                       const int32_t *subset_rows, int32_t n_subsets, void *cuda_stream,
                       aiwcrf_forest **out);

/* Predict (Sec. I, Sec. V). Xq: F x Q column-major float32; page-locked host memory is read in
 * place by the device (no staging copy) and must stay unchanged until the stream has passed
 * the call, pageable host memory is copied as usual. out_pred[q] = floor((2P + T)/(2T))
 * with P the exact sum of the T leaf values reached (x <= threshold goes left; a NaN feature
 * goes right). out_var (or NULL): per query two uint64 words (low, high) of the exact
 * unsigned 128-bit V = T * sum(v^2) - P^2 (T^2 times the ensemble variance). */
int aiwcrf_predict(const aiwcrf_forest *forest, const float *Xq, int64_t n_queries,
                   int64_t *out_pred, uint64_t *out_var, void *cuda_stream);

/* Raw per-query sums P over this forest's trees (for forests split across processes by
 * tree: add the shards' sums, then aiwcrf_round_mean with the total tree count). */
int aiwcrf_predict_sum(const aiwcrf_forest *forest, const float *Xq, int64_t n_queries,
                       int64_t *out_sum, void *cuda_stream);

/* Out-of-bag evaluation (Sec. III-B: the tuning minimises the out-of-bag prediction error).
 * X: the F x n_rows training matrix the forest was fitted on by aiwcrf_fit in this process
 * (AIWCRF_E_INVALID_ARG otherwise). For each row r: out_sum[r] = exact sum of the leaf values
 * reached in the trees whose bootstrap did not draw r, out_count[r] = their number. The
 * out-of-bag prediction is floor((2 out_sum + c) / (2 c)) for c = out_count > 0. */
int aiwcrf_oob(const aiwcrf_forest *forest, const float *X, int64_t n_rows, int64_t *out_sum,
               int32_t *out_count, void *cuda_stream);

/* Out-of-bag error (Sec. III-B: the parameters are tuned by the out-of-bag prediction error).
 * X and y: the F x n_rows training matrix and its int64 Q32.32 targets that the forest was
 * fitted on by aiwcrf_fit in this process (host or device arrays; AIWCRF_E_INVALID_ARG for
 * another forest or another row count, or a |y| above 2^40). For a row r with c_r > 0 trees
 * whose bootstrap did not draw it and leaf sum s_r over those trees, its out-of-bag prediction
 * is p_r = floor((2 s_r + c_r) / (2 c_r)). out_pred (or NULL): int64[n_rows], p_r, 0 where
 * c_r = 0. *out_mse (host): the mean of (p_r - y_r)^2 over the rows with c_r > 0, in the
 * target's units squared (Q32.32 differences divided by 2^32): the squared errors are summed
 * exactly in 128-bit integers on the device and divided once in double precision. *out_rows
 * (host, or NULL): the number of those rows. Synchronises the stream. */
int aiwcrf_oob_error(const aiwcrf_forest *forest, const float *X, const int64_t *y, int64_t n_rows,
                     int64_t *out_pred, double *out_mse, int64_t *out_rows, void *cuda_stream);

/* Tuning of num.trees, mtry and min.node.size at once against the out-of-bag error (Sec. III-C:
 * the paper minimises the out-of-bag prediction error by simulated annealing over the three
 * parameters; its annealer is an R package's, this one is stated here). Every evaluation is
 * aiwcrf_fit with the candidate's three parameters (the rest from *start) followed by
 * aiwcrf_oob_error on the same rows; a setting already evaluated is not fitted again.
 *  - start: the first state, clamped into the bounds; its error E_0 sets the temperature
 *    t_1 = t0 * E_0, and t_{i+1} = cooling * t_i.
 *  - step i = 1..steps: one of the three parameters, chosen uniformly, moves to a value uniform in
 *    [v - r, v + r] clamped into its bounds, r = max(1, ceil(0.25 * (max - min) * t_i / t_1));
 *    a proposal equal to the current value moves by one instead (up if it can). The candidate is
 *    accepted if its error E <= the current one, or if u < exp(-(E - E_cur) / t_i).
 *  - random numbers: SplitMix64 from seed; u and the choices from its top 53 bits.
 * trace (host, steps + 1 entries, or NULL): entry 0 the start, entry i the i-th candidate and
 * whether it was accepted. *best receives *start with the lowest-error candidate's three
 * parameters (the earliest on ties), *best_mse its error. X, y: as aiwcrf_fit (host or device). */
typedef struct {
    int32_t steps;                  /* candidates after the start (>= 0) */
    int32_t trees_min, trees_max;   /* num.trees bounds (1 <= min <= max) */
    int32_t mtry_min, mtry_max;     /* mtry bounds */
    int32_t node_min, node_max;     /* min.node.size bounds */
    int32_t reserved;               /* must be 0 */
    double t0;                      /* initial temperature relative to the start's error (> 0) */
    double cooling;                 /* temperature factor per step, (0, 1] */
    uint64_t seed;
} aiwcrf_tune_params;

typedef struct {
    int32_t num_trees, mtry, min_node_size;
    int32_t accepted;               /* 1: the walk moved to this candidate */
    double oob_mse;                 /* aiwcrf_oob_error's mean squared error */
} aiwcrf_tune_step;

int aiwcrf_tune_sa(const aiwcrf_tune_params *params, const aiwcrf_fit_params *start, const float *X,
                   const int64_t *y, int64_t n_rows, int32_t n_features, void *cuda_stream,
                   aiwcrf_tune_step *trace, aiwcrf_fit_params *best, double *best_mse);

/* out[q] = floor((2 sums[q] + total_trees) / (2 total_trees)). */
int aiwcrf_round_mean(const int64_t *sums, int64_t n, int64_t total_trees, int64_t *out,
                      void *cuda_stream);

/* Device selection (Sec. VI: which device runs a kernel fastest). kfeat: (F-2) x K
 * column-major kernel features; query (k, j) is kfeat[:, k] with device_ids[j] and
 * size_class appended as the last two features. out_best[k] = the device id with the
 * smallest prediction (ties: lower device id). out_pred (or NULL): K x D row-major
 * predictions. device_ids: host array of D ids. */
int aiwcrf_select_device(const aiwcrf_forest *forest, const float *kfeat, int32_t n_kernels,
                         int32_t size_class, const int32_t *device_ids, int32_t n_devices,
                         int32_t *out_best, int64_t *out_pred, void *cuda_stream);

/* Device selection that allocates no device memory (the paper has no counterpart; this is for
 * callers that cannot allocate). aiwcrf_select_device allocates scratch on the stream; a
 * caller such as a scheduler hook living inside another application, whose device memory is
 * owned by that application's allocator and which must not trigger the device-wide
 * synchronisation a cudaMalloc/cudaFree can cause, uses this variant instead. Same inputs,
 * outputs and results as aiwcrf_select_device, except:
 *  - kfeat, out_best and out_pred (or NULL) must be memory of the current device
 *    (AIWCRF_E_BAD_POINTER otherwise); device_ids may be a host or a device array.
 *  - Scratch is one static device array of AIWCRF_NOALLOC_SCRATCH_BYTES that every GPU loading
 *    the library holds until the process exits. A request needs about
 *    (4F + 8 + 4 * code words) bytes per (kernel, device) pair (F = 32: 172 bytes, so about
 *    6,000 pairs fit); a larger request fails with AIWCRF_E_LIMIT before launching anything.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture.
 *  - Every call reuses the same array: calls that overlap on the GPU (other streams, other
 *    host threads) race on it. The call synchronises its stream before returning, also when
 *    it fails after enqueuing work, so that no work of a returned call still uses the array. */
#define AIWCRF_NOALLOC_SCRATCH_BYTES (1 << 20)
int aiwcrf_select_device_noalloc(const aiwcrf_forest *forest, const float *kfeat, int32_t n_kernels,
                                 int32_t size_class, const int32_t *device_ids, int32_t n_devices,
                                 int32_t *out_best, int64_t *out_pred, void *cuda_stream);

/* Tensor-core primitive of the learned surrogate (the paper has no surrogate; the model queried
 * in Sec. VI is the forest): C (M x N, FP32, row-major, device) = A * B^T for BF16 A (M x K)
 * and B (N x K), on tcgen05 with an FP32 accumulator in tensor memory. Element (m, k) of A is
 * A[m * lda + k], or A[k * lda + m] with a_trans; likewise B with b_trans. N is a multiple of 16
 * in [16, 256]; lda and ldb are multiples of 8; device pointers, 16-byte aligned. ksplit > 1
 * spreads K over that many CTAs per 128-row slab and sums their FP32 partials in a fixed order. */
int aiwcrf_tc_gemm_bf16(const void *A, int32_t lda, int32_t a_trans, const void *B, int32_t ldb,
                        int32_t b_trans, float *C, int32_t M, int32_t N, int32_t K, int32_t ksplit,
                        void *cuda_stream);

/* ---------------------------------------------------------------------------------------------
 * Learned surrogate (not in the paper: its model is the forest of Sec. III-B). A small MLP
 * distilled from a forest's own predictions, for cheaper queries: inputs are the first F-2
 * (AIWC) columns standardised -- after log2 for columns of values >= 1 that span three orders
 * of magnitude -- then one-hot device (column F-2) and size class (column F-1), zero-padded to
 * 64; layers 64 -> 256 -> 256 -> 1 with GELU; BF16 weights and activations, FP32 accumulation
 * on the tensor cores (tcgen05); output log10 seconds as float. Trained with Adam on the mean
 * squared error against the forest's predictions.
 * Parameter vector (float32, aiwcrf_surrogate_num_params() of them): W1[256][64], b1[256],
 * W2[256][256], b2[256], w3[256], b3. */
typedef struct aiwcrf_surrogate aiwcrf_surrogate;

typedef struct {
    int32_t epochs;      /* passes over the samples (20) */
    int32_t batch;       /* samples per Adam step, a multiple of 128 (4096) */
    float lr;            /* Adam step size (1e-3) */
    float beta1;         /* 0.9 */
    float beta2;         /* 0.999 */
    float eps;           /* 1e-8 */
    uint64_t seed;       /* weight initialisation and shuffling */
    int32_t n_devices;   /* one-hot width of the device column (15) */
    int32_t n_sizes;     /* one-hot width of the size-class column (4) */
} aiwcrf_surrogate_params;

typedef struct {
    int64_t steps;
    float first_batch_loss;   /* mean of (out - y)^2 / 2 over the first batch */
    float last_batch_loss;    /* ... over the last batch */
} aiwcrf_surrogate_fit_stats;

/* Distil: label X (device, F x n column-major) with the teacher forest's predictions and train. */
int aiwcrf_surrogate_fit(const aiwcrf_surrogate_params *params, const aiwcrf_forest *teacher,
                         const float *X, int64_t n, int32_t n_features, void *cuda_stream,
                         aiwcrf_surrogate **out);

/* out[q] = surrogate prediction of log10 seconds for query q (device pointers). One fused
 * persistent kernel: weights resident in shared memory, both layers on the tensor cores. */
int aiwcrf_surrogate_predict(const aiwcrf_surrogate *surrogate, const float *Xq, int64_t n,
                             float *out, void *cuda_stream);

/* Loss (sum over the batch of (out - y)^2 / 2) and its gradient with respect to every
 * parameter divided by n (the training step's gradient), for X (F x n) and float targets y;
 * n a multiple of 128; device pointers; grad has aiwcrf_surrogate_num_params() floats. */
int aiwcrf_surrogate_grad(const aiwcrf_surrogate *surrogate, const float *X, const float *y,
                          int32_t n, float *grad, float *loss, void *cuda_stream);

/* Build a surrogate from a host parameter vector and feature transform (mean, standard
 * deviation and log2 flag of each of the F-2 AIWC columns). */
int aiwcrf_surrogate_create(int32_t n_features, int32_t n_devices, int32_t n_sizes,
                            const float *params, const float *mu, const float *sd,
                            const uint8_t *log2_cols, aiwcrf_surrogate **out);

/* Copy out parameters and feature transform (host arrays; any may be NULL). */
int aiwcrf_surrogate_export(const aiwcrf_surrogate *surrogate, float *params, float *mu,
                            float *sd, uint8_t *log2_cols);
int aiwcrf_surrogate_stats(const aiwcrf_surrogate *surrogate, aiwcrf_surrogate_fit_stats *out);
int32_t aiwcrf_surrogate_num_params(void);

/* Waits for the device (work reading the network may be in flight on any stream), then returns
 * its memory to the stream-ordered pool: no cudaFree, so no device-wide wait inside the free.
 * NULL is accepted. */
int aiwcrf_surrogate_free(aiwcrf_surrogate *surrogate);

/* ---------------------------------------------------------------------------------------------
 * Device-selection server. Sec. VI's use of the model is a scheduler that asks, for kernels about
 * to run, which device will be fastest; Sec. I notes the model is retrained only when the set of
 * devices changes. The server keeps a forest resident on the device and answers requests
 * (1..max_request_kernels kernels of one size class, each against every server device) by
 * continuous batching:
 *  - A dispatcher thread owns n_streams stream slots. Whenever a slot is free it takes the
 *    pending requests in arrival order, as many as fit in one batch (batch_kernels kernels) and
 *    in the device arena, and launches them as one batch: a host-to-device copy of the features,
 *    one selection kernel (trees spread over warps, exact int64 sums, argmin with ties to the
 *    lower device id), a device-to-host copy of the results. Batches on different slots run
 *    concurrently; requests arriving meanwhile queue for the next free slot.
 *  - Admission by device memory: every batch's inputs and outputs live in a first-fit arena of
 *    arena_bytes carved from one allocation made at creation. A batch takes requests only while
 *    their bytes fit the arena's free space; the rest wait for batches to complete and release
 *    theirs. A request that could never fit, has more than max_request_kernels kernels, or
 *    arrives while max_pending requests wait, is refused with AIWCRF_E_LIMIT.
 *  - Refit: rows appended with aiwcrf_server_append are held on the host. Every refit_every
 *    completed requests (and on aiwcrf_server_refit) a refit thread moves refit_rows of them
 *    (all when 0) into the training set, fits a new forest with the creation's fit parameters on
 *    its own low-priority stream as a background fit (ctas_per_sm = 1, the same forest), and
 *    swaps it in. Each batch uses the forest current when it was formed, and
 *    each result reports that forest's generation (0 = the forest fitted at creation). A result
 *    equals aiwcrf_select_device on a forest fitted by aiwcrf_fit on the same rows.
 * Host pointers throughout; the server copies what it keeps. The device is the calling thread's
 * current device at creation.
 * The GPU runs the server's n_streams + 1 streams, and any other stream of the process, on a
 * fixed number of hardware queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless set in the process
 * environment before CUDA initialises). A selection stream that shares a queue with the refit
 * stream waits in order behind the refit's queued kernels; a refit enqueues one tree level at a
 * time to bound that wait, and a process that serves while refitting should set
 * CUDA_DEVICE_MAX_CONNECTIONS=32. */
typedef struct aiwcrf_server aiwcrf_server;

typedef struct {
    int32_t n_streams;            /* batches in flight at once, 1..16 (4) */
    int32_t max_request_kernels;  /* kernels of one request, 1..4096 (64) */
    int32_t batch_kernels;        /* kernels of one batch, max_request_kernels..65536 (1024) */
    int32_t max_pending;          /* requests waiting for a slot, >= 1 (65536) */
    int64_t arena_bytes;          /* device arena for batch inputs and outputs (64 MiB) */
    int64_t refit_every;          /* completed requests between automatic refits; 0 = never */
    int64_t refit_rows;           /* appended rows one refit consumes; 0 = all appended */
} aiwcrf_server_params;

typedef struct {
    int64_t submitted;            /* requests accepted */
    int64_t rejected;             /* requests refused with AIWCRF_E_LIMIT */
    int64_t completed;
    int64_t failed;               /* completed with an error */
    int64_t batches;
    int64_t batch_kernels_total;  /* sum over batches of their kernels */
    int64_t batch_kernels_max;
    int64_t arena_waits;          /* batches cut short because the arena was full */
    int64_t arena_bytes;
    int64_t arena_peak_bytes;     /* most arena bytes held at once */
    int64_t refits;               /* forests swapped in after creation */
    int64_t refit_failures;
    int64_t generation;           /* generation of the current forest */
    int64_t training_rows;        /* rows the current forest was fitted on */
    int64_t appended_rows;        /* appended rows not yet consumed by a refit */
    int64_t forest_bytes;         /* device bytes of the current forest */
    int64_t refit_us_total;       /* wall time of all refits (rows staged, fit, swap) */
    int64_t refit_us_max;
    int64_t gated_kernels;        /* kernels of completed gated requests */
    int64_t gated_fallback;       /* ... answered by the forest */
    int64_t gated_fallback_ood;   /* ... with an out-of-range feature */
    int64_t gated_fallback_var;   /* ... whose surrogate margin was within z deviations */
    int64_t surrogate_bytes;      /* device bytes of the resident surrogate (0: none) */
} aiwcrf_server_counters;

typedef struct {
    int64_t n_requests;
    int64_t n_kernels;            /* sum of the requests' kernels */
    double offered_rate;          /* requests per second of the Poisson arrival process */
    double wall_s;                /* first arrival to last completion */
    double requests_per_s;        /* n_requests / wall_s */
    double kernels_per_s;
    double p50_us, p99_us, mean_us, max_us;   /* arrival to completion */
    int64_t batches;              /* batches launched during the run */
    double mean_batch_kernels;
    int64_t refits;               /* refits finished during the run */
    int64_t failed;               /* requests that completed with an error or were abandoned */
    int64_t rejected;             /* requests refused on arrival (AIWCRF_E_LIMIT) */
} aiwcrf_load_report;

/* X: host, F x n_rows column-major training matrix (columns F-2 and F-1 are the device id and
 * the size class); y: host Q32.32 targets; device_ids: host, the n_devices (1..64) devices
 * every request is answered for. Fits the generation-0 forest before returning. */
int aiwcrf_server_create(const aiwcrf_server_params *params, const aiwcrf_fit_params *fit,
                         const float *X, const int64_t *y, int64_t n_rows, int32_t n_features,
                         const int32_t *device_ids, int32_t n_devices, aiwcrf_server **out);

/* Queue one request: kfeat is a host (F-2) x n_kernels column-major matrix (copied before
 * returning). *ticket identifies it for aiwcrf_server_wait. */
int aiwcrf_server_submit(aiwcrf_server *server, const float *kfeat, int32_t n_kernels,
                         int32_t size_class, int64_t *ticket);

/* Wait up to timeout_ms (< 0: without limit) for a request; AIWCRF_E_TIMEOUT if it is still
 * running (the ticket stays valid). On completion writes best (host, n_kernels device ids),
 * pred (host n_kernels x n_devices row-major Q32.32, or NULL) and generation (or NULL), and
 * retires the ticket; returns the request's status. */
int aiwcrf_server_wait(aiwcrf_server *server, int64_t ticket, int32_t timeout_ms, int32_t *best,
                       int64_t *pred, int64_t *generation);

/* Append training rows (host, F x n_rows column-major, and targets) for later refits. */
int aiwcrf_server_append(aiwcrf_server *server, const float *X, const int64_t *y, int64_t n_rows);

/* Ask for a refit now; with wait != 0 return once it finished (its status). */
int aiwcrf_server_refit(aiwcrf_server *server, int32_t wait);

/* While paused != 0 the dispatcher forms no new batch (queued requests wait; batches in flight
 * complete). */
int aiwcrf_server_pause(aiwcrf_server *server, int32_t paused);

int aiwcrf_server_stats(aiwcrf_server *server, aiwcrf_server_counters *out);

/* Open-loop load generator: request i arrives at the i-th event of a Poisson process of
 * rate_per_s (exponential gaps from a SplitMix64 stream of seed) and asks for kernels
 * pool[:, first[i] .. first[i] + n_kernels[i]) of size class size_class[i]; pool is a host
 * (F-2) x pool_kernels column-major matrix. Latency runs from the scheduled arrival to the
 * dispatcher seeing the batch complete, so a late submission counts against it. Optional host
 * outputs: best (sum of n_kernels entries, in request order), generation and latency_ns (one per
 * request; a refused request keeps its best entries and gets latency -1). Returns the first failing request's status, or AIWCRF_E_TIMEOUT if requests were
 * still running after timeout_ms (they are then abandoned without writing the outputs). */
int aiwcrf_server_run_load(aiwcrf_server *server, const float *pool, int64_t pool_kernels,
                           const int64_t *first, const int32_t *n_kernels, const int32_t *size_class,
                           int64_t n_requests, double rate_per_s, uint64_t seed, int32_t timeout_ms,
                           int32_t *best, int64_t *generation, int64_t *latency_ns,
                           aiwcrf_load_report *report);

/* Trace of the most recent batches and refits (steady-clock nanoseconds, oldest first): the
 * server keeps the last 65,536 batches and 256 refits. A batch was formed (requests taken from
 * the queue), enqueued (its copies and kernel handed to the stream) and done (completion seen by
 * the dispatcher). A refit started (rows taken), staged its rows on the device, finished the fit
 * and swapped the forest in. */
/* One batch: when it was formed, when its copies, kernel and event had been enqueued, and when
 * the dispatcher saw it complete (steady-clock ns). Where a slow batch's time went:
 *  - enqueue_cpu_ns: CPU time of the dispatcher thread while enqueuing (against the wall time
 *    t_enqueued_ns - t_formed_ns: a large gap means the thread waited);
 *  - enqueue_voluntary_switches / enqueue_involuntary_switches: the thread's context switches
 *    while enqueuing (voluntary: it blocked, e.g. on a driver lock; involuntary: the operating
 *    system preempted it for another thread or process);
 *  - poll_gap_max_ns: the longest interval between two consecutive completion polls of the
 *    batch by the dispatcher (a gap near the batch's time means the completion was seen late,
 *    not that the GPU was slow). */
typedef struct {
    int64_t t_formed_ns, t_enqueued_ns, t_done_ns;
    int32_t kernels, generation;
    int64_t enqueue_cpu_ns;
    int32_t enqueue_voluntary_switches, enqueue_involuntary_switches;
    int64_t poll_gap_max_ns;
    int32_t gated_kernels;        /* kernels of gated requests in the batch */
    int32_t fallback_kernels;     /* ... of which the forest answered */
} aiwcrf_batch_trace;

typedef struct {
    int64_t t_start_ns, t_staged_ns, t_fitted_ns, t_swapped_ns;
    int64_t rows, generation;
} aiwcrf_refit_trace;

/* Copies up to cap batch records into batches and up to rcap refit records into refits (either
 * may be NULL with cap 0); *n and *rn receive the numbers copied. */
int aiwcrf_server_trace(aiwcrf_server *server, aiwcrf_batch_trace *batches, int64_t cap, int64_t *n,
                        aiwcrf_refit_trace *refits, int64_t rcap, int64_t *rn);

/* Stop the dispatcher and refit threads (queued requests fail with AIWCRF_E_INVALID_ARG; batches
 * in flight complete first) and free everything. */
int aiwcrf_server_destroy(aiwcrf_server *server);

/* Device selection through the surrogate with the forest as fallback and judge (the paper has no
 * surrogate; its selection of Sec. VI queries the forest). For each kernel k the D queries
 * (k, device_ids[j]) are predicted by the surrogate, s_j (NaN counts as +infinity); b is the
 * argmin and r the runner-up (ties: lower device id). The kernel falls back to the forest when
 *  - gate->ood = 1 and a feature of one of its queries lies outside [smallest, largest] of the
 *    forest's training values of that column, or is NaN; or
 *  - the surrogate's margin is within z standard deviations of the ensemble spread of the two
 *    contenders: with V_j = var_trees * sum_t v_t^2 - (sum_t v_t)^2 over the forest's first
 *    var_trees trees' leaf values v_t (Q32.32, exact), the test is
 *        ((s_r - s_b)^2 * var_trees^2) * 2^64  <=  (z * z) * (V_b + V_r)
 *    evaluated in IEEE double with round-to-nearest in exactly this order, V_b + V_r converted
 *    as double(high 64 bits) * 2^64 + double(low 64 bits); or
 *  - the surrogate's margin is below a fixed threshold: double(s_r) - double(s_b) < tau (log10
 *    seconds; tau = 0 never holds).
 * With one device there is no runner-up and only the range test applies.
 * A kernel that falls back gets exactly aiwcrf_select_device's device and the forest's
 * predictions (converted to float log10 s); the others get b and the surrogate's predictions.
 * kfeat ((F-2) x K), out_best (K), out_pred (K x D float, or NULL) and out_fallback (K bytes,
 * 1 = forest, or NULL) are device memory; device_ids and stats (or NULL) are host memory. The
 * call synchronises its stream. */
typedef struct {
    int32_t var_trees;      /* 1..num_trees (32) */
    float z;                /* margin in ensemble standard deviations, 0 <= z < 2^20 (1) */
    int32_t ood;            /* 1: out-of-range features fall back (1) */
    float tau;              /* margin threshold in log10 seconds, 0 <= tau < 2^20 (0: none) */
} aiwcrf_gate_params;

typedef struct {
    int64_t kernels;
    int64_t fallback;       /* kernels answered by the forest */
    int64_t fallback_ood;   /* ... with an out-of-range feature */
    int64_t fallback_var;   /* ... whose surrogate margin was within z deviations or below tau */
} aiwcrf_gate_stats;

int aiwcrf_select_device_gated(const aiwcrf_forest *forest, const aiwcrf_surrogate *surrogate,
                               const aiwcrf_gate_params *gate, const float *kfeat, int32_t n_kernels,
                               int32_t size_class, const int32_t *device_ids, int32_t n_devices,
                               int32_t *out_best, float *out_pred, uint8_t *out_fallback,
                               aiwcrf_gate_stats *stats, void *cuda_stream);

/* Gated requests in the device-selection server: the surrogate resident beside the forest.
 * aiwcrf_server_set_surrogate copies the surrogate (the caller may free its own afterwards) and
 * keeps gate (checked as for aiwcrf_select_device_gated against the server's forest); NULL
 * removes it, and gated requests still queued then fail with AIWCRF_E_INVALID_ARG. The surrogate
 * must have the server's n_features and live on the server's device. Batches already formed keep
 * the surrogate they were formed with; a refit replaces the forest but not the surrogate (the gate
 * and the fallback use the new forest).
 * A gated request (aiwcrf_server_submit_gated: as aiwcrf_server_submit; refused with
 * AIWCRF_E_INVALID_ARG while no surrogate is held, and with AIWCRF_E_LIMIT if its batch bytes can
 * never fit the arena) is answered as aiwcrf_select_device_gated answers the same kernels on the
 * forest of its batch's generation: the surrogate's device, or the forest's where the gate
 * falls back. It shares batches with exact requests: a batch puts its gated requests' kernels
 * first, runs the surrogate, the prefix variances and the gate on those, then one selection kernel
 * for the exact kernels and the gated kernels that fell back, with no host synchronisation in
 * between. aiwcrf_server_wait_gated writes best (host, n_kernels device ids), pred (host
 * n_kernels x n_devices row-major float log10 seconds, or NULL) and fallback (host n_kernels bytes,
 * 1 = the forest answered, or NULL); aiwcrf_server_wait refuses a gated ticket and
 * aiwcrf_server_wait_gated an exact one, without retiring it.
 * aiwcrf_server_run_load_gated is aiwcrf_server_run_load with request i gated where gated[i] != 0
 * (gated may be NULL: none). */
int aiwcrf_server_set_surrogate(aiwcrf_server *server, const aiwcrf_surrogate *surrogate,
                                const aiwcrf_gate_params *gate);
int aiwcrf_server_submit_gated(aiwcrf_server *server, const float *kfeat, int32_t n_kernels,
                               int32_t size_class, int64_t *ticket);
int aiwcrf_server_wait_gated(aiwcrf_server *server, int64_t ticket, int32_t timeout_ms, int32_t *best,
                             float *pred, uint8_t *fallback, int64_t *generation);
int aiwcrf_server_run_load_gated(aiwcrf_server *server, const float *pool, int64_t pool_kernels,
                                 const int64_t *first, const int32_t *n_kernels,
                                 const int32_t *size_class, const uint8_t *gated, int64_t n_requests,
                                 double rate_per_s, uint64_t seed, int32_t timeout_ms, int32_t *best,
                                 int64_t *generation, int64_t *latency_ns, aiwcrf_load_report *report);

/* Fit plan: the whole fit of aiwcrf_fit / aiwcrf_fit_subsets captured once as a CUDA graph and
 * replayed (the batched leave-one-kernel-out fits of Alg. 1 run as one graph launch). The graph
 * holds the presort, ranks and groups, the bootstrap, and a device-side loop over the tree
 * levels (a conditional WHILE node whose body grows two levels; a kernel ends it when no node
 * is left), so no host synchronisation happens inside the fit; the host then packs the forests.
 * X ((n_features x n_rows), y and subset_rows (or NULL for one forest on all rows) are device
 * memory bound to the plan and read at every run: a run fits the data they hold then. The plan
 * sizes its tables from the data at creation (rank width, number of distinct feature vectors);
 * a run on data that outgrows them fails with AIWCRF_E_LIMIT. subset_offsets is a host array.
 * Results equal aiwcrf_fit / aiwcrf_fit_subsets on the same data, bit for bit, for every
 * schedule. The plan owns its device tables (about 150 bytes per (tree, distinct row) pair)
 * until aiwcrf_fit_plan_free. */
typedef struct aiwcrf_fit_plan aiwcrf_fit_plan;

/* A launch schedule of the level loop: resident CTAs per SM of the grid-stride level kernels. */
typedef struct {
    int32_t level_big_ctas_per_sm;     /* 1..the CTAs per SM the big-node kernel is built for */
    int32_t level_small_ctas_per_sm;   /* 1..the same for the small-node kernel */
    float ms;                          /* median wall time of a run with this schedule (tuning) */
    int32_t reserved;
} aiwcrf_fit_schedule;

int aiwcrf_fit_plan_create(const aiwcrf_fit_params *params, const float *X, const int64_t *y, int64_t n_rows,
                           int32_t n_features, const int64_t *subset_offsets, const int32_t *subset_rows,
                           int32_t n_subsets, void *cuda_stream, aiwcrf_fit_plan **out);

/* Replay the fit; out receives n_subsets forests (1 without subsets). Synchronises the stream. */
int aiwcrf_fit_plan_run(aiwcrf_fit_plan *plan, void *cuda_stream, aiwcrf_forest **out);

/* Autotuner: times every schedule (reps runs each, median) on the plan's data, keeps the
 * fastest, and reports them (tried: host array of cap entries or NULL; *n_tried the number
 * tried; chosen or NULL). */
int aiwcrf_fit_plan_tune(aiwcrf_fit_plan *plan, int32_t reps, void *cuda_stream, aiwcrf_fit_schedule *tried,
                         int32_t cap, int32_t *n_tried, aiwcrf_fit_schedule *chosen);

/* Set a schedule explicitly (the graph is captured again). */
int aiwcrf_fit_plan_set_schedule(aiwcrf_fit_plan *plan, const aiwcrf_fit_schedule *schedule);

/* Waits for the device, destroys the captured graph and returns the plan's tables to the
 * stream-ordered pool (no cudaFree, so no device-wide wait inside the free). NULL is accepted. */
int aiwcrf_fit_plan_free(aiwcrf_fit_plan *plan);

/* Bounds checks of a debug build (no counterpart in the paper; the stand-in for an external
 * memory checker). A library built with -DAIWCRF_DEBUG_BOUNDS (libaiwcrf_debug.so) checks every
 * gathered entry row or group id, node id of a level's tables and of a tree walk, split
 * feature, histogram bin and output position of the fit, predict and selection kernels
 * against its array's extent; a violation is recorded and the access redirected to index 0.
 * Returns the OR of the violated sites since the last call (1 row/group, 2 node, 4 walk node,
 * 8 feature, 16 bin, 32 output position; 0 = none) and clears it; -1 in a release build, which
 * compiles the checks away. Reading the flags synchronises the device. */
int64_t aiwcrf_debug_bounds(void);

/* Which kernels grow the trees of the following fits in this process (the paper has no
 * counterpart: both give the same forest, node for node, for the model of Sec. III-B).
 *  AIWCRF_GROWER_AUTO (default): tree-resident when it fits, else level-synchronous with
 *    presorted lists when a column has more than 4,096 distinct values, else level-synchronous.
 *  AIWCRF_GROWER_LEVEL: level-synchronous, every depth of every tree as three launches
 *    (big-node CTAs, small-node warps, a finalize pass); a big node's search builds shared-memory
 *    histograms over every rank of its tried features.
 *  AIWCRF_GROWER_LISTS: level-synchronous, a big node's search scans presorted lists instead:
 *    every tree keeps its entries in rank order per feature (4 bytes per entry and feature, twice,
 *    and 12 bytes per tree and row) and each depth partitions them with the entries. Its cost per
 *    node follows the node's entries, not the columns' value counts.
 *  AIWCRF_GROWER_TREE: tree-resident, one CTA grows a whole tree with its entries in shared
 *    memory; a fit whose trees do not fit (ranks wider than one byte, more than 32 features,
 *    more than 65,535 groups, or too many entries per tree for shared memory) fails with
 *    AIWCRF_E_LIMIT. Fit plans always use the level-synchronous kernels.
 * AIWCRF_E_INVALID_ARG for another value. The forest's aiwcrf_fit_stats.grower says which
 * ran. */
#define AIWCRF_GROWER_AUTO 0
#define AIWCRF_GROWER_LEVEL 1
#define AIWCRF_GROWER_TREE 2
#define AIWCRF_GROWER_LISTS 3
int aiwcrf_set_grower(int32_t grower);

/* Counters of the fit that produced the forest (zeros for a deserialized forest). The paper has
 * no counterpart: these count the work of the fit (Sec. III-B) for measurement. */
int aiwcrf_forest_stats(const aiwcrf_forest *forest, aiwcrf_fit_stats *out);

/* Number of trees, packed nodes (including alignment padding) and features (the fitted model of
 * Sec. III-B; its layout is this library's). */
int aiwcrf_forest_info(const aiwcrf_forest *forest, int64_t *num_trees, int64_t *num_nodes,
                       int32_t *n_features);

/* Checkpoint of a fitted forest. The paper's model is fitted once and needs refitting only when
 * a new kind of device is added (Sec. I); keeping it between processes is this library's, with
 * no counterpart in the paper.
 * Versioned little-endian blob of the packed forest, into a host buffer. With buf == NULL or
 * cap too small, *needed receives the size and AIWCRF_E_INVALID_ARG is returned for a short
 * non-NULL buffer. Layout: "AIWCRF01", u32 version (1), u32 n_features, i64 num_trees,
 * i64 num_nodes, i64 tree_offset[num_trees + 1], u64 node[num_nodes]. Node encoding: bit 63
 * set = leaf with value bits 0..62 (sign-extended); else bits 0..31 threshold (float32),
 * bits 32..55 left-child index within the tree (right = left + 1), bits 56..62 feature.
 * Trees are padded to an even node count with one unreachable leaf of value 0. */
int aiwcrf_forest_serialize(const aiwcrf_forest *forest, void *buf, size_t cap, size_t *needed);

/* Resume from a checkpoint (see aiwcrf_forest_serialize): rebuild a forest on the current device
 * from a blob (validated: AIWCRF_E_CORRUPT). Out-of-bag evaluation is not available on it. */
int aiwcrf_forest_deserialize(const void *buf, size_t len, aiwcrf_forest **out);

/* Releases a forest (library resource management; no counterpart in the paper). Waits for the
 * device (work reading the forest may be in flight on any stream), then returns the forest's
 * memory to the stream-ordered pool. NULL is accepted. */
int aiwcrf_forest_free(aiwcrf_forest *forest);

/* Message of the last failing call on this host thread ("" if none; every call clears it on
 * entry). Error reporting of this library; no counterpart in the paper. */
const char *aiwcrf_last_error(void);

/* Optional per-kernel timing with CUDA events recorded on the launching stream around each
 * library kernel launch. Off by default. aiwcrf_profile_read synchronises the events and
 * returns, per kernel class k < n (names via aiwcrf_profile_name), the launch count and the
 * summed duration in milliseconds; it then clears the record. */
int aiwcrf_profile_enable(int32_t on);
/* Restrict the timing to the kernel classes whose bit k is set in mask (all by default): each
 * recorded pair of events costs the stream a little time. */
int aiwcrf_profile_classes(uint32_t mask);
int aiwcrf_profile_read(int32_t n, int64_t *launches, double *total_ms);
const char *aiwcrf_profile_name(int32_t k);
int32_t aiwcrf_profile_num_classes(void);

/* Number of CUDA kernels this library has launched in this process (all devices). */
int64_t aiwcrf_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* AIWCRF_H */
