/*
 * aiwcrf_oracle.c -- plain, slow CPU restatement of the random-forest regression the paper fits
 * (ranger random forest with num.trees / mtry / min.node.size, Sec. III-B) and of how it is
 * queried (predict a kernel's time on each device, Sec. I and Sec. VI).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load this file. It shares no code with the CUDA library: it has its own Philox, its own
 * split search (sorting node rows by feature value, not ranks), its own exact big-integer
 * arithmetic (base 2^32 limbs) and its own tree layout.
 *
 * The paper only names the model (ranger, Breiman's random forest) and its three parameters.
 * Every step below is the reading fixed for this library:
 *
 *  1. Bootstrap (ranger's default, sampling with replacement, fraction 1). Tree t draws n_pool
 *     rows: draw k takes word (k & 3) of Philox4x32-10(key = seed, ctr = (t, k >> 2, 0xB007, 0))
 *     and maps it to pool index (u * n_pool) >> 32. w[row] = number of times drawn.
 *     With bootstrap off every row has w = 1.
 *  2. Nodes are grown breadth first. Node i at depth d (0-based, BFS order within the depth)
 *     creates its children left then right; depth d+1 is numbered in that order.
 *  3. A node with n = sum(w) <= min_node_size, or at depth == max_depth (max_depth > 0), is a leaf.
 *  4. mtry features: key_f = word (f & 3) of Philox4x32-10(seed, (t, d, i, 0x3779 << 16 | f >> 2));
 *     the mtry features with the smallest (key_f, f) are tried ("mtry, the number of features
 *     tried to possibly split within each node", Sec. III-B).
 *  5. For a tried feature the node's rows are sorted by value; every boundary between two
 *     consecutive distinct values v_a < v_b is a candidate "x <= v_a goes left". The CART
 *     regression criterion G = S_L^2/n_L + S_R^2/n_R (n = sum w, S = sum w*y) is maximised,
 *     compared exactly as rationals with big integers. Ties: lowest feature, then lowest
 *     threshold. The split is made only if G > S^2/n strictly; otherwise the node is a leaf.
 *  6. The stored threshold is v_a itself (the largest value sent left), with -0 read as +0.
 *  7. Leaf value = round(S/n) half up, i.e. floor((2S + n) / (2n)), in Q32.32.
 *  8. Forest prediction = floor((2P + T) / (2T)) with P the exact int64 sum of the T leaf values
 *     reached (random forest regression averages its trees). The ensemble variance numerator
 *     V = T * sum(v^2) - P^2 is reported exactly as an unsigned 128-bit integer.
 *  9. Device selection (Sec. VI): the device with the smallest predicted time; ties go to the
 *     lower device id.
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle_aiwcrf.so aiwcrf_oracle.c
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------------------------------ */
/* Philox-4xW-R, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"   */
/* (SC'11). One round multiplies words 0 and 2 by the round multipliers, XORs the high halves */
/* with the other two words and the round key, and permutes; the key is bumped by the Weyl    */
/* constants between rounds.                                                                  */
/* ------------------------------------------------------------------------------------------ */
/* One implementation for both word widths: words are held in 64-bit variables, products in
 * 128 bits, and every result is masked to the width. */
static void philox4xW(int bits, const uint64_t M[2], const uint64_t W[2], const uint64_t ctr_in[4],
                      const uint64_t key_in[2], int rounds, uint64_t out[4])
{
    const uint64_t mask = bits == 64 ? ~0ull : ((1ull << bits) - 1);
    uint64_t c[4] = {ctr_in[0] & mask, ctr_in[1] & mask, ctr_in[2] & mask, ctr_in[3] & mask};
    uint64_t k0 = key_in[0] & mask, k1 = key_in[1] & mask;
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) { k0 = (k0 + W[0]) & mask; k1 = (k1 + W[1]) & mask; }
        u128 p0 = (u128)M[0] * c[0];
        u128 p1 = (u128)M[1] * c[2];
        uint64_t hi0 = (uint64_t)(p0 >> bits) & mask, lo0 = (uint64_t)p0 & mask;
        uint64_t hi1 = (uint64_t)(p1 >> bits) & mask, lo1 = (uint64_t)p1 & mask;
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    for (int j = 0; j < 4; ++j) out[j] = c[j];
}

/* Philox4x32: multipliers and Weyl key increments of the 32-bit member. */
void orc_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], int rounds, uint32_t out[4])
{
    const uint64_t M[2] = {0xD2511F53u, 0xCD9E8D57u};
    const uint64_t W[2] = {0x9E3779B9u, 0xBB67AE85u};
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]}, k[2] = {key_in[0], key_in[1]}, o[4];
    philox4xW(32, M, W, c, k, rounds, o);
    for (int j = 0; j < 4; ++j) out[j] = (uint32_t)o[j];
}

/* Philox4x64: the 64-bit member; exported so the shared round code can be checked against an
 * independent library implementation of Philox4x64-10. */
void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], int rounds, uint64_t out[4])
{
    const uint64_t M[2] = {0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull};
    const uint64_t W[2] = {0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull};
    philox4xW(64, M, W, ctr_in, key_in, rounds, out);
}

#define DOM_BOOT 0xB007u
#define DOM_MTRY 0x3779u

static uint32_t draw_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32(ctr, key, 10, out);
    return out[word];
}

/* Step 1: bootstrap multiplicities over a pool of n_pool rows for tree t. */
void orc_bootstrap_counts(uint64_t seed, int64_t t, int64_t n_pool, uint32_t *counts)
{
    for (int64_t j = 0; j < n_pool; ++j) counts[j] = 0;
    for (int64_t k = 0; k < n_pool; ++k) {
        uint32_t u = draw_word(seed, (uint32_t)t, (uint32_t)(k >> 2), DOM_BOOT, 0, (int)(k & 3));
        uint64_t j = ((uint64_t)u * (uint64_t)n_pool) >> 32;
        counts[j] += 1;
    }
}

/* Step 4: the mtry features tried at node (t, d, i); written in increasing feature order. */
void orc_mtry_draw(uint64_t seed, int64_t t, int64_t d, int64_t i, int32_t F, int32_t mtry, int32_t *out)
{
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)F);
    for (int32_t f = 0; f < F; ++f)
        key[f] = draw_word(seed, (uint32_t)t, (uint32_t)d, (uint32_t)i,
                           (DOM_MTRY << 16) | (uint32_t)(f >> 2), f & 3);
    int32_t m = mtry < F ? mtry : F;
    int32_t nout = 0;
    /* feature f is chosen iff fewer than m features have a smaller (key, index) pair */
    for (int32_t f = 0; f < F; ++f) {
        int32_t smaller = 0;
        for (int32_t g = 0; g < F; ++g)
            if (key[g] < key[f] || (key[g] == key[f] && g < f)) ++smaller;
        if (smaller < m) out[nout++] = f;
    }
    free(key);
}

/* ------------------------------------------------------------------------------------------ */
/* Exact unsigned big integers, base 2^32, fixed width. Plain schoolbook arithmetic.          */
/* ------------------------------------------------------------------------------------------ */
#define BIG_LIMBS 12
typedef struct { uint32_t w[BIG_LIMBS]; } big;

static big big_u64(uint64_t v)
{
    big r; memset(&r, 0, sizeof r);
    r.w[0] = (uint32_t)v; r.w[1] = (uint32_t)(v >> 32);
    return r;
}

static big big_mul(big a, big b)
{
    big r; memset(&r, 0, sizeof r);
    for (int i = 0; i < BIG_LIMBS; ++i) {
        uint64_t carry = 0;
        for (int j = 0; i + j < BIG_LIMBS; ++j) {
            uint64_t cur = (uint64_t)r.w[i + j] + (uint64_t)a.w[i] * b.w[j] + carry;
            r.w[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
    }
    return r;
}

static big big_add(big a, big b)
{
    big r; uint64_t carry = 0;
    for (int i = 0; i < BIG_LIMBS; ++i) {
        uint64_t cur = (uint64_t)a.w[i] + b.w[i] + carry;
        r.w[i] = (uint32_t)cur;
        carry = cur >> 32;
    }
    return r;
}

static int big_cmp(big a, big b)
{
    for (int i = BIG_LIMBS - 1; i >= 0; --i) {
        if (a.w[i] < b.w[i]) return -1;
        if (a.w[i] > b.w[i]) return 1;
    }
    return 0;
}

static uint64_t abs_i64(int64_t v) { return v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v; }

/* G = S_L^2/n_L + S_R^2/n_R held as the fraction num/den, num = S_L^2 n_R + S_R^2 n_L,
 * den = n_L n_R. */
typedef struct { big num, den; } gain_t;

static gain_t gain_of(int64_t nL, int64_t SL, int64_t nR, int64_t SR)
{
    big sl = big_u64(abs_i64(SL)), sr = big_u64(abs_i64(SR));
    gain_t g;
    g.num = big_add(big_mul(big_mul(sl, sl), big_u64((uint64_t)nR)),
                    big_mul(big_mul(sr, sr), big_u64((uint64_t)nL)));
    g.den = big_mul(big_u64((uint64_t)nL), big_u64((uint64_t)nR));
    return g;
}

/* sign of G_a - G_b */
static int gain_cmp(gain_t a, gain_t b)
{
    return big_cmp(big_mul(a.num, b.den), big_mul(b.num, a.den));
}

/* exported for tests: sign(G(a) - G(b)) for two candidate splits */
int orc_gain_cmp(int64_t nLa, int64_t SLa, int64_t nRa, int64_t SRa,
                 int64_t nLb, int64_t SLb, int64_t nRb, int64_t SRb)
{
    return gain_cmp(gain_of(nLa, SLa, nRa, SRa), gain_of(nLb, SLb, nRb, SRb));
}

/* G > S^2 / n  <=>  num * n > S^2 * den */
static int gain_beats_parent(gain_t g, int64_t n, int64_t S)
{
    big s = big_u64(abs_i64(S));
    return big_cmp(big_mul(g.num, big_u64((uint64_t)n)), big_mul(big_mul(s, s), g.den)) > 0;
}

/* floor(a / b) for b > 0 */
static i128 floor_div(i128 a, i128 b)
{
    i128 q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

int64_t orc_round_mean(int64_t S, int64_t n)
{
    return (int64_t)floor_div((i128)2 * S + n, (i128)2 * n);
}

/* ------------------------------------------------------------------------------------------ */
/* Trees                                                                                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t feature;     /* -1 for a leaf */
    float thr;           /* x <= thr goes left */
    int64_t left;        /* BFS index of the left child (right = left + 1); -1 for a leaf */
    int64_t value;       /* leaf value, Q32.32 */
    int64_t n;           /* sum of w */
    int64_t S;           /* sum of w*y */
    int64_t nrows;       /* distinct in-bag rows in the node */
    int32_t depth;
    int32_t evaluated;   /* 1 if a split was searched for (not stopped by size or depth) */
    int64_t *rows;       /* rows in the node while growing; freed afterwards */
} onode;

typedef struct {
    onode *nodes;
    int64_t count, cap;
} otree;

struct orc_forest {
    int64_t t0, t1;      /* global tree indices [t0, t1) */
    int32_t F;
    otree *trees;
    uint64_t seed;       /* the fit's bootstrap, kept for out-of-bag evaluation */
    int32_t bootstrap;
    int64_t N;
};
typedef struct orc_forest orc_forest;

static int64_t push_node(otree *tr)
{
    if (tr->count == tr->cap) {
        tr->cap = tr->cap ? 2 * tr->cap : 64;
        tr->nodes = (onode *)realloc(tr->nodes, sizeof(onode) * (size_t)tr->cap);
    }
    memset(&tr->nodes[tr->count], 0, sizeof(onode));
    return tr->count++;
}

/* sort context for qsort: one per host thread, so trees may be grown on several threads */
static _Thread_local const float *g_col;
static int cmp_rows_by_value(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    float va = g_col[a], vb = g_col[b];
    if (va < vb) return -1;
    if (vb < va) return 1;
    return (a > b) - (a < b);
}

/* Grow tree t (global index) on rows 0..N-1. */
static void grow_tree(otree *tr, const float *X, const int64_t *y, int64_t N, int32_t F,
                      int64_t t, int32_t mtry, int32_t min_node, int32_t max_depth,
                      uint64_t seed, int32_t bootstrap)
{
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    if (bootstrap) orc_bootstrap_counts(seed, t, N, w);
    else for (int64_t r = 0; r < N; ++r) w[r] = 1;

    int64_t root = push_node(tr);
    onode *nd = &tr->nodes[root];
    nd->rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t r = 0; r < N; ++r)
        if (w[r] > 0) nd->rows[nd->nrows++] = r;
    for (int64_t k = 0; k < nd->nrows; ++k) {
        nd->n += w[nd->rows[k]];
        nd->S += (int64_t)w[nd->rows[k]] * y[nd->rows[k]];
    }
    nd->depth = 0;

    int32_t *feats = (int32_t *)malloc(sizeof(int32_t) * (size_t)F);
    int64_t *sorted = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));

    int64_t level_begin = 0, level_end = 1;
    for (int32_t d = 0; level_begin < level_end; ++d) {
        for (int64_t id = level_begin; id < level_end; ++id) {
            int64_t i = id - level_begin;          /* BFS index within depth d */
            onode *node = &tr->nodes[id];
            int64_t n = node->n, S = node->S;
            int split = 0;
            int32_t best_f = -1;
            float best_thr = 0.0f;
            gain_t best_g;
            int64_t best_nL = 0, best_SL = 0;

            if (n > min_node && !(max_depth > 0 && d == max_depth)) {
                node->evaluated = 1;
                int32_t m = mtry < F ? mtry : F;
                orc_mtry_draw(seed, t, d, i, F, mtry, feats);
                for (int32_t q = 0; q < m; ++q) {
                    int32_t f = feats[q];
                    const float *col = X + (size_t)f * (size_t)N;
                    memcpy(sorted, node->rows, sizeof(int64_t) * (size_t)node->nrows);
                    g_col = col;
                    qsort(sorted, (size_t)node->nrows, sizeof(int64_t), cmp_rows_by_value);
                    int64_t nL = 0, SL = 0;
                    for (int64_t p = 0; p + 1 < node->nrows; ++p) {
                        int64_t r = sorted[p];
                        nL += w[r];
                        SL += (int64_t)w[r] * y[r];
                        float va = col[r], vb = col[sorted[p + 1]];
                        if (!(va < vb)) continue;       /* not a boundary between distinct values */
                        gain_t g = gain_of(nL, SL, n - nL, S - SL);
                        if (best_f < 0 || gain_cmp(g, best_g) > 0) {
                            /* strictly better only: earlier (lower f, lower thr) wins ties */
                            best_f = f; best_thr = va + 0.0f; best_g = g;
                            best_nL = nL; best_SL = SL;
                        }
                    }
                }
                if (best_f >= 0 && gain_beats_parent(best_g, n, S)) split = 1;
            }

            if (!split) {
                node->feature = -1;
                node->left = -1;
                node->value = orc_round_mean(S, n);
                free(node->rows); node->rows = NULL;
                continue;
            }

            node->feature = best_f;
            node->thr = best_thr;
            const float *col = X + (size_t)best_f * (size_t)N;
            int64_t lid = push_node(tr);
            int64_t rid = push_node(tr);
            node = &tr->nodes[id];                 /* push_node may move the array */
            onode *L = &tr->nodes[lid], *R = &tr->nodes[rid];
            node->left = lid;
            L->rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)node->nrows);
            R->rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)node->nrows);
            for (int64_t k = 0; k < node->nrows; ++k) {
                int64_t r = node->rows[k];
                onode *c = (col[r] <= best_thr) ? L : R;
                c->rows[c->nrows++] = r;
                c->n += w[r];
                c->S += (int64_t)w[r] * y[r];
            }
            L->depth = R->depth = d + 1;
            /* the children's sums equal the chosen candidate's prefix sums */
            if (L->n != best_nL || L->S != best_SL) abort();
            free(node->rows); node->rows = NULL;
        }
        level_begin = level_end;
        level_end = tr->count;
    }
    free(sorted);
    free(feats);
    free(w);
}

/* Fit trees with global indices [t0, t1) on X (column-major F x N) and y (Q32.32). */
int orc_fit(const float *X, const int64_t *y, int64_t N, int32_t F,
            int64_t t0, int64_t t1, int32_t mtry, int32_t min_node, int32_t max_depth,
            uint64_t seed, int32_t bootstrap, orc_forest **out)
{
    if (!X || !y || !out || N < 1 || F < 1 || t1 <= t0 || mtry < 1 || min_node < 1 || max_depth < 0)
        return -1;
    orc_forest *fr = (orc_forest *)calloc(1, sizeof(orc_forest));
    fr->t0 = t0; fr->t1 = t1; fr->F = F;
    fr->seed = seed; fr->bootstrap = bootstrap; fr->N = N;
    fr->trees = (otree *)calloc((size_t)(t1 - t0), sizeof(otree));
    for (int64_t t = t0; t < t1; ++t)
        grow_tree(&fr->trees[t - t0], X, y, N, F, t, mtry, min_node, max_depth, seed, bootstrap);
    *out = fr;
    return 0;
}

void orc_forest_free(orc_forest *fr)
{
    if (!fr) return;
    for (int64_t t = 0; t < fr->t1 - fr->t0; ++t) free(fr->trees[t].nodes);
    free(fr->trees);
    free(fr);
}

int64_t orc_forest_num_trees(const orc_forest *fr) { return fr->t1 - fr->t0; }
int64_t orc_tree_num_nodes(const orc_forest *fr, int64_t k) { return fr->trees[k].count; }

/* Copy out tree k (local index) node by node, in BFS order. Any pointer may be NULL. */
void orc_tree_export(const orc_forest *fr, int64_t k, int32_t *feature, float *thr, int64_t *left,
                     int64_t *value, int64_t *n, int64_t *S, int64_t *nrows, int32_t *depth,
                     int32_t *evaluated)
{
    const otree *tr = &fr->trees[k];
    for (int64_t j = 0; j < tr->count; ++j) {
        const onode *nd = &tr->nodes[j];
        if (feature) feature[j] = nd->feature;
        if (thr) thr[j] = nd->thr;
        if (left) left[j] = nd->left;
        if (value) value[j] = nd->value;
        if (n) n[j] = nd->n;
        if (S) S[j] = nd->S;
        if (nrows) nrows[j] = nd->nrows;
        if (depth) depth[j] = nd->depth;
        if (evaluated) evaluated[j] = nd->evaluated;
    }
}

static int64_t tree_leaf(const otree *tr, const float *Xq, int64_t Q, int64_t q)
{
    int64_t j = 0;
    while (tr->nodes[j].feature >= 0) {
        float x = Xq[(size_t)tr->nodes[j].feature * (size_t)Q + (size_t)q];
        j = tr->nodes[j].left + (x <= tr->nodes[j].thr ? 0 : 1);
    }
    return tr->nodes[j].value;
}

/* Queries Xq column-major F x Q. out_sum: exact sum of leaf values over this forest's trees
 * (may be NULL). out_pred: floor((2P + T)/(2T)) with T = total_trees (the whole forest's tree
 * count, so shards can be combined by summing out_sum). out_var: V = T*sum(v^2) - P^2 as
 * (lo, hi) 64-bit words (may be NULL; only meaningful when this forest is the whole forest). */
int orc_predict(const orc_forest *fr, const float *Xq, int64_t Q, int64_t total_trees,
                int64_t *out_sum, int64_t *out_pred, uint64_t *out_var)
{
    int64_t T = fr->t1 - fr->t0;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t P = 0;
        u128 sq = 0;
        for (int64_t k = 0; k < T; ++k) {
            int64_t v = tree_leaf(&fr->trees[k], Xq, Q, q);
            P += v;
            sq += (u128)((i128)v * v);
        }
        if (out_sum) out_sum[q] = P;
        if (out_pred) out_pred[q] = (int64_t)floor_div((i128)2 * P + total_trees, (i128)2 * total_trees);
        if (out_var) {
            u128 V = (u128)total_trees * sq - (u128)((i128)P * P);
            out_var[2 * q] = (uint64_t)V;
            out_var[2 * q + 1] = (uint64_t)(V >> 64);
        }
    }
    return 0;
}

/* Out-of-bag evaluation (Sec. III-B: the tuning objective). For each training row r of the
 * fit's X: out_sum[r] = sum of the leaf values of the trees whose bootstrap did not draw r,
 * out_count[r] = their number. Without bootstrap every row is in every tree's sample. */
int orc_oob(const orc_forest *fr, const float *X, int64_t N, int64_t *out_sum, int32_t *out_count)
{
    if (N != fr->N) return -1;
    uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    for (int64_t r = 0; r < N; ++r) { out_sum[r] = 0; out_count[r] = 0; }
    for (int64_t k = 0; k < fr->t1 - fr->t0; ++k) {
        if (!fr->bootstrap) break;
        orc_bootstrap_counts(fr->seed, fr->t0 + k, N, w);
        for (int64_t r = 0; r < N; ++r) {
            if (w[r] > 0) continue;
            out_sum[r] += tree_leaf(&fr->trees[k], X, N, r);
            out_count[r] += 1;
        }
    }
    free(w);
    return 0;
}

/* Device selection (Sec. VI). kfeat: column-major (F-2) x K kernel features; the query for
 * (kernel k, device j) is kfeat[:, k] followed by device_ids[j] and size_class as floats.
 * out_best[k] = device id with the smallest prediction (ties: lower device id);
 * out_pred[k*D + j] = the prediction (may be NULL). */
int orc_select_device(const orc_forest *fr, const float *kfeat, int32_t K, int32_t size_class,
                      const int32_t *device_ids, int32_t D, int32_t *out_best, int64_t *out_pred)
{
    int32_t F = fr->F;
    int64_t T = fr->t1 - fr->t0;
    float *q = (float *)malloc(sizeof(float) * (size_t)F);
    for (int32_t k = 0; k < K; ++k) {
        int64_t best_pred = 0;
        int32_t best_dev = -1;
        for (int32_t j = 0; j < D; ++j) {
            for (int32_t f = 0; f < F - 2; ++f) q[f] = kfeat[(size_t)f * (size_t)K + (size_t)k];
            q[F - 2] = (float)device_ids[j];
            q[F - 1] = (float)size_class;
            int64_t pred;
            orc_predict(fr, q, 1, T, NULL, &pred, NULL);
            if (out_pred) out_pred[(size_t)k * (size_t)D + (size_t)j] = pred;
            if (best_dev < 0 || pred < best_pred || (pred == best_pred && device_ids[j] < best_dev)) {
                best_pred = pred;
                best_dev = device_ids[j];
            }
        }
        out_best[k] = best_dev;
    }
    free(q);
    return 0;
}
