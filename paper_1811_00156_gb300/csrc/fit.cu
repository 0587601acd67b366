// fit.cu -- random-forest growth on the GPU (the model of Sec. III-B, fitted breadth first).
//
// Pipeline of one fit (all trees of all forests of the batch grow together, level by level):
//   presort            every column's float keys sorted by the segmented radix sort (sort.cu);
//                      dense ranks and the rank -> value table; ranks copied to row-major
//                      records of F bytes (u8 when every column has <= 256 values, else u16)
//   grouping           rows with identical rank records (identical feature vectors) form a
//                      group: such rows fall on the same side of every threshold, so a tree
//                      can carry one entry per group with the summed multiplicity and target.
//                      Groups are ordered by a hash of their record.
//   boot_groups_kernel Philox draws per tree, each adding 1 and its row's y to the row's
//                      group sums in shared memory -> one entry {row, sum w, sum w*y} per
//                      group that has an in-bag row (bootstrap_kernel: the same through per-row
//                      multiplicities, when the group sums do not fit shared memory)
//   per depth d:
//     level_big_kernel   one CTA per node with > 32 entries: mtry draw, shared-memory histogram
//                        (sum w, sum w*y) per rank of every tried feature, block scan, exact
//                        argmax of the gain, stable partition of the entries
//     level_small_kernel one warp per node with <= 32 entries: the same search with a register
//                        bitonic sort per feature instead of a histogram (runs concurrently with
//                        level_big_kernel; both count each tile's splits)
//     finalize_kernel    exclusive scan of the split flags, then encodes each node, numbers the
//                        children breadth first, writes the next depth's node table and its
//                        warp/CTA work lists; its last CTA advances the per-tree node counts,
//                        next-depth offsets and level counts
//   pack_kernel        scatters every finished node to its forest / tree / BFS position
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.cuh"

namespace aiwcrf {

// runs the statement with RT the rank type of rank_bytes (1, 2 or 4 bytes per stored rank)
#define AIWCRF_BY_RANK(rank_bytes, ...)                                       \
    switch (rank_bytes) {                                                     \
    case 1: { using RT = uint8_t; __VA_ARGS__; } break;                       \
    case 2: { using RT = uint16_t; __VA_ARGS__; } break;                      \
    default: { using RT = uint32_t; __VA_ARGS__; } break;                     \
    }

inline int rank_bytes_for(uint32_t max_card)
{
    return max_card <= 256u ? 1 : (max_card <= 65536u ? 2 : 4);
}

// Small device-to-host reads (sizes, counts, error flags) staged through the host thread's
// page-locked buffer, from byte 1,024 on (the level loop keeps its counts below that): the
// copies are then asynchronous and one stream wait covers them all (a copy into pageable memory
// waits by itself). Copies that do not fit go to their pageable destinations directly.
struct HostReads {
    struct Item { void *dst; const void *src; size_t bytes, off; };
    Item items[8];
    int n = 0;
    size_t used = 1024;
    void add(void *dst, const void *src, size_t bytes) { items[n++] = Item{dst, src, bytes, 0}; }
    int run(cudaStream_t s)
    {
        unsigned char *pin = static_cast<unsigned char *>(pinned_scratch());
        for (int i = 0; i < n; ++i) {
            Item &it = items[i];
            const size_t off = (used + 15) & ~(size_t)15;
            const bool staged = pin && off + it.bytes <= kPinnedScratchBytes;
            it.off = staged ? off : (size_t)-1;
            if (staged) used = off + it.bytes;
            const cudaError_t e = cudaMemcpyAsync(staged ? pin + off : it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_fail(e, "device-to-host read");
        }
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host read");
        for (int i = 0; i < n; ++i)
            if (items[i].off != (size_t)-1) std::memcpy(items[i].dst, pin + items[i].off, items[i].bytes);
        return AIWCRF_OK;
    }
};

struct Entry {            // one group of identical in-bag rows of one tree
    uint32_t row;         // a row of the group (all its rows have the same features)
    uint32_t w;           // summed bootstrap multiplicity
    int64_t wy;           // summed w * y
};
static_assert(sizeof(Entry) == 16, "Entry is one 16-byte vector");

__device__ __forceinline__ Entry load_entry(const Entry *p)
{
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    Entry e;
    e.row = v.x; e.w = v.y; e.wy = (int64_t)(((uint64_t)v.w << 32) | v.z);
    return e;
}

__device__ __forceinline__ void store_entry(Entry *p, const Entry &e)
{
    *reinterpret_cast<uint4 *>(p) = make_uint4(e.row, e.w, (uint32_t)(uint64_t)e.wy, (uint32_t)((uint64_t)e.wy >> 32));
}

// ------------------------------------------------------------------------------------------
// a1: presort and rank
// ------------------------------------------------------------------------------------------
__global__ void key_init_kernel(const float *__restrict__ X, int64_t N, uint32_t *keys, uint32_t *vals, uint32_t *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (i >= N) return;
    const float x = X[(size_t)f * (size_t)N + i];
    if (x != x) atomicOr(err, kErrNaN);
    keys[(size_t)f * (size_t)N + i] = float_key(x);
    vals[(size_t)f * (size_t)N + i] = (uint32_t)i;
}

// Dense ranks of the sorted columns (equal keys share a rank; the rank -> value table and every
// column's value count), with the columns cut into chunks of kRankChunk sorted keys (many CTAs
// per column): rank_count_kernel counts each chunk's distinct-value starts, rank_write_kernel
// adds the counts of the column's earlier chunks to its own block scan.
constexpr int kRankThreads = 1024;
constexpr int kRankChunk = 4 * kRankThreads;

__global__ void __launch_bounds__(kRankThreads) rank_count_kernel(const uint32_t *__restrict__ keys, int64_t N,
                                                                  uint32_t *__restrict__ chunk_count)
{
    __shared__ uint32_t warp_tmp[32];
    const int f = blockIdx.y;
    const size_t off = (size_t)f * (size_t)N;
    const int64_t i0 = (int64_t)blockIdx.x * kRankChunk;
    uint32_t c = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * kRankThreads + threadIdx.x;
        if (i < N && (i == 0 || keys[off + i - 1] != keys[off + i])) ++c;
    }
    uint32_t tot;
    block_incl_scan(c, warp_tmp, tot);
    if (threadIdx.x == 0) chunk_count[(size_t)f * gridDim.x + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRankThreads) rank_write_kernel(const uint32_t *__restrict__ keys,
                                                                  const uint32_t *__restrict__ idx, int64_t N,
                                                                  const uint32_t *__restrict__ chunk_count,
                                                                  uint32_t *__restrict__ Rcol, float *__restrict__ vals,
                                                                  uint32_t *__restrict__ card)
{
    __shared__ uint32_t warp_tmp[32];
    __shared__ uint32_t s_base;
    const int f = blockIdx.y, tid = threadIdx.x;
    const size_t off = (size_t)f * (size_t)N;
    if (tid < 32) {                        // distinct values before this chunk
        uint32_t b = 0;
        for (uint32_t c = tid; c < blockIdx.x; c += 32) b += chunk_count[(size_t)f * gridDim.x + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(kFull, b, o);
        if (tid == 0) s_base = b;
    }
    __syncthreads();
    uint32_t running = s_base;
    const int64_t i0 = (int64_t)blockIdx.x * kRankChunk;
    for (int u = 0; u < 4; ++u) {                                  // block-uniform
        const int64_t i = i0 + u * kRankThreads + tid;
        const bool valid = i < N;
        const uint32_t k = valid ? keys[off + i] : 0u;
        const uint32_t flag = (valid && (i == 0 || keys[off + i - 1] != k)) ? 1u : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan(flag, warp_tmp, tot);
        if (valid) {
            const uint32_t r = running + incl - 1u;                 // < N < 2^22
            Rcol[off + idx[off + i]] = r;
            if (flag) vals[off + r] = key_float(k);
        }
        running += tot;
    }
    if (tid == 0 && blockIdx.x == gridDim.x - 1) card[f] = running;
}

int dense_ranks(const uint32_t *keys, const uint32_t *idx, int64_t N, int F, uint32_t *chunk_count, uint32_t *Rcol,
                float *vals, uint32_t *card, cudaStream_t s)
{
    const dim3 grid((unsigned)((N + kRankChunk - 1) / kRankChunk), (unsigned)F);
    rank_count_kernel<<<grid, kRankThreads, 0, s>>>(keys, N, chunk_count);
    rank_write_kernel<<<grid, kRankThreads, 0, s>>>(keys, idx, N, chunk_count, Rcol, vals, card);
    count_launches(2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dense rank launch");
    return AIWCRF_OK;
}

size_t dense_rank_chunk_words(int64_t N, int F)
{
    return (size_t)((N + kRankChunk - 1) / kRankChunk) * (size_t)F;
}

// Row-major copy of the ranks: the tried features of one row share one record.
template <typename RT>
__global__ void rank_rows_kernel(const uint32_t *__restrict__ Rcol, int64_t N, int F, RT *__restrict__ Rr)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    for (int f = 0; f < F; ++f) Rr[(size_t)row * (size_t)F + f] = (RT)Rcol[(size_t)f * (size_t)N + row];
}

// ------------------------------------------------------------------------------------------
// grouping of rows with identical rank records
// ------------------------------------------------------------------------------------------
// 32-bit hash of a row's rank record (FNV-style steps, then a final mix)
template <typename RT>
__device__ __forceinline__ uint32_t record_hash(const RT *r, int F)
{
    uint32_t h = 0x811C9DC5u;
    for (int f = 0; f < F; ++f) {
        h ^= (uint32_t)r[f];
        h *= 0x01000193u;
        h ^= h >> 13;
    }
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    return h;
}

template <typename RT>
__global__ void hash_rows_kernel(const RT *__restrict__ Rr, int64_t N, int F, uint32_t *keys, uint32_t *vals)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    keys[row] = record_hash(Rr + (size_t)row * (size_t)F, F);
    vals[row] = (uint32_t)row;
}

template <typename RT>
__device__ __forceinline__ bool same_record(const RT *Rr, int F, uint32_t a, uint32_t b)
{
    const RT *ra = Rr + (size_t)a * (size_t)F, *rb = Rr + (size_t)b * (size_t)F;
    for (int f = 0; f < F; ++f)
        if (ra[f] != rb[f]) return false;
    return true;
}

// rows sorted by hash -> groups of adjacent rows with the same hash and the same record:
// flag[i] = 1 where sorted position i starts a group
template <typename RT>
__global__ void group_flags_kernel(const RT *__restrict__ Rr, int64_t N, int F, const uint32_t *__restrict__ hkeys,
                                   const uint32_t *__restrict__ rows, uint32_t *__restrict__ flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    flags[i] = (i == 0 || hkeys[i] != hkeys[i - 1] || !same_record(Rr, F, rows[i], rows[i - 1])) ? 1u : 0u;
}

// grp_off[g] = first sorted position of group g, grp_off[G] = N, *n_groups = G
__global__ void group_offsets_kernel(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ excl, int64_t N,
                                     uint32_t *__restrict__ grp_off, uint32_t *n_groups)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && flags[i]) grp_off[excl[i]] = (uint32_t)i;
    if (i == 0) {
        grp_off[excl[N]] = (uint32_t)N;
        *n_groups = excl[N];
    }
}

// group order: y of every position (rows in group order) and the group it belongs to (flags
// mark group starts, excl is their exclusive scan)
__global__ void group_order_kernel(const uint32_t *__restrict__ rows, const uint32_t *__restrict__ flags,
                                   const uint32_t *__restrict__ excl, const int64_t *__restrict__ y, int64_t N,
                                   int64_t *__restrict__ y_g, uint32_t *__restrict__ grp_of, uint4 *__restrict__ rowrec)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t row = rows[k];
    const int64_t yr = y[row];
    const uint32_t g = excl[k] + flags[k] - 1u;
    y_g[k] = yr;
    grp_of[k] = g;
    // per row: y and its group, one 16-byte record (read by boot_groups_kernel's draws)
    if (rowrec) rowrec[row] = make_uint4((uint32_t)(uint64_t)yr, (uint32_t)((uint64_t)yr >> 32), g, 0u);
}

// Grouping through a hash table instead of a sort (the fit's usual path). Open addressing over
// a power-of-two table of 64-bit slots {hash, first row}: a row claims an empty slot with a
// compare-and-swap or joins the slot whose row has the same record (compared in full when the
// hashes agree), probing linearly, at most table-size probes. Groups are then numbered in slot
// order; which row claims a slot, and so the numbering and the rows' order within a group, can
// differ between runs, which changes no sum and no forest (entries are summed per group, and
// splits and partitions do not depend on the entries' order).
constexpr unsigned long long kSlotEmpty = ~0ull;

template <typename RT>
__global__ void group_insert_kernel(const RT *__restrict__ Rr, int64_t N, int F, unsigned long long *table,
                                    uint32_t mask, uint32_t *__restrict__ slot_of_row, uint32_t *err)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const uint32_t h = record_hash(Rr + (size_t)r * (size_t)F, F);
    const unsigned long long mine = ((unsigned long long)h << 32) | (uint32_t)r;
    uint32_t i = h & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = table[i];
        if (cur == kSlotEmpty) {
            cur = atomicCAS(&table[i], kSlotEmpty, mine);
            if (cur == kSlotEmpty) { slot_of_row[r] = i; return; }
        }
        if ((uint32_t)(cur >> 32) == h && same_record(Rr, F, (uint32_t)cur, (uint32_t)r)) {
            slot_of_row[r] = i;
            return;
        }
        i = (i + 1u) & mask;
    }
    atomicOr(err, kErrCapacity);                       // a full table (it holds at least 2N slots)
    slot_of_row[r] = 0u;
}

__global__ void slot_flags_kernel(const unsigned long long *__restrict__ table, int64_t n, uint32_t *__restrict__ flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = table[i] != kSlotEmpty ? 1u : 0u;
}

// the row's group (its slot's rank among the occupied slots), the groups' row counts, and G
__global__ void row_group_kernel(const uint32_t *__restrict__ slot_of_row, const uint32_t *__restrict__ slot_excl,
                                 int64_t n_slots, int64_t N, uint32_t *__restrict__ group_of_row, uint32_t *cnt,
                                 uint32_t *n_groups)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) *n_groups = slot_excl[n_slots];
    if (r >= N) return;
    const uint32_t g = slot_excl[slot_of_row[r]];
    group_of_row[r] = g;
    atomicAdd(&cnt[g], 1u);
}

// rows in group order: each row takes the next place of its group
__global__ void group_scatter_kernel(const uint32_t *__restrict__ group_of_row, const uint32_t *__restrict__ grp_off,
                                     int64_t N, uint32_t *fill, uint32_t *__restrict__ grp_rows)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const uint32_t g = group_of_row[r];
    grp_rows[grp_off[g] + atomicAdd(&fill[g], 1u)] = (uint32_t)r;
}

// as group_order_kernel, with each row's group given
__global__ void group_order_rows_kernel(const uint32_t *__restrict__ rows, const uint32_t *__restrict__ group_of_row,
                                        const int64_t *__restrict__ y, int64_t N, int64_t *__restrict__ y_g,
                                        uint32_t *__restrict__ grp_of, uint4 *__restrict__ rowrec)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t row = rows[k];
    const int64_t yr = y[row];
    const uint32_t g = group_of_row[row];
    y_g[k] = yr;
    grp_of[k] = g;
    if (rowrec) rowrec[row] = make_uint4((uint32_t)(uint64_t)yr, (uint32_t)((uint64_t)yr >> 32), g, 0u);
}

// ------------------------------------------------------------------------------------------
// a2: bootstrap, one CTA per tree. Multiplicities are byte counters per row, packed four to a
// word, in shared memory when they fit, else in a per-tree global scratch. Entries are then
// formed group by group, in group order.
// ------------------------------------------------------------------------------------------
constexpr int kBootThreads = 1024;

struct BootArgs {
    const int64_t *tree_pool_off;   // per tree: offset into sub_rows, or -1 for rows 0..len-1
    const uint32_t *tree_pool_len;  // per tree: pool size
    const uint32_t *tree_rng;       // per tree: global tree index used as Philox counter word 0
    const int32_t *sub_rows;
    const int64_t *y;
    int64_t N;
    const uint32_t *grp_off;        // G + 1
    const uint32_t *grp_rows;       // rows in group order
    uint32_t G;
    const uint32_t *G_ptr;          // when set, the group count is read here
    uint32_t seed_lo, seed_hi;
    int bootstrap;
    uint32_t *gcnt;                 // global byte counters (may be null)
    int64_t gcnt_stride;            // words per tree
    int smem_words;
    Entry *rows_out;
    int64_t row_cap;
    NodeRec *root;
    int32_t *small_list, *big_list;
    uint32_t *counters;             // [0] small count, [1] big count (depth 0's list counts)
    uint32_t *err;
    uint32_t *inbag;                // per tree ceil(N / 32) words: bit r set = row r drawn (or null)
    int64_t inbag_words;
    int store_group;                // entries name their group (tree-resident growth) instead of a row
    // group-ordered pass (when set): y in group order and the group of every group-ordered
    // position; the per-group sums (sum w, sum w*y) go to gsum, 2 * G words per tree
    const int64_t *y_g;
    const uint32_t *grp_of;
    unsigned long long *gsum;
};

__global__ void __launch_bounds__(kBootThreads) bootstrap_kernel(BootArgs a)
{
    extern __shared__ uint32_t sm_cnt[];
    __shared__ uint32_t warp_tmp[32];
    __shared__ unsigned long long red_n[32];
    __shared__ long long red_s[32];

    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = a.tree_pool_len[t];
    const int64_t poff = a.tree_pool_off[t];
    const uint32_t words = (uint32_t)((a.N + 3) / 4);
    uint32_t *cnt = ((int)words <= a.smem_words) ? sm_cnt : a.gcnt + (size_t)t * (size_t)a.gcnt_stride;

    for (uint32_t k = tid; k < words; k += kBootThreads) cnt[k] = 0u;
    __syncthreads();
    if (a.bootstrap) {
        const uint32_t tg = a.tree_rng[t];
        int overflow = 0;
        for (uint32_t b = tid; b < (n + 3u) / 4u; b += kBootThreads) {
            const uint4 u = philox10(make_uint4(tg, b, kDomBoot, 0u), a.seed_lo, a.seed_hi);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t k = 4u * b + (uint32_t)w;
                if (k < n) {
                    const uint32_t j = __umulhi(uint4_word(u, w), n);
                    const uint32_t row = poff < 0 ? j : (uint32_t)a.sub_rows[poff + j];
                    const uint32_t sh = 8u * (row & 3u);
                    const uint32_t old = atomicAdd(&cnt[row >> 2], 1u << sh);
                    if (((old >> sh) & 255u) == 255u) overflow = 1;
                }
            }
        }
        if (overflow) atomicOr(a.err, kErrBootOverflow);
    } else {
        for (uint32_t j = tid; j < n; j += kBootThreads) {
            const uint32_t row = poff < 0 ? j : (uint32_t)a.sub_rows[poff + j];
            atomicOr(&cnt[row >> 2], 1u << (8u * (row & 3u)));
        }
    }
    __syncthreads();

    if (a.inbag) {                  // in-bag bitmap for out-of-bag evaluation
        uint32_t *bits = a.inbag + (size_t)t * (size_t)a.inbag_words;
        for (int64_t wd = tid; wd < a.inbag_words; wd += kBootThreads) {
            uint32_t v = 0;
            for (int b = 0; b < 32; ++b) {
                const int64_t row = wd * 32 + b;
                if (row < a.N && ((cnt[row >> 2] >> (8u * (uint32_t)(row & 3))) & 255u)) v |= 1u << b;
            }
            bits[wd] = v;
        }
    }

    uint32_t running = 0;
    unsigned long long acc_n = 0;
    long long acc_s = 0;
    Entry *out = a.rows_out + (size_t)t * (size_t)a.row_cap;
    const uint32_t G = a.G_ptr ? *a.G_ptr : a.G;
    // group-ordered pass: every position k of the group order (coalesced row and y reads) adds
    // its row's w and w*y to its group's shared-memory sums, one atomic per run of a group
    // within a warp (groups are contiguous in that order)
    unsigned long long *gsum = nullptr;
    if (a.y_g) {
        gsum = a.gsum + (size_t)t * 2 * (size_t)G;
        for (uint32_t g = tid; g < 2 * G; g += kBootThreads) gsum[g] = 0ull;
        __syncthreads();
        // kBootIlp positions per thread per round: their loads are issued before any is reduced
        constexpr int kBootIlp = 4;
        for (int64_t k0 = 0; k0 < a.N; k0 += (int64_t)kBootThreads * kBootIlp) {
            uint32_t rw[kBootIlp], rg[kBootIlp];
            long long ry[kBootIlp];
#pragma unroll
            for (int u = 0; u < kBootIlp; ++u) {
                const int64_t k = k0 + (int64_t)u * kBootThreads + tid;
                rg[u] = 0xFFFFFFFFu; rw[u] = 0u; ry[u] = 0ll;
                if (k < a.N) {
                    const uint32_t row = a.grp_rows[k];
                    rg[u] = a.grp_of[k];
                    ry[u] = a.y_g[k];
                    rw[u] = (cnt[row >> 2] >> (8u * (row & 3u))) & 255u;
                }
            }
#pragma unroll
            for (int u = 0; u < kBootIlp; ++u) {
                uint32_t w = rw[u];
                const uint32_t g = rg[u];
                long long wy = w ? (long long)w * ry[u] : 0ll;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t tw = __shfl_up_sync(kFull, w, o);
                    const long long ty = __shfl_up_sync(kFull, wy, o);
                    const uint32_t tg = __shfl_up_sync(kFull, g, o);
                    if (lane >= o && tg == g) { w += tw; wy += ty; }
                }
                const uint32_t ng = __shfl_down_sync(kFull, g, 1);
                if (g != 0xFFFFFFFFu && w && (lane == 31 || ng != g)) {
                    atomicAdd(&gsum[2 * (size_t)g], (unsigned long long)w);
                    atomicAdd(&gsum[2 * (size_t)g + 1], (unsigned long long)wy);
                }
            }
        }
        __syncthreads();
    }
    for (uint32_t g0 = 0; g0 < G; g0 += kBootThreads) {
        const uint32_t g = g0 + tid;
        uint32_t sw = 0, rep = 0;
        long long swy = 0;
        if (g < G) {
            rep = a.grp_rows[a.grp_off[g]];
            if (gsum) {                 // the sums were made by L2 atomics: read them from L2
                sw = (uint32_t)__ldcg(&gsum[2 * (size_t)g]);
                swy = (long long)__ldcg(&gsum[2 * (size_t)g + 1]);
            } else {
                const uint32_t e = a.grp_off[g + 1];
                for (uint32_t k = a.grp_off[g]; k < e; ++k) {
                    const uint32_t row = a.grp_rows[k];
                    const uint32_t w = (cnt[row >> 2] >> (8u * (row & 3u))) & 255u;
                    if (w) {
                        sw += w;
                        swy += (long long)w * a.y[row];
                    }
                }
            }
        }
        uint32_t tot;
        const uint32_t incl = block_incl_scan(sw > 0 ? 1u : 0u, warp_tmp, tot);
        if (sw > 0) {
            Entry en;
            en.row = a.store_group ? g : rep; en.w = sw; en.wy = swy;
            // entries never outnumber the row capacity when it was sized from this data; a
            // replayed plan on data with more groups than it was built for flags it instead
            if ((int64_t)(running + incl - 1u) < a.row_cap) store_entry(&out[running + incl - 1u], en);
            else atomicOr(a.err, kErrCapacity);
            acc_n += sw;
            acc_s += swy;
        }
        running += tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_n += __shfl_xor_sync(kFull, acc_n, o);
        acc_s += __shfl_xor_sync(kFull, acc_s, o);
    }
    if (lane == 0) { red_n[warp] = acc_n; red_s[warp] = acc_s; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long sn = 0;
        long long ss = 0;
        for (int w = 0; w < kBootThreads / 32; ++w) { sn += red_n[w]; ss += red_s[w]; }
        NodeRec r;
        // (a flagged overflow keeps the node inside its tree's slice; the fit then fails)
        r.tree = (uint32_t)t; r.idx = 0u; r.start = 0u; r.len = (uint32_t)min((int64_t)running, a.row_cap);
        r.n = (uint32_t)sn;
        r.pad = 0u; r.S = ss;
        a.root[t] = r;
        if (running <= (uint32_t)kSmallNodeRows) a.small_list[atomicAdd(&a.counters[0], 1u)] = t;
        else a.big_list[atomicAdd(&a.counters[1], 1u)] = t;
    }
}

// The bootstrap with the draws summed per group directly (the fit's usual case: the groups'
// sums and the in-bag bitmap fit shared memory). Each draw reads its row's 16-byte record
// {y, group} and adds 1 and y to the group's shared-memory sums; no per-row counters and no
// pass over the rows follow. Integer sums, so the entries equal bootstrap_kernel's.
constexpr int kBootGThreads = 512;      // 40 registers: three CTAs per SM
constexpr int kBootGIlp = 4;            // draws whose record loads a thread issues together
constexpr int kBootGroupsSmemMax = 96 * 1024;      // at least two CTAs per SM
#ifndef AIWCRF_GROUP_HASH
#define AIWCRF_GROUP_HASH 1            // 0: the fit groups rows through a radix sort of their hashes
#endif
#ifndef AIWCRF_BOOT_GROUPS
#define AIWCRF_BOOT_GROUPS 1           // 0: always the per-row counters of bootstrap_kernel
#endif

__host__ __forceinline__ size_t boot_groups_smem(uint32_t G, int64_t inbag_words)
{
    return (size_t)G * 12u + (size_t)inbag_words * 4u;
}

__global__ void __launch_bounds__(kBootGThreads) boot_groups_kernel(BootArgs a, const uint4 *__restrict__ rowrec)
{
    extern __shared__ __align__(16) unsigned char boot_sm[];
    __shared__ uint32_t warp_tmp[32];
    __shared__ unsigned long long red_n[32];
    __shared__ long long red_s[32];

    const uint32_t G = a.G;
    unsigned long long *gwy = reinterpret_cast<unsigned long long *>(boot_sm);     // G sums of y
    uint32_t *gw = reinterpret_cast<uint32_t *>(gwy + G);                           // G draw counts
    uint32_t *bits = gw + G;                                                        // in-bag bitmap
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = a.tree_pool_len[t];
    const int64_t poff = a.tree_pool_off[t];
    const int64_t nbits = a.inbag ? a.inbag_words : 0;

    for (uint32_t g = tid; g < G; g += kBootGThreads) { gwy[g] = 0ull; gw[g] = 0u; }
    for (int64_t k = tid; k < nbits; k += kBootGThreads) bits[k] = 0u;
    __syncthreads();
    const uint32_t tg = a.tree_rng[t];
    const uint32_t nb4 = (n + 3u) / 4u;               // Philox blocks of four draws
    constexpr int U = kBootGIlp / 4;                  // blocks per thread per round
    for (uint32_t b0 = tid; b0 < nb4; b0 += kBootGThreads * U) {
        uint32_t row[4 * U];
        uint4 rec[4 * U];
#pragma unroll
        for (int v = 0; v < U; ++v) {           // all the round's record loads are issued together
            const uint32_t b = b0 + (uint32_t)(v * kBootGThreads);
            const uint4 u = philox10(make_uint4(tg, b, kDomBoot, 0u), a.seed_lo, a.seed_hi);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t k = 4u * b + (uint32_t)w;
                row[4 * v + w] = 0xFFFFFFFFu;
                rec[4 * v + w] = make_uint4(0u, 0u, 0u, 0u);
                if (b < nb4 && k < n) {
                    const uint32_t j = __umulhi(uint4_word(u, w), n);
                    row[4 * v + w] = AIWCRF_IDX(poff < 0 ? j : (uint32_t)a.sub_rows[poff + j], (uint32_t)a.N, kBoundRow);
                    rec[4 * v + w] = __ldg(&rowrec[row[4 * v + w]]);
                }
            }
        }
#pragma unroll
        for (int w = 0; w < 4 * U; ++w) {
            if (row[w] != 0xFFFFFFFFu) {
                const uint32_t g = AIWCRF_IDX(rec[w].z, G, kBoundRow);
                atomicAdd(&gw[g], 1u);
                // the 64-bit sum as two 32-bit shared atomics (low word, then the high word
                // plus the low word's carry): a 64-bit shared atomic add costs more
                uint32_t *h = reinterpret_cast<uint32_t *>(&gwy[g]);
                const uint32_t old = atomicAdd(&h[0], rec[w].x);
                const uint32_t hi = rec[w].y + ((old + rec[w].x < old) ? 1u : 0u);
                if (hi) atomicAdd(&h[1], hi);
                if (nbits) atomicOr(&bits[row[w] >> 5], 1u << (row[w] & 31u));
            }
        }
    }
    __syncthreads();
    if (nbits) {
        uint32_t *out_bits = a.inbag + (size_t)t * (size_t)a.inbag_words;
        for (int64_t k = tid; k < nbits; k += kBootGThreads) out_bits[k] = bits[k];
    }

    // entries in group order: one per group with a draw
    uint32_t running = 0;
    unsigned long long acc_n = 0;
    long long acc_s = 0;
    Entry *out = a.rows_out + (size_t)t * (size_t)a.row_cap;
    for (uint32_t g0 = 0; g0 < G; g0 += kBootGThreads) {
        const uint32_t g = g0 + tid;
        uint32_t sw = 0;
        long long swy = 0;
        if (g < G) { sw = gw[g]; swy = (long long)gwy[g]; }
        uint32_t tot;
        const uint32_t incl = block_incl_scan(sw > 0 ? 1u : 0u, warp_tmp, tot);
        if (sw > 0) {
            Entry en;
            en.row = a.store_group ? g : a.grp_rows[a.grp_off[g]];
            en.w = sw; en.wy = swy;
            if ((int64_t)(running + incl - 1u) < a.row_cap) store_entry(&out[running + incl - 1u], en);
            else atomicOr(a.err, kErrCapacity);
            acc_n += sw;
            acc_s += swy;
        }
        running += tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_n += __shfl_xor_sync(kFull, acc_n, o);
        acc_s += __shfl_xor_sync(kFull, acc_s, o);
    }
    if (lane == 0) { red_n[warp] = acc_n; red_s[warp] = acc_s; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long sn = 0;
        long long ss = 0;
        for (int w = 0; w < kBootGThreads / 32; ++w) { sn += red_n[w]; ss += red_s[w]; }
        NodeRec r;
        r.tree = (uint32_t)t; r.idx = 0u; r.start = 0u; r.len = (uint32_t)min((int64_t)running, a.row_cap);
        r.n = (uint32_t)sn;
        r.pad = 0u; r.S = ss;
        a.root[t] = r;
        if (running <= (uint32_t)kSmallNodeRows) a.small_list[atomicAdd(&a.counters[0], 1u)] = t;
        else a.big_list[atomicAdd(&a.counters[1], 1u)] = t;
    }
}

// ------------------------------------------------------------------------------------------
// a3/a4/a5: one depth of growth. Every per-depth kernel reads its sizes from LevelCounts in
// device memory, so the host can enqueue several depths without waiting for their results.
// ------------------------------------------------------------------------------------------
struct LevelCounts {
    uint32_t n_list[2][2];        // by depth parity: [0] nodes searched by a warp, [1] by a CTA
    uint32_t C;                   // nodes of the current depth
    uint32_t levels;              // depths that held nodes so far
    unsigned long long packed_off;    // finished nodes of the earlier depths
};

constexpr int kScanThreads = 1024;
constexpr int kFinThreads = 256;
constexpr int kScanTile = kFinThreads;   // nodes per tile of the split-flag scan (one per thread)

struct LevelArgs {
    const NodeRec *nodes;
    const int32_t *list;
    const uint32_t *list_n;       // the depth's warp or CTA list count in LevelCounts
    const Entry *rows_in;
    Entry *rows_out;
    int64_t row_cap;
    const void *Rr;             // row-major ranks [N][F], uint8_t or uint16_t
    const float *vals;
    const uint32_t *card;
    int64_t N;
    const uint32_t *tree_rng;
    int32_t F, mtry, min_node, max_depth, depth;
    uint32_t seed_lo, seed_hi;
    SplitRes *res;
    uint32_t *tile_splits;      // per tile of kScanTile nodes: nodes that split (zero on entry)
    const uint32_t *depth_ptr;  // when set, the depth is read here (a graph replays one level body)
    uint32_t node_cap;          // entries of the node table (bounds checks of debug builds)
    // presorted lists (the list kernel): per feature f, per tree t, a node's segment of
    // lists_in[f * list_stride + t * row_cap + ...] holds the positions of its entries within its
    // segment of rows_in, in increasing rank of f; newpos[t * row_cap + start + p] receives the
    // position in rows_out of the entry at position p when the node splits
    const uint32_t *lists_in = nullptr;
    uint32_t *lists_out = nullptr;
    int64_t list_stride = 0;
    uint32_t *newpos = nullptr;
};

__device__ __forceinline__ int level_depth(const LevelArgs &a)
{
    return a.depth_ptr ? (int)*a.depth_ptr : a.depth;
}

__device__ __forceinline__ bool node_stops(const LevelArgs &a, const NodeRec &nd)
{
    return nd.n <= (uint32_t)a.min_node || (a.max_depth > 0 && level_depth(a) >= a.max_depth);
}

#ifndef AIWCRF_MTRY_REDUX
#define AIWCRF_MTRY_REDUX 1            // 1: the mtry smallest keys by warp min-reductions
#endif
// a3: the tried features of node (tree, depth, idx). Lane l of the warp evaluates the keys of
// features l, l+32, ...; feature f is tried iff fewer than mtry features have a smaller
// (key, index). Result: bit (f & 31) of mask[f >> 5].
__device__ __forceinline__ void warp_mtry_s(int F, int mtry, uint32_t depth, uint32_t seed_lo, uint32_t seed_hi,
                                            uint32_t tg, uint32_t idx, uint32_t mask[4])
{
    const int lane = threadIdx.x & 31;
    const int nch = (F + 31) >> 5;
    uint32_t key[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        key[c] = 0xFFFFFFFFu;
        mask[c] = 0u;
        const int f = c * 32 + lane;
        if (c < nch && f < F) {
            const uint4 u = philox10(make_uint4(tg, depth, idx, (kDomMtry << 16) | (uint32_t)(f >> 2)), seed_lo, seed_hi);
            key[c] = uint4_word(u, f & 3);
        }
    }
    if (mtry >= F) {
#pragma unroll
        for (int c = 0; c < 4; ++c) mask[c] = __ballot_sync(kFull, c < nch && c * 32 + lane < F);
        return;
    }
    if (nch == 1) {
#if AIWCRF_MTRY_REDUX
        // F <= 32: mtry rounds, each taking the smallest key not yet taken (the lowest lane on
        // a tie: lanes >= F hold 0xFFFFFFFF and come after every feature of the same key)
        uint32_t k = key[0], sel = 0u;
        bool taken = false;
        for (int r = 0; r < mtry; ++r) {
            const uint32_t mn = __reduce_min_sync(kFull, k);
            const uint32_t who = (uint32_t)__ffs(__ballot_sync(kFull, !taken && k == mn)) - 1u;
            sel |= 1u << who;
            if ((uint32_t)lane == who) { taken = true; k = 0xFFFFFFFFu; }
        }
        mask[0] = sel;
        return;
#endif
        // F <= 32: one key per lane; lanes >= F hold 0xFFFFFFFF, which never ranks below a
        // feature's key (on an equal key the higher index loses)
        uint32_t cnt0 = 0u;
#pragma unroll
        for (int g = 0; g < 32; ++g) {
            const uint32_t kg = __shfl_sync(kFull, key[0], g);
            cnt0 += (kg < key[0] || (kg == key[0] && g < lane)) ? 1u : 0u;
        }
        mask[0] = __ballot_sync(kFull, lane < F && cnt0 < (uint32_t)mtry);
        return;
    }
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    for (int c2 = 0; c2 < nch; ++c2) {
        for (int s = 0; s < 32; ++s) {
            const int g = c2 * 32 + s;
            if (g >= F) break;
            const uint32_t kg = __shfl_sync(kFull, key[c2], s);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int f = c * 32 + lane;
                if (kg < key[c] || (kg == key[c] && g < f)) cnt[c]++;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int f = c * 32 + lane;
        mask[c] = __ballot_sync(kFull, c < nch && f < F && cnt[c] < (uint32_t)mtry);
    }
}

__device__ __forceinline__ void warp_mtry(const LevelArgs &a, uint32_t tg, uint32_t idx, uint32_t mask[4])
{
    warp_mtry_s(a.F, a.mtry, (uint32_t)level_depth(a), a.seed_lo, a.seed_hi, tg, idx, mask);
}

__device__ __forceinline__ long long shfl_xor_ll(long long v, int m)
{
    return __shfl_xor_sync(kFull, v, m);
}

__device__ __forceinline__ long long shfl_up_ll(long long v, int m)
{
    return __shfl_up_sync(kFull, v, m);
}

__device__ __forceinline__ void write_leaf(SplitRes *res, int j, int kind, int64_t value)
{
    SplitRes r;
    r.feature = kind; r.rank = 0u; r.thr_bits = 0u; r.nL = 0u; r.lenL = 0u; r.pad = 0u; r.v = value;
    res[j] = r;
}


constexpr int kSmallThreads = 256;
constexpr int kSmallCtasPerSm = 4;     // resident CTAs per SM the small-node kernel is compiled for
constexpr int kLevelChunk = 32;        // depths enqueued between two host reads of the node count

// the n-th (from 0) set bit of the 128-bit feature mask, or -1
__device__ __forceinline__ int nth_feature(const uint32_t (&mask)[4], int n)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int pc = __popc(mask[c]);
        if (n < pc) {
            uint32_t m = mask[c];
            for (int i = 0; i < n; ++i) m &= m - 1;
            return c * 32 + __ffs(m) - 1;
        }
        n -= pc;
    }
    return -1;
}

// One warp per node of at most 32 entries. The node's entries are sorted by each tried feature's
// rank with a bitonic network of width K (the smallest power of two >= the entry count), and
// 32 / K features are sorted side by side in K-lane segments: segment s of pass q takes the
// (q * 32 / K + s)-th tried feature, lane p of a segment entry p. The best candidate is kept
// per lane and reduced over the warp at the end; ties resolve on (gain, feature, rank), so the
// order in which features are visited does not matter.
template <typename RT>
__device__ __forceinline__ void small_node(const LevelArgs &a, const RT *__restrict__ Rr, int j, int lane)
{
    j = AIWCRF_IDX(j, a.node_cap, kBoundNode);
    const NodeRec nd = a.nodes[j];
    if (node_stops(a, nd)) {
        if (lane == 0) write_leaf(a.res, j, -2, 0);
        return;
    }
    if (nd.len == 1) {                  // one entry: every candidate is its last rank, a leaf
        if (lane == 0) write_leaf(a.res, j, -1, 0);
        return;
    }
    const size_t tb = (size_t)nd.tree * (size_t)a.row_cap + nd.start;
    const int K = nd.len <= 2 ? 2 : (int)(1u << (32 - __clz((int)nd.len - 1)));
    const int P = 32 / K;                                        // features per pass
    const int pos = lane & (K - 1), seg = lane / K;
    const bool valid = pos < (int)nd.len;
    Entry e;
    e.row = 0u; e.w = 0u; e.wy = 0;
    if (valid) e = load_entry(a.rows_in + tb + pos);
    const size_t rec = (size_t)AIWCRF_IDX(e.row, (uint32_t)a.N, kBoundRow) * (size_t)a.F;

    uint32_t mask[4];
    warp_mtry(a, a.tree_rng[nd.tree], nd.idx, mask);
    const int n_tried = __popc(mask[0]) + __popc(mask[1]) + __popc(mask[2]) + __popc(mask[3]);
    const int f_lane = lane < n_tried ? nth_feature(mask, lane) : -1;     // lane p: p-th tried feature

    Cand best = cand_none();
    for (int q0 = 0; q0 < n_tried; q0 += P) {
        const int qf = q0 + seg;
        const int fs = __shfl_sync(kFull, f_lane, qf & 31);
        const int f = qf < n_tried ? (qf < 32 ? fs : nth_feature(mask, qf)) : -1;
        const bool live = valid && f >= 0;
        const uint32_t rank = live ? (uint32_t)__ldg(&Rr[rec + f]) : kRankSentinel;
        // a pass whose features are all constant over the node has no boundary (lane seg*K
        // always holds an entry; the shuffle runs in every lane before the vote)
        const uint32_t rank0 = __shfl_sync(kFull, rank, lane & ~(K - 1));
        if (__all_sync(kFull, !live || rank == rank0)) continue;
        uint32_t key = (rank << 5) | (uint32_t)pos;                  // unique within a segment
        // bitonic sort of the keys within each segment, ascending; the low five bits name the
        // entry's lane, whose w and w*y are fetched once the order is known
        for (int k = 2; k <= K; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const uint32_t ok = __shfl_xor_sync(kFull, key, jj);
                const bool asc = (pos & k) == 0;
                const bool lower = (pos & jj) == 0;
                key = ((lower == asc) ? (ok < key) : (ok > key)) ? ok : key;
            }
        }
        const int src = (lane & ~(K - 1)) | (int)(key & 31u);
        const uint32_t r = key >> 5;
        uint32_t cw = __shfl_sync(kFull, live ? e.w : 0u, src);
        long long cs = __shfl_sync(kFull, live ? (long long)e.wy : 0ll, src);
        for (int o = 1; o < K; o <<= 1) {
            const uint32_t tw = __shfl_up_sync(kFull, cw, o);
            const long long ts = __shfl_up_sync(kFull, cs, o);
            if (pos >= o) { cw += tw; cs += ts; }
        }
        uint32_t nr = __shfl_down_sync(kFull, r, 1);
        if (pos == K - 1) nr = kRankSentinel;
        if (f >= 0 && r != kRankSentinel && nr != kRankSentinel && r != nr) {
            const i128_t delta = cand_delta(nd.n, nd.S, cw, cs);
            if (delta != 0) {
                Cand cd;
                cd.h = cand_h(delta, nd.n, cw);
                cd.f = f; cd.r = r; cd.nL = cw; cd.SL = cs;
                if (cand_better(cd, best, nd.n, nd.S)) best = cd;
            }
        }
    }
    best = warp_best(best, nd.n, nd.S);
    if (best.h < 0.0f) {
        if (lane == 0) write_leaf(a.res, j, -1, 0);
        return;
    }
    // partition: entry i on lane i
    const bool lv = lane < (int)nd.len;
    Entry el = e;
    if (K != 32) {
        el.row = 0u; el.w = 0u; el.wy = 0;
        if (lv) el = load_entry(a.rows_in + tb + lane);
    }
    const uint32_t rk =
        lv ? (uint32_t)__ldg(&Rr[(size_t)AIWCRF_IDX(el.row, (uint32_t)a.N, kBoundRow) * (size_t)a.F + best.f]) : kRankSentinel;
    const bool left = lv && rk <= best.r;
    const uint32_t bl = __ballot_sync(kFull, left), bv = __ballot_sync(kFull, lv);
    const uint32_t lenL = __popc(bl), lt = lanemask_lt();
    const uint32_t pos_out = left ? __popc(bl & lt) : lenL + __popc(bv & ~bl & lt);
    if (lv) store_entry(a.rows_out + tb + AIWCRF_IDX(pos_out, nd.len, kBoundOut), el);
    if (lane == 0) {
        SplitRes sr;
        sr.feature = best.f; sr.rank = best.r;
        sr.thr_bits = 0u;                                   // looked up where the node is encoded
        sr.nL = best.nL; sr.lenL = lenL; sr.pad = 0u; sr.v = best.SL;
        a.res[j] = sr;
        atomicAdd(&a.tile_splits[(uint32_t)j / (uint32_t)kScanTile], 1u);
    }
}

// one warp per node with at most 32 entries
template <typename RT>
__global__ void __launch_bounds__(kSmallThreads, kSmallCtasPerSm) level_small_kernel(LevelArgs a)
{
    const RT *__restrict__ Rr = static_cast<const RT *>(a.Rr);
    const int lane = threadIdx.x & 31;
    const uint32_t list_n = *a.list_n;
    const uint32_t wstride = gridDim.x * (kSmallThreads / 32);
    for (uint32_t gw = blockIdx.x * (kSmallThreads / 32) + (threadIdx.x >> 5); gw < list_n; gw += wstride) {
        small_node(a, Rr, a.list[gw], lane);         // warp-uniform trip count
    }
}


// ------------------------------------------------------------------------------------------
// Presorted lists: the level-synchronous search for columns with many distinct values. A
// histogram over every rank of the tried features costs a node O(sum of their cardinalities)
// whatever its size; instead every tree keeps, per feature, its entries in increasing rank of
// that feature, and each depth partitions these lists stably together with the entries. A node's
// segment of a list is then its entries sorted by that feature, and its split search is one
// ordered scan per tried feature. The candidates (every present rank but the largest) and their
// exact comparison are those of the histogram search, so the trees are the same node for node.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kListMinCard = 4096;   // automatic choice: lists above this many values in a column

__global__ void rep_mark_kernel(const uint32_t *__restrict__ grp_rows, const uint32_t *__restrict__ grp_off,
                                uint32_t G, uint8_t *__restrict__ is_rep)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) is_rep[grp_rows[grp_off[g]]] = 1u;
}

// one CTA per feature: the groups' representative rows in the column's sorted row order
__global__ void __launch_bounds__(1024) rep_order_kernel(const uint32_t *__restrict__ ordF, int64_t N,
                                                         const uint8_t *__restrict__ is_rep, uint32_t G,
                                                         uint32_t *__restrict__ ordG)
{
    __shared__ uint32_t warp_tmp[32];
    const uint32_t *src = ordF + (size_t)blockIdx.x * (size_t)N;
    uint32_t *dst = ordG + (size_t)blockIdx.x * (size_t)G;
    uint32_t running = 0;
    for (int64_t b0 = 0; b0 < N; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t row = i < N ? src[i] : 0u;
        const bool keep = i < N && is_rep[row];
        uint32_t tot;
        const uint32_t incl = block_incl_scan(keep ? 1u : 0u, warp_tmp, tot);
        if (keep && running + incl - 1u < G) dst[running + incl - 1u] = row;
        running += tot;
    }
}

// every tree's entry position (plus one) by representative row ([T][N], zero elsewhere)
__global__ void list_pos_kernel(const Entry *__restrict__ rows, int64_t row_cap, const NodeRec *__restrict__ root,
                                int64_t N, uint32_t *__restrict__ P)
{
    const int64_t t = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)root[t].len) return;
    const Entry e = load_entry(rows + (size_t)t * (size_t)row_cap + (size_t)i);
    P[(size_t)t * (size_t)N + AIWCRF_IDX(e.row, (uint32_t)N, kBoundRow)] = (uint32_t)i + 1u;
}

// CTA (tree, feature): the positions of the tree's entries in increasing rank of the feature
__global__ void __launch_bounds__(1024) list_build_kernel(const uint32_t *__restrict__ ordG, uint32_t G,
                                                          const uint32_t *__restrict__ P, int64_t N, int64_t row_cap,
                                                          int64_t stride, uint32_t *__restrict__ lists)
{
    __shared__ uint32_t warp_tmp[32];
    const int64_t t = blockIdx.x;
    const uint32_t *src = ordG + (size_t)blockIdx.y * (size_t)G;
    const uint32_t *Pt = P + (size_t)t * (size_t)N;
    uint32_t *dst = lists + (size_t)blockIdx.y * (size_t)stride + (size_t)t * (size_t)row_cap;
    uint32_t running = 0;
    for (uint32_t b0 = 0; b0 < G; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t pos = i < G ? Pt[src[i]] : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan(pos > 0u ? 1u : 0u, warp_tmp, tot);
        if (pos > 0u && (int64_t)(running + incl - 1u) < row_cap) dst[running + incl - 1u] = pos - 1u;
        running += tot;
    }
}

constexpr int kBigThreads = 128;
constexpr int kBigCtasPerSm = 6;       // resident CTAs per SM the big-node kernel is compiled for
constexpr int kRowsPerIter = 4;   // rows per thread per pass: independent gathers in flight
constexpr int kFeatChunk = 8;     // tried features whose ranks are loaded before their atomics

// bins the big-node kernel needs so that every tried feature's values fit in one pass (at most
// 4,096; more is handled in groups of that size)
inline int big_bin_cap(int mtry, int F, uint32_t max_card)
{
    const int64_t need = (int64_t)std::min(mtry, F) * (int64_t)std::max<uint32_t>(max_card, 1u);
    return (int)std::min<int64_t>(4096, (need + 31) & ~(int64_t)31);
}

// A big node's split search from the presorted lists. The warps take the tried features in
// turn; a warp scans (w, w*y) along the node's segment of its feature's list (entry positions,
// read from the node's own entry segment), 32 entries a step and kListIlp steps' loads in
// flight, so the left sums of every threshold come without block barriers. A candidate sits at
// the last entry of each run of equal ranks but the last run.
// With AIWCRF_LIST_STAGE > 0, a node of at most that many entries is staged in shared memory
// first (its entries, then per warp the ranks of the feature it scans, gathered in entry order
// with no dependence on the list), so that each scan step reads one list position from HBM and
// the rest from shared memory. Off by default: on the per-row fit the staging passes and the
// smaller L1 cost more than the dependent loads they remove.
constexpr int kListIlp = 4;
#ifndef AIWCRF_LIST_STAGE
#define AIWCRF_LIST_STAGE 0            // entries staged per node (0: none; 768 and 1536 were slower)
#endif
constexpr int kListStage = AIWCRF_LIST_STAGE;

template <int NW>
constexpr int list_stage_bytes() { return kListStage > 0 ? kListStage * 16 + NW * kListStage * 4 : 0; }

template <typename RT, int NW>
__device__ __forceinline__ Cand list_search(const LevelArgs &a, const NodeRec &nd, const int *feats, int m,
                                            unsigned char *stage)
{
    const RT *__restrict__ Rr = static_cast<const RT *>(a.Rr);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t tb = (size_t)nd.tree * (size_t)a.row_cap + nd.start;
    const Entry *__restrict__ rin = a.rows_in + tb;
    const bool staged = kListStage > 0 && nd.len <= (uint32_t)kListStage;   // block-uniform
    long long *s_wy = reinterpret_cast<long long *>(stage);
    uint32_t *s_w = reinterpret_cast<uint32_t *>(stage + 8 * kListStage);
    uint32_t *s_row = s_w + kListStage;
    uint32_t *s_rk = s_row + kListStage + warp * kListStage;     // this warp's ranks
    if (staged) {
        for (uint32_t q = threadIdx.x; q < nd.len; q += 32u * NW) {
            const Entry e = load_entry(rin + q);
            s_wy[q] = (long long)e.wy;
            s_w[q] = e.w;
            s_row[q] = AIWCRF_IDX(e.row, (uint32_t)a.N, kBoundRow);
        }
        __syncthreads();
    }
    Cand best = cand_none();
    for (int k = warp; k < m; k += NW) {
        const int f = feats[k];
        const uint32_t *__restrict__ L = a.lists_in + (size_t)f * (size_t)a.list_stride + tb;
        uint32_t cw = 0u;                       // sums of the earlier steps (warp-uniform)
        long long cs = 0ll;
        if (staged) {
            __syncwarp();                       // the previous feature's ranks are no longer read
#pragma unroll 8
            for (uint32_t q = (uint32_t)lane; q < nd.len; q += 32u) s_rk[q] = (uint32_t)__ldg(&Rr[(size_t)s_row[q] * (size_t)a.F + f]);
            __syncwarp();
        }
        for (uint32_t b0 = 0; b0 < nd.len; b0 += 32u * kListIlp) {
            uint32_t w[kListIlp], rank[kListIlp], nrank[kListIlp];
            long long wy[kListIlp];
#pragma unroll
            for (int u = 0; u < kListIlp; ++u) {
                const uint32_t i = b0 + 32u * u + (uint32_t)lane;
                w[u] = 0u; wy[u] = 0ll; rank[u] = 0u; nrank[u] = 0u;
                if (staged) {
                    if (i < nd.len) {
                        const uint32_t q = AIWCRF_IDX(__ldg(&L[i]), nd.len, kBoundOut);
                        w[u] = s_w[q];
                        wy[u] = s_wy[q];
                        rank[u] = s_rk[q];
                    }
                    if (lane == 31 && i + 1u < nd.len) nrank[u] = s_rk[AIWCRF_IDX(__ldg(&L[i + 1u]), nd.len, kBoundOut)];
                } else if (i < nd.len) {
                    const Entry e = load_entry(rin + AIWCRF_IDX(__ldg(&L[i]), nd.len, kBoundOut));
                    w[u] = e.w;
                    wy[u] = (long long)e.wy;
                    rank[u] = (uint32_t)__ldg(&Rr[(size_t)AIWCRF_IDX(e.row, (uint32_t)a.N, kBoundRow) * (size_t)a.F + f]);
                }
                // the rank after the warp's last entry of this step
                if (!staged && lane == 31 && i + 1u < nd.len) {
                    const uint32_t row2 = __ldg(&rin[AIWCRF_IDX(__ldg(&L[i + 1u]), nd.len, kBoundOut)].row);
                    nrank[u] = (uint32_t)__ldg(&Rr[(size_t)AIWCRF_IDX(row2, (uint32_t)a.N, kBoundRow) * (size_t)a.F + f]);
                }
            }
#pragma unroll
            for (int u = 0; u < kListIlp; ++u) {
                const uint32_t i = b0 + 32u * u + (uint32_t)lane;
                const uint32_t nr_lane = __shfl_down_sync(kFull, rank[u], 1);
                const uint32_t nr = lane == 31 ? nrank[u] : nr_lane;
                uint32_t pw = w[u];
                long long ps = wy[u];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t tw = __shfl_up_sync(kFull, pw, o);
                    const long long tsum = __shfl_up_sync(kFull, ps, o);
                    if (lane >= o) { pw += tw; ps += tsum; }
                }
                if (i + 1u < nd.len && nr != rank[u]) {        // the last entry of a rank's run
                    const uint32_t nL = cw + pw;
                    const long long SL = cs + ps;
                    const i128_t delta = cand_delta(nd.n, nd.S, nL, SL);
                    if (delta != 0) {
                        Cand cd;
                        cd.h = cand_h(delta, nd.n, nL);
                        cd.f = f; cd.r = rank[u]; cd.nL = nL; cd.SL = SL;
                        if (cand_better(cd, best, nd.n, nd.S)) best = cd;
                    }
                }
                cw += __shfl_sync(kFull, pw, 31);
                cs += __shfl_sync(kFull, ps, 31);
            }
        }
    }
    return best;
}

// Stable partition of a split big node's segment of one feature's list, by one warp: ballots
// give each entry its place, so the children's segments stay in rank order. An entry's new
// position, written by the entry partition, also says its side; the list receives the positions
// within the child's own segment.
constexpr int kPartIlp = 8;

// needL / needR: whether the left / right child will search its lists (the other side's entries
// are not written: a child of at most 32 entries is searched from the entries, a stopping one not
// at all).
__device__ __forceinline__ void list_partition_feature(const LevelArgs &a, const NodeRec &nd, int f, uint32_t lenL,
                                                       const uint32_t *np, bool needL, bool needR)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const size_t tb = (size_t)nd.tree * (size_t)a.row_cap + nd.start;
    const uint32_t *__restrict__ Li = a.lists_in + (size_t)f * (size_t)a.list_stride + tb;
    uint32_t *__restrict__ Lo = a.lists_out + (size_t)f * (size_t)a.list_stride + tb;
    uint32_t rl = 0u, rr = 0u;
    for (uint32_t b0 = 0; b0 < nd.len; b0 += 32u * kPartIlp) {
        uint32_t p[kPartIlp], d[kPartIlp];
#pragma unroll
        for (int u = 0; u < kPartIlp; ++u) {
            const uint32_t i = b0 + 32u * u + (uint32_t)lane;
            p[u] = i < nd.len ? AIWCRF_IDX(__ldg(&Li[i]), nd.len, kBoundOut) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kPartIlp; ++u) {
            const uint32_t i = b0 + 32u * u + (uint32_t)lane;
            d[u] = i < nd.len ? AIWCRF_IDX(np[p[u]], nd.len, kBoundOut) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kPartIlp; ++u) {
            const uint32_t s0 = b0 + 32u * u;
            if (s0 >= nd.len) break;                                // warp-uniform
            const uint32_t i = s0 + (uint32_t)lane;
            const bool left = i < nd.len && d[u] < lenL;
            const uint32_t bal = __ballot_sync(kFull, left);
            const uint32_t before = (uint32_t)__popc(bal & lt);
            if (i < nd.len && (left ? needL : needR))
                Lo[AIWCRF_IDX(left ? rl + before : lenL + rr + ((uint32_t)lane - before), nd.len, kBoundOut)] =
                    left ? d[u] : d[u] - lenL;
            const uint32_t nl = (uint32_t)__popc(bal);
            rl += nl;
            rr += min(32u, nd.len - s0) - nl;
        }
    }
}

// After the list kernel of a depth: one CTA per split big node, its warps taking the features
// in turn. A node of at most kPartStage entries first copies its new positions into shared
// memory, so each step's second load is a shared-memory read.
constexpr int kPartThreads = 256;
constexpr int kPartCtasPerSm = 4;
constexpr int kPartStage = 8192;
__global__ void __launch_bounds__(kPartThreads, kPartCtasPerSm) list_partition_kernel(LevelArgs a)
{
    __shared__ uint32_t s_np[kPartStage];
    const uint32_t list_n = *a.list_n;
    const int warp = threadIdx.x >> 5;
    for (uint32_t k = blockIdx.x; k < list_n; k += gridDim.x) {
        const int j = AIWCRF_IDX(a.list[k], a.node_cap, kBoundNode);
        const SplitRes sr = a.res[j];
        if (sr.feature < 0) continue;                                // block-uniform: a leaf
        const NodeRec nd = a.nodes[j];
        // a child needs its lists only if it is searched by the list kernel next depth
        const int d1 = level_depth(a) + 1;
        const bool deep = a.max_depth > 0 && d1 >= a.max_depth;
        const bool needL = !deep && sr.lenL > (uint32_t)kSmallNodeRows && sr.nL > (uint32_t)a.min_node;
        const bool needR = !deep && nd.len - sr.lenL > (uint32_t)kSmallNodeRows && nd.n - sr.nL > (uint32_t)a.min_node;
        if (!needL && !needR) continue;                              // block-uniform
        const uint32_t *np = a.newpos + (size_t)nd.tree * (size_t)a.row_cap + nd.start;
        const bool staged = nd.len <= (uint32_t)kPartStage;
        __syncthreads();                                             // the previous node's copy is read
        if (staged) {
            for (uint32_t q = threadIdx.x; q < nd.len; q += kPartThreads) s_np[q] = __ldg(&np[q]);
            __syncthreads();
        }
        for (int f = warp; f < a.F; f += kPartThreads / 32)
            list_partition_feature(a, nd, f, sr.lenL, staged ? s_np : np, needL, needR);
    }
}

// One CTA per node with more than 32 entries. Shared bins, bin_cap of them, hold per rank
// of every tried feature: sum w (u32) and sum w*y as an exact (low u32, high i32) pair. All
// updates are native 32-bit shared atomics; a wrap of the low word carries into the high word.
template <typename RT, bool LISTS, int NT = kBigThreads>
__device__ __forceinline__ void big_node(const LevelArgs &a, int bin_cap, int j)
{
    const RT *__restrict__ Rr = static_cast<const RT *>(a.Rr);
    extern __shared__ uint32_t sm_bins[];
    uint32_t *bw = sm_bins;                                       // sum w, then its prefix
    uint32_t *blo = sm_bins + bin_cap;                            // sum w*y: low word
    int32_t *bhi = reinterpret_cast<int32_t *>(sm_bins + 2 * bin_cap);   // high word
    uint16_t *cand_l = reinterpret_cast<uint16_t *>(sm_bins + 3 * bin_cap);  // present bins, per warp
    __shared__ int feats[AIWCRF_MAX_FEATURES];
    __shared__ uint32_t fbase[AIWCRF_MAX_FEATURES + 1];
    __shared__ uint32_t carry_w[AIWCRF_MAX_FEATURES];
    __shared__ long long carry_s[AIWCRF_MAX_FEATURES];
    __shared__ uint32_t tot_w[NT];
    __shared__ long long tot_s[NT];
    __shared__ int m_sh;
    __shared__ Cand wbest[(NT / 32)];
    __shared__ Cand winner;
    __shared__ uint32_t warp_tmp[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    j = AIWCRF_IDX(j, a.node_cap, kBoundNode);
    const NodeRec nd = a.nodes[j];
    if (node_stops(a, nd)) {
        if (tid == 0) write_leaf(a.res, j, -2, 0);
        return;
    }
    const size_t tb = (size_t)nd.tree * (size_t)a.row_cap + nd.start;
    const Entry *rin = a.rows_in + tb;

    if (warp == 0) {
        uint32_t mask[4];
        warp_mtry(a, a.tree_rng[nd.tree], nd.idx, mask);
        // tried features in increasing order and the first bin of each
        int m = 0;
        for (int c = 0; c < 4; ++c) {
            const uint32_t mm = mask[c];
            const int f = c * 32 + lane;
            const bool sel = (mm >> lane) & 1u;
            const int pos = m + __popc(mm & ((1u << lane) - 1u));
            if (sel) { feats[pos] = f; carry_w[pos] = 0u; carry_s[pos] = 0ll; }
            m += __popc(mm);
        }
        __syncwarp();
        // exclusive prefix of the tried features' cardinalities
        uint32_t run = 0;
        for (int k0 = 0; k0 < m; k0 += 32) {
            const int k = k0 + lane;
            const uint32_t c = k < m ? a.card[feats[k]] : 0u;
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += t;
            }
            if (k < m) fbase[k] = run + x - c;
            run += __shfl_sync(kFull, x, 31);
        }
        if (lane == 0) { fbase[m] = run; m_sh = m; }
    }
    __syncthreads();
    const int m = m_sh;
    const uint32_t total_bins = fbase[m];
    Cand best = cand_none();

    if constexpr (LISTS) best = list_search<RT, NT / 32>(a, nd, feats, m, reinterpret_cast<unsigned char *>(sm_bins));
    else for (uint32_t g0 = 0; g0 < total_bins; g0 += (uint32_t)bin_cap) {
        const uint32_t g1 = min(total_bins, g0 + (uint32_t)bin_cap);
        const int nb = (int)(g1 - g0);
        for (int b = tid; b < nb; b += NT) { bw[b] = 0u; blo[b] = 0u; bhi[b] = 0; }
        int k_lo = 0;
        while (fbase[k_lo + 1] <= g0) ++k_lo;
        int k_hi = k_lo;
        while (k_hi + 1 < m && fbase[k_hi + 1] < g1) ++k_hi;
        __syncthreads();

        // histogram: per pass a thread loads kRowsPerIter entries and gathers the tried
        // features' ranks of their rows, then adds them to the shared bins
        for (uint32_t base = 0; base < nd.len; base += NT * kRowsPerIter) {
            uint32_t rowv[kRowsPerIter], wv[kRowsPerIter], lov[kRowsPerIter];
            int32_t hiv[kRowsPerIter];
#pragma unroll
            for (int u = 0; u < kRowsPerIter; ++u) {
                const uint32_t i = base + (uint32_t)(u * NT + tid);
                Entry e;
                e.row = 0u; e.w = 0u; e.wy = 0;                           // w = 0: no entry
                if (i < nd.len) e = load_entry(rin + i);
                rowv[u] = e.row;
                wv[u] = e.w;
                lov[u] = (uint32_t)(uint64_t)e.wy;
                hiv[u] = (int32_t)(e.wy >> 32);
            }
            for (int k0 = k_lo; k0 <= k_hi; k0 += kFeatChunk) {
                uint32_t rk[kRowsPerIter][kFeatChunk];
#pragma unroll
                for (int c = 0; c < kFeatChunk; ++c) {
                    const bool kv = k0 + c <= k_hi;
                    const int fk = kv ? feats[k0 + c] : 0;
#pragma unroll
                    for (int u = 0; u < kRowsPerIter; ++u)
                        rk[u][c] = (kv && wv[u])
                                       ? (uint32_t)__ldg(&Rr[(size_t)AIWCRF_IDX(rowv[u], (uint32_t)a.N, kBoundRow) * (size_t)a.F + fk])
                                       : 0u;
                }
#pragma unroll
                for (int c = 0; c < kFeatChunk; ++c) {
                    if (k0 + c > k_hi) break;
                    const uint32_t fb = fbase[k0 + c];
#pragma unroll
                    for (int u = 0; u < kRowsPerIter; ++u) {
                        const uint32_t b = fb + rk[u][c];
                        if (wv[u] && b >= g0 && b < g1) {
                            const uint32_t q = b - g0;
                            atomicAdd(&bw[q], wv[u]);
                            const uint32_t old = atomicAdd(&blo[q], lov[u]);
                            const int32_t carry = (old + lov[u] < old) ? 1 : 0;
                            if (hiv[u] + carry != 0) atomicAdd(&bhi[q], hiv[u] + carry);
                        }
                    }
                }
            }
        }
        __syncthreads();

        // block inclusive prefix over the group's bins (unsegmented), in place
        const int per = (nb + NT - 1) / NT;
        const int lo = min(nb, tid * per), hi = min(nb, lo + per);
        uint32_t lw = 0;
        long long ls = 0;
        for (int b = lo; b < hi; ++b) {
            lw += bw[b];
            ls += ((long long)bhi[b] << 32) + (long long)blo[b];
        }
        tot_w[tid] = lw;
        tot_s[tid] = ls;
        __syncthreads();
        if (warp == 0) {            // exclusive scan of the thread totals by one warp
            constexpr int kPer = NT / 32;
            uint32_t w8[kPer];
            long long s8[kPer];
            uint32_t ws = 0;
            long long ss = 0;
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                w8[k] = ws; s8[k] = ss; ws += tot_w[lane * kPer + k]; ss += tot_s[lane * kPer + k];
            }
            uint32_t xw = ws;
            long long xs = ss;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t tw = __shfl_up_sync(kFull, xw, o);
                const long long ts = __shfl_up_sync(kFull, xs, o);
                if (lane >= o) { xw += tw; xs += ts; }
            }
            xw -= ws;
            xs -= ss;
#pragma unroll
            for (int k = 0; k < kPer; ++k) { tot_w[lane * kPer + k] = xw + w8[k]; tot_s[lane * kPer + k] = xs + s8[k]; }
        }
        __syncthreads();
        {
            uint32_t rw = tot_w[tid];
            long long rs = tot_s[tid];
            for (int b = lo; b < hi; ++b) {
                rw += bw[b];
                rs += ((long long)bhi[b] << 32) + (long long)blo[b];
                bw[b] = rw;
                blo[b] = (uint32_t)(unsigned long long)rs;
                bhi[b] = (int32_t)(rs >> 32);
            }
        }
        __syncthreads();

        // candidates: each warp first lists the present ranks (bins holding entries) of its
        // threads' bins, by ballots, in its own part of cand_l (warp w's part starts at its first
        // bin and holds at most its bins); then its lanes evaluate the listed bins one each
        {
            uint16_t *wl = cand_l + (size_t)warp * 32u * (size_t)per;
            uint32_t n_w = 0u;
            for (int i = 0; i < per; ++i) {
                const int b = lo + i;
                const bool pres = b < hi && bw[b] != (b > 0 ? bw[b - 1] : 0u);
                const uint32_t bal = __ballot_sync(kFull, pres);
                if (pres) wl[n_w + __popc(bal & lanemask_lt())] = (uint16_t)b;
                n_w += (uint32_t)__popc(bal);
            }
            __syncwarp();
            for (uint32_t ix = (uint32_t)lane; ix < n_w; ix += 32u) {
                const int b = wl[ix];
                const uint32_t gb = g0 + (uint32_t)b;
                int k = k_lo;
                while (fbase[k + 1] <= gb) ++k;
                const uint32_t pw = bw[b];
                const int fs = (int)(max(fbase[k], g0) - g0);          // feature's first bin here
                const uint32_t nL = pw - (fs > 0 ? bw[fs - 1] : 0u) + carry_w[k];
                if (nL >= nd.n) continue;                               // last present rank
                const long long pS = ((long long)bhi[b] << 32) + (long long)blo[b];
                const long long baseS = fs > 0 ? ((long long)bhi[fs - 1] << 32) + (long long)blo[fs - 1] : 0ll;
                const long long SL = pS - baseS + carry_s[k];
                const i128_t delta = cand_delta(nd.n, nd.S, nL, SL);
                if (delta == 0) continue;
                Cand cd;
                cd.h = cand_h(delta, nd.n, nL);
                cd.f = feats[k]; cd.r = gb - fbase[k]; cd.nL = nL; cd.SL = SL;
                if (cand_better(cd, best, nd.n, nd.S)) best = cd;
            }
        }
        __syncthreads();
        if (tid == 0 && fbase[k_hi + 1] > g1) {                        // feature continues
            const int fs = (int)(max(fbase[k_hi], g0) - g0);
            carry_w[k_hi] += bw[nb - 1] - (fs > 0 ? bw[fs - 1] : 0u);
            const long long lastS = ((long long)bhi[nb - 1] << 32) + (long long)blo[nb - 1];
            carry_s[k_hi] += lastS - (fs > 0 ? ((long long)bhi[fs - 1] << 32) + (long long)blo[fs - 1] : 0ll);
        }
        __syncthreads();
    }

    best = warp_best(best, nd.n, nd.S);
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (warp == 0) {
        Cand c = lane < (NT / 32) ? wbest[lane] : cand_none();
        c = warp_best(c, nd.n, nd.S);
        if (lane == 0) winner = c;
    }
    __syncthreads();
    const Cand win = winner;
    if (win.h < 0.0f) {
        if (tid == 0) write_leaf(a.res, j, -1, 0);
        return;
    }

    // a5: stable partition of the node's entries into [left | right] at the same offsets; a
    // first pass counts the entries that go left
    uint32_t cnt = 0;
    for (uint32_t i = tid; i < nd.len; i += NT) {
        const uint32_t row = AIWCRF_IDX(__ldg(&rin[i].row), (uint32_t)a.N, kBoundRow);
        cnt += (uint32_t)__ldg(&Rr[(size_t)row * (size_t)a.F + win.f]) <= win.r ? 1u : 0u;
    }
    uint32_t lenL;
    block_incl_scan(cnt, warp_tmp, lenL);
    uint32_t run_l = 0u, run_r = 0u;           // block-uniform running counts
    Entry *rout = a.rows_out + tb;
    for (uint32_t b0 = 0; b0 < nd.len; b0 += NT) {
        const uint32_t i = b0 + tid;
        const bool valid = i < nd.len;
        Entry e;
        e.row = 0u; e.w = 0u; e.wy = 0;
        if (valid) e = load_entry(rin + i);
        const bool left =
            valid && (uint32_t)__ldg(&Rr[(size_t)AIWCRF_IDX(e.row, (uint32_t)a.N, kBoundRow) * (size_t)a.F + win.f]) <= win.r;
        uint32_t tot;
        const uint32_t incl = block_incl_scan(left ? 1u : 0u, warp_tmp, tot);
        if (valid) {
            const uint32_t before_l = incl - (left ? 1u : 0u);
            const uint32_t dst = AIWCRF_IDX(left ? run_l + before_l : lenL + run_r + ((uint32_t)tid - before_l), nd.len, kBoundOut);
            store_entry(&rout[dst], e);
            if constexpr (LISTS) a.newpos[tb + i] = dst;
        }
        run_l += tot;
        run_r += min((uint32_t)NT, nd.len - b0) - tot;
    }

    if (tid == 0) {
        SplitRes sr;
        sr.feature = win.f; sr.rank = win.r;
        sr.thr_bits = 0u;                                   // looked up where the node is encoded
        sr.nL = win.nL; sr.lenL = lenL; sr.pad = 0u; sr.v = win.SL;
        a.res[j] = sr;
        atomicAdd(&a.tile_splits[(uint32_t)j / (uint32_t)kScanTile], 1u);
    }
}

// one CTA per node with more than 32 entries, strided over the depth's CTA list
template <typename RT>
__global__ void __launch_bounds__(kBigThreads, kBigCtasPerSm) level_big_kernel(LevelArgs a, int bin_cap)
{
    const uint32_t list_n = *a.list_n;
    for (uint32_t k = blockIdx.x; k < list_n; k += gridDim.x) {
        __syncthreads();                 // the previous node's shared state is no longer read
        big_node<RT, false>(a, bin_cap, a.list[k]);
    }
}

// the same with the presorted-list search (a.lists_in set): wider CTAs (a node's lists are
// shared among more warps: the top depths hold few, long nodes) with 128 registers per thread
// for the loads the warps keep in flight
#ifndef AIWCRF_LIST_THREADS
#define AIWCRF_LIST_THREADS 128
#endif
constexpr int kListThreads = AIWCRF_LIST_THREADS;
constexpr int kListCtasPerSm = 65536 / (kListThreads * 128);
template <typename RT>
__global__ void __launch_bounds__(kListThreads, kListCtasPerSm) level_list_kernel(LevelArgs a)
{
    const uint32_t list_n = *a.list_n;
    for (uint32_t k = blockIdx.x; k < list_n; k += gridDim.x) {
        __syncthreads();
        big_node<RT, true, kListThreads>(a, 0, a.list[k]);
    }
}

// ------------------------------------------------------------------------------------------
// Tree-resident growth. One CTA grows a whole tree, depth after depth, with the tree's entries
// (sum w, sum w*y, group) in shared memory and a permutation of them that each depth
// partitions into the children's segments. Node tables of the current and the next depth,
// split results and the big nodes' per-feature candidates live in a global scratch slot of the
// CTA. Per depth:
//   A  work items, taken by the warps in turn: (big node, k-th tried feature) -- a warp-private
//      shared-memory histogram of (sum w, sum w*y) per rank of that feature, a scan and the
//      best candidate of that feature; then every small node (<= 32 entries), searched whole
//      by one warp with the bitonic method of level_small_kernel;
//   B  per big node, one warp: the best of its features' candidates, and the stable partition
//      of its entries;
//   C  all threads: an exclusive scan of the split flags numbers the children breadth first;
//      every node is encoded into the tree's output and the next depth's nodes and big-node
//      list are written.
// It is used when every tree's entries fit in shared memory (grouped rows, one-byte ranks,
// F <= 32) and replaces the level-synchronous path's three launches per depth. Trees are the
// same node for node: the same BFS numbering, mtry draws, exact candidate comparison,
// tie-breaks and leaf values.
// ------------------------------------------------------------------------------------------
// build-time tuning of the tree kernel (the forest does not depend on them)
#ifndef AIWCRF_TREE_THREADS
#define AIWCRF_TREE_THREADS 256        // threads per CTA
#endif
#ifndef AIWCRF_TREE_UNROLL
#define AIWCRF_TREE_UNROLL 0           // 1: small-node sort and scan unrolled per segment width
#endif
#ifndef AIWCRF_TREE_PREFETCH
#define AIWCRF_TREE_PREFETCH 1         // small-node passes whose ranks are loaded together
#endif
#ifndef AIWCRF_TREE_DYN
#define AIWCRF_TREE_DYN 1              // 1: phase-A items handed out by a shared counter
#endif
constexpr int kTreeThreads = AIWCRF_TREE_THREADS;
constexpr int kTreeWarps = kTreeThreads / 32;
constexpr int kTreeCtasPerSm = 4;      // resident CTAs per SM the tree kernel is compiled for
constexpr int kTreeIlp = 8;            // rank loads in flight per lane in a histogram pass

struct TNode {            // an active node of a CTA's tree at the current depth
    uint16_t start, len;  // segment of the tree's entry permutation
    uint32_t n;           // sum of multiplicities
    int64_t S;            // sum of w*y
    uint32_t idx;         // BFS index within the depth
    uint32_t pad;
};
static_assert(sizeof(TNode) == 24, "TNode layout");

// a group's rank record in the tree-resident grower: one byte per feature, padded to 32 bytes
// (the grower needs F <= 32; a record is one 32-byte sector)
constexpr int kRecBytes = 32;

struct TreeArgs {
    const Entry *rows;            // bootstrap entries (row = group id), tree t at t * row_cap
    const NodeRec *root;          // bootstrap root record per tree (entry count, n, S)
    int64_t row_cap;
    const uint8_t *Rg;            // group-major rank records [groups][kRecBytes] (F <= 32, zero padded)
    const uint8_t *RgT;           // the same ranks feature-major [F][groups] (a big item's gathers
                                  // for one feature then stay within groups bytes)
    const float *vals;            // rank -> value tables [F][N]
    int64_t N;
    const uint32_t *card;         // values per feature (<= bins)
    const uint32_t *tree_rng;     // global tree index per tree (Philox counter word 0)
    uint32_t n_groups;            // rows of Rg (debug bounds checks)
    int T, F, mtry, min_node, max_depth;
    uint32_t seed_lo, seed_hi;
    int ecap;                     // entry capacity of the shared-memory arrays (>= row_cap)
    int bins;                     // histogram bins per warp (>= every card)
    int big_cap;                  // big nodes per depth at most (ecap / 33 + 1)
    TNode *nodes;                 // per CTA: 2 * ecap
    SplitRes *res;                // per CTA: ecap
    Cand *cands;                  // per CTA: big_cap * 32
    uint64_t *out_nodes, *out_cnodes;   // per tree t at t * node_cap, BFS order
    int64_t node_cap;
    uint32_t *out_count;          // nodes per tree
    GrowStats *stats;
    uint32_t *levels;             // the deepest tree's depth count (atomicMax)
};

size_t tree_smem_bytes(int ecap, int bins, int big_cap)
{
    const size_t e = (size_t)ecap;
    return 8 * e + 4 * e + ((2 * e + 15) & ~(size_t)15) + 2 * ((2 * e + 15) & ~(size_t)15) + ((e + 15) & ~(size_t)15) +
           (size_t)kTreeWarps * (size_t)bins * 12 + 2 * (((size_t)big_cap * 2 + 15) & ~(size_t)15);
}

struct TreeSmem {
    int64_t *wy;
    uint32_t *w;
    uint16_t *g;
    uint16_t *ix[2];
    uint8_t *flag;
    uint32_t *bins;
    uint16_t *big[2];
    uint32_t *big_mask;      // tried features of the depth's big nodes (aliases flag)
};

__device__ __forceinline__ TreeSmem tree_smem(unsigned char *base, const TreeArgs &a)
{
    const size_t e = (size_t)a.ecap;
    TreeSmem m;
    unsigned char *p = base;
    m.wy = reinterpret_cast<int64_t *>(p); p += 8 * e;
    m.w = reinterpret_cast<uint32_t *>(p); p += 4 * e;
    m.g = reinterpret_cast<uint16_t *>(p); p += (2 * e + 15) & ~(size_t)15;
    m.ix[0] = reinterpret_cast<uint16_t *>(p); p += (2 * e + 15) & ~(size_t)15;
    m.ix[1] = reinterpret_cast<uint16_t *>(p); p += (2 * e + 15) & ~(size_t)15;
    m.flag = p; p += (e + 15) & ~(size_t)15;
    m.bins = reinterpret_cast<uint32_t *>(p); p += (size_t)kTreeWarps * (size_t)a.bins * 12;
    m.big[0] = reinterpret_cast<uint16_t *>(p); p += ((size_t)a.big_cap * 2 + 15) & ~(size_t)15;
    m.big[1] = reinterpret_cast<uint16_t *>(p);
    // the big nodes' masks are read in phase A only, the partition flags written in phase B only:
    // they share the flag array (4 * big_cap <= its 16-byte-rounded ecap bytes)
    m.big_mask = reinterpret_cast<uint32_t *>(m.flag);
    return m;
}

__device__ __forceinline__ bool tnode_stops(const TreeArgs &a, uint32_t n, uint32_t depth)
{
    return n <= (uint32_t)a.min_node || (a.max_depth > 0 && (int)depth >= a.max_depth);
}

__device__ __forceinline__ bool tnode_big(const TreeArgs &a, const TNode &nd, uint32_t depth)
{
    return nd.len > (uint32_t)kSmallNodeRows && !tnode_stops(a, nd.n, depth);
}

// One pass of a small node's search with K-entry segments (K a power of two): the keys
// (rank, entry lane) of every segment sorted by a bitonic network, then the prefix of (w, w*y)
// in that order. r: this lane's rank in sorted order; nr: the next lane's (sentinel at the end).
template <int K>
__device__ __forceinline__ void small_sort_scan(uint32_t rank, int pos, int lane, uint32_t w_live, long long wy_live,
                                                uint32_t &r, uint32_t &cw, long long &cs, uint32_t &nr)
{
    uint32_t key = (rank << 5) | (uint32_t)pos;
#pragma unroll
    for (int k = 2; k <= K; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            const uint32_t ok = __shfl_xor_sync(kFull, key, jj);
            const bool asc = (pos & k) == 0;
            const bool lower = (pos & jj) == 0;
            key = ((lower == asc) ? (ok < key) : (ok > key)) ? ok : key;
        }
    }
    const int src = (lane & ~(K - 1)) | (int)(key & 31u);
    r = key >> 5;
    cw = __shfl_sync(kFull, w_live, src);
    cs = __shfl_sync(kFull, wy_live, src);
#pragma unroll
    for (int o = 1; o < K; o <<= 1) {
        const uint32_t tw = __shfl_up_sync(kFull, cw, o);
        const long long ts = __shfl_up_sync(kFull, cs, o);
        if (pos >= o) { cw += tw; cs += ts; }
    }
    nr = __shfl_down_sync(kFull, r, 1);
    if (pos == K - 1) nr = kRankSentinel;
}

constexpr int kSmallPrefetch = AIWCRF_TREE_PREFETCH;   // passes whose ranks a small node loads at once

// the same pass with the segment width a runtime value (one loop for every width)
__device__ __forceinline__ void small_sort_scan_rt(int K, uint32_t rank, int pos, int lane, uint32_t w_live,
                                                   long long wy_live, uint32_t &r, uint32_t &cw, long long &cs,
                                                   uint32_t &nr)
{
    uint32_t key = (rank << 5) | (uint32_t)pos;
    for (int k = 2; k <= K; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            const uint32_t ok = __shfl_xor_sync(kFull, key, jj);
            const bool asc = (pos & k) == 0;
            const bool lower = (pos & jj) == 0;
            key = ((lower == asc) ? (ok < key) : (ok > key)) ? ok : key;
        }
    }
    const int src = (lane & ~(K - 1)) | (int)(key & 31u);
    r = key >> 5;
    cw = __shfl_sync(kFull, w_live, src);
    cs = __shfl_sync(kFull, wy_live, src);
    for (int o = 1; o < K; o <<= 1) {
        const uint32_t tw = __shfl_up_sync(kFull, cw, o);
        const long long ts = __shfl_up_sync(kFull, cs, o);
        if (pos >= o) { cw += tw; cs += ts; }
    }
    nr = __shfl_down_sync(kFull, r, 1);
    if (pos == K - 1) nr = kRankSentinel;
}

// A small node (or a node that stops) searched whole by one warp: as small_node, on the tree's
// shared-memory entries and the group records, with the passes' rank loads issued together and
// the sort and scan unrolled for the node's segment width.
__device__ __forceinline__ void tree_small_node(const TreeArgs &a, const TreeSmem &sm, const uint16_t *ix, uint16_t *ox,
                                                const TNode &nd, uint32_t tg, uint32_t depth, SplitRes *res_j, int lane)
{
    if (tnode_stops(a, nd.n, depth)) {
        if (lane == 0) write_leaf(res_j, 0, -2, 0);
        return;
    }
    if (nd.len == 1) {                  // one entry: every candidate is its last rank, a leaf
        if (lane == 0) write_leaf(res_j, 0, -1, 0);
        return;
    }
    const int len = nd.len;
    const int K = len <= 2 ? 2 : (int)(1u << (32 - __clz(len - 1)));
    const int P = 32 / K;
    const int pos = lane & (K - 1), seg = lane / K;
    const bool valid = pos < len;
    uint32_t ew = 0u, eg = 0u;
    long long ewy = 0ll;
    if (valid) {
        const int ei = AIWCRF_IDX(ix[nd.start + pos], a.ecap, kBoundRow);
        ew = sm.w[ei]; ewy = sm.wy[ei]; eg = sm.g[ei];
    }
    const uint8_t *rec = a.Rg + (size_t)AIWCRF_IDX(eg, a.n_groups, kBoundRow) * kRecBytes;

    uint32_t mask[4];
    warp_mtry_s(a.F, a.mtry, depth, a.seed_lo, a.seed_hi, tg, nd.idx, mask);
    const int n_tried = __popc(mask[0]);
    const int f_lane = lane < n_tried ? nth_feature(mask, lane) : -1;

    Cand best = cand_none();
    for (int q0 = 0; q0 < n_tried; q0 += kSmallPrefetch * P) {
        uint32_t rk[kSmallPrefetch];
#pragma unroll
        for (int u = 0; u < kSmallPrefetch; ++u) {
            const int qf = q0 + u * P + seg;
            const int fs = __shfl_sync(kFull, f_lane, qf & 31);
            rk[u] = (valid && qf < n_tried) ? (uint32_t)__ldg(&rec[fs]) : kRankSentinel;
        }
#pragma unroll
        for (int u = 0; u < kSmallPrefetch; ++u) {
            if (q0 + u * P >= n_tried) break;                       // warp-uniform
            const int qf = q0 + u * P + seg;
            const int fs = __shfl_sync(kFull, f_lane, qf & 31);
            const int f = qf < n_tried ? fs : -1;
            const bool live = valid && f >= 0;
            const uint32_t rank = rk[u];
            // a pass whose features are all constant over the node has no boundary (lane seg*K
            // always holds an entry; the shuffle runs in every lane before the vote)
            const uint32_t rank0 = __shfl_sync(kFull, rank, lane & ~(K - 1));
            if (__all_sync(kFull, !live || rank == rank0)) continue;
            uint32_t r, cw, nr;
            long long cs;
            const uint32_t wl = live ? ew : 0u;
            const long long yl = live ? ewy : 0ll;
#if AIWCRF_TREE_UNROLL
            switch (K) {                                            // warp-uniform
            case 2: small_sort_scan<2>(rank, pos, lane, wl, yl, r, cw, cs, nr); break;
            case 4: small_sort_scan<4>(rank, pos, lane, wl, yl, r, cw, cs, nr); break;
            case 8: small_sort_scan<8>(rank, pos, lane, wl, yl, r, cw, cs, nr); break;
            case 16: small_sort_scan<16>(rank, pos, lane, wl, yl, r, cw, cs, nr); break;
            default: small_sort_scan<32>(rank, pos, lane, wl, yl, r, cw, cs, nr); break;
            }
#else
            small_sort_scan_rt(K, rank, pos, lane, wl, yl, r, cw, cs, nr);
#endif
            if (f >= 0 && r != kRankSentinel && nr != kRankSentinel && r != nr) {
                const i128_t delta = cand_delta(nd.n, nd.S, cw, cs);
                if (delta != 0) {
                    Cand cd;
                    cd.h = cand_h(delta, nd.n, cw);
                    cd.f = f; cd.r = r; cd.nL = cw; cd.SL = cs;
                    if (cand_better(cd, best, nd.n, nd.S)) best = cd;
                }
            }
        }
    }
    best = warp_best(best, nd.n, nd.S);
    if (best.h < 0.0f) {
        if (lane == 0) write_leaf(res_j, 0, -1, 0);
        return;
    }
    // partition: entry i on lane i
    // (lane i < len holds entry i: segment 0, position i, and that entry's record)
    const bool lv = lane < len;
    const int el = lv ? AIWCRF_IDX(ix[nd.start + lane], a.ecap, kBoundRow) : 0;
    const uint32_t rk = lv ? (uint32_t)__ldg(&rec[best.f]) : kRankSentinel;
    const bool left = lv && rk <= best.r;
    const uint32_t bl = __ballot_sync(kFull, left), bv = __ballot_sync(kFull, lv);
    const uint32_t lenL = __popc(bl), lt = lanemask_lt();
    const uint32_t pos_out = left ? __popc(bl & lt) : lenL + __popc(bv & ~bl & lt);
    if (lv) ox[nd.start + AIWCRF_IDX(pos_out, (uint32_t)len, kBoundOut)] = (uint16_t)el;
    if (lane == 0) {
        SplitRes sr;
        sr.feature = best.f; sr.rank = best.r;
        sr.thr_bits = 0u;                                   // looked up where the node is encoded
        sr.nL = best.nL; sr.lenL = lenL; sr.pad = 0u; sr.v = best.SL;
        *res_j = sr;
    }
}

// Work item (big node, k-th tried feature): a warp-private histogram over the feature's ranks,
// its scan, and the best candidate of the feature.
__device__ __forceinline__ void tree_big_item(const TreeArgs &a, const TreeSmem &sm, const uint16_t *ix, const TNode &nd,
                                              uint32_t tried, int k, uint32_t *bins, Cand *out, int lane,
                                              uint32_t card_lane)
{
    uint32_t mask[4] = {tried, 0u, 0u, 0u};
    const int f = nth_feature(mask, k);
    const int card = (int)__shfl_sync(kFull, card_lane, f);       // lane f holds feature f's value count
    uint32_t *bw = bins, *blo = bins + a.bins;
    int32_t *bhi = reinterpret_cast<int32_t *>(bins + 2 * a.bins);
    for (int b = lane; b < card; b += 32) { bw[b] = 0u; blo[b] = 0u; bhi[b] = 0; }
    __syncwarp();
    const int len = nd.len;
    const uint8_t *Rf = a.RgT + (size_t)f * a.n_groups;          // this feature's ranks, by group
    for (int base = 0; base < len; base += 32 * kTreeIlp) {
        uint32_t rk[kTreeIlp], wv[kTreeIlp], lov[kTreeIlp];
        int32_t hiv[kTreeIlp];
#pragma unroll
        for (int u = 0; u < kTreeIlp; ++u) {
            const int i = base + u * 32 + lane;
            wv[u] = 0u; rk[u] = 0u; lov[u] = 0u; hiv[u] = 0;
            if (i < len) {
                const int e = AIWCRF_IDX(ix[nd.start + i], a.ecap, kBoundRow);
                const int64_t y = sm.wy[e];
                wv[u] = sm.w[e];
                lov[u] = (uint32_t)(uint64_t)y;
                hiv[u] = (int32_t)(y >> 32);
                rk[u] = AIWCRF_IDX((uint32_t)__ldg(&Rf[AIWCRF_IDX(sm.g[e], a.n_groups, kBoundRow)]),
                                   (uint32_t)card, kBoundBin);
            }
        }
#pragma unroll
        for (int u = 0; u < kTreeIlp; ++u) {
            if (wv[u]) {
                atomicAdd(&bw[rk[u]], wv[u]);
                const uint32_t old = atomicAdd(&blo[rk[u]], lov[u]);
                const int32_t carry = (old + lov[u] < old) ? 1 : 0;
                if (hiv[u] + carry != 0) atomicAdd(&bhi[rk[u]], hiv[u] + carry);
            }
        }
    }
    __syncwarp();
    // lane l scans bins [l * per, (l + 1) * per): its totals, a warp exclusive scan, then its
    // present bins in order
    const int per = (card + 31) >> 5;
    const int b0 = min(card, lane * per), b1 = min(card, b0 + per);
    uint32_t lw = 0u;
    long long ls = 0ll;
    for (int b = b0; b < b1; ++b) {
        lw += bw[b];
        ls += ((long long)bhi[b] << 32) + (long long)blo[b];
    }
    uint32_t xw = lw;
    long long xs = ls;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t tw = __shfl_up_sync(kFull, xw, o);
        const long long ts = __shfl_up_sync(kFull, xs, o);
        if (lane >= o) { xw += tw; xs += ts; }
    }
    uint32_t nL = xw - lw;
    long long SL = xs - ls;
    Cand best = cand_none();
    for (int b = b0; b < b1; ++b) {
        const uint32_t cw = bw[b];
        if (!cw) continue;
        nL += cw;
        SL += ((long long)bhi[b] << 32) + (long long)blo[b];
        if (nL >= nd.n) continue;                               // the last present rank
        const i128_t delta = cand_delta(nd.n, nd.S, nL, SL);
        if (delta == 0) continue;
        Cand cd;
        cd.h = cand_h(delta, nd.n, nL);
        cd.f = f; cd.r = (uint32_t)b; cd.nL = nL; cd.SL = SL;
        if (cand_better(cd, best, nd.n, nd.S)) best = cd;
    }
    best = warp_best(best, nd.n, nd.S);
    if (lane == 0) *out = best;
    __syncwarp();                                               // the bins are reused next
}

// A big node's decision from its features' candidates, then the stable partition of its entries.
__device__ __forceinline__ void tree_big_split(const TreeArgs &a, const TreeSmem &sm, const uint16_t *ix, uint16_t *ox,
                                               const TNode &nd, int m, const Cand *cands, SplitRes *res_j, int lane)
{
    Cand c = lane < m ? cands[lane] : cand_none();
    c = warp_best(c, nd.n, nd.S);
    if (c.h < 0.0f) {
        if (lane == 0) write_leaf(res_j, 0, -1, 0);
        return;
    }
    const int len = nd.len;
    const uint8_t *Rf = a.RgT + (size_t)c.f * a.n_groups;
    uint32_t cnt = 0u;
    for (int base = 0; base < len; base += 32 * kTreeIlp) {
        uint32_t rk[kTreeIlp];
#pragma unroll
        for (int u = 0; u < kTreeIlp; ++u) {
            const int i = base + u * 32 + lane;
            rk[u] = i < len ? (uint32_t)__ldg(&Rf[(size_t)AIWCRF_IDX(sm.g[AIWCRF_IDX(ix[nd.start + i], a.ecap, kBoundRow)],
                                                                     a.n_groups, kBoundRow)])
                            : kRankSentinel;
        }
#pragma unroll
        for (int u = 0; u < kTreeIlp; ++u) {
            const int i = base + u * 32 + lane;
            if (i < len) {
                const bool l = rk[u] <= c.r;
                sm.flag[nd.start + i] = l ? 1 : 0;
                cnt += l ? 1u : 0u;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    __syncwarp();
    const uint32_t lenL = cnt, lt = lanemask_lt();
    uint32_t run_l = 0u, run_r = 0u;
    for (int b0 = 0; b0 < len; b0 += 32) {
        const int i = b0 + lane;
        const bool v = i < len;
        const bool l = v && sm.flag[nd.start + i];
        const uint32_t bl = __ballot_sync(kFull, l), bv = __ballot_sync(kFull, v);
        if (v) {
            const uint32_t p = l ? run_l + __popc(bl & lt) : lenL + run_r + __popc(bv & ~bl & lt);
            ox[nd.start + p] = ix[nd.start + i];
        }
        run_l += __popc(bl);
        run_r += __popc(bv & ~bl);
    }
    if (lane == 0) {
        SplitRes sr;
        sr.feature = c.f; sr.rank = c.r;
        sr.thr_bits = 0u;                                   // looked up where the node is encoded
        sr.nL = c.nL; sr.lenL = lenL; sr.pad = 0u; sr.v = c.SL;
        *res_j = sr;
    }
}

// Phase B when the depth has fewer big nodes than warps: the W = warps / nb warps of a node
// split its entries into W consecutive chunks; each flags and counts its chunk, the counts meet
// in shared memory across one CTA barrier, and each writes its chunk's entries after the left
// (or right) entries of the chunks before it: the same stable partition as one warp's.
// Every warp of the CTA calls this once (it holds the depth's one barrier).
__device__ __forceinline__ void tree_big_split_w(const TreeArgs &a, const TreeSmem &sm, const uint16_t *ix, uint16_t *ox,
                                                 const TNode *cn, const uint16_t *big, uint32_t nb, int m,
                                                 const Cand *cands, SplitRes *res, uint32_t *counts, int warp, int lane)
{
    const uint32_t W = (uint32_t)kTreeWarps / nb, bi = (uint32_t)warp / W, q = (uint32_t)warp % W;
    const bool act = bi < nb;
    Cand c = cand_none();
    TNode nd;
    uint32_t i = 0u, c0 = 0u, c1 = 0u, cnt = 0u;
    if (act) {
        i = AIWCRF_IDX(big[bi], a.ecap, kBoundNode);
        nd = cn[i];
        c = lane < m ? cands[(size_t)bi * 32 + lane] : cand_none();
        c = warp_best(c, nd.n, nd.S);                   // the same in every warp of the node
        if (c.h >= 0.0f) {
            const uint32_t len = nd.len, chunk = ((len + W - 1u) / W + 31u) & ~31u;
            c0 = min(len, q * chunk);
            c1 = min(len, c0 + chunk);
            const uint8_t *Rf = a.RgT + (size_t)c.f * a.n_groups;
            for (uint32_t base = c0; base < c1; base += 32u * kTreeIlp) {
                uint32_t rk[kTreeIlp];
#pragma unroll
                for (int u = 0; u < kTreeIlp; ++u) {
                    const uint32_t e = base + 32u * u + (uint32_t)lane;
                    rk[u] = e < c1 ? (uint32_t)__ldg(&Rf[AIWCRF_IDX(sm.g[AIWCRF_IDX(ix[nd.start + e], a.ecap, kBoundRow)],
                                                                    a.n_groups, kBoundRow)])
                                   : kRankSentinel;
                }
#pragma unroll
                for (int u = 0; u < kTreeIlp; ++u) {
                    const uint32_t e = base + 32u * u + (uint32_t)lane;
                    if (e < c1) {
                        const bool l = rk[u] <= c.r;
                        sm.flag[nd.start + e] = l ? 1 : 0;
                        cnt += l ? 1u : 0u;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        } else if (q == 0 && lane == 0) {
            write_leaf(&res[i], 0, -1, 0);
        }
    }
    if (lane == 0) counts[warp] = cnt;
    __syncthreads();
    if (!act || c.h < 0.0f) return;
    uint32_t lenL = 0u, offL = 0u;
    for (uint32_t k = 0; k < W; ++k) {
        const uint32_t ck = counts[bi * W + k];
        lenL += ck;
        if (k < q) offL += ck;
    }
    const uint32_t lt = lanemask_lt();
    uint32_t run_l = offL, run_r = c0 - offL;           // the chunks before this one hold c0 entries
    for (uint32_t b0 = c0; b0 < c1; b0 += 32u) {
        const uint32_t e = b0 + (uint32_t)lane;
        const bool v = e < c1;
        const bool l = v && sm.flag[nd.start + e];
        const uint32_t bl = __ballot_sync(kFull, l), bv = __ballot_sync(kFull, v);
        if (v) {
            const uint32_t p = l ? run_l + __popc(bl & lt) : lenL + run_r + __popc(bv & ~bl & lt);
            ox[nd.start + AIWCRF_IDX(p, (uint32_t)nd.len, kBoundOut)] = ix[nd.start + e];
        }
        run_l += __popc(bl);
        run_r += __popc(bv & ~bl);
    }
    if (q == 0 && lane == 0) {
        SplitRes sr;
        sr.feature = c.f; sr.rank = c.r;
        sr.thr_bits = 0u;                                   // looked up where the node is encoded
        sr.nL = c.nL; sr.lenL = lenL; sr.pad = 0u; sr.v = c.SL;
        res[i] = sr;
    }
}

__global__ void __launch_bounds__(kTreeThreads, kTreeCtasPerSm) tree_grow_kernel(TreeArgs a)
{
    extern __shared__ __align__(16) unsigned char tree_sm[];
    __shared__ uint32_t warp_tmp[32];
    __shared__ unsigned long long red[6][kTreeWarps];
    __shared__ uint32_t s_nb[2];
    __shared__ uint32_t s_next;                                 // the next phase-A item to hand out
    const TreeSmem sm = tree_smem(tree_sm, a);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    TNode *const nodes0 = a.nodes + (size_t)blockIdx.x * 2 * (size_t)a.ecap;
    TNode *const nodes1 = nodes0 + a.ecap;
    SplitRes *const res = a.res + (size_t)blockIdx.x * (size_t)a.ecap;
    Cand *const cands = a.cands + (size_t)blockIdx.x * (size_t)a.big_cap * 32;
    uint32_t *const wbins = sm.bins + (size_t)warp * (size_t)a.bins * 3;
    const int m = a.mtry < a.F ? a.mtry : a.F;
    const uint32_t card_lane = lane < a.F ? __ldg(&a.card[lane]) : 0u;   // F <= 32 here
    // fit counters: 32-bit per thread within a tree, folded into per-warp 64-bit sums in
    // shared memory after each tree (fewer live registers than 64-bit per-thread sums)
    uint32_t v[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    if (lane < 6) red[lane][warp] = 0ull;
    uint32_t max_levels = 0u;

    for (int t = blockIdx.x; t < a.T; t += gridDim.x) {
        __syncthreads();                                        // the previous tree is done
        const NodeRec root = a.root[t];
        const int len0 = (int)root.len;
        const Entry *rin = a.rows + (size_t)t * (size_t)a.row_cap;
        for (int i = tid; i < len0; i += kTreeThreads) {
            const Entry e = load_entry(rin + i);
            sm.wy[i] = e.wy; sm.w[i] = e.w; sm.g[i] = (uint16_t)e.row; sm.ix[0][i] = (uint16_t)i;
        }
        if (tid == 0) {
            TNode r;
            r.start = 0; r.len = (uint16_t)len0; r.n = root.n; r.S = root.S; r.idx = 0u; r.pad = 0u;
            nodes0[0] = r;
            const bool big = tnode_big(a, r, 0u);
            s_nb[0] = big ? 1u : 0u;
            sm.big[0][0] = 0;
            s_next = kTreeWarps;
        }
        const uint32_t tg = a.tree_rng[t];
        uint64_t *onodes = a.out_nodes + (size_t)t * (size_t)a.node_cap;
        uint64_t *ocnodes = a.out_cnodes + (size_t)t * (size_t)a.node_cap;
        uint32_t C = 1u, base = 0u, depth = 0u;
        int p = 0;
        __syncthreads();
        while (C > 0u) {
            const TNode *cn = p ? nodes1 : nodes0;
            TNode *nx = p ? nodes0 : nodes1;
            const uint16_t *ix = sm.ix[p];
            uint16_t *ox = sm.ix[p ^ 1];
            const uint16_t *big = sm.big[p];
            const uint32_t nb = s_nb[p];
            // the big nodes' tried features, once per node (their items share them)
            if (nb) {
                for (uint32_t bi = (uint32_t)warp; bi < nb; bi += kTreeWarps) {
                    const TNode nd = cn[AIWCRF_IDX(big[bi], a.ecap, kBoundNode)];
                    uint32_t mask[4];
                    warp_mtry_s(a.F, a.mtry, depth, a.seed_lo, a.seed_hi, tg, nd.idx, mask);
                    if (lane == 0) sm.big_mask[bi] = mask[0];
                }
                __syncthreads();
            }
            // A: big-node feature items first (they are the long ones), then the small nodes; a
            // warp that finishes an item takes the next one not yet handed out
            const uint32_t items = nb * (uint32_t)m + C;
            for (uint32_t j = (uint32_t)warp; j < items;) {
                if (j < nb * (uint32_t)m) {
                    const uint32_t bi = j / (uint32_t)m, k = j - bi * (uint32_t)m;
                    const TNode nd = cn[AIWCRF_IDX(big[bi], a.ecap, kBoundNode)];
                    tree_big_item(a, sm, ix, nd, sm.big_mask[bi], (int)k, wbins, &cands[(size_t)bi * 32 + k], lane,
                                  card_lane);
                } else {
                    const uint32_t i = j - nb * (uint32_t)m;
                    const TNode nd = cn[i];
                    if (!tnode_big(a, nd, depth)) tree_small_node(a, sm, ix, ox, nd, tg, depth, &res[i], lane);
                }
#if AIWCRF_TREE_DYN
                uint32_t jn = 0u;
                if (lane == 0) jn = atomicAdd(&s_next, 1u);
                j = __shfl_sync(kFull, jn, 0);
#else
                j += kTreeWarps;
#endif
            }
            __syncthreads();
            // B: big nodes' decisions and partitions (a node per warp, or several warps per
            // node when the depth has fewer big nodes than warps)
            if (nb > 0u && nb < (uint32_t)kTreeWarps) {
                tree_big_split_w(a, sm, ix, ox, cn, big, nb, m, cands, res, warp_tmp, warp, lane);
            } else {
                for (uint32_t bi = (uint32_t)warp; bi < nb; bi += kTreeWarps) {
                    const uint32_t i = AIWCRF_IDX(big[bi], a.ecap, kBoundNode);
                    tree_big_split(a, sm, ix, ox, cn[i], m, &cands[(size_t)bi * 32], &res[i], lane);
                }
            }
            __syncthreads();
            // C: number the children, encode every node, list the next depth
            uint32_t run_split = 0u, run_big = 0u;
            uint16_t *nbig = sm.big[p ^ 1];
            for (uint32_t i0 = 0; i0 < C; i0 += kTreeThreads) {
                const uint32_t i = i0 + (uint32_t)tid;
                const bool valid = i < C;
                SplitRes r;
                TNode nd;
                r.feature = -2;
                if (valid) { r = res[i]; nd = cn[i]; }
                const bool split = valid && r.feature >= 0;
                uint32_t tot;
                const uint32_t loc = run_split + block_incl_scan(split ? 1u : 0u, warp_tmp, tot) - (split ? 1u : 0u);
                TNode L, R;
                bool bigL = false, bigR = false;
                if (valid) {
                    const uint32_t pos = base + i;
                    const uint32_t left = base + C + 2u * loc;
                    const uint64_t node =
                        split ? encode_split(r.feature, left, __float_as_uint(a.vals[(size_t)r.feature * (size_t)a.N + r.rank]))
                              : encode_leaf(round_mean(nd.S, nd.n));
                    onodes[AIWCRF_IDX(pos, a.node_cap, kBoundOut)] = node;
                    ocnodes[AIWCRF_IDX(pos, a.node_cap, kBoundOut)] = split ? encode_split_coded(r.feature, left, r.rank) : node;
                    if (split) {
                        L.start = nd.start; L.len = (uint16_t)r.lenL; L.n = r.nL; L.S = r.v; L.idx = 2u * loc; L.pad = 0u;
                        R.start = (uint16_t)(nd.start + r.lenL); R.len = (uint16_t)(nd.len - r.lenL); R.n = nd.n - r.nL;
                        R.S = nd.S - r.v; R.idx = 2u * loc + 1u; R.pad = 0u;
                        nx[AIWCRF_IDX(2u * loc, a.ecap, kBoundOut)] = L;
                        nx[AIWCRF_IDX(2u * loc + 1u, a.ecap, kBoundOut)] = R;
                        bigL = tnode_big(a, L, depth + 1u);
                        bigR = tnode_big(a, R, depth + 1u);
                    }
                    const bool evald = r.feature != -2;
                    const bool small = nd.len <= (uint32_t)kSmallNodeRows;
                    v[0] += evald ? nd.len : 0u;
                    v[1] += split ? nd.len : 0u;
                    v[2] += evald ? 1u : 0u;
                    v[3] += (evald && small) ? 1u : 0u;
                    v[4] += (evald && small) ? nd.len : 0u;
                    v[5] += (split && small) ? nd.len : 0u;
                }
                const uint32_t nbi = (bigL ? 1u : 0u) + (bigR ? 1u : 0u);
                uint32_t totb;
                uint32_t bpos = run_big + block_incl_scan(nbi, warp_tmp, totb) - nbi;
                if (bigL) nbig[AIWCRF_IDX(bpos++, a.big_cap, kBoundOut)] = (uint16_t)(2u * loc);
                if (bigR) nbig[AIWCRF_IDX(bpos, a.big_cap, kBoundOut)] = (uint16_t)(2u * loc + 1u);
                run_split += tot;
                run_big += totb;
            }
            if (tid == 0) { s_nb[p ^ 1] = run_big; s_next = kTreeWarps; }
            base += C;
            C = 2u * run_split;
            ++depth;
            p ^= 1;
            __syncthreads();
        }
        if (tid == 0) a.out_count[t] = base;
        max_levels = max(max_levels, depth);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            unsigned long long x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            if (lane == 0) red[k][warp] += x;
            v[k] = 0u;
        }
    }
    __syncthreads();
    if (tid < 6) {
        unsigned long long sum = 0;
        for (int w = 0; w < kTreeWarps; ++w) sum += red[tid][w];
        if (sum) atomicAdd(&a.stats->entries_evaluated + tid, sum);   // GrowStats field order
    }
    if (tid == 0 && max_levels) atomicMax(a.levels, max_levels);
}

// Rg[g][f] = the rank record of group g (all its rows share it), kRecBytes per group, zero past F;
// RgT[f][g] the same ranks feature-major
__global__ void group_records_kernel(const uint8_t *__restrict__ Rr, int F, const uint32_t *__restrict__ grp_off,
                                     const uint32_t *__restrict__ grp_rows, const uint32_t *n_groups, uint8_t *__restrict__ Rg,
                                     uint8_t *__restrict__ RgT)
{
    const uint32_t G = *n_groups;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * kRecBytes) return;
    const uint32_t g = (uint32_t)(i / kRecBytes), f = (uint32_t)(i - (int64_t)g * kRecBytes);
    const uint8_t r = (int)f < F ? Rr[(size_t)grp_rows[grp_off[g]] * (size_t)F + f] : (uint8_t)0;
    Rg[i] = r;
    if ((int)f < F) RgT[(size_t)f * G + g] = r;
}

// copy each tree's nodes from its output slot into the forest (and pad an odd count)
__global__ void tree_place_kernel(const uint64_t *slot_nodes, const uint64_t *slot_cnodes, int64_t node_cap,
                                  const uint32_t *counts, uint64_t *const *tree_dst, uint64_t *const *tree_cdst)
{
    const int t = blockIdx.x;
    const uint32_t c = (uint32_t)AIWCRF_IDX(counts[t], (uint64_t)node_cap, kBoundOut);
    const uint64_t *sn = slot_nodes + (size_t)t * (size_t)node_cap, *sc = slot_cnodes + (size_t)t * (size_t)node_cap;
    uint64_t *dn = tree_dst[t], *dc = tree_cdst[t];
    for (uint32_t i = threadIdx.x; i < c; i += blockDim.x) { dn[i] = sn[i]; dc[i] = sc[i]; }
    if (threadIdx.x == 0 && (c & 1u)) { dn[c] = 1ull << 63; dc[c] = 1ull << 63; }
}

// ------------------------------------------------------------------------------------------
// exclusive scans of flag arrays (the grouping of identical feature vectors)
// ------------------------------------------------------------------------------------------

// exclusive scan of nblocks block sums, the grand total at [nblocks]
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(uint32_t *block_sums, int nblocks)
{
    __shared__ uint32_t warp_tmp[32];
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nblocks ? block_sums[b] : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan(v, warp_tmp, tot);
        if (b < nblocks) block_sums[b] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) block_sums[nblocks] = carry;
}

// exclusive scan of a u32 flag array in three passes (4 flags per thread, tiles of kFlagTile)
constexpr int kFlagPer = 4;
constexpr int kFlagTile = kScanThreads * kFlagPer;

__global__ void __launch_bounds__(kScanThreads) flag_scan_reduce_kernel(const uint32_t *flags, int64_t n, uint32_t *block_sums)
{
    __shared__ uint32_t warp_tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kFlagTile + (int64_t)threadIdx.x * kFlagPer;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kFlagPer; ++k) c += base + k < n ? flags[base + k] : 0u;
    uint32_t tot;
    block_incl_scan(c, warp_tmp, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) flag_scan_write_kernel(const uint32_t *flags, int64_t n,
                                                                       const uint32_t *block_sums, int nblocks,
                                                                       uint32_t *excl)
{
    __shared__ uint32_t warp_tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kFlagTile + (int64_t)threadIdx.x * kFlagPer;
    uint32_t fl[kFlagPer], c = 0;
#pragma unroll
    for (int k = 0; k < kFlagPer; ++k) {
        fl[k] = base + k < n ? flags[base + k] : 0u;
        c += fl[k];
    }
    uint32_t tot;
    const uint32_t incl = block_incl_scan(c, warp_tmp, tot);
    uint32_t run = block_sums[blockIdx.x] + incl - c;
#pragma unroll
    for (int k = 0; k < kFlagPer; ++k) {
        if (base + k < n) excl[base + k] = run;
        run += fl[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) excl[n] = block_sums[nblocks];
}

// ------------------------------------------------------------------------------------------
// finalize one depth
// ------------------------------------------------------------------------------------------
struct FinalArgs {
    const NodeRec *nodes;
    const SplitRes *res;
    const uint32_t *tree_off;      // T + 1: first node of each tree at this depth
    uint32_t *tree_base;           // T: nodes of each tree at lower depths
    LevelCounts *cnt;              // C and packed_off of this depth; list counts of the next
    NodeRec *next;
    int32_t *small_list, *big_list;
    PackedRec *packed;             // all finished nodes; this depth starts at cnt->packed_off
    GrowStats *stats;
    uint32_t *next_tree_off;       // T + 1: first node of each tree at the next depth
    int T;
    uint32_t *done;                // CTAs finished (zero on entry, left zero)
    uint32_t *tile_splits;         // the level kernels' split counts per tile, cleared for the next depth
    uint32_t *excl_out;            // n + 1: exclusive split count of every node (written here)
    int parity;                    // this depth's parity: its list counts, cleared at the end
    uint32_t next_cap;             // entries of the next depth's node table (debug bounds checks)
    const float *vals;             // rank -> value tables [F][N]: thresholds of the splits
    int64_t N;
};

__device__ __forceinline__ void push_list(int32_t *list, uint32_t *counter, bool want, int32_t value)
{
    const uint32_t b = __ballot_sync(kFull, want);
    if (!b) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(b) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(b));
    base = __shfl_sync(kFull, base, leader);
    if (want) list[base + __popc(b & lanemask_lt())] = value;
}

// One depth's close, one node per thread, tiles of kScanTile nodes strided over the CTAs:
//  - the exclusive scan of the split flags: the tile's base from the level kernels' per-tile
//    split counts, then a block scan; written to excl_out;
//  - every node finished: its packed record, its children and their list entries in the next
//    depth's parity. A tree's split count before its first node comes from this tile's scan,
//    or, for the one tree that reaches into the tile from an earlier tile, from that tile's base
//    and a count of its flags before the tree's first node;
//  - the last CTA (atomic counter) advances the per-tree bookkeeping and the level counts, and
//    clears this depth's tile and list counts.
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(FinalArgs a)
{
    __shared__ uint32_t sx[kScanTile];
    __shared__ uint32_t warp_tmp[32];
    __shared__ unsigned long long red[6][kFinThreads / 32];
    __shared__ int last;
    const uint32_t n = a.cnt->C;
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *n_next = a.cnt->n_list[a.parity ^ 1];
    unsigned long long v[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    PackedRec *packed = a.packed + a.cnt->packed_off;
    for (uint32_t b = blockIdx.x; b < ntiles; b += gridDim.x) {     // block-uniform
        const uint32_t t0 = b * (uint32_t)kScanTile;
        uint32_t part = 0, base;
        for (uint32_t i = (uint32_t)tid; i < b; i += kFinThreads) part += a.tile_splits[i];
        block_incl_scan(part, warp_tmp, base);          // splits before the tile
        const uint32_t jj = t0 + (uint32_t)tid;
        const bool active = jj < n;
        const uint32_t j = active ? jj : t0;
        const NodeRec nd = a.nodes[j];
        const SplitRes r = a.res[j];
        const bool split = active && r.feature >= 0;
        uint32_t tot;
        const uint32_t g = base + block_incl_scan(split ? 1u : 0u, warp_tmp, tot) - (split ? 1u : 0u);
        sx[tid] = g;
        if (active) a.excl_out[j] = g;
        // the tree of the tile's first node: its split count before its first node
        const uint32_t tf = a.nodes[t0].tree;
        const uint32_t ff = a.tree_off[tf];
        uint32_t span = 0u;
        if (ff < t0) {                                  // block-uniform
            const uint32_t fb = ff / (uint32_t)kScanTile, fs = fb * (uint32_t)kScanTile;
            uint32_t p2 = 0, before;
            for (uint32_t i = (uint32_t)tid; i < fb; i += kFinThreads) p2 += a.tile_splits[i];
            block_incl_scan(p2, warp_tmp, before);
            const uint32_t k = fs + (uint32_t)tid;
            uint32_t cnt_k;
            block_incl_scan((k < ff && a.res[k].feature >= 0) ? 1u : 0u, warp_tmp, cnt_k);
            span = before + cnt_k;
        }
        __syncthreads();
        const uint32_t t = nd.tree;
        const uint32_t first = a.tree_off[t];
        const uint32_t cnt_t = a.tree_off[t + 1] - first;
        const uint32_t local = g - (first >= t0 ? sx[first - t0] : span);
        const uint32_t base_t = a.tree_base[t];
        NodeRec L, Rn;
        if (active) {
            PackedRec pr;
            pr.tree = t;
            pr.pos = base_t + nd.idx;
            // a leaf's value: one thread per node, here (the searches leave it to this pass)
            pr.node = split ? encode_split(r.feature, base_t + cnt_t + 2u * local,
                                           __float_as_uint(a.vals[(size_t)r.feature * (size_t)a.N + r.rank]))
                            : encode_leaf(round_mean(nd.S, nd.n));
            pr.cnode = split ? encode_split_coded(r.feature, base_t + cnt_t + 2u * local, r.rank) : pr.node;
            packed[j] = pr;
        }
        if (split) {
            L.tree = t; L.idx = 2u * local; L.start = nd.start; L.len = r.lenL; L.n = r.nL; L.pad = 0u; L.S = r.v;
            Rn.tree = t; Rn.idx = 2u * local + 1u; Rn.start = nd.start + r.lenL; Rn.len = nd.len - r.lenL;
            Rn.n = nd.n - r.nL; Rn.pad = 0u; Rn.S = nd.S - r.v;
            a.next[AIWCRF_IDX(2u * g, a.next_cap, kBoundOut)] = L;
            a.next[AIWCRF_IDX(2u * g + 1u, a.next_cap, kBoundOut)] = Rn;
        }
        push_list(a.small_list, &n_next[0], split && L.len <= (uint32_t)kSmallNodeRows, (int32_t)(2u * g));
        push_list(a.big_list, &n_next[1], split && L.len > (uint32_t)kSmallNodeRows, (int32_t)(2u * g));
        push_list(a.small_list, &n_next[0], split && Rn.len <= (uint32_t)kSmallNodeRows, (int32_t)(2u * g + 1u));
        push_list(a.big_list, &n_next[1], split && Rn.len > (uint32_t)kSmallNodeRows, (int32_t)(2u * g + 1u));

        const bool evald = active && r.feature != -2;
        const bool small = nd.len <= (uint32_t)kSmallNodeRows;
        v[0] += evald ? nd.len : 0u;
        v[1] += split ? nd.len : 0u;
        v[2] += evald ? 1u : 0u;
        v[3] += (evald && small) ? 1u : 0u;
        v[4] += (evald && small) ? nd.len : 0u;
        v[5] += (split && small) ? nd.len : 0u;
        __syncthreads();                                // sx is rewritten by the next tile
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) red[k][warp] = v[k];
    }
    __syncthreads();
    if (tid < 6) {
        unsigned long long sum = 0;
        for (int w = 0; w < kFinThreads / 32; ++w) sum += red[tid][w];
        if (sum) atomicAdd(&a.stats->entries_evaluated + tid, sum);   // GrowStats field order
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(a.done, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint32_t part = 0, total;
    for (uint32_t i = (uint32_t)tid; i < ntiles; i += kFinThreads) part += a.tile_splits[i];
    block_incl_scan(part, warp_tmp, total);
    for (int t = tid; t <= a.T; t += kFinThreads) {
        const uint32_t o = a.tree_off[t];
        if (t < a.T) a.tree_base[t] += a.tree_off[t + 1] - o;
        a.next_tree_off[t] = 2u * (o < n ? a.excl_out[o] : total);
    }
    // this depth's and the next depth's tiles, and this depth's list counts, start from zero
    const uint32_t nt = (max(n, 2u * total) + (uint32_t)kScanTile - 1u) / (uint32_t)kScanTile;
    for (uint32_t i = (uint32_t)tid; i < nt; i += kFinThreads) a.tile_splits[i] = 0u;
    if (tid == 0) {
        a.cnt->n_list[a.parity][0] = 0u;
        a.cnt->n_list[a.parity][1] = 0u;
        a.cnt->packed_off += n;
        a.cnt->levels += n > 0 ? 1u : 0u;
        a.cnt->C = 2u * total;
        *a.done = 0u;
    }
}

// per tree: nodes below the next depth and where the tree's nodes start in the next depth's
// table; thread 0 then advances the depth counters (after every reader of them has finished)
__global__ void iota_kernel(uint32_t *v, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) v[i] = (uint32_t)i;
}

__global__ void pack_kernel(const PackedRec *packed, int64_t n, uint64_t *const *tree_dst, uint64_t *const *tree_cdst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PackedRec p = packed[i];
    tree_dst[p.tree][p.pos] = p.node;
    tree_cdst[p.tree][p.pos] = p.cnode;
}

// a tree with an odd node count is padded by one never-reached leaf of value 0
__global__ void pad_kernel(const uint32_t *counts, int64_t T, uint64_t *const *tree_dst, uint64_t *const *tree_cdst)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t c = counts[t];
    if (c & 1u) { tree_dst[t][c] = 1ull << 63; tree_cdst[t][c] = 1ull << 63; }
}

__global__ void check_y_kernel(const int64_t *y, int64_t n, uint32_t *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long v = y[i];
    if (v > AIWCRF_MAX_ABS_Y || v < -AIWCRF_MAX_ABS_Y) atomicOr(err, kErrY);
}

// ------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------
static std::atomic<int> g_grower{AIWCRF_GROWER_AUTO};

int set_grower_mode(int mode)
{
    if (mode != AIWCRF_GROWER_AUTO && mode != AIWCRF_GROWER_LEVEL && mode != AIWCRF_GROWER_TREE &&
        mode != AIWCRF_GROWER_LISTS)
        return fail(AIWCRF_E_INVALID_ARG,
                    "grower: 0 (automatic), 1 (level-synchronous), 2 (tree-resident) or 3 (presorted lists)");
    g_grower.store(mode);
    return AIWCRF_OK;
}

int grower_mode() { return g_grower.load(); }

namespace {

struct DevBuf {                // stream-ordered scratch allocation
    void *p = nullptr;
    size_t bytes = 0;
};

// A fit's scratch. Requests up to kArenaPiece bytes are carved from the calling host thread's
// arena: device memory kept between fits and bump-allocated, so that a fit makes a few
// allocation calls instead of dozens (each a host round trip while the device may be idle).
// The arena grows, at the start of a later fit, to the largest carved total a fit asked for,
// up to kArenaCap. Larger requests, and those past the arena, are stream-ordered allocations
// freed at release. Scratches on one thread nest (last in, first out); release() returns the
// carved part to the arena and first waits for the stream, so that no later fit on this thread
// writes memory that queued work still reads.
constexpr size_t kArenaPiece = (size_t)64 << 20;
constexpr size_t kArenaCap = (size_t)512 << 20;

struct Arena {
    void *base = nullptr;
    size_t cap = 0, used = 0, want = 0;
    int device = -1;
    ~Arena() { if (base) cudaFree(base); }
};

inline Arena &thread_arena()
{
    static thread_local Arena a;
    return a;
}

class Scratch {
public:
    explicit Scratch(cudaStream_t s) : s_(s)
    {
        Arena &a = thread_arena();
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
        if (a.used == 0 && (a.device != dev || a.want > a.cap)) {
            // nothing of this thread's arena is in use: (re)size it on the current device
            const size_t want = std::min(std::max(a.want, a.cap), kArenaCap);
            if (a.base) { cudaFreeAsync(a.base, s_); a.base = nullptr; a.cap = 0; }
            a.device = dev;
            if (want && cudaMallocAsync(&a.base, want, s_) == cudaSuccess) a.cap = want;
            else { cudaGetLastError(); a.base = nullptr; a.cap = 0; }
        }
        arena_ = a.device == dev ? &a : nullptr;
        mark_ = arena_ ? arena_->used : 0;
    }
    ~Scratch() { release(); }
    template <class T>
    T *get(size_t count, int *rc)
    {
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        const size_t up = (bytes + 255) & ~(size_t)255;
        if (arena_ && up <= kArenaPiece) {
            carved_ += up;
            arena_->want = std::max(arena_->want, mark_ + carved_);
            if (arena_->used + up <= arena_->cap) {
                void *p = static_cast<unsigned char *>(arena_->base) + arena_->used;
                arena_->used += up;
                return static_cast<T *>(p);
            }
        }
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, bytes, s_);
        if (e != cudaSuccess) {
            *rc = fail(AIWCRF_E_OOM, std::string("device allocation of ") + std::to_string(bytes) +
                                         " bytes failed: " + cudaGetErrorString(e));
            return nullptr;
        }
        bufs_.push_back(p);
        return static_cast<T *>(p);
    }
    // a buffer no longer needed (carved ones stay until release)
    void drop(void *p)
    {
        for (auto &b : bufs_)
            if (b == p) { cudaFreeAsync(b, s_); b = nullptr; }
    }
    void release()
    {
        for (auto b : bufs_)
            if (b) cudaFreeAsync(b, s_);
        bufs_.clear();
        if (arena_ && arena_->used > mark_) {
            cudaStreamSynchronize(s_);
            arena_->used = mark_;
        }
        carved_ = 0;
    }

private:
    cudaStream_t s_;
    std::vector<void *> bufs_;
    Arena *arena_ = nullptr;
    size_t mark_ = 0, carved_ = 0;
};

#define AIWCRF_LAUNCH_CHECK(what)                                   \
    do {                                                            \
        count_launches(1);                                          \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);          \
    } while (0)

#define AIWCRF_CUDA(call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
    } while (0)

int check_err_flags(uint32_t err)
{
    if (err & kErrNaN) return fail(AIWCRF_E_NAN_INPUT, "NaN in the training features");
    if (err & kErrY) return fail(AIWCRF_E_INVALID_ARG, "a target value exceeds |y| <= 2^40");
    if (err & kErrBootOverflow) return fail(AIWCRF_E_LIMIT, "a bootstrap multiplicity exceeded 255");
    if (err & kErrTimeout) return fail(AIWCRF_E_TIMEOUT, "a bounded device wait gave up");
    if (err & kErrCapacity)
        return fail(AIWCRF_E_LIMIT, "the data outgrew the fit plan (more groups, wider ranks or deeper trees)");
    return AIWCRF_OK;
}

// what the level loop leaves behind, for packing into forests
struct PackIn {
    const aiwcrf_fit_params *p;
    int64_t T, Tper;
    int32_t G;
    int64_t N;
    int32_t F;
    int device;
    const uint32_t *tree_base;     // nodes per tree
    const GrowStats *d_stats;
    const PackedRec *packed;
    size_t packed_n;
    int levels;
    const uint32_t *d_inbag;       // or null
    int64_t inbag_words;
    const float *d_vals;
    const uint32_t *d_card;
    uint32_t max_card;
    int rank_bytes;
    uint32_t n_groups;
    // tree-resident growth: nodes in per-tree slots of slot_cap (BFS order), counts in tree_base
    const uint64_t *slot_nodes = nullptr, *slot_cnodes = nullptr;
    int64_t slot_cap = 0;
    const uint32_t *d_levels = nullptr;   // when set, the level count is read here
    int grower = 1;                       // 1 level-synchronous, 2 tree-resident
    const uint32_t *d_err = nullptr;      // when set, the growth's error flags: read with the sizes
};

// One forest per tree group, trees padded to an even node count (16-byte aligned); nodes placed
// by pack_kernel, padding by pad_kernel, compact copies built. Enqueued on s; the caller
// synchronises before using the forests.
int package_forests(const PackIn &in, cudaStream_t s, std::vector<aiwcrf_forest *> &out)
{
    int rc = AIWCRF_OK;
    const int64_t T = in.T, Tper = in.Tper;
    const int32_t G = in.G, F = in.F;
    std::vector<uint32_t> h_tot((size_t)T);
    GrowStats hs;
    uint32_t h_levels = (uint32_t)in.levels;
    uint32_t h_err = 0;
    {
        HostReads hr;
        hr.add(h_tot.data(), in.tree_base, sizeof(uint32_t) * (size_t)T);
        hr.add(&hs, in.d_stats, sizeof(GrowStats));
        if (in.d_levels) hr.add(&h_levels, in.d_levels, sizeof(uint32_t));
        if (in.d_err) hr.add(&h_err, in.d_err, sizeof(uint32_t));
        if ((rc = hr.run(s)) != AIWCRF_OK) return rc;
    }
    if (in.d_err && (rc = check_err_flags(h_err)) != AIWCRF_OK) return rc;     // before any size is used

    std::vector<aiwcrf_forest *> forests((size_t)G, nullptr);
    struct Guard {
        std::vector<aiwcrf_forest *> *v;
        bool keep = false;
        ~Guard() {
            if (keep) return;
            for (auto f : *v) forest_release(f);
        }
    } guard{&forests};
    std::vector<uint64_t *> h_dst((size_t)T), h_cdst((size_t)T);
    for (int32_t g = 0; g < G; ++g) {
        aiwcrf_forest *fr = new aiwcrf_forest();
        forests[(size_t)g] = fr;
        fr->F = F; fr->T = Tper; fr->device = in.device;
        fr->tree_off.assign((size_t)Tper + 1, 0);
        for (int64_t k = 0; k < Tper; ++k) {
            const int64_t cnt = h_tot[(size_t)(g * Tper + k)];
            fr->tree_off[(size_t)k + 1] = fr->tree_off[(size_t)k] + ((cnt + 1) & ~(int64_t)1);
            fr->max_tree_nodes = std::max(fr->max_tree_nodes, (cnt + 1) & ~(int64_t)1);
        }
        fr->num_nodes = fr->tree_off[(size_t)Tper];
        // the training value tables code the queries at predict time
        fr->max_card = in.max_card;
        fr->fstride = std::max<int64_t>(in.max_card, 1);
        if (in.d_inbag) { fr->oob_rows = in.N; fr->inbag_words = in.inbag_words; }
        AIWCRF_CUDA(forest_alloc(fr, s));
        if (in.d_inbag)
            AIWCRF_CUDA(cudaMemcpyAsync(fr->d_inbag, in.d_inbag + (size_t)g * (size_t)Tper * (size_t)in.inbag_words,
                                        sizeof(uint32_t) * (size_t)Tper * (size_t)in.inbag_words, cudaMemcpyDeviceToDevice, s));
        AIWCRF_CUDA(cudaMemcpy2DAsync(fr->d_fvals, sizeof(float) * (size_t)fr->fstride, in.d_vals,
                                      sizeof(float) * (size_t)in.N, sizeof(float) * (size_t)in.max_card, (size_t)F,
                                      cudaMemcpyDeviceToDevice, s));
        AIWCRF_CUDA(cudaMemcpyAsync(fr->d_fcard, in.d_card, sizeof(uint32_t) * (size_t)F, cudaMemcpyDeviceToDevice, s));
        AIWCRF_CUDA(cudaMemcpyAsync(fr->d_tree_off, fr->tree_off.data(), sizeof(int64_t) * (size_t)(Tper + 1),
                                    cudaMemcpyHostToDevice, s));
        for (int64_t k = 0; k < Tper; ++k) {
            h_dst[(size_t)(g * Tper + k)] = fr->d_nodes + fr->tree_off[(size_t)k];
            h_cdst[(size_t)(g * Tper + k)] = fr->d_cnodes + fr->tree_off[(size_t)k];
        }
        fr->stats.num_trees = Tper;
        fr->stats.total_nodes = 0;
        for (int64_t k = 0; k < Tper; ++k) fr->stats.total_nodes += h_tot[(size_t)(g * Tper + k)];
        fr->stats.levels = (int64_t)h_levels;
        fr->stats.grower = in.grower;
        fr->stats.n_features = F;
        fr->stats.mtry = in.p->mtry;
        fr->stats.rank_bytes = in.rank_bytes;
        fr->stats.groups = in.n_groups;
        if (G == 1) {
            fr->stats.entries_evaluated = (int64_t)hs.entries_evaluated;
            fr->stats.entries_partitioned = (int64_t)hs.entries_partitioned;
            fr->stats.nodes_evaluated = (int64_t)hs.nodes_evaluated;
            fr->stats.nodes_small = (int64_t)hs.nodes_small;
            fr->stats.entries_evaluated_small = (int64_t)hs.entries_evaluated_small;
            fr->stats.entries_partitioned_small = (int64_t)hs.entries_partitioned_small;
        }
    }
    Scratch sc(s);
    uint64_t **d_dst = sc.get<uint64_t *>(2 * (size_t)T, &rc); if (rc) return rc;
    AIWCRF_CUDA(cudaMemcpyAsync(d_dst, h_dst.data(), sizeof(uint64_t *) * (size_t)T, cudaMemcpyHostToDevice, s));
    AIWCRF_CUDA(cudaMemcpyAsync(d_dst + T, h_cdst.data(), sizeof(uint64_t *) * (size_t)T, cudaMemcpyHostToDevice, s));
    prof_begin(s, kProfPack);
    if (in.slot_nodes) {
        tree_place_kernel<<<(unsigned)T, 256, 0, s>>>(in.slot_nodes, in.slot_cnodes, in.slot_cap, in.tree_base, d_dst,
                                                      d_dst + T);
        AIWCRF_LAUNCH_CHECK("tree_place_kernel");
    } else {
        pack_kernel<<<(unsigned)((in.packed_n + 255) / 256), 256, 0, s>>>(in.packed, (int64_t)in.packed_n, d_dst, d_dst + T);
        AIWCRF_LAUNCH_CHECK("pack_kernel");
        pad_kernel<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(in.tree_base, T, d_dst, d_dst + T);
        AIWCRF_LAUNCH_CHECK("pad_kernel");
    }
    prof_end(s, kProfPack);
    for (auto fr : forests)
        if ((rc = forest_build_compact(fr, s)) != AIWCRF_OK) return rc;
    guard.keep = true;
    out = forests;
    return AIWCRF_OK;
}

}  // namespace

int fit_batch(const aiwcrf_fit_params &p, const float *dX, const int64_t *dy, int64_t N, int32_t F,
              const std::vector<int64_t> &sub_off, const int32_t *d_sub_rows, int32_t G,
              cudaStream_t s, std::vector<aiwcrf_forest *> &out)
{
    int rc = AIWCRF_OK;
    Scratch sc(s);
    const int64_t Tper = p.num_trees;
    const int64_t T = Tper * (int64_t)G;
    if (T > (int64_t)AIWCRF_MAX_TREES * 16)
        return fail(AIWCRF_E_LIMIT, "too many trees in one batch");

    int device = 0;
    AIWCRF_CUDA(cudaGetDevice(&device));
    keep_pool_memory(device);
    int max_smem_optin = 0;
    AIWCRF_CUDA(cudaDeviceGetAttribute(&max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));

    // per-tree pools
    std::vector<int64_t> h_pool_off((size_t)T);
    std::vector<uint32_t> h_pool_len((size_t)T), h_rng((size_t)T);
    int64_t row_cap = 1;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t off = d_sub_rows ? sub_off[(size_t)g] : -1;
        const int64_t len = d_sub_rows ? sub_off[(size_t)g + 1] - sub_off[(size_t)g] : N;
        row_cap = std::max(row_cap, len);
        for (int64_t k = 0; k < Tper; ++k) {
            const size_t t = (size_t)(g * Tper + k);
            h_pool_off[t] = off;
            h_pool_len[t] = (uint32_t)len;
            h_rng[t] = (uint32_t)(p.first_tree + k);
        }
    }

    uint32_t *d_err = sc.get<uint32_t>(1, &rc); if (rc) return rc;
    GrowStats *d_stats = sc.get<GrowStats>(1, &rc); if (rc) return rc;
    uint32_t *d_counters = sc.get<uint32_t>(4, &rc); if (rc) return rc;
    AIWCRF_CUDA(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
    AIWCRF_CUDA(cudaMemsetAsync(d_stats, 0, sizeof(GrowStats), s));
    AIWCRF_CUDA(cudaMemsetAsync(d_counters, 0, 4 * sizeof(uint32_t), s));

    // a1: presort and rank. The first kernels are enqueued before the rest of the scratch is
    // allocated, so that the device works while the host allocates.
    // sort buffers (one spare word: the grouping's scan writes its total at [N])
    uint32_t *kA = sc.get<uint32_t>((size_t)F * (size_t)N + 1, &rc); if (rc) return rc;
    uint32_t *vA = sc.get<uint32_t>((size_t)F * (size_t)N + 1, &rc); if (rc) return rc;
    const unsigned yblocks = (unsigned)((N + 255) / 256);
    check_y_kernel<<<yblocks, 256, 0, s>>>(dy, N, d_err);
    AIWCRF_LAUNCH_CHECK("check_y_kernel");
    prof_begin(s, kProfRank);
    key_init_kernel<<<dim3(yblocks, (unsigned)F), 256, 0, s>>>(dX, N, kA, vA, d_err);
    AIWCRF_LAUNCH_CHECK("key_init_kernel");
    uint32_t *d_R = sc.get<uint32_t>((size_t)F * (size_t)N, &rc); if (rc) return rc;
    float *d_vals = sc.get<float>((size_t)F * (size_t)N, &rc); if (rc) return rc;
    uint32_t *d_card = sc.get<uint32_t>((size_t)F, &rc); if (rc) return rc;
    uint32_t *kB = sc.get<uint32_t>((size_t)F * (size_t)N + 1, &rc); if (rc) return rc;
    uint32_t *vB = sc.get<uint32_t>((size_t)F * (size_t)N + 1, &rc); if (rc) return rc;
    uint32_t *hist = sc.get<uint32_t>(radix_sort_hist_words(N, F), &rc); if (rc) return rc;
    int64_t *d_pool_off = sc.get<int64_t>((size_t)T, &rc); if (rc) return rc;
    uint32_t *d_pool_len = sc.get<uint32_t>((size_t)T, &rc); if (rc) return rc;
    uint32_t *d_rng = sc.get<uint32_t>((size_t)T, &rc); if (rc) return rc;
    LevelCounts *d_cnt = sc.get<LevelCounts>(1, &rc); if (rc) return rc;
    LevelCounts c0;
    c0.n_list[0][0] = c0.n_list[0][1] = c0.n_list[1][0] = c0.n_list[1][1] = 0u;
    c0.C = (uint32_t)T; c0.levels = 0u; c0.packed_off = 0ull;
    uint32_t max_card = 0;
    {
        if ((rc = radix_sort_segments(kA, vA, kB, vB, N, F, N, hist, s)) != AIWCRF_OK) return rc;
        // the sort's histogram scratch is free again: it holds the chunk counts
        if ((rc = dense_ranks(kA, vA, N, F, hist, d_R, d_vals, d_card, s)) != AIWCRF_OK) return rc;
        prof_end(s, kProfRank);
        // the per-tree pools and the first level's counts are staged while the presort runs
        // (a copy from pageable memory costs host time, not a device wait)
        AIWCRF_CUDA(cudaMemcpyAsync(d_pool_off, h_pool_off.data(), sizeof(int64_t) * (size_t)T, cudaMemcpyHostToDevice, s));
        AIWCRF_CUDA(cudaMemcpyAsync(d_pool_len, h_pool_len.data(), sizeof(uint32_t) * (size_t)T, cudaMemcpyHostToDevice, s));
        AIWCRF_CUDA(cudaMemcpyAsync(d_rng, h_rng.data(), sizeof(uint32_t) * (size_t)T, cudaMemcpyHostToDevice, s));
        AIWCRF_CUDA(cudaMemcpyAsync(d_cnt, &c0, sizeof(LevelCounts), cudaMemcpyHostToDevice, s));
        std::vector<uint32_t> h_card((size_t)F);
        uint32_t h_err = 0;
        HostReads hr;
        hr.add(h_card.data(), d_card, sizeof(uint32_t) * (size_t)F);
        hr.add(&h_err, d_err, sizeof(uint32_t));
        if ((rc = hr.run(s)) != AIWCRF_OK) return rc;
        if ((rc = check_err_flags(h_err)) != AIWCRF_OK) return rc;
        max_card = *std::max_element(h_card.begin(), h_card.end());
    }
    const int rank_bytes = rank_bytes_for(max_card);
    const bool rank8 = rank_bytes == 1;
    void *d_Rr = sc.get<uint8_t>((size_t)F * (size_t)N * (size_t)rank_bytes, &rc);
    if (rc) return rc;
    // presorted lists for columns with many values (or when asked for): keep every column's
    // sorted row order before the grouping reuses the sort buffers
    const int gmode = grower_mode();
    const bool use_lists = gmode == AIWCRF_GROWER_LISTS || (gmode == AIWCRF_GROWER_AUTO && max_card > kListMinCard);
    uint32_t *d_ordF = nullptr;
    if (use_lists) {
        d_ordF = sc.get<uint32_t>((size_t)F * (size_t)N, &rc); if (rc) return rc;
        AIWCRF_CUDA(cudaMemcpyAsync(d_ordF, vA, sizeof(uint32_t) * (size_t)F * (size_t)N, cudaMemcpyDeviceToDevice, s));
    }

    // grouping of identical feature vectors
    uint32_t *grp_off = sc.get<uint32_t>((size_t)N + 1, &rc); if (rc) return rc;
    uint32_t n_groups = 0;
    int64_t *d_y_g = nullptr;
    uint32_t *d_grp_of = nullptr;
    uint4 *d_rowrec = nullptr;
    const uint32_t *grp_rows = vA;            // rows in group order
    {
        const unsigned rb = (unsigned)((N + 255) / 256);
        prof_begin(s, kProfRank);
        AIWCRF_BY_RANK(rank_bytes, rank_rows_kernel<RT><<<rb, 256, 0, s>>>(d_R, N, F, (RT *)d_Rr))
        AIWCRF_LAUNCH_CHECK("rank_rows_kernel");
        uint32_t *group_of_row = nullptr;
        if (AIWCRF_GROUP_HASH) {
            // the hash table (at least 2N slots), groups numbered in slot order, then a counting
            // sort of the rows by group
            int64_t n_slots = 1024;
            while (n_slots < 2 * N) n_slots *= 2;
            unsigned long long *table = sc.get<unsigned long long>((size_t)n_slots, &rc); if (rc) return rc;
            uint32_t *slot_of_row = sc.get<uint32_t>((size_t)N, &rc); if (rc) return rc;
            uint32_t *slot_flags = sc.get<uint32_t>((size_t)n_slots + 1, &rc); if (rc) return rc;
            uint32_t *slot_excl = sc.get<uint32_t>((size_t)n_slots + 1, &rc); if (rc) return rc;
            uint32_t *cnt = sc.get<uint32_t>((size_t)N + 1, &rc); if (rc) return rc;
            uint32_t *fill = sc.get<uint32_t>((size_t)N, &rc); if (rc) return rc;
            uint32_t *rows_g = sc.get<uint32_t>((size_t)N, &rc); if (rc) return rc;
            uint32_t *sblock = sc.get<uint32_t>((size_t)((std::max<int64_t>(n_slots, N) + kFlagTile - 1) / kFlagTile) + 2, &rc);
            if (rc) return rc;
            group_of_row = sc.get<uint32_t>((size_t)N, &rc); if (rc) return rc;
            AIWCRF_CUDA(cudaMemsetAsync(table, 0xFF, sizeof(unsigned long long) * (size_t)n_slots, s));
            AIWCRF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * ((size_t)N + 1), s));
            AIWCRF_CUDA(cudaMemsetAsync(fill, 0, sizeof(uint32_t) * (size_t)N, s));
            AIWCRF_BY_RANK(rank_bytes, group_insert_kernel<RT><<<rb, 256, 0, s>>>((const RT *)d_Rr, N, F, table,
                                                                                 (uint32_t)(n_slots - 1), slot_of_row, d_err))
            const unsigned sb = (unsigned)((n_slots + 255) / 256);
            slot_flags_kernel<<<sb, 256, 0, s>>>(table, n_slots, slot_flags);
            const int sblocks = (int)((n_slots + kFlagTile - 1) / kFlagTile);
            flag_scan_reduce_kernel<<<sblocks, kScanThreads, 0, s>>>(slot_flags, n_slots, sblock);
            scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(sblock, sblocks);
            flag_scan_write_kernel<<<sblocks, kScanThreads, 0, s>>>(slot_flags, n_slots, sblock, sblocks, slot_excl);
            row_group_kernel<<<rb, 256, 0, s>>>(slot_of_row, slot_excl, n_slots, N, group_of_row, cnt, d_counters + 2);
            // group offsets: the exclusive scan of the counts (past the last group it stays N)
            const int gblocks = (int)((N + kFlagTile - 1) / kFlagTile);
            flag_scan_reduce_kernel<<<gblocks, kScanThreads, 0, s>>>(cnt, N, sblock);
            scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(sblock, gblocks);
            flag_scan_write_kernel<<<gblocks, kScanThreads, 0, s>>>(cnt, N, sblock, gblocks, grp_off);
            group_scatter_kernel<<<rb, 256, 0, s>>>(group_of_row, grp_off, N, fill, rows_g);
            count_launches(9);
            AIWCRF_LAUNCH_CHECK("grouping kernels");
            grp_rows = rows_g;
        } else {
            AIWCRF_BY_RANK(rank_bytes, hash_rows_kernel<RT><<<rb, 256, 0, s>>>((const RT *)d_Rr, N, F, kA, vA))
            AIWCRF_LAUNCH_CHECK("hash_rows_kernel");
            if ((rc = radix_sort_segments(kA, vA, kB, vB, N, 1, N, hist, s)) != AIWCRF_OK) return rc;
            // group starts (flags in kB), their exclusive scan (in vB), offsets
            AIWCRF_BY_RANK(rank_bytes, group_flags_kernel<RT><<<rb, 256, 0, s>>>((const RT *)d_Rr, N, F, kA, vA, kB))
            const int gblocks = (int)((N + kFlagTile - 1) / kFlagTile);
            flag_scan_reduce_kernel<<<gblocks, kScanThreads, 0, s>>>(kB, N, hist);
            scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(hist, gblocks);
            flag_scan_write_kernel<<<gblocks, kScanThreads, 0, s>>>(kB, N, hist, gblocks, vB);
            group_offsets_kernel<<<rb, 256, 0, s>>>(kB, vB, N, grp_off, d_counters + 2);
            count_launches(4);
            AIWCRF_LAUNCH_CHECK("grouping kernels");
        }
        prof_end(s, kProfRank);
        // y in group order, every position's group and every row's {y, group} record (for the
        // bootstrap), enqueued before the group count is read
        d_y_g = sc.get<int64_t>((size_t)N, &rc); if (rc) return rc;
        d_grp_of = sc.get<uint32_t>((size_t)N, &rc); if (rc) return rc;
        if (AIWCRF_BOOT_GROUPS && p.bootstrap) { d_rowrec = sc.get<uint4>((size_t)N, &rc); if (rc) return rc; }
        if (group_of_row)
            group_order_rows_kernel<<<rb, 256, 0, s>>>(grp_rows, group_of_row, dy, N, d_y_g, d_grp_of, d_rowrec);
        else
            group_order_kernel<<<rb, 256, 0, s>>>(vA, kB, vB, dy, N, d_y_g, d_grp_of, d_rowrec);
        AIWCRF_LAUNCH_CHECK("group_order_kernel");
        HostReads hr;
        hr.add(&n_groups, d_counters + 2, sizeof(uint32_t));
        if ((rc = hr.run(s)) != AIWCRF_OK) return rc;
    }
    // the groups' representative rows in every column's order
    uint32_t *d_ordG = nullptr;
    if (use_lists) {
        uint8_t *is_rep = sc.get<uint8_t>((size_t)N, &rc); if (rc) return rc;
        d_ordG = sc.get<uint32_t>((size_t)F * (size_t)n_groups, &rc); if (rc) return rc;
        AIWCRF_CUDA(cudaMemsetAsync(is_rep, 0, (size_t)N, s));
        rep_mark_kernel<<<(unsigned)((n_groups + 255) / 256), 256, 0, s>>>(grp_rows, grp_off, n_groups, is_rep);
        rep_order_kernel<<<(unsigned)F, 1024, 0, s>>>(d_ordF, N, is_rep, n_groups, d_ordG);
        count_launches(1);
        AIWCRF_LAUNCH_CHECK("rep_mark / rep_order");
        sc.drop(is_rep);
        sc.drop(d_ordF);
    }
    // the bootstrap sums its draws per group in shared memory when the groups' sums and the
    // in-bag bitmap fit there (it then reads one {y, group} record per drawn row)
    const int64_t boot_inbag_words = d_sub_rows ? 0 : (N + 31) / 32;
    const bool boot_groups = d_rowrec && boot_groups_smem(n_groups, boot_inbag_words) <= (size_t)kBootGroupsSmemMax;
    sc.drop(d_R); sc.drop(kA); sc.drop(kB); sc.drop(vB); sc.drop(hist);
    row_cap = std::min<int64_t>(row_cap, (int64_t)n_groups);

    // Tree-resident growth when every tree's entries fit in shared memory: one-byte ranks,
    // F <= 32, group ids and entry offsets in 16 bits
    const int tree_bins = (int)std::max<uint32_t>(max_card, 1u);
    const int tree_ecap = (int)std::max<int64_t>(row_cap, 1);
    const int tree_big_cap = tree_ecap / (kSmallNodeRows + 1) + 1;
    const size_t tree_smem = tree_smem_bytes(tree_ecap, tree_bins, tree_big_cap);
    const bool tree_fits = rank8 && F <= 32 && n_groups <= 65535u && row_cap <= 65535 &&
                           tree_smem + 1024 <= (size_t)max_smem_optin;
    if (gmode == AIWCRF_GROWER_TREE && !tree_fits)
        return fail(AIWCRF_E_LIMIT, "tree-resident growth needs one-byte ranks, F <= 32 and a tree's entries in shared memory");
    const bool use_tree = tree_fits && !use_lists && gmode != AIWCRF_GROWER_LEVEL;

    // a2: bootstrap (what it needs is allocated first; the growth's scratch is allocated while
    // it runs)
    Entry *rows_a = sc.get<Entry>((size_t)T * (size_t)row_cap, &rc); if (rc) return rc;
    Entry *rows_b = nullptr;               // the level loop's second entry buffer
    if (!use_tree) { rows_b = sc.get<Entry>((size_t)T * (size_t)row_cap, &rc); if (rc) return rc; }

    // Level-loop capacities. A depth holds at most C_max = T * row_cap nodes (each holds an
    // entry) and a tree at most 2 * row_cap - 1 nodes. Depths are enqueued in chunks without
    // waiting; after each chunk the host reads the node count and grows the buffers so that
    // they hold the next chunk whatever its growth (at most doubling per depth).
    const int64_t C_max = T * row_cap;
    const int64_t nodes_max = T * (2 * row_cap - 1);
    const size_t per_node_bytes = 2 * sizeof(NodeRec) + sizeof(SplitRes) + 4 * sizeof(int32_t) + 8;
    const size_t budget = (size_t)4 << 30;                      // level-table budget per fit
    int dev_sms = 0;
    AIWCRF_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, device));

    size_t node_cap = 0, packed_cap = 0;
    NodeRec *nodes_cur = nullptr, *nodes_nxt = nullptr;
    SplitRes *res = nullptr;
    uint32_t *excl = nullptr, *block_sums = nullptr;
    int32_t *small_a = nullptr, *big_a = nullptr;
    PackedRec *packed = nullptr;
    // (re)allocate the per-depth tables for up to cap nodes per depth; the current depth's
    // nodes and lists are carried over
    auto grow_tables = [&](size_t cap, uint32_t carry_nodes) -> int {
        if (cap <= node_cap) return AIWCRF_OK;
        int rc2 = AIWCRF_OK;
        NodeRec *nc = sc.get<NodeRec>(cap, &rc2); if (rc2) return rc2;
        NodeRec *nn = sc.get<NodeRec>(2 * cap, &rc2); if (rc2) return rc2;
        SplitRes *nr = sc.get<SplitRes>(cap, &rc2); if (rc2) return rc2;
        uint32_t *ne = sc.get<uint32_t>(cap + 1, &rc2); if (rc2) return rc2;
        uint32_t *nbs = sc.get<uint32_t>(cap / kScanTile + 2, &rc2); if (rc2) return rc2;
        int32_t *ns = sc.get<int32_t>(2 * cap, &rc2); if (rc2) return rc2;
        int32_t *nb = sc.get<int32_t>(2 * cap, &rc2); if (rc2) return rc2;
        if (nodes_cur) {
            cudaError_t e1 = cudaMemcpyAsync(nc, nodes_cur, sizeof(NodeRec) * carry_nodes, cudaMemcpyDeviceToDevice, s);
            if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(ns, small_a, sizeof(int32_t) * carry_nodes, cudaMemcpyDeviceToDevice, s);
            if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(nb, big_a, sizeof(int32_t) * carry_nodes, cudaMemcpyDeviceToDevice, s);
            if (e1 != cudaSuccess) return cuda_fail(e1, "growing level tables");
            sc.drop(nodes_cur); sc.drop(nodes_nxt); sc.drop(res); sc.drop(excl); sc.drop(block_sums);
            sc.drop(small_a); sc.drop(big_a);
        }
        nodes_cur = nc; nodes_nxt = nn; res = nr; excl = ne; block_sums = nbs; small_a = ns; big_a = nb;
        node_cap = cap;
        // the level kernels count splits per tile into block_sums: zero before the next depth
        const cudaError_t e2 = cudaMemsetAsync(nbs, 0, sizeof(uint32_t) * (cap / kScanTile + 2), s);
        if (e2 != cudaSuccess) return cuda_fail(e2, "growing level tables");
        return AIWCRF_OK;
    };
    if (use_tree) {
        // the tree-resident grower reads only the roots and the bootstrap's list counts
        nodes_cur = sc.get<NodeRec>((size_t)T, &rc); if (rc) return rc;
        small_a = sc.get<int32_t>((size_t)T, &rc); if (rc) return rc;
        big_a = sc.get<int32_t>((size_t)T, &rc); if (rc) return rc;
        node_cap = (size_t)T;
    } else if ((rc = grow_tables((size_t)std::max<int64_t>(T, 1024), 0)) != AIWCRF_OK) {
        return rc;
    }
    auto grow_packed = [&](size_t need, size_t keep) -> int {
        if (need <= packed_cap) return AIWCRF_OK;
        int rc2 = AIWCRF_OK;
        const size_t ncap = std::max(need, packed_cap * 2);
        PackedRec *np = sc.get<PackedRec>(ncap, &rc2); if (rc2) return rc2;
        if (packed && keep) {
            cudaError_t e1 = cudaMemcpyAsync(np, packed, sizeof(PackedRec) * keep, cudaMemcpyDeviceToDevice, s);
            if (e1 != cudaSuccess) return cuda_fail(e1, "growing node records");
        }
        if (packed) sc.drop(packed);
        packed = np;
        packed_cap = ncap;
        return AIWCRF_OK;
    };

    // in-bag bitmaps (forests fitted on all rows keep them for out-of-bag evaluation)
    const int64_t inbag_words = (N + 31) / 32;
    uint32_t *d_inbag = nullptr;
    if (!d_sub_rows) {
        d_inbag = sc.get<uint32_t>((size_t)T * (size_t)inbag_words, &rc); if (rc) return rc;
    }


    {
        const int boot_smem_words = std::min<int>((max_smem_optin - 2048) / 4, 56 * 1024);
        const uint32_t words = (uint32_t)((N + 3) / 4);
        uint32_t *gcnt = nullptr;
        int64_t gstride = 0;
        if (!boot_groups && (int)words > boot_smem_words) {
            gstride = words;
            gcnt = sc.get<uint32_t>((size_t)T * (size_t)words, &rc); if (rc) return rc;
        }
        // the group-ordered pass (counters in shared memory, per-group sums in a global scratch)
        const bool grouped = !gcnt && !boot_groups;
        unsigned long long *d_gsum = nullptr;
        if (grouped) { d_gsum = sc.get<unsigned long long>((size_t)T * 2 * (size_t)n_groups, &rc); if (rc) return rc; }
        const int smem_bytes = (gcnt || boot_groups) ? 0 : (int)words * 4;
        AIWCRF_CUDA(cudaFuncSetAttribute(bootstrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         std::max(smem_bytes, 1)));
        BootArgs ba;
        ba.tree_pool_off = d_pool_off; ba.tree_pool_len = d_pool_len; ba.tree_rng = d_rng;
        ba.sub_rows = d_sub_rows; ba.y = dy; ba.N = N; ba.grp_off = grp_off; ba.grp_rows = grp_rows; ba.G = n_groups;
        ba.seed_lo = (uint32_t)p.seed; ba.seed_hi = (uint32_t)(p.seed >> 32);
        ba.bootstrap = p.bootstrap; ba.gcnt = gcnt; ba.gcnt_stride = gstride;
        ba.smem_words = gcnt ? 0 : (int)words;
        ba.rows_out = rows_a; ba.row_cap = row_cap; ba.root = nodes_cur;
        ba.small_list = small_a; ba.big_list = big_a; ba.counters = d_cnt->n_list[0]; ba.err = d_err;
        ba.inbag = d_inbag; ba.inbag_words = inbag_words;
        ba.G_ptr = nullptr;
        ba.store_group = use_tree ? 1 : 0;
        ba.y_g = grouped ? d_y_g : nullptr;
        ba.grp_of = grouped ? d_grp_of : nullptr;
        ba.gsum = d_gsum;
        prof_begin(s, kProfBoot);
        if (boot_groups) {
            const size_t gsmem = boot_groups_smem(n_groups, boot_inbag_words);
            AIWCRF_CUDA(cudaFuncSetAttribute(boot_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             std::max((int)gsmem, 1)));
            boot_groups_kernel<<<(unsigned)T, kBootGThreads, gsmem, s>>>(ba, d_rowrec);
            AIWCRF_LAUNCH_CHECK("boot_groups_kernel");
        } else {
            bootstrap_kernel<<<(unsigned)T, kBootThreads, smem_bytes, s>>>(ba);
            AIWCRF_LAUNCH_CHECK("bootstrap_kernel");
        }
        prof_end(s, kProfBoot);
    }
    uint8_t *d_Rg = nullptr, *d_RgT = nullptr;
    if (use_tree) {
        d_Rg = sc.get<uint8_t>((size_t)n_groups * kRecBytes, &rc); if (rc) return rc;
        d_RgT = sc.get<uint8_t>((size_t)n_groups * (size_t)F, &rc); if (rc) return rc;
        const int64_t cells = (int64_t)n_groups * kRecBytes;
        group_records_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>((const uint8_t *)d_Rr, F, grp_off, grp_rows,
                                                                           d_counters + 2, d_Rg, d_RgT);
        AIWCRF_LAUNCH_CHECK("group_records_kernel");
    }

    // presorted lists of every tree: its entries by representative row, then per feature in rank order
    const int64_t list_stride = T * row_cap;
    uint32_t *lists_a = nullptr, *lists_b = nullptr, *newpos = nullptr;
    if (use_lists) {
        uint32_t *P = sc.get<uint32_t>((size_t)T * (size_t)N, &rc); if (rc) return rc;
        lists_a = sc.get<uint32_t>((size_t)F * (size_t)list_stride, &rc); if (rc) return rc;
        lists_b = sc.get<uint32_t>((size_t)F * (size_t)list_stride, &rc); if (rc) return rc;
        newpos = sc.get<uint32_t>((size_t)list_stride, &rc); if (rc) return rc;
        prof_begin(s, kProfBoot);
        AIWCRF_CUDA(cudaMemsetAsync(P, 0, sizeof(uint32_t) * (size_t)T * (size_t)N, s));
        list_pos_kernel<<<dim3((unsigned)((row_cap + 255) / 256), (unsigned)T), 256, 0, s>>>(rows_a, row_cap, nodes_cur, N, P);
        AIWCRF_LAUNCH_CHECK("list_pos_kernel");
        list_build_kernel<<<dim3((unsigned)T, (unsigned)F), 1024, 0, s>>>(d_ordG, n_groups, P, N, row_cap, list_stride,
                                                                         lists_a);
        AIWCRF_LAUNCH_CHECK("list_build_kernel");
        prof_end(s, kProfBoot);
        sc.drop(d_ordG);
        sc.drop(P);
    }

    if (use_tree) {
        // one CTA per tree at a time, as many as fit (a background fit: at most ctas_per_sm per SM)
        AIWCRF_CUDA(cudaFuncSetAttribute(tree_grow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tree_smem));
        // shared memory over L1: the occupancy (and one wave of trees) depends on it
        AIWCRF_CUDA(cudaFuncSetAttribute(tree_grow_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared));
        int occ = 0;
        AIWCRF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tree_grow_kernel, kTreeThreads, tree_smem));
        if (occ < 1) return fail(AIWCRF_E_LIMIT, "tree-resident growth: no CTA fits on an SM");
        if (p.ctas_per_sm > 0) occ = std::min<int>(occ, p.ctas_per_sm);
        const int64_t grid = std::min<int64_t>(T, (int64_t)occ * dev_sms);
        const int64_t node_cap = 2 * (int64_t)tree_ecap;
        TNode *t_nodes = sc.get<TNode>((size_t)grid * 2 * (size_t)tree_ecap, &rc); if (rc) return rc;
        SplitRes *t_res = sc.get<SplitRes>((size_t)grid * (size_t)tree_ecap, &rc); if (rc) return rc;
        Cand *t_cands = sc.get<Cand>((size_t)grid * (size_t)tree_big_cap * 32, &rc); if (rc) return rc;
        uint64_t *slot_nodes = sc.get<uint64_t>((size_t)T * (size_t)node_cap, &rc); if (rc) return rc;
        uint64_t *slot_cnodes = sc.get<uint64_t>((size_t)T * (size_t)node_cap, &rc); if (rc) return rc;
        uint32_t *counts = sc.get<uint32_t>((size_t)T + 1, &rc); if (rc) return rc;
        uint32_t *levels = counts + T;
        AIWCRF_CUDA(cudaMemsetAsync(levels, 0, sizeof(uint32_t), s));
        TreeArgs ta;
        ta.rows = rows_a; ta.root = nodes_cur; ta.row_cap = row_cap; ta.Rg = d_Rg; ta.RgT = d_RgT; ta.vals = d_vals; ta.N = N;
        ta.card = d_card; ta.tree_rng = d_rng; ta.n_groups = n_groups; ta.T = (int)T; ta.F = F; ta.mtry = p.mtry;
        ta.min_node = p.min_node_size; ta.max_depth = p.max_depth;
        ta.seed_lo = (uint32_t)p.seed; ta.seed_hi = (uint32_t)(p.seed >> 32);
        ta.ecap = tree_ecap; ta.bins = tree_bins; ta.big_cap = tree_big_cap;
        ta.nodes = t_nodes; ta.res = t_res; ta.cands = t_cands;
        ta.out_nodes = slot_nodes; ta.out_cnodes = slot_cnodes; ta.node_cap = node_cap; ta.out_count = counts;
        ta.stats = d_stats; ta.levels = levels;
        prof_begin(s, kProfTree);
        tree_grow_kernel<<<(unsigned)grid, kTreeThreads, tree_smem, s>>>(ta);
        AIWCRF_LAUNCH_CHECK("tree_grow_kernel");
        prof_end(s, kProfTree);
        // the error flags are read with the tree sizes (one wait instead of two)
        PackIn pin;
        pin.p = &p; pin.T = T; pin.Tper = Tper; pin.G = G; pin.N = N; pin.F = F; pin.device = device;
        pin.tree_base = counts; pin.d_stats = d_stats; pin.packed = nullptr; pin.packed_n = 0;
        pin.levels = 0; pin.d_inbag = d_inbag; pin.inbag_words = inbag_words;
        pin.d_vals = d_vals; pin.d_card = d_card; pin.max_card = max_card; pin.rank_bytes = rank_bytes; pin.n_groups = n_groups;
        pin.slot_nodes = slot_nodes; pin.slot_cnodes = slot_cnodes; pin.slot_cap = node_cap; pin.d_levels = levels;
        pin.grower = AIWCRF_GROWER_TREE;
        pin.d_err = d_err;
        rc = package_forests(pin, s, out);
        sc.release();
        if (rc == AIWCRF_OK) AIWCRF_CUDA(cudaStreamSynchronize(s));
        return rc;
    }

    // per-tree level bookkeeping
    uint32_t *tree_off = sc.get<uint32_t>((size_t)T + 1, &rc); if (rc) return rc;
    uint32_t *tree_off_nxt = sc.get<uint32_t>((size_t)T + 1, &rc); if (rc) return rc;
    uint32_t *tree_base = sc.get<uint32_t>((size_t)T, &rc); if (rc) return rc;
    uint32_t *d_done = sc.get<uint32_t>(1, &rc); if (rc) return rc;
    iota_kernel<<<(unsigned)((T + 256) / 256), 256, 0, s>>>(tree_off, (int)T);
    AIWCRF_LAUNCH_CHECK("iota_kernel");
    AIWCRF_CUDA(cudaMemsetAsync(tree_base, 0, sizeof(uint32_t) * (size_t)T, s));
    AIWCRF_CUDA(cudaMemsetAsync(d_done, 0, sizeof(uint32_t), s));

    LevelCounts *h_cnt = static_cast<LevelCounts *>(pinned_scratch());
    if (!h_cnt) return fail(AIWCRF_E_OOM, "pinned host buffer");
    uint32_t *h_err = reinterpret_cast<uint32_t *>(h_cnt + 1);

    // bins: the tried features' value counts side by side (one pass over the entries)
    const int bin_cap = big_bin_cap(p.mtry, F, max_card);
    const int big_smem = bin_cap * 14;
    {
        cudaError_t e_ = cudaSuccess;
        AIWCRF_BY_RANK(rank_bytes, e_ = cudaFuncSetAttribute(level_big_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                             big_smem))
        if (e_ != cudaSuccess) return cuda_fail(e_, "level_big_kernel attribute");
        if (use_lists) {
            AIWCRF_BY_RANK(rank_bytes, e_ = cudaFuncSetAttribute(level_list_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                 list_stage_bytes<kListThreads / 32>()))
            if (e_ != cudaSuccess) return cuda_fail(e_, "level_list_kernel attribute");
        }
    }

    LevelArgs la;
    la.row_cap = row_cap; la.Rr = d_Rr; la.vals = d_vals; la.card = d_card; la.N = N;
    la.tree_rng = d_rng; la.F = F; la.mtry = p.mtry; la.min_node = p.min_node_size;
    la.max_depth = p.max_depth; la.seed_lo = (uint32_t)p.seed; la.seed_hi = (uint32_t)(p.seed >> 32);
    la.depth_ptr = nullptr;
    la.node_cap = 0;
    la.list_stride = list_stride; la.newpos = newpos;

    // The two level kernels of a depth are independent (disjoint nodes, disjoint entry
    // segments): a foreground fit runs the small-node kernel on a second stream of the same
    // priority, forked after the previous depth's finalize and joined before the scan, so that
    // either kernel's tail overlaps the other's work. (A background fit stays on one stream.)
    struct Fork {
        cudaStream_t side = nullptr;
        cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
        ~Fork()
        {
            if (ev_fork) cudaEventDestroy(ev_fork);
            if (ev_join) cudaEventDestroy(ev_join);
            if (side) cudaStreamDestroy(side);
        }
    } fk;
    const bool fork = p.ctas_per_sm == 0;
    if (fork) {
        int prio = 0;
        AIWCRF_CUDA(cudaStreamGetPriority(s, &prio));
        AIWCRF_CUDA(cudaStreamCreateWithPriority(&fk.side, cudaStreamNonBlocking, prio));
        AIWCRF_CUDA(cudaEventCreateWithFlags(&fk.ev_fork, cudaEventDisableTiming));
        AIWCRF_CUDA(cudaEventCreateWithFlags(&fk.ev_join, cudaEventDisableTiming));
    }
    cudaStream_t s_small = fork ? fk.side : s;

    Entry *rin = rows_a, *rout = rows_b;
    uint32_t *lin = lists_a, *lout = lists_b;
    int depth = 0;
    int64_t C_known = T;                 // node count at the start of the next chunk (exact)
    uint64_t packed_known = 0;           // finished nodes before it (exact)
    while (C_known > 0) {
        // largest chunk whose bound fits the budget; a background fit enqueues one level at a
        // time, so that work of other streams sharing a hardware queue with it waits at most
        // one level behind it
        int chunk = p.ctas_per_sm > 0 ? 1 : kLevelChunk;
        auto bound = [&](int k) { return std::min<int64_t>(C_known << k, C_max); };
        while (chunk > 1 && (size_t)bound(chunk) * per_node_bytes > budget) chunk >>= 1;
        if ((rc = grow_tables((size_t)bound(chunk), (uint32_t)C_known)) != AIWCRF_OK) return rc;
        int64_t packed_need = (int64_t)packed_known;
        for (int k = 0; k < chunk; ++k) packed_need += bound(k);
        packed_need = std::min<int64_t>(packed_need, nodes_max + T);
        if ((rc = grow_packed((size_t)packed_need, (size_t)packed_known)) != AIWCRF_OK) return rc;

        for (int k = 0; k < chunk; ++k, ++depth) {
            const int64_t Cb = bound(k);                        // bound on this depth's nodes
            la.nodes = nodes_cur; la.rows_in = rin; la.rows_out = rout; la.depth = depth; la.res = res;
            la.tile_splits = block_sums; la.node_cap = (uint32_t)node_cap;
            la.lists_in = lin; la.lists_out = lout;
            if (fork) {
                AIWCRF_CUDA(cudaEventRecord(fk.ev_fork, s));
                AIWCRF_CUDA(cudaStreamWaitEvent(fk.side, fk.ev_fork, 0));
            }
            {
                la.list = big_a; la.list_n = &d_cnt->n_list[depth & 1][1];
                const int64_t cps_big = p.ctas_per_sm > 0 ? p.ctas_per_sm : kBigCtasPerSm;
                const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(Cb, cps_big * dev_sms));
                prof_begin(s, kProfLevelBig);
                if (use_lists) {
                    const int64_t cps_list = p.ctas_per_sm > 0 ? p.ctas_per_sm : kListCtasPerSm;
                    const unsigned lgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(Cb, cps_list * dev_sms));
                    AIWCRF_BY_RANK(rank_bytes, level_list_kernel<RT><<<lgrid, kListThreads, list_stage_bytes<kListThreads / 32>(), s>>>(la))
                    AIWCRF_LAUNCH_CHECK("level_list_kernel");
                    prof_end(s, kProfLevelBig);
                    prof_begin(s, kProfListPart);
                    const int64_t cps_part = p.ctas_per_sm > 0 ? p.ctas_per_sm : kPartCtasPerSm;
                    const unsigned pgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(Cb, cps_part * dev_sms));
                    list_partition_kernel<<<pgrid, kPartThreads, 0, s>>>(la);
                    AIWCRF_LAUNCH_CHECK("list_partition_kernel");
                    prof_end(s, kProfListPart);
                } else {
                    AIWCRF_BY_RANK(rank_bytes, level_big_kernel<RT><<<grid, kBigThreads, big_smem, s>>>(la, bin_cap))
                    AIWCRF_LAUNCH_CHECK("level_big_kernel");
                    prof_end(s, kProfLevelBig);
                }
            }
            {
                la.list = small_a; la.list_n = &d_cnt->n_list[depth & 1][0];
                const int64_t wpb = kSmallThreads / 32;
                const int64_t cps_small = p.ctas_per_sm > 0 ? p.ctas_per_sm : kSmallCtasPerSm;
                const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Cb + wpb - 1) / wpb, cps_small * dev_sms));
                prof_begin(s_small, kProfLevelSmall);
                AIWCRF_BY_RANK(rank_bytes, level_small_kernel<RT><<<grid, kSmallThreads, 0, s_small>>>(la))
                AIWCRF_LAUNCH_CHECK("level_small_kernel");
                prof_end(s_small, kProfLevelSmall);
            }
            if (fork) {
                AIWCRF_CUDA(cudaEventRecord(fk.ev_join, fk.side));
                AIWCRF_CUDA(cudaStreamWaitEvent(s, fk.ev_join, 0));
            }
            FinalArgs fa;
            fa.nodes = nodes_cur; fa.res = res; fa.excl_out = excl; fa.tree_off = tree_off; fa.tree_base = tree_base;
            fa.cnt = d_cnt; fa.next = nodes_nxt; fa.small_list = small_a; fa.big_list = big_a;
            fa.packed = packed; fa.stats = d_stats;
            fa.next_tree_off = tree_off_nxt; fa.T = (int)T; fa.done = d_done; fa.tile_splits = block_sums;
            fa.parity = depth & 1; fa.next_cap = (uint32_t)(2 * node_cap); fa.vals = d_vals; fa.N = N;
            // tiles of the depth's (bounded) node count, at most four (256-thread) CTAs per SM
            const unsigned fgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Cb + kScanTile - 1) / kScanTile, 4 * (int64_t)dev_sms));
            prof_begin(s, kProfFinalize);
            finalize_kernel<<<fgrid, kFinThreads, 0, s>>>(fa);
            AIWCRF_LAUNCH_CHECK("finalize_kernel");
            prof_end(s, kProfFinalize);

            std::swap(nodes_cur, nodes_nxt);
            std::swap(rin, rout);
            std::swap(lin, lout);
            std::swap(tree_off, tree_off_nxt);
        }
        AIWCRF_CUDA(cudaMemcpyAsync(h_cnt, d_cnt, sizeof(LevelCounts), cudaMemcpyDeviceToHost, s));
        AIWCRF_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        AIWCRF_CUDA(cudaStreamSynchronize(s));
        if ((rc = check_err_flags(*h_err)) != AIWCRF_OK) return rc;
        C_known = h_cnt->C;
        packed_known = h_cnt->packed_off;
    }
    PackIn pin;
    pin.p = &p; pin.T = T; pin.Tper = Tper; pin.G = G; pin.N = N; pin.F = F; pin.device = device;
    pin.tree_base = tree_base; pin.d_stats = d_stats; pin.packed = packed; pin.packed_n = (size_t)packed_known;
    pin.levels = (int)h_cnt->levels; pin.d_inbag = d_inbag; pin.inbag_words = inbag_words;
    pin.d_vals = d_vals; pin.d_card = d_card; pin.max_card = max_card; pin.rank_bytes = rank_bytes; pin.n_groups = n_groups;
    pin.grower = use_lists ? AIWCRF_GROWER_LISTS : AIWCRF_GROWER_LEVEL;
    rc = package_forests(pin, s, out);
    sc.release();
    if (rc == AIWCRF_OK) AIWCRF_CUDA(cudaStreamSynchronize(s));
    return rc;
}


// ------------------------------------------------------------------------------------------
// Fit plan: the whole fit as one CUDA graph. The presort, ranks and groups, the bootstrap and a
// device-side WHILE loop whose body grows two tree levels (even and odd halves of the ping-pong
// buffers) and then lets a one-thread kernel decide, from the device's node count, whether the
// loop continues. No host synchronisation happens between the first kernel and the last level;
// the host then reads the counts and packs the forests. Sizes the graph cannot learn without
// the host (one- or two-byte ranks, the number of groups) are taken from a probe of the data at
// creation; a replay on data that outgrows them sets kErrCapacity instead of writing out of
// bounds, and the tables are sized for the worst case of that capacity.
// ------------------------------------------------------------------------------------------
// the plan's value tables (and one-byte ranks) hold max_card values per column
__global__ void plan_check_kernel(const uint32_t *card, int F, uint32_t max_card, uint32_t *err)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F && card[f] > max_card) atomicOr(err, kErrCapacity);
}

__global__ void level_counts_init_kernel(LevelCounts *cnt, uint32_t T)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        cnt->n_list[0][0] = cnt->n_list[0][1] = cnt->n_list[1][0] = cnt->n_list[1][1] = 0u;
        cnt->C = T; cnt->levels = 0u; cnt->packed_off = 0ull;
    }
}

__global__ void level_loop_cond_kernel(cudaGraphConditionalHandle h, const LevelCounts *cnt, uint32_t limit,
                                       uint32_t *err)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool more = cnt->C > 0u;
    if (more && cnt->levels >= limit) atomicOr(err, kErrCapacity);
    if (!more || cnt->levels >= limit) cudaGraphSetConditional(h, 0u);
}

struct FitPlan {
    aiwcrf_fit_params p{};
    const float *dX = nullptr;
    const int64_t *dy = nullptr;
    int64_t N = 0;
    int32_t F = 0, G = 1;
    std::vector<int64_t> sub_off;
    const int32_t *d_sub_rows = nullptr;
    int device = 0, sms = 0;
    int64_t T = 0, Tper = 0, row_cap = 0, C_max = 0, packed_cap = 0, inbag_words = 0;
    int rank_bytes = 1;
    uint32_t max_card = 0, probe_groups = 0;
    int boot_smem = 0;
    int64_t gstride = 0;
    std::vector<void *> bufs;
    // device buffers
    uint32_t *d_err = nullptr, *d_counters = nullptr, *d_card = nullptr;
    GrowStats *d_stats = nullptr;
    uint32_t *d_R = nullptr;
    float *d_vals = nullptr;
    uint32_t *kA = nullptr, *vA = nullptr, *kB = nullptr, *vB = nullptr, *hist = nullptr;
    void *d_Rr = nullptr;
    uint32_t *grp_off = nullptr;
    int64_t *d_pool_off = nullptr;
    uint32_t *d_pool_len = nullptr, *d_rng = nullptr;
    Entry *rows_a = nullptr, *rows_b = nullptr;
    NodeRec *nodes_a = nullptr, *nodes_b = nullptr;
    SplitRes *res = nullptr;
    uint32_t *excl = nullptr, *block_sums = nullptr;
    int32_t *small_l = nullptr, *big_l = nullptr;
    PackedRec *packed = nullptr;
    LevelCounts *d_cnt = nullptr;
    uint32_t *d_inbag = nullptr, *gcnt = nullptr;
    uint32_t *toff_a = nullptr, *toff_b = nullptr, *tree_base = nullptr, *d_done = nullptr;
    // schedule and graph
    int cps_big = kBigCtasPerSm, cps_small = kSmallCtasPerSm;
    cudaGraphExec_t exec = nullptr;
    int64_t prefix_launches = 0, body_launches = 0;

    // buffers come from the stream-ordered pool: freeing them never waits for the whole
    // device (a selection server may be busy on other streams)
    template <class U>
    int alloc(U **ptr, size_t count)
    {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(U), cudaStreamPerThread);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
        if (e != cudaSuccess)
            return fail(AIWCRF_E_OOM, std::string("fit plan: device allocation of ") +
                                          std::to_string(count * sizeof(U)) + " bytes failed");
        bufs.push_back(q);
        *ptr = static_cast<U *>(q);
        return AIWCRF_OK;
    }
    ~FitPlan()
    {
        // a run returns only after its work has finished, so nothing reads these any more
        if (exec) cudaGraphExecDestroy(exec);
        for (auto b : bufs) cudaFreeAsync(b, cudaStreamPerThread);
        cudaStreamSynchronize(cudaStreamPerThread);
    }
};

namespace {

// phase A (presort, ranks, groups) on s; with `probe` the host reads back what sizes the rest
int plan_phase_a(FitPlan &P, cudaStream_t s, bool probe)
{
    const int64_t N = P.N;
    const int32_t F = P.F;
    const unsigned yblocks = (unsigned)((N + 255) / 256);
    AIWCRF_CUDA(cudaMemsetAsync(P.d_err, 0, sizeof(uint32_t), s));
    AIWCRF_CUDA(cudaMemsetAsync(P.d_stats, 0, sizeof(GrowStats), s));
    AIWCRF_CUDA(cudaMemsetAsync(P.d_counters, 0, 4 * sizeof(uint32_t), s));
    check_y_kernel<<<yblocks, 256, 0, s>>>(P.dy, N, P.d_err);
    AIWCRF_LAUNCH_CHECK("check_y_kernel");
    key_init_kernel<<<dim3(yblocks, (unsigned)F), 256, 0, s>>>(P.dX, N, P.kA, P.vA, P.d_err);
    AIWCRF_LAUNCH_CHECK("key_init_kernel");
    int rc;
    if ((rc = radix_sort_segments(P.kA, P.vA, P.kB, P.vB, N, F, N, P.hist, s)) != AIWCRF_OK) return rc;
    if ((rc = dense_ranks(P.kA, P.vA, N, F, P.hist, P.d_R, P.d_vals, P.d_card, s)) != AIWCRF_OK) return rc;
    if (probe) {
        std::vector<uint32_t> h_card((size_t)F);
        uint32_t h_err = 0;
        AIWCRF_CUDA(cudaMemcpyAsync(h_card.data(), P.d_card, sizeof(uint32_t) * (size_t)F, cudaMemcpyDeviceToHost, s));
        AIWCRF_CUDA(cudaMemcpyAsync(&h_err, P.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        AIWCRF_CUDA(cudaStreamSynchronize(s));
        if ((rc = check_err_flags(h_err)) != AIWCRF_OK) return rc;
        P.max_card = *std::max_element(h_card.begin(), h_card.end());
        P.rank_bytes = rank_bytes_for(P.max_card);
        if ((rc = P.alloc(reinterpret_cast<uint8_t **>(&P.d_Rr), (size_t)F * (size_t)N * (size_t)P.rank_bytes))) return rc;
    } else {
        plan_check_kernel<<<(unsigned)((F + 127) / 128), 128, 0, s>>>(P.d_card, F, P.max_card, P.d_err);
        AIWCRF_LAUNCH_CHECK("plan_check_kernel");
    }
    const unsigned rb = (unsigned)((N + 255) / 256);
    AIWCRF_BY_RANK(P.rank_bytes, rank_rows_kernel<RT><<<rb, 256, 0, s>>>(P.d_R, N, F, (RT *)P.d_Rr);
                                 hash_rows_kernel<RT><<<rb, 256, 0, s>>>((const RT *)P.d_Rr, N, F, P.kA, P.vA))
    count_launches(1);
    AIWCRF_LAUNCH_CHECK("rank_rows / hash_rows");
    if ((rc = radix_sort_segments(P.kA, P.vA, P.kB, P.vB, N, 1, N, P.hist, s)) != AIWCRF_OK) return rc;
    AIWCRF_BY_RANK(P.rank_bytes, group_flags_kernel<RT><<<rb, 256, 0, s>>>((const RT *)P.d_Rr, N, F, P.kA, P.vA, P.kB))
    const int gblocks = (int)((N + kFlagTile - 1) / kFlagTile);
    flag_scan_reduce_kernel<<<gblocks, kScanThreads, 0, s>>>(P.kB, N, P.hist);
    scan_blocks_kernel<<<1, kScanThreads, 0, s>>>(P.hist, gblocks);
    flag_scan_write_kernel<<<gblocks, kScanThreads, 0, s>>>(P.kB, N, P.hist, gblocks, P.vB);
    group_offsets_kernel<<<rb, 256, 0, s>>>(P.kB, P.vB, N, P.grp_off, P.d_counters + 2);
    count_launches(4);
    AIWCRF_LAUNCH_CHECK("grouping kernels");
    if (probe) {
        AIWCRF_CUDA(cudaMemcpyAsync(&P.probe_groups, P.d_counters + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        AIWCRF_CUDA(cudaStreamSynchronize(s));
    }
    return AIWCRF_OK;
}

// the bootstrap and the per-tree bookkeeping (captured)
int plan_bootstrap(FitPlan &P, cudaStream_t s)
{
    level_counts_init_kernel<<<1, 32, 0, s>>>(P.d_cnt, (uint32_t)P.T);
    AIWCRF_LAUNCH_CHECK("level_counts_init_kernel");
    AIWCRF_CUDA(cudaMemsetAsync(P.block_sums, 0, sizeof(uint32_t) * ((size_t)P.C_max / kScanTile + 2), s));
    BootArgs ba;
    ba.tree_pool_off = P.d_pool_off; ba.tree_pool_len = P.d_pool_len; ba.tree_rng = P.d_rng;
    ba.sub_rows = P.d_sub_rows; ba.y = P.dy; ba.N = P.N; ba.grp_off = P.grp_off; ba.grp_rows = P.vA;
    ba.G = 0u; ba.G_ptr = P.d_counters + 2;
    ba.seed_lo = (uint32_t)P.p.seed; ba.seed_hi = (uint32_t)(P.p.seed >> 32);
    ba.bootstrap = P.p.bootstrap; ba.gcnt = P.gcnt; ba.gcnt_stride = P.gstride;
    ba.smem_words = P.gcnt ? 0 : (int)((P.N + 3) / 4);
    ba.rows_out = P.rows_a; ba.row_cap = P.row_cap; ba.root = P.nodes_a;
    ba.small_list = P.small_l; ba.big_list = P.big_l; ba.counters = P.d_cnt->n_list[0]; ba.err = P.d_err;
    ba.inbag = P.d_inbag; ba.inbag_words = P.inbag_words;
    ba.store_group = 0;
    ba.y_g = nullptr;
    ba.grp_of = nullptr;
    ba.gsum = nullptr;
    bootstrap_kernel<<<(unsigned)P.T, kBootThreads, P.boot_smem, s>>>(ba);
    AIWCRF_LAUNCH_CHECK("bootstrap_kernel");
    iota_kernel<<<(unsigned)((P.T + 256) / 256), 256, 0, s>>>(P.toff_a, (int)P.T);
    AIWCRF_LAUNCH_CHECK("iota_kernel");
    AIWCRF_CUDA(cudaMemsetAsync(P.tree_base, 0, sizeof(uint32_t) * (size_t)P.T, s));
    AIWCRF_CUDA(cudaMemsetAsync(P.d_done, 0, sizeof(uint32_t), s));
    return AIWCRF_OK;
}

// one level from (nodes_in, rin, toff_in) to (nodes_out, rout, toff_out), at the depth the
// device's level counter holds; fixed grids (the kernels stride over the device's counts)
// one depth; the small-node kernel is captured on `side` (forked and joined through the two
// events), so the graph runs the depth's two level kernels as parallel branches
int plan_level(FitPlan &P, cudaStream_t s, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join, int parity,
               NodeRec *nodes_in, NodeRec *nodes_out, Entry *rin, Entry *rout, uint32_t *toff_in, uint32_t *toff_out)
{
    LevelArgs la;
    la.row_cap = P.row_cap; la.Rr = P.d_Rr; la.vals = P.d_vals; la.card = P.d_card; la.N = P.N;
    la.tree_rng = P.d_rng; la.F = P.F; la.mtry = P.p.mtry; la.min_node = P.p.min_node_size;
    la.max_depth = P.p.max_depth; la.seed_lo = (uint32_t)P.p.seed; la.seed_hi = (uint32_t)(P.p.seed >> 32);
    la.depth = 0; la.depth_ptr = &P.d_cnt->levels;
    la.nodes = nodes_in; la.rows_in = rin; la.rows_out = rout; la.res = P.res; la.tile_splits = P.block_sums;
    la.node_cap = (uint32_t)P.C_max;
    const int bin_cap = big_bin_cap(P.p.mtry, P.F, P.max_card), big_smem = bin_cap * 14;
    la.list = P.big_l; la.list_n = &P.d_cnt->n_list[parity][1];
    const unsigned gbig = (unsigned)(P.cps_big * P.sms), gsmall = (unsigned)(P.cps_small * P.sms);
    AIWCRF_CUDA(cudaEventRecord(ev_fork, s));
    AIWCRF_CUDA(cudaStreamWaitEvent(side, ev_fork, 0));
    AIWCRF_BY_RANK(P.rank_bytes, level_big_kernel<RT><<<gbig, kBigThreads, big_smem, s>>>(la, bin_cap))
    AIWCRF_LAUNCH_CHECK("level_big_kernel");
    la.list = P.small_l; la.list_n = &P.d_cnt->n_list[parity][0];
    AIWCRF_BY_RANK(P.rank_bytes, level_small_kernel<RT><<<gsmall, kSmallThreads, 0, side>>>(la))
    AIWCRF_LAUNCH_CHECK("level_small_kernel");
    AIWCRF_CUDA(cudaEventRecord(ev_join, side));
    AIWCRF_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
    FinalArgs fa;
    fa.nodes = nodes_in; fa.res = P.res; fa.excl_out = P.excl; fa.tree_off = toff_in; fa.tree_base = P.tree_base;
    fa.cnt = P.d_cnt; fa.next = nodes_out; fa.small_list = P.small_l; fa.big_list = P.big_l;
    fa.packed = P.packed; fa.stats = P.d_stats;
    fa.next_tree_off = toff_out; fa.T = (int)P.T; fa.done = P.d_done; fa.tile_splits = P.block_sums;
    fa.parity = parity; fa.next_cap = (uint32_t)P.C_max; fa.vals = P.d_vals; fa.N = P.N;
    finalize_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((P.C_max + kScanTile - 1) / kScanTile, 4 * (int64_t)P.sms)), kFinThreads, 0, s>>>(fa);
    AIWCRF_LAUNCH_CHECK("finalize_kernel");
    return AIWCRF_OK;
}

// capture the graph for the plan's current schedule and instantiate it
int plan_capture(FitPlan &P)
{
    cudaStream_t cs = nullptr, bs = nullptr, ss = nullptr;
    cudaEvent_t evf = nullptr, evj = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evf, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evj, cudaEventDisableTiming);
    struct Streams {
        cudaStream_t a, b, c;
        cudaEvent_t f, j;
        ~Streams()
        {
            if (f) cudaEventDestroy(f);
            if (j) cudaEventDestroy(j);
            if (a) cudaStreamDestroy(a);
            if (b) cudaStreamDestroy(b);
            if (c) cudaStreamDestroy(c);
        }
    } st{cs, bs, ss, evf, evj};
    if (e != cudaSuccess) return cuda_fail(e, "fit plan: streams");
    cudaGraph_t g = nullptr;
    struct G { cudaGraph_t *g; ~G() { if (*g) cudaGraphDestroy(*g); } } gg{&g};
    const int64_t l0 = aiwcrf_launch_count();
    AIWCRF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = plan_phase_a(P, cs, false);
    if (rc == AIWCRF_OK) rc = plan_bootstrap(P, cs);
    cudaGraphConditionalHandle h = 0;
    if (rc == AIWCRF_OK) {
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, cg, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&cn, cg, deps, nullptr, ndeps, &np);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fit plan: level loop node");
        } else {
            P.prefix_launches = aiwcrf_launch_count() - l0;
            // the body grows an even and then an odd depth (the loop starts at depth 0)
            rc = plan_level(P, bs, ss, evf, evj, 0, P.nodes_a, P.nodes_b, P.rows_a, P.rows_b, P.toff_a, P.toff_b);
            if (rc == AIWCRF_OK)
                rc = plan_level(P, bs, ss, evf, evj, 1, P.nodes_b, P.nodes_a, P.rows_b, P.rows_a, P.toff_b, P.toff_a);
            if (rc == AIWCRF_OK) {
                level_loop_cond_kernel<<<1, 32, 0, bs>>>(h, P.d_cnt, (uint32_t)(P.row_cap + 2), P.d_err);
                count_launches(1);
                const cudaError_t e2 = cudaGetLastError();
                if (e2 != cudaSuccess) rc = cuda_fail(e2, "level_loop_cond_kernel launch");
            }
            cudaGraph_t body = nullptr;
            const cudaError_t e3 = cudaStreamEndCapture(bs, &body);
            if (rc == AIWCRF_OK && e3 != cudaSuccess) rc = cuda_fail(e3, "fit plan: level body capture");
        }
    }
    const cudaError_t e4 = cudaStreamEndCapture(cs, &g);
    if (rc != AIWCRF_OK) return rc;
    if (e4 != cudaSuccess) return cuda_fail(e4, "fit plan: capture");
    P.body_launches = aiwcrf_launch_count() - l0 - P.prefix_launches;
    count_launches(-(int)(P.prefix_launches + P.body_launches));     // captured, not run
    if (P.exec) { cudaGraphExecDestroy(P.exec); P.exec = nullptr; }
    AIWCRF_CUDA(cudaGraphInstantiate(&P.exec, g, 0));
    return AIWCRF_OK;
}

}  // namespace

int fit_plan_create(const aiwcrf_fit_params &p, const float *dX, const int64_t *dy, int64_t N, int32_t F,
                    const std::vector<int64_t> &sub_off, const int32_t *d_sub_rows, int32_t G, cudaStream_t s,
                    FitPlan **out)
{
    std::unique_ptr<FitPlan> P(new FitPlan());
    P->p = p; P->dX = dX; P->dy = dy; P->N = N; P->F = F; P->G = G; P->sub_off = sub_off; P->d_sub_rows = d_sub_rows;
    P->Tper = p.num_trees;
    P->T = P->Tper * (int64_t)G;
    if (P->T > (int64_t)AIWCRF_MAX_TREES * 16) return fail(AIWCRF_E_LIMIT, "too many trees in one batch");
    AIWCRF_CUDA(cudaGetDevice(&P->device));
    AIWCRF_CUDA(cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device));
    keep_pool_memory(P->device);
    int rc;
    FitPlan &Q = *P;
    if ((rc = Q.alloc(&Q.d_err, 1)) || (rc = Q.alloc(&Q.d_stats, 1)) || (rc = Q.alloc(&Q.d_counters, 4)) ||
        (rc = Q.alloc(&Q.d_R, (size_t)F * (size_t)N)) || (rc = Q.alloc(&Q.d_vals, (size_t)F * (size_t)N)) ||
        (rc = Q.alloc(&Q.d_card, (size_t)F)) || (rc = Q.alloc(&Q.kA, (size_t)F * (size_t)N + 1)) ||
        (rc = Q.alloc(&Q.vA, (size_t)F * (size_t)N + 1)) || (rc = Q.alloc(&Q.kB, (size_t)F * (size_t)N + 1)) ||
        (rc = Q.alloc(&Q.vB, (size_t)F * (size_t)N + 1)) || (rc = Q.alloc(&Q.hist, radix_sort_hist_words(N, F))) ||
        (rc = Q.alloc(&Q.grp_off, (size_t)N + 1)))
        return rc;
    // probe: the sizes the graph is built for
    if ((rc = plan_phase_a(Q, s, true))) return rc;

    std::vector<int64_t> h_pool_off((size_t)Q.T);
    std::vector<uint32_t> h_pool_len((size_t)Q.T), h_rng((size_t)Q.T);
    int64_t max_pool = 1;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t off = d_sub_rows ? sub_off[(size_t)g] : -1;
        const int64_t len = d_sub_rows ? sub_off[(size_t)g + 1] - sub_off[(size_t)g] : N;
        max_pool = std::max(max_pool, len);
        for (int64_t k = 0; k < Q.Tper; ++k) {
            const size_t t = (size_t)(g * Q.Tper + k);
            h_pool_off[t] = off;
            h_pool_len[t] = (uint32_t)len;
            h_rng[t] = (uint32_t)(p.first_tree + k);
        }
    }
    Q.row_cap = std::min<int64_t>(max_pool, (int64_t)Q.probe_groups);
    Q.C_max = Q.T * Q.row_cap;
    Q.packed_cap = Q.T * (2 * Q.row_cap - 1) + Q.T;
    const size_t table_bytes = (size_t)Q.C_max * (2 * sizeof(NodeRec) + sizeof(SplitRes) + 4 * sizeof(int32_t) + 8) +
                               (size_t)Q.packed_cap * sizeof(PackedRec) + 2 * (size_t)Q.C_max * sizeof(Entry);
    if (table_bytes > ((size_t)16 << 30))
        return fail(AIWCRF_E_LIMIT, "fit plan: worst-case level tables exceed 16 GiB; use aiwcrf_fit");
    if ((rc = Q.alloc(&Q.d_pool_off, (size_t)Q.T)) || (rc = Q.alloc(&Q.d_pool_len, (size_t)Q.T)) ||
        (rc = Q.alloc(&Q.d_rng, (size_t)Q.T)) || (rc = Q.alloc(&Q.rows_a, (size_t)Q.C_max)) ||
        (rc = Q.alloc(&Q.rows_b, (size_t)Q.C_max)) || (rc = Q.alloc(&Q.nodes_a, (size_t)Q.C_max)) ||
        (rc = Q.alloc(&Q.nodes_b, (size_t)Q.C_max)) || (rc = Q.alloc(&Q.res, (size_t)Q.C_max)) ||
        (rc = Q.alloc(&Q.excl, (size_t)Q.C_max + 1)) || (rc = Q.alloc(&Q.block_sums, (size_t)Q.C_max / kScanTile + 2)) ||
        (rc = Q.alloc(&Q.small_l, (size_t)Q.C_max)) || (rc = Q.alloc(&Q.big_l, (size_t)Q.C_max)) ||
        (rc = Q.alloc(&Q.packed, (size_t)Q.packed_cap)) || (rc = Q.alloc(&Q.d_cnt, 1)) ||
        (rc = Q.alloc(&Q.toff_a, (size_t)Q.T + 1)) || (rc = Q.alloc(&Q.toff_b, (size_t)Q.T + 1)) ||
        (rc = Q.alloc(&Q.tree_base, (size_t)Q.T)) || (rc = Q.alloc(&Q.d_done, 1)))
        return rc;
    Q.inbag_words = (N + 31) / 32;
    if (!d_sub_rows && (rc = Q.alloc(&Q.d_inbag, (size_t)Q.T * (size_t)Q.inbag_words))) return rc;
    int optin = 0;
    AIWCRF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, Q.device));
    const int boot_smem_words = std::min<int>((optin - 2048) / 4, 56 * 1024);
    const uint32_t words = (uint32_t)((N + 3) / 4);
    if ((int)words > boot_smem_words) {
        Q.gstride = words;
        if ((rc = Q.alloc(&Q.gcnt, (size_t)Q.T * (size_t)words))) return rc;
    }
    Q.boot_smem = Q.gcnt ? 0 : (int)words * 4;
    AIWCRF_CUDA(cudaMemcpyAsync(Q.d_pool_off, h_pool_off.data(), sizeof(int64_t) * (size_t)Q.T, cudaMemcpyHostToDevice, s));
    AIWCRF_CUDA(cudaMemcpyAsync(Q.d_pool_len, h_pool_len.data(), sizeof(uint32_t) * (size_t)Q.T, cudaMemcpyHostToDevice, s));
    AIWCRF_CUDA(cudaMemcpyAsync(Q.d_rng, h_rng.data(), sizeof(uint32_t) * (size_t)Q.T, cudaMemcpyHostToDevice, s));
    AIWCRF_CUDA(cudaStreamSynchronize(s));
    AIWCRF_CUDA(cudaFuncSetAttribute(bootstrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(Q.boot_smem, 1)));
    const int big_smem = big_bin_cap(p.mtry, F, Q.max_card) * 14;
    {
        cudaError_t e_ = cudaSuccess;
        AIWCRF_BY_RANK(Q.rank_bytes, e_ = cudaFuncSetAttribute(level_big_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               big_smem))
        if (e_ != cudaSuccess) return cuda_fail(e_, "level_big_kernel attribute");
    }
    if ((rc = plan_capture(Q))) return rc;
    *out = P.release();
    return AIWCRF_OK;
}

int fit_plan_run(FitPlan *P, cudaStream_t s, std::vector<aiwcrf_forest *> &out)
{
    AIWCRF_CUDA(cudaGraphLaunch(P->exec, s));
    LevelCounts *h_cnt = static_cast<LevelCounts *>(pinned_scratch());
    if (!h_cnt) return fail(AIWCRF_E_OOM, "pinned host buffer");
    uint32_t *h_err = reinterpret_cast<uint32_t *>(h_cnt + 1);
    AIWCRF_CUDA(cudaMemcpyAsync(h_cnt, P->d_cnt, sizeof(LevelCounts), cudaMemcpyDeviceToHost, s));
    AIWCRF_CUDA(cudaMemcpyAsync(h_err, P->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AIWCRF_CUDA(cudaMemcpyAsync(h_err + 1, P->d_counters + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AIWCRF_CUDA(cudaStreamSynchronize(s));
    int rc = check_err_flags(*h_err);
    if (rc) return rc;
    const uint32_t n_groups = h_err[1];
    const int64_t iters = ((int64_t)h_cnt->levels + 1) / 2;
    count_launches((int)(P->prefix_launches + P->body_launches * iters));    // the body ran iters times
    PackIn pin;
    pin.p = &P->p; pin.T = P->T; pin.Tper = P->Tper; pin.G = P->G; pin.N = P->N; pin.F = P->F; pin.device = P->device;
    pin.tree_base = P->tree_base; pin.d_stats = P->d_stats; pin.packed = P->packed; pin.packed_n = (size_t)h_cnt->packed_off;
    pin.levels = (int)h_cnt->levels; pin.d_inbag = P->d_inbag; pin.inbag_words = P->inbag_words;
    pin.d_vals = P->d_vals; pin.d_card = P->d_card; pin.max_card = P->max_card; pin.rank_bytes = P->rank_bytes;
    pin.n_groups = n_groups;
    pin.grower = AIWCRF_GROWER_LEVEL;
    rc = package_forests(pin, s, out);
    if (rc == AIWCRF_OK) AIWCRF_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int fit_plan_set_schedule(FitPlan *P, int cps_big, int cps_small)
{
    if (cps_big < 1 || cps_big > kBigCtasPerSm || cps_small < 1 || cps_small > kSmallCtasPerSm)
        return fail(AIWCRF_E_INVALID_ARG, "schedule: CTAs per SM out of the range the level kernels are built for");
    P->cps_big = cps_big;
    P->cps_small = cps_small;
    return plan_capture(*P);
}

void fit_plan_schedule(const FitPlan *P, int *cps_big, int *cps_small)
{
    *cps_big = P->cps_big;
    *cps_small = P->cps_small;
}

void fit_plan_limits(int *cps_big, int *cps_small)
{
    *cps_big = kBigCtasPerSm;
    *cps_small = kSmallCtasPerSm;
}

void fit_plan_free(FitPlan *P)
{
    delete P;
}

}  // namespace aiwcrf

namespace aiwcrf {
AIWCRF_BOUNDS_READER(bounds_flags_fit)
}  // namespace aiwcrf
