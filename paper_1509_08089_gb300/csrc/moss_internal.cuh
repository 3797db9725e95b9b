// moss_internal.cuh -- shared definitions of the libmoss translation units.
//
// Device layout of a loaded graph (all arrays in HBM, owned by moss_graph):
//   vert[n]   uint4 {off, deg, S_v, 0}           S_v = sum_{x in N_v} (d_x - 1)
//   col[nnz]  uint32 sorted neighbour lists N_v   (the CSR, Table 1)
//   slot[2 nnz] two uint4 per position, one 32-byte sector:
//             {col, nb, thr, alias} {off, alias col, alias nb, alias off} --
//             per-list alias table of sigma^(v) (eq. 1): keep the column when
//             y < thr for y uniform in [0, S_v), else take position alias --
//             with what a draw needs of the picked neighbour x = col: its
//             list N_x (off, d_x) and twin = position of v in N_x (POS of
//             Sec. 4.1.3, used to exclude v from N_x).  nb packs
//             twin | d_x << 16 when d_x < 2^16; for a larger list nb is
//             kSlotHub, off holds twin and N_x comes from vert[x].
//   acc[nnz]  uint32 ACC_sigma^(v) exclusive prefix of (d_x - 1) within N_v
//   sq[nnz]   uint64 exclusive prefix of (d_x - 1)^2 within N_v: with ACC it
//             gives the prefix of tau^(v) weights (d_x - 1)(S_v - d_x + 1) as
//             S_v ACC - sq, so the Path-5 fallback draws u by binary search;
//             Q_v = sum (d_x - 1)^2 is the list's total (Gamma^(2)_v = S_v^2 - Q_v)
//   gam[l][n] u128 vertex weights Gamma_v, Gamma^(1)_v, Gamma^(2)_v
//   seed[l][2n] two uint4 per column c, one 32-byte sector: {T lo, T hi,
//             alias, 0} -- vertex alias table of weight l, keep the column when
//             x < T for a 64-bit word x -- and a copy of the alias's vertex
//             record (vert, or mvert for MOSS-4Min), so that a draw that takes
//             the alias (most draws for skewed weights) needs no second load.
// MOSS-4Min (Sec. 4.2), built on request:
//   mvert[n]  uint4 {off, deg, Gamma-check_v lo, hi}
//   mslot[2 nnz] two uint4 per slot (v -> u), one 32-byte sector:
//             {thr lo, thr hi, alias, u} -- per-list alias table of
//             sigma-check^(v) (eq. 3): keep the column when y < thr for y
//             uniform in [0, Gamma-check_v), else take position alias --
//             and {off_u, d_u, d_{v,u}, d_{u,v}}
//   mpick[2 nnz] two uint4 per slot, one 32-byte sector, read instead of
//             mslot by a draw from a list with Gamma-check_v < 2^32:
//             {thr, u, off_u, d_{v,u} | d_{u,v} << 16} {alias's u, off_u,
//             d_{v,u} | d_{u,v} << 16, d_u | alias's d_u << 16} -- the draw
//             and both possible picks in one load; the last word is
//             kSlotHub when a field does not fit 16 bits (mslot then serves)
//   rlist[nnz] uint2 {x, d_x}: N_v ordered by the total order (degree, then
//             id; Sec. 3.2), highest first, so N_{v,u} is its first d_{v,u}
//             entries
//   gam[3], seed[3]: Gamma-check_v and its vertex alias table
// nnz < 2^32 bounds every S_v, ACC entry and sigma threshold below 2^32, and
// every Gamma-check_v = sum d_{v,x} d_{x,v} <= d_v * nnz below 2^64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned __int128 u128;

namespace moss {

constexpr int kSlots = 22;            // [0] collisions, [1..21] classes

constexpr int kMethods = 4;          // MOSS-4, T-5, Path-5, MOSS-4Min
// slot record: nb of a neighbour with 2^16 or more neighbours of its own
constexpr uint32_t kSlotHub = 0xffffffffu;
constexpr uint32_t kSlotDegLimit = 1u << 16;

// nb and off words of a slot record for neighbour degree dx and twin tw
__host__ __device__ __forceinline__ uint32_t slot_nb(uint32_t dx, uint32_t tw) {
    return dx < kSlotDegLimit ? (tw | dx << 16) : kSlotHub;
}
// twin of position p from the 32-bit view of the slot records
__device__ __forceinline__ uint32_t slot_twin(const uint32_t *s32, uint64_t p) {
    const uint32_t nb = s32[8 * p + 1];
    return nb == kSlotHub ? s32[8 * p + 4] : (nb & (kSlotDegLimit - 1));
}
// Path-5 samples run in chunks of kDeferChunk ids; a sample whose first pair
// of sigma draws collides is flagged in a bitmap and redone by a second launch
constexpr uint64_t kDeferChunk = 1ull << 26;

// The split of a vertex table into its two levels: the heavy vertices
// (w_v >= ceil(W / 2^split)) take columns [0, nh) in ascending id order, the
// light ones columns [nh, n); a draw takes the light level when its level
// word is below tl = floor(W_L 2^64 / W) (always when nh = 0).
struct alignas(16) SeedLevel {
    u128 WH, WL;                      // the levels' total weights
    uint64_t tl;
    uint32_t nh, pad;
};

struct alignas(16) DevTotals {
    u128 gamma[kMethods];             // Gamma, Gamma^(1), Gamma^(2), Gamma-check
    u128 lambda3, lambda4;            // Lambda_3, Lambda_4
    uint32_t d_max;
    uint32_t pad[3];
    SeedLevel level[kMethods];        // the vertex tables' levels
};

struct DevGraph {
    const uint4 *vert;
    const uint32_t *col;
    const uint4 *slot;
    const uint32_t *acc;
    const uint64_t *sq;
    const uint4 *seed[kMethods];
    const uint4 *mvert;     // MOSS-4Min tables (null until built)
    const uint4 *mslot;
    const uint4 *mpick;
    const uint2 *rlist;
    const uint4 *hash;      // hashed edge set (4 keys per 32 B bucket), or null: probe by search
    const uint32_t *filter; // Bloom filter in front of the hash, or null
    uint32_t *defer;        // Path-5 deferral bitmap, kDeferChunk bits
    uint32_t hash_mask;     // buckets - 1
    uint32_t hash_shift;    // 64 - log2(buckets)
    uint32_t filter_shift;  // 64 - log2(filter words)
    uint32_t n;
    uint32_t rng;           // word generator: kRngSplitMix or kRngPhilox
    uint32_t nheavy[kMethods];   // heavy columns of each vertex table (SeedLevel)
    uint64_t tlight[kMethods];   // light-level bound of each vertex table
    const uint2 *hub_rank;       // behind the filter: per 32 vertices {hubs before them, hub bits}, or null
    const uint32_t *hub_bits;    // the hubs' H x H adjacency bits
    uint32_t hubs;               // H
};

// ------------------------------------------------------- hub adjacency --
// Behind the edge filter (graphs whose edge set leaves the L2), pairs of hubs
// -- every vertex of degree >= D, D the smallest degree with at most
// H = min(8192, max(16, n / 16)) of them -- are answered from an H x H bitmap
// of their adjacency (bit i H + j: hubs i and j adjacent), exactly and from
// the L2.  Hub i is the i-th hub in ascending id order; its index comes from
// one 8-byte load of the rank table: entry x / 32 = {hubs below 32 (x / 32),
// bit t set iff vertex 32 (x / 32) + t is a hub}.
constexpr uint32_t kNoHub = 0xFFFFFFFFu;
constexpr uint32_t kMaxHubs = 8192;

inline uint32_t hub_capacity(uint32_t n) {
    const uint32_t h = n / 16 < 16 ? 16 : n / 16;
    return h < kMaxHubs ? h : kMaxHubs;
}
__device__ __forceinline__ uint32_t hub_index(uint2 e, uint32_t x) {
    const uint32_t bit = 1u << (x & 31u);
    return (e.y & bit) ? e.x + (uint32_t)__popc(e.y & (bit - 1u)) : kNoHub;
}

// ------------------------------------------------------- hashed edge set --
// Key of the undirected edge {a, b}: (min << 32) | max; empty slot: ~0.
// Buckets hold four keys (32 B, one sector, read by one 256-bit load); a
// bucket's slot k is filled only after its slot k-1, and keys are never
// removed, so a lookup walking from the home bucket can stop at the first
// bucket whose last slot is empty.
constexpr uint64_t kEmptyKey = ~0ULL;
constexpr int kBucketKeys = 4;

__host__ __device__ inline uint64_t edge_key(uint32_t a, uint32_t b) {
    return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}

// home bucket: the top bits of a 64-bit finaliser (MurmurHash3 fmix64 steps)
__host__ __device__ inline uint32_t edge_bucket(uint64_t k, uint32_t shift) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return (uint32_t)(k >> shift);
}

// ----------------------------------------------------------- edge filter --
// Blocked Bloom filter over the same keys: word = top bits of a second
// 64-bit finaliser (different constants), three bit positions from its low
// bits; a key is possibly present when all three bits of its word are set.
__host__ __device__ inline uint64_t filter_hash(uint64_t k) {
    k ^= 0x9e3779b97f4a7c15ULL;
    k ^= k >> 31;
    k *= 0xbf58476d1ce4e5b9ULL;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebULL;
    k ^= k >> 31;
    return k;
}

__host__ __device__ inline uint32_t filter_mask(uint64_t h) {
    return (1u << (h & 31u)) | (1u << ((h >> 5) & 31u)) | (1u << ((h >> 10) & 31u));
}

// Status flags raised by kernels (bitwise OR into a device word).
enum : uint32_t {
    kErrRowPtr = 1u << 0,     // row_ptr not monotone / wrong ends
    kErrRange = 1u << 1,      // neighbour id >= n
    kErrSelf = 1u << 2,       // self loop
    kErrOrder = 1u << 3,      // list not strictly increasing (or duplicate)
    kErrAsym = 1u << 4,       // (v,u) without (u,v)
    kErrOverflow = 1u << 5,   // exact total out of range
};

// ------------------------------------------------------------ arithmetic --
__host__ __device__ inline uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((u128)a * b) >> 64);
#endif
}

// floor(x * m / 2^64): a uniform index in [0, m) from a 64-bit word
__device__ __forceinline__ uint64_t word_index(uint64_t x, uint64_t m) { return __umul64hi(x, m); }

// ------------------------------------------------------------ warp scans --
__device__ __forceinline__ uint64_t shfl_up64(uint64_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }

__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t t = shfl_up64(v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
    uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)v, d);
    uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(v >> 64), d);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
    uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)v, d);
    uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(v >> 64), d);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_idx_u128(u128 v, int src) {
    uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)v, src);
    uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(v >> 64), src);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 warp_incl_scan128(u128 v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u128 t = shfl_up_u128(v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ u128 warp_sum128(u128 v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += shfl_down_u128(v, d);
    return v;
}

// ------------------------------------------------------------ SplitMix64 --
// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) in counter form: word i (0 <= i < 16) of sample s
// of method t under seed k is output number (4 s + t) 16 + i + 1 of the
// generator seeded with k: the state k advanced by that many Weyl increments,
// through the generator's mixing function.  Every word is independent of the
// others, so a sample computes only the words it reads.
struct Words2 { uint64_t x[2]; };

constexpr uint64_t kSplitMixGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// --------------------------------------------------------- Philox4x32-10 --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds on a 128-bit counter (c0..c3) under
// a 64-bit key (k0, k1).  A round forms the 64-bit products p = M0 c0 and
// q = M1 c2 and makes the counter (hi q ^ c1 ^ k0, lo q, hi p ^ c3 ^ k1,
// lo p); the key grows by the Weyl increments between rounds.  Words 2b and
// 2b+1 of sample s of method t under seed k are the outputs of block
// (s lo, s hi, t, b) under the key (k lo, k hi), low output first.
constexpr int kRngSplitMix = 0, kRngPhilox = 1;
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint32_t p_hi = __umulhi(kPhiloxM0, c.x), p_lo = kPhiloxM0 * c.x;
        const uint32_t q_hi = __umulhi(kPhiloxM1, c.z), q_lo = kPhiloxM1 * c.z;
        c = make_uint4(q_hi ^ c.y ^ k0, q_lo, p_hi ^ c.w ^ k1, p_lo);
    }
    return c;
}

// words 2 p and 2 p + 1 of sample s of method t under generator RNG: one
// Philox block, or two SplitMix64 outputs.  Samplers fetch each pair where
// they first read it, which keeps the words' live ranges short (a word the
// caller never reads is not computed: everything is inlined).
template <int RNG>
__device__ __forceinline__ Words2 sample_words2(uint64_t seed, uint32_t t, uint64_t s, uint32_t p) {
    Words2 w;
    if (RNG == kRngPhilox) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), t, p), (uint32_t)seed,
                                      (uint32_t)(seed >> 32));
        w.x[0] = (uint64_t)o.x | ((uint64_t)o.y << 32);
        w.x[1] = (uint64_t)o.z | ((uint64_t)o.w << 32);
    } else {
        const uint64_t base = seed + ((4 * s + t) * 16 + 2 * p + 1) * kSplitMixGamma;
        w.x[0] = splitmix_mix(base);
        w.x[1] = splitmix_mix(base + kSplitMixGamma);
    }
    return w;
}

// word i of sample s of method t under generator RNG alone
template <int RNG>
__device__ __forceinline__ uint64_t sample_word(uint64_t seed, uint32_t t, uint64_t s, uint32_t i) {
    const Words2 w = sample_words2<RNG>(seed, t, s, i >> 1);
    return w.x[i & 1];
}

// ----------------------------------------------------- host-side launches --
// Auxiliary streams of the calling host thread on one device, with the
// events of one fork (a[0..2] each wait for what was queued on s), one join
// (s waits for all of them) and one hand-over (s waits for one of them
// mid-chain), for independent chains of the table build; a[3], a[4] and the
// sub_* events serve the chains' own inner forks (the MOSS-4Min tables).
constexpr int kAuxStreams = 5;
constexpr int kAuxOuter = 3;
struct AuxStreams {
    cudaStream_t a[kAuxStreams] = {};
    cudaEvent_t forked = nullptr, done[kAuxStreams] = {}, mid = nullptr;
    cudaEvent_t sub_fork = nullptr, sub_done[2] = {}, sub_mid = nullptr;
    cudaError_t fork(cudaStream_t s) const;
    cudaError_t join(cudaStream_t s) const;
    cudaError_t wait_for(cudaStream_t s, int i) const;   // s waits for what is queued on a[i] so far
};
// the calling thread's auxiliary streams on the current device (created on
// first use; null when they cannot be created: callers then stay on s)
const AuxStreams *aux_streams();

// SM count of a device (of the current device), queried once per device
int device_sms(int device);
int current_sms();

// moss_tables.cu
cudaError_t launch_vertices(const void *row_ptr, int is64, uint32_t n, uint64_t nnz, uint4 *vert,
                            uint32_t *flags, cudaStream_t s);
// flags[0]: kErr* bits; flags[1]: slots whose twin was matched (must reach nnz)
cudaError_t launch_slots(uint32_t n, uint64_t nnz, const uint32_t *col, uint4 *vert, uint4 *slot, uint32_t *acc,
                         uint32_t *owner, uint64_t *sq, u128 *gam0, u128 *gam1, u128 *gam2, u128 *partials,
                         int blocks, uint32_t *flags, cudaStream_t s, const AuxStreams *aux);
cudaError_t launch_totals(const u128 *partials, int blocks, DevTotals *tot, cudaStream_t s);
cudaError_t launch_edge_hash(uint64_t nnz, const uint32_t *col, const uint32_t *owner, unsigned long long *table,
                             uint32_t mask, uint32_t shift, cudaStream_t s);
// filter of 2^(64 - shift) words, zeroed beforehand
cudaError_t launch_edge_filter(uint64_t nnz, const uint32_t *col, const uint32_t *owner, uint32_t *filter,
                               uint32_t shift, cudaStream_t s);
// hub adjacency of the edge filter in `mem` (hub_bytes(n) bytes, kept with the
// filter): the rank table, the bitmap and the hub list (ascending ids,
// kNoHub past the last) come back through the out pointers; `mem` also
// holds the scratch of the build
uint64_t hub_bytes(uint32_t n);
cudaError_t launch_hub_tables(uint32_t n, const uint4 *vert, const uint32_t *col, void *mem, uint2 **rank_out,
                              uint32_t **bits_out, uint32_t **list_out, cudaStream_t s);
// aux (nullable, already forked from s): the long lists go to aux->a[long_stream]
cudaError_t launch_sigma_alias(uint32_t n, uint64_t nnz, const uint4 *vert, const uint32_t *acc, const uint32_t *owner,
                               uint4 *slot, uint32_t *scratch_idx, uint64_t *scratch_pre, cudaStream_t s,
                               const AuxStreams *aux, int long_stream);
// two-level vertex alias tables of up to 3 weights in the same launches
// (seed[t]: 2n uint4, vrec[t]: the n vertex records copied beside each
// alias; the levels go to tot->level[which[t]]; heavy: w_v 2^split >= W;
// split 64: one table over all vertices); scratch of seed_scratch_bytes(n) bytes
cudaError_t launch_seed_alias(uint32_t n, DevTotals *tot, int ntables, const int *which, u128 *const *w,
                              uint4 *const *seed, const uint4 *const *vrec, void *scratch, uint32_t *flags, int split,
                              cudaStream_t s);
uint64_t seed_scratch_bytes(uint32_t n);
int table_blocks(uint32_t n);
int slot_partial_rows(uint32_t n);   // rows of 6 u128 totals launch_slots writes (launch_totals sums them)

// moss_min.cu: the MOSS-4Min tables (ordered lists, d_{v,u}, Gamma-check_v,
// the sigma-check alias tables, tot->gamma[3] and its vertex alias table)
uint64_t min_scratch_bytes(uint32_t n, uint64_t nnz);
cudaError_t launch_min_tables(uint32_t n, uint64_t nnz, const uint4 *vert, const uint32_t *col,
                              const uint32_t *owner, const uint4 *slot, uint4 *mvert, uint4 *mslot, uint4 *mpick,
                              uint2 *rlist, u128 *gmin, uint4 *seed_min, DevTotals *tot, void *scratch,
                              uint32_t *flags, int split, cudaStream_t s, const AuxStreams *aux);

// moss_sample.cu
// class of each 4- and 5-vertex edge mask; c(s) of MOSS-4Min by (mask << 6 | order bits)
void upload_luts(const uint8_t *lut4, const uint8_t *lut5, const uint8_t *lutc);
// Counts (22 uint64 at counts_dev) of samples [first, first+count) of one
// method, with optional per-sample records (classes, verts: count and 5*count
// entries); partials holds sample_rows(method) rows of 22 uint64.  Path-5 runs
// in chunks of kDeferChunk ids: a launch that defers the samples whose first
// sigma attempt collides, one that redoes them, and a reduce that accumulates.
cudaError_t launch_counts(int method, const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed,
                          uint64_t *partials, uint8_t *classes, uint32_t *verts, uint64_t *counts_dev,
                          cudaStream_t s);
int sample_blocks(int method, int device);   // the most blocks any variant of a sampler launches
int sample_launch_blocks(int method, int device, const DevGraph &g);   // blocks of the variant g uses
int sample_rows(int method, int device);     // partial-count rows launch_counts needs

// moss_finalize.cu
struct FinalizeIn {
    int k;
    int mix = 0;      // k = 4 only: MOSS-4 (K[0], hits[0]) with MOSS-4Min (K[1], hits[1])
    uint64_t K[2];
};
cudaError_t launch_finalize(const FinalizeIn &in, const uint64_t *hits_dev, const DevTotals *tot,
                            void *result_dev, cudaStream_t s);
cudaError_t launch_covariance(const FinalizeIn &in, const uint64_t *hits_dev, const DevTotals *tot,
                              void *result_dev, double *cov_dev, cudaStream_t s);

// ---------------------------------------------------------------- batches --
// One task = one sub-method of one request: sample ids [first, first+count)
// of `method` on graph `graph`, cut into tiles of the batch's tile size,
// starting at tile `tile0` of the batch.
struct BatchTask {
    uint64_t seed;
    uint64_t first;
    uint64_t count;
    uint64_t tile0;
    uint32_t graph;
    uint32_t method;
};
struct BatchRequest {
    FinalizeIn in;
    const DevTotals *tot;
    int task[2];      // task index per sub-method, -1 when it draws nothing
};
// persistent sampler over a batch: tile_counts[t][22] per tile; threads per
// block 128, 256 or 512; tile_cycles (nullable) receives each tile's SM
// cycles; rngs: the generators of the batch's graphs (kBatch*)
constexpr int kBatchSplitMix = 0, kBatchPhilox = 1, kBatchBoth = 2;
cudaError_t launch_sample_batch(const DevGraph *graphs, const BatchTask *tasks, int ntasks, uint64_t ntiles,
                                uint32_t tile_samples, unsigned long long *next_tile, uint32_t *tile_counts,
                                int threads, int blocks, unsigned long long *tile_cycles, int rngs, cudaStream_t s);
// the batch generator mode of a set of graph views
inline int batch_rngs(const DevGraph *views, size_t n) {
    bool sm = false, ph = false;
    for (size_t i = 0; i < n; ++i) (views[i].rng == kRngPhilox ? ph : sm) = true;
    return sm && ph ? kBatchBoth : ph ? kBatchPhilox : kBatchSplitMix;
}
// task_counts[task][22] = sum of the task's tile rows, in tile order
cudaError_t launch_batch_reduce(const BatchTask *tasks, int ntasks, uint32_t tile_samples,
                                const uint32_t *tile_counts, uint64_t *task_counts, cudaStream_t s);
int batch_max_per_sm(int threads, int rngs);                    // resident blocks per SM at most
int batch_blocks(int device, int threads, int per_sm, int rngs);  // grid; per_sm <= 0: the most that fit
cudaError_t launch_finalize_batch(const BatchRequest *reqs, int nreq, const uint64_t *task_counts, void *results,
                                  cudaStream_t s);

// moss_capi.cu: what another translation unit needs of a moss_graph
struct GraphInfo {
    DevGraph view;
    const DevTotals *tot;
    int device;
    unsigned built;          // bit l: vertex table l; bit 3: sigma tables; bit 4: edge hash; bit 5: MOSS-4Min;
                             // bit 6: edge filter
    bool total_nonzero[kMethods];   // Gamma, Gamma^(1), Gamma^(2), Gamma-check > 0
    bool ready[kMethods];    // the method can sample: its tables and the probe tables of the graph's
                             // probe strategy are built (what moss_sample_counts requires)
};
}  // namespace moss

struct moss_graph;
namespace moss {
int graph_info(const moss_graph *g, GraphInfo *out);
// the device view of g with the given probe strategy (MOSS_PROBE_*; AUTO: the
// graph's own); MOSS_ESTATE when the tables it needs are not built
int graph_view_for(const moss_graph *g, int strategy, DevGraph *out);
int set_error(int code, const char *detail);   // records the thread's error detail
}  // namespace moss
