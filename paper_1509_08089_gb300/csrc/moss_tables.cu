// moss_tables.cu -- the initialization step on the device.
//
// Paper: Sec. 4.1.3 ("Initialization", WeightRandomVertex) and Sec. 5.1.4.
//   * vertex weights Gamma_v = (d_v-1) S_v (Sec. 4.1.1), Gamma^(1)_v =
//     (d_v-1)(d_v-2) S_v (Sec. 5.1.1), Gamma^(2)_v = S_v^2 - Q_v (Sec. 5.1.2),
//     S_v = sum_{x in N_v} (d_x-1), Q_v = sum (d_x-1)^2; exact totals (Table 1)
//     and Lambda_3 = sum C(d,3), Lambda_4 = sum C(d,4) in 128-bit integers.
//   * WeightRandomVertex is realised with alias tables (O(1) per draw) instead
//     of the paper's prefix-array binary search (O(log d)).
//
// Alias construction.  m items, weights w_j, W = sum w, q_j = w_j m.  Every
// column holds W: item j keeps thr_j, the rest goes to alias_j.  Light items
// (q_j < W) carry a deficit D = W - q_j, heavy ones (q_j >= W) an excess
// E = q_j - W, both taken in index order.  With A_i the exclusive prefix of
// the light deficits and P_k the inclusive prefix of the heavy excesses, the
// table equals the one of the sequential sweep that fills lights in order
// from the current heavy item and moves on when the heavy item's residue
// falls below W:
//   light i : thr = q, alias = heavy k(i), k(i) = min{k : P_k >= A_i}
//   heavy k : if P_k < P_total: alias = heavy k+1, thr = W + P_k - A_{i'},
//             i' = min{i : A_i > P_k} (A_{#lights} = P_total);
//             else thr = W, alias = itself.
// Both prefix sums and every search are parallel, so the per-list tables
// (a warp per list) and the vertex tables (a block scan over V, then one
// thread per item) are built without a sequential pass.
#include <algorithm>
#include <atomic>

#include "moss_alias.cuh"
#include "moss_internal.cuh"

namespace moss {

namespace {

constexpr int kWarp = 32;
constexpr int kTableThreads = 256;
constexpr uint32_t kLongList = 256;   // longer lists get a block each in the alias passes
constexpr int kUnroll = 1;            // chunks of 32 slots per round in k_slots
constexpr int kLongThreads = 256;

// ------------------------------------------------------------ vertices ---
template <typename IdxT>
__global__ void k_vertices(const IdxT *row_ptr, uint32_t n, uint64_t nnz, uint4 *vert, uint32_t *flags) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = row_ptr[v], b = row_ptr[v + 1];
        bool bad = b < a || b > nnz || (v == 0 && a != 0) || (v + 1 == n && b != nnz);
        if (bad) {
            atomicOr(flags, kErrRowPtr);
            a = b = 0;
        }
        vert[v] = make_uint4((uint32_t)a, (uint32_t)(b - a), 0u, 0u);
    }
}

// --------------------------------------------------------------- slots ---
// Three passes.  k_owner: the vertex of each slot (warp per vertex, stores
// only).  k_slot_weights: one thread per slot validates the neighbour id and
// order and gathers w = d_x - 1 into acc -- every gather of the graph in
// flight at once.  k_slots: one warp per vertex scans its w (coalesced
// loads) into the ACC prefix and the prefix of squares, then S_v, Q_v, the
// three vertex weights and the block's share of the exact totals.
__global__ void k_owner(uint32_t n, const uint4 *__restrict__ vert, uint32_t *owner) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    for (uint64_t v = (uint64_t)blockIdx.x * wpb + warp; v < n; v += (uint64_t)gridDim.x * wpb) {
        const uint4 vr = vert[v];
        for (uint32_t i = lane; i < vr.y; i += kWarp) owner[vr.x + i] = (uint32_t)v;
    }
}

__global__ void k_slot_weights(uint32_t n, uint64_t nnz, const uint32_t *__restrict__ col,
                               const uint4 *__restrict__ vert, const uint32_t *__restrict__ owner, uint4 *slot,
                               uint32_t *acc, uint32_t *flags) {
    uint32_t err = 0;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = owner[p], x = col[p];
        uint32_t w = 0, ox = 0, dx = 0;
        if (x >= n) {
            err |= kErrRange;
        } else {
            if (x == v) err |= kErrSelf;
            if (p > 0 && owner[p - 1] == v && col[p - 1] >= x) err |= kErrOrder;
            const uint4 xr = vert[x];
            w = xr.y ? xr.y - 1 : 0;
            ox = xr.x;
            dx = xr.y;
        }
        acc[p] = w;    // turned into the prefix by k_slots
        // words 2 and 3 (the sigma threshold and alias, written by the table
        // build) hold x's {off, deg} until then, for k_twin
        slot[2 * p] = make_uint4(x, 0u, ox, dx);
        slot[2 * p + 1] = make_uint4(ox, 0u, 0u, 0u);   // nb and, for a hub, off: k_twin
    }
    if (err) atomicOr(flags, err);
}

// exact totals of a share of the vertices: Gamma, Gamma^(1), Gamma^(2),
// Lambda_3, Lambda_4 and the maximum degree
struct Totals {
    u128 g0, g1, g2, l3, l4;
    uint32_t dmax;
    __device__ void add(const Totals &o) {
        g0 += o.g0; g1 += o.g1; g2 += o.g2; l3 += o.l3; l4 += o.l4;
        dmax = o.dmax > dmax ? o.dmax : dmax;
    }
    __device__ void store(u128 *row) const {
        row[0] = g0; row[1] = g1; row[2] = g2; row[3] = l3; row[4] = l4; row[5] = dmax;
    }
};

// S_v, the vertex weights Gamma_v = (d-1) S_v, Gamma^(1)_v = (d-1)(d-2) S_v,
// Gamma^(2)_v = S_v^2 - Q_v, and v's share of the totals
__device__ __forceinline__ void vertex_weights(uint64_t v, uint32_t d, uint64_t S, uint64_t Q, u128 *gam0,
                                               u128 *gam1, u128 *gam2, Totals &t) {
    const u128 g0 = d >= 1 ? (u128)(d - 1) * S : 0;
    const u128 g1 = d >= 2 ? (u128)(d - 1) * (d - 2) * S : 0;
    const u128 g2 = (u128)S * S - Q;
    gam0[v] = g0;
    gam1[v] = g1;
    gam2[v] = g2;
    t.g0 += g0;
    t.g1 += g1;
    t.g2 += g2;
    if (d >= 3) {
        // C(d,3) and C(d,4) without a 128-bit division: d(d-1)/2 is exact in
        // 64 bits, 3 divides it or d-2, and 4 C(d,4) = C(d,3)(d-3)
        const uint64_t h = (uint64_t)d * (d - 1) / 2;
        const u128 c3 = (d - 2) % 3 == 0 ? (u128)h * ((d - 2) / 3) : (u128)(h / 3) * (d - 2);
        t.l3 += c3;
        if (d >= 4) t.l4 += (c3 * (d - 3)) >> 2;
    }
    t.dmax = d > t.dmax ? d : t.dmax;
}

__device__ __forceinline__ uint32_t warp_incl_scan32(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kTableThreads, 8) k_slots(uint32_t n, uint4 *vert, uint32_t *acc, uint64_t *sq,
                                                           u128 *gam2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * wpb;
    uint64_t v = (uint64_t)blockIdx.x * wpb + warp;
    uint4 next = v < n ? vert[v] : make_uint4(0u, 0u, 0u, 0u);
    for (; v < n; v += stride) {
        // the next vertex's record is loaded while this list is scanned
        const uint4 vr = next;
        if (v + stride < n) next = vert[v + stride];
        const uint32_t o = vr.x, d = vr.y;
        if (d > kLongList) continue;   // k_slots_long
        uint64_t run = 0, qsum = 0;
        // kUnroll chunks of 32 per round, their loads issued together
        for (uint32_t base = 0; base < d; base += kWarp * kUnroll) {
            uint32_t w[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const uint32_t i = base + u * kWarp + lane;
                w[u] = i < d ? acc[o + i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (base + u * kWarp >= d) break;   // warp-uniform
                const uint32_t i = base + u * kWarp + lane;
                const uint64_t w2 = (uint64_t)w[u] * w[u];
                const uint64_t incl = warp_incl_scan32(w[u], lane);   // S_v < 2^32
                const uint64_t incl2 = warp_incl_scan64(w2, lane);
                if (i < d) {
                    acc[o + i] = (uint32_t)(run + incl - w[u]);
                    sq[o + i] = qsum + incl2 - w2;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
                qsum += __shfl_sync(0xffffffffu, incl2, 31);
            }
        }
        if (lane == 0) {   // S_v, and Q_v until k_vertex_weights turns it into Gamma^(2)_v
            vert[v].z = (uint32_t)run;
            gam2[v] = qsum;
        }
    }
}

// lists longer than kLongList: a block per list scans NT x 4 entries a round
// (each thread 4 consecutive ones, then a block scan of the thread sums)
__global__ void __launch_bounds__(kLongThreads) k_slots_long(uint32_t n, uint4 *vert, uint32_t *acc, uint64_t *sq,
                                                            u128 *gam2) {
    __shared__ uint64_t s_w[kLongThreads / kWarp], s_q[kLongThreads / kWarp];
    for_each_vertex<kLongThreads>(n, vert, [](uint4 vr) { return vr.y > kLongList; }, [&](uint32_t v) {
        const uint4 vr = vert[v];
        const uint32_t o = vr.x, d = vr.y;
        uint64_t run = 0, qsum = 0;
        for (uint32_t base = 0; base < d; base += kLongThreads * 4) {
            const uint32_t i0 = base + 4 * threadIdx.x;
            uint32_t w[4];
            uint64_t lw = 0, lq = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                w[k] = i0 + k < d ? acc[o + i0 + k] : 0u;
                lw += w[k];
                lq += (uint64_t)w[k] * w[k];
            }
            uint64_t tw, tq;
            const uint64_t iw = block_incl_scan<uint64_t, kLongThreads>(lw, tw, s_w);
            const uint64_t iq = block_incl_scan<uint64_t, kLongThreads>(lq, tq, s_q);
            uint64_t ew = run + iw - lw, eq = qsum + iq - lq;   // exclusive prefixes at i0
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (i0 + k < d) {
                    acc[o + i0 + k] = (uint32_t)ew;
                    sq[o + i0 + k] = eq;
                }
                ew += w[k];
                eq += (uint64_t)w[k] * w[k];
            }
            run += tw;
            qsum += tq;
        }
        if (threadIdx.x == 0) {   // S_v, and Q_v until k_vertex_weights turns it into Gamma^(2)_v
            vert[v].z = (uint32_t)run;
            gam2[v] = qsum;
        }
        __syncthreads();
    });
}

// Gamma_v, Gamma^(1)_v, Gamma^(2)_v from d_v, S_v and Q_v (left in gam2 by
// the list scans), one thread per vertex, and each block's share of the
// exact totals (the 128-bit arithmetic of a vertex on one lane each, instead
// of on the first lane of a warp per list)
__global__ void __launch_bounds__(kTableThreads) k_vertex_weights(uint32_t n, const uint4 *__restrict__ vert,
                                                                  u128 *gam0, u128 *gam1, u128 *gam2, u128 *partials) {
    Totals t = {};
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = vert[v];
        vertex_weights(v, r.y, r.z, (uint64_t)gam2[v], gam0, gam1, gam2, t);
    }
    __shared__ Totals sh[kTableThreads / kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        Totals o;
        o.g0 = shfl_down_u128(t.g0, k);
        o.g1 = shfl_down_u128(t.g1, k);
        o.g2 = shfl_down_u128(t.g2, k);
        o.l3 = shfl_down_u128(t.l3, k);
        o.l4 = shfl_down_u128(t.l4, k);
        o.dmax = __shfl_down_sync(0xffffffffu, t.dmax, k);
        t.add(o);
    }
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        Totals b = {};
        for (int w = 0; w < kTableThreads / kWarp; ++w) b.add(sh[w]);
        b.store(partials + (uint64_t)blockIdx.x * 6);
    }
}

// One block of kTotalsThreads: each thread adds a strided share of the rows,
// then warps and the block combine (exact integer sums and a maximum, so the
// order does not matter).
constexpr int kTotalsThreads = 1024;

__device__ __forceinline__ void warp_totals(u128 (&s)[6]) {
    for (int j = 0; j < 5; ++j) s[j] = warp_sum128(s[j]);
    for (int d = 16; d > 0; d >>= 1) {
        const u128 o = shfl_down_u128(s[5], d);
        s[5] = o > s[5] ? o : s[5];
    }
}

__global__ void __launch_bounds__(kTotalsThreads) k_totals(const u128 *partials, int blocks, DevTotals *tot) {
    __shared__ u128 w_tot[kTotalsThreads / kWarp][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u128 s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < blocks; b += kTotalsThreads)
        for (int j = 0; j < 6; ++j) {
            u128 x = partials[(uint64_t)b * 6 + j];
            s[j] = j == 5 ? (x > s[j] ? x : s[j]) : s[j] + x;
        }
    warp_totals(s);
    if (lane == 0)
        for (int j = 0; j < 6; ++j) w_tot[warp][j] = s[j];
    __syncthreads();
    if (warp != 0) return;
    for (int j = 0; j < 6; ++j) s[j] = w_tot[lane][j];   // kTotalsThreads / kWarp == 32 rows
    warp_totals(s);
    if (lane == 0) {
        tot->gamma[0] = s[0];
        tot->gamma[1] = s[1];
        tot->gamma[2] = s[2];
        tot->gamma[3] = 0;    // Gamma-check: set when the MOSS-4Min tables are built
        tot->lambda3 = s[3];
        tot->lambda4 = s[4];
        tot->d_max = (uint32_t)s[5];
    }
}

// --------------------------------------------------------------- twins ---
// One thread per slot.  Each undirected edge {v, x} is handled once, by the
// endpoint with the larger degree (the smaller id on ties), which searches
// itself in the other endpoint's (shorter) sorted list and writes both
// twins: twin(v->x) = POS of v in N_x and twin(x->v) = POS of x in N_v.  For
// a symmetric graph every edge is matched once, so the matched slots add up
// to nnz; a reverse that is missing leaves the sum short.
__global__ void k_twin(uint32_t n, uint64_t nnz, const uint4 *__restrict__ vert, const uint32_t *__restrict__ col,
                       const uint32_t *__restrict__ owner, uint4 *slot, uint32_t *flags) {
    uint32_t matched = 0, err = 0;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = owner[p], x = col[p];
        if (x >= n || x == v) continue;  // flagged by the slot pass
        // {off, deg} only: k_slots may be writing S_v into the same records;
        // x's comes from words 2 and 3 of the slot record (k_slot_weights), a
        // streamed read instead of a random one
        const uint2 vr = reinterpret_cast<const uint2 *>(vert)[2 * (uint64_t)v];
        const uint2 xr = reinterpret_cast<const uint2 *>(slot)[4 * p + 1];
        const bool mine = vr.y > xr.y || (vr.y == xr.y && v < x);
        if (!mine) continue;
        uint32_t lo = xr.x, len = xr.y;
        while (len > 0) {
            const uint32_t half = len >> 1;
            if (col[lo + half] < v) { lo += half + 1; len -= half + 1; } else { len = half; }
        }
        if (lo >= xr.x + xr.y || col[lo] != v) {
            err |= kErrAsym;
            continue;
        }
        uint32_t *s32 = reinterpret_cast<uint32_t *>(slot);
        const uint32_t tp = lo - xr.x;                 // POS of v in N_x
        const uint32_t tl = (uint32_t)(p - vr.x);      // POS of x in N_v
        s32[8 * p + 1] = slot_nb(xr.y, tp);
        if (xr.y >= kSlotDegLimit) s32[8 * p + 4] = tp;
        s32[8 * (uint64_t)lo + 1] = slot_nb(vr.y, tl);
        if (vr.y >= kSlotDegLimit) s32[8 * (uint64_t)lo + 4] = tl;
        matched += 2;
    }
    if (err) atomicOr(flags, err);
    // warp sum of the matched slots, one atomic per warp
#pragma unroll
    for (int sft = 16; sft > 0; sft >>= 1) matched += __shfl_down_sync(0xffffffffu, matched, sft);
    if ((threadIdx.x & 31) == 0 && matched) atomicAdd(flags + 1, matched);
}

// ----------------------------------------------------- hashed edge set ---
// One thread per slot inserts the edge {v, x} with v < x by compare-and-swap
// into the first free slot from the home bucket on, slots of a bucket in
// order.  The table has at least four slots per edge, so a free slot always
// exists and the walk is bounded by the bucket count.
__global__ void k_edge_hash(uint64_t nnz, const uint32_t *__restrict__ col, const uint32_t *__restrict__ owner,
                            unsigned long long *table, uint32_t mask, uint32_t shift) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = owner[p], x = col[p];
        if (x <= v) continue;
        const unsigned long long key = edge_key(v, x);
        uint32_t b = edge_bucket(key, shift);
        bool done = false;
        for (uint64_t it = 0; it <= mask && !done; ++it) {
            for (int k = 0; k < kBucketKeys && !done; ++k) {
                const unsigned long long old =
                    atomicCAS(table + (uint64_t)kBucketKeys * b + k, (unsigned long long)kEmptyKey, key);
                done = old == kEmptyKey || old == key;
            }
            b = (b + 1) & mask;
        }
    }
}

// --------------------------------------------------------- edge filter ---
// One thread per slot sets the three bits of each edge {v, x}, v < x.
__global__ void k_edge_filter(uint64_t nnz, const uint32_t *__restrict__ col, const uint32_t *__restrict__ owner,
                              uint32_t *filter, uint32_t shift) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = owner[p], x = col[p];
        if (x <= v) continue;
        const uint64_t h = filter_hash(edge_key(v, x));
        atomicOr(filter + (h >> shift), filter_mask(h));
    }
}

// ------------------------------------------------ per-list sigma tables ---
// Slot record (32 bytes) of position j of N_v: {col, nb, thr, alias} {off,
// alias col, alias nb, alias off}, so a draw that takes the alias needs no
// second load.  col, nb and off were set at load; the alias passes write thr
// and alias (one 8-byte store), and k_slot_alias_fill then copies col, nb
// and off of the alias position into words 5..7.
__device__ __forceinline__ void set_sigma(uint32_t *slot32, uint32_t o, uint32_t j, uint32_t thr, uint32_t alias) {
    *reinterpret_cast<uint2 *>(slot32 + 8 * (uint64_t)(o + j) + 2) = make_uint2(thr, alias);
}
// weight of position p of N_v from the ACC prefix
// (read-only loads: acc is not written while the alias tables are built, so
// they need not wait for the passes' stores to the slot records)
__device__ __forceinline__ uint32_t acc_weight(const uint32_t *acc, uint32_t o, uint32_t d, uint32_t S, uint32_t p) {
    return (p + 1 < d ? __ldg(acc + o + p + 1) : S) - __ldg(acc + o + p);
}

// A warp per list of at most kLongList entries; the split (idx, pre) of the
// list being built lives in the warp's share of shared memory, so the
// searches and merges of pass 2 wait on shared rather than global loads.
__global__ void __launch_bounds__(kTableThreads) k_sigma_alias(uint32_t n, const uint4 *__restrict__ vert,
                                                              const uint32_t *__restrict__ acc, uint4 *slot) {
    __shared__ uint64_t s_pre[kTableThreads / kWarp][kLongList];
    __shared__ uint32_t s_idx[kTableThreads / kWarp][kLongList];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint64_t *pre = s_pre[warp];
    uint32_t *idx = s_idx[warp];
    const uint32_t below = (1u << lane) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * wpb;
    uint64_t v = (uint64_t)blockIdx.x * wpb + warp;
    uint4 next = v < n ? vert[v] : make_uint4(0u, 0u, 0u, 0u);
    for (; v < n; v += stride) {
        // the next list's record is loaded while this one is built
        const uint4 vr = next;
        if (v + stride < n) next = vert[v + stride];
        const uint32_t o = vr.x, d = vr.y, S = vr.z;
        if (d == 0 || (d > kLongList && S != 0)) continue;   // long lists: k_sigma_alias_long
        uint32_t *slot32 = reinterpret_cast<uint32_t *>(slot);
        if (S == 0) {  // never drawn (Gamma_v = 0): keep every column
            for (uint32_t p = lane; p < d; p += kWarp) set_sigma(slot32, o, p, 0, p);
            continue;
        }
        const uint64_t W = S;
        // pass 1: split into lights (front) and heavies (back) with prefixes
        uint32_t nl = 0, nh = 0;
        uint64_t Arun = 0, Prun = 0;
        for (uint32_t base = 0; base < d; base += kWarp) {
            const uint32_t j = base + lane;
            uint64_t qj = 0;
            bool valid = j < d, light = false;
            if (valid) {
                qj = (uint64_t)acc_weight(acc, o, d, S, j) * d;
                light = qj < W;
            }
            const uint32_t lmask = __ballot_sync(0xffffffffu, valid && light);
            const uint32_t hmask = __ballot_sync(0xffffffffu, valid && !light);
            const uint64_t D = valid && light ? W - qj : 0;
            const uint64_t E = valid && !light ? qj - W : 0;
            const uint64_t Dincl = warp_incl_scan64(D, lane);
            const uint64_t Eincl = warp_incl_scan64(E, lane);
            if (valid && light) {
                const uint32_t r = nl + __popc(lmask & below);
                idx[r] = j;
                pre[r] = Arun + Dincl - D;            // exclusive A_i
            } else if (valid) {
                const uint32_t r = nh + __popc(hmask & below);
                idx[d - 1 - r] = j;
                pre[d - 1 - r] = Prun + Eincl;        // inclusive P_k
            }
            nl += __popc(lmask);
            nh += __popc(hmask);
            Arun += __shfl_sync(0xffffffffu, Dincl, 31);
            Prun += __shfl_sync(0xffffffffu, Eincl, 31);
        }
        __syncwarp();
        const uint64_t Ptot = Prun;  // == Arun
        // pass 2: thresholds and aliases.  Lights take the first heavy whose
        // inclusive excess reaches their exclusive deficit, heavies the first
        // light whose deficit exceeds their excess; both sequences are sorted,
        // so each lane merges a contiguous run after one binary search.
        {
            const uint32_t cl = (nl + kWarp - 1) / kWarp;
            const uint32_t i0 = lane * cl, i1 = min(nl, i0 + cl);
            if (i0 < i1) {
                const uint64_t A0 = pre[i0];
                uint32_t k = 0, len = nh;           // first heavy k with P_k >= A
                while (len > 0) {
                    const uint32_t half = len >> 1;
                    if (pre[d - 1 - (k + half)] < A0) { k += half + 1; len -= half + 1; } else { len = half; }
                }
                for (uint32_t i = i0; i < i1; ++i) {
                    const uint64_t A = pre[i];
                    while (pre[d - 1 - k] < A) ++k;
                    const uint32_t j = idx[i];
                    set_sigma(slot32, o, j, acc_weight(acc, o, d, S, j) * d, idx[d - 1 - k]);
                }
            }
        }
        {
            const uint32_t ch = (nh + kWarp - 1) / kWarp;
            const uint32_t k0 = lane * ch, k1 = min(nh, k0 + ch);
            if (k0 < k1) {
                const uint64_t P0 = pre[d - 1 - k0];
                uint32_t i = 0, len = nl;           // first light i with A_i > P_k
                while (len > 0) {
                    const uint32_t half = len >> 1;
                    if (pre[i + half] <= P0) { i += half + 1; len -= half + 1; } else { len = half; }
                }
                for (uint32_t k = k0; k < k1; ++k) {
                    const uint64_t Pk = pre[d - 1 - k];
                    while (i < nl && pre[i] <= Pk) ++i;
                    const uint32_t j = idx[d - 1 - k];
                    uint32_t thr, alias;
                    if (Pk < Ptot) {
                        const uint64_t Ai = i < nl ? pre[i] : Ptot;
                        thr = (uint32_t)(W + Pk - Ai);
                        alias = idx[d - 1 - (k + 1)];
                    } else {
                        thr = (uint32_t)W;
                        alias = j;
                    }
                    set_sigma(slot32, o, j, thr, alias);
                }
            }
        }
        __syncwarp();
    }
}

// lists longer than kLongList: a block per list (moss_alias.cuh); a list of
// at most kLongSmemList entries keeps its split in dynamic shared memory, a
// longer one in its range of the global scratch (idx, pre).  The grid has a
// block per kSigmaChunk vertices, so the hardware scheduler spreads the long
// lists over the SMs as blocks finish instead of a fixed share per block.
constexpr uint32_t kLongSmemList = 4096;
constexpr size_t kLongSmemBytes = (size_t)kLongSmemList * (sizeof(uint64_t) + sizeof(uint32_t));
constexpr int kSigmaChunk = 32;

__global__ void __launch_bounds__(kLongThreads) k_sigma_alias_long(uint32_t n, const uint4 *__restrict__ vert,
                                                                  const uint32_t *__restrict__ acc, uint4 *slot,
                                                                  uint32_t *idx, uint64_t *pre) {
    extern __shared__ uint64_t s_split[];   // kLongSmemList pre, then kLongSmemList idx
    uint32_t *slot32 = reinterpret_cast<uint32_t *>(slot);
    for_each_vertex<kLongThreads, kSigmaChunk>(
        n, vert, [](uint4 vr) { return vr.y > kLongList && vr.z != 0; },
        [&](uint32_t v) {
            const uint4 vr = vert[v];
            const uint32_t o = vr.x, d = vr.y, S = vr.z;
            const bool fits = d <= kLongSmemList;
            block_alias<uint64_t, kLongThreads>(
                d, (uint64_t)S, [&](uint32_t j) { return (uint64_t)acc_weight(acc, o, d, S, j); },
                fits ? reinterpret_cast<uint32_t *>(s_split + kLongSmemList) : idx + o, fits ? s_split : pre + o,
                [&](uint32_t j, uint64_t thr, uint32_t alias) {
                    set_sigma(slot32, o, j, (uint32_t)thr, alias);
                });
        });
}

// One thread per slot: words 5..7 of each record from words 0, 1 and 4 of
// its alias position's record (written before this launch, read only here).
__global__ void k_slot_alias_fill(uint64_t nnz, const uint4 *__restrict__ vert, const uint32_t *__restrict__ owner,
                                  uint4 *slot) {
    uint32_t *s32 = reinterpret_cast<uint32_t *>(slot);
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = (uint64_t)vert[owner[p]].x + s32[8 * p + 3];
        const uint32_t col = s32[8 * a], nb = s32[8 * a + 1], off = s32[8 * a + 4];
        s32[8 * p + 5] = col;
        *reinterpret_cast<uint2 *>(s32 + 8 * p + 6) = make_uint2(nb, off);
    }
}

// ---------------------------------------------------- vertex (seed) tables ---
constexpr int kSeedThreads = 256;
constexpr int kSeedRounds = 16;                              // items per thread per block
constexpr uint32_t kSeedChunk = kSeedThreads * kSeedRounds;  // items per block

struct SeedSplit {
    uint32_t nl, nh;
    u128 total;  // sum of deficits == sum of excesses
};

// per-block aggregate of one contiguous chunk: lights, heavies, sum D, sum E
struct alignas(16) SeedAgg {
    u128 D, E;
    uint32_t nl, nh, pad0, pad1;
};

// One level of one vertex table being built: weights, output, and its
// scratch.  Items are the level's columns: item j is column base + j, the
// vertex perm[base + j], with weight w[vertex]; base, the item count and the
// level's total are read from the table's SeedLevel (filled by the split
// kernels before).
struct SeedTask {
    const u128 *w;
    uint4 *seed;           // 2 per column: {T lo, T hi, alias, self} and the alias's vertex record
    const uint4 *vrec;     // vertex records copied into seed
    const uint32_t *perm;  // column -> vertex (heavy ids ascending, then light ids ascending); null: identity
    int level;             // 0: the heavy columns [0, nh); 1: the light ones [nh, n); 2: one level, all n
    uint32_t *idx;         // items: lights from the front, heavies from the back (of the level's count)
    u128 *pre;             // A_i (lights) / P_k (heavies)
    SeedSplit *split;
    SeedAgg *agg;          // one per chunk
    int which;             // 0 Gamma, 1 Gamma^(1), 2 Gamma^(2), 3 Gamma-check
};
struct SeedTasks {
    SeedTask t[2 * 3];
};

__device__ __forceinline__ uint32_t task_base(const SeedTask &T, const DevTotals *tot) {
    return T.level == 1 ? tot->level[T.which].nh : 0u;
}
__device__ __forceinline__ uint32_t task_items(const SeedTask &T, const DevTotals *tot, uint32_t n) {
    return T.level == 2 ? n : T.level == 1 ? n - tot->level[T.which].nh : tot->level[T.which].nh;
}
__device__ __forceinline__ u128 task_total(const SeedTask &T, const DevTotals *tot) {
    return T.level == 2 ? tot->gamma[T.which] : T.level == 1 ? tot->level[T.which].WL : tot->level[T.which].WH;
}
__device__ __forceinline__ uint32_t task_vertex(const SeedTask &T, uint32_t column) {
    return T.perm ? T.perm[column] : column;
}

__device__ __forceinline__ void seed_item(const SeedTask &T, uint64_t j, uint32_t m, uint32_t base, u128 W,
                                          bool &light, bool &heavy, u128 &D, u128 &E) {
    light = heavy = false;
    D = E = 0;
    if (j < m) {
        const u128 q = T.w[task_vertex(T, base + (uint32_t)j)] * (u128)m;
        light = q < W;
        heavy = !light;
        if (light) D = W - q; else E = q - W;
    }
}

// exclusive block scan of per-thread counts (lights, heavies) and sums
// (deficits D, excesses E); returns the block totals
__device__ __forceinline__ void block_scan_counts(uint32_t cl, uint32_t ch, u128 D, u128 E, uint32_t &xl,
                                                  uint32_t &xh, u128 &xD, u128 &xE, SeedAgg &tot) {
    __shared__ uint32_t s_l[kSeedThreads / kWarp], s_h[kSeedThreads / kWarp];
    __shared__ u128 s_D[kSeedThreads / kWarp], s_E[kSeedThreads / kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t il = cl, ih = ch;
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, il, d), b = __shfl_up_sync(0xffffffffu, ih, d);
        if (lane >= d) { il += a; ih += b; }
    }
    const u128 Di = warp_incl_scan128(D, lane), Ei = warp_incl_scan128(E, lane);
    if (lane == 31) {
        s_l[warp] = il;
        s_h[warp] = ih;
        s_D[warp] = Di;
        s_E[warp] = Ei;
    }
    __syncthreads();
    uint32_t wl = 0, wh = 0;
    u128 wD = 0, wE = 0;
    tot.nl = tot.nh = 0;
    tot.D = tot.E = 0;
    for (int k = 0; k < kSeedThreads / kWarp; ++k) {
        if (k < warp) {
            wl += s_l[k];
            wh += s_h[k];
            wD += s_D[k];
            wE += s_E[k];
        }
        tot.nl += s_l[k];
        tot.nh += s_h[k];
        tot.D += s_D[k];
        tot.E += s_E[k];
    }
    xl = wl + il - cl;
    xh = wh + ih - ch;
    xD = wD + Di - D;
    xE = wE + Ei - E;
    __syncthreads();
}

// floor(thr 2^64 / W) for thr < W by binary long division
__device__ __noinline__ uint64_t quantize64_long(u128 thr, u128 W) {
    uint64_t qq = 0;
    u128 r = thr;
    for (int i = 0; i < 64; ++i) {
        const bool carry = (uint64_t)(r >> 127) != 0;
        r <<= 1;
        qq <<= 1;
        if (carry || r >= W) { r -= W; qq |= 1; }
    }
    return qq;
}

__device__ __forceinline__ double u128_to_double(u128 x) {
    return (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x;
}

// thr 2^64 - q W as a signed 192-bit number: (hi, lo), hi's sign its sign
__device__ __forceinline__ void quantize_rem(u128 thr, u128 W, uint64_t q, int64_t &hi, u128 &lo) {
    const u128 p0 = (u128)q * (uint64_t)W, p1 = (u128)q * (uint64_t)(W >> 64);
    const u128 blo = p0 + (p1 << 64);
    const uint64_t bhi = (uint64_t)(p1 >> 64) + (blo < p0 ? 1u : 0u);
    const u128 alo = (u128)(uint64_t)thr << 64;
    const uint64_t ahi = (uint64_t)(thr >> 64);
    lo = alo - blo;
    hi = (int64_t)(ahi - bhi - (alo < blo ? 1u : 0u));
}

// floor(thr 2^64 / W) for thr <= W, saturated: a double estimate (53 good
// bits), one correction from the exact remainder, then at most a few unit
// steps -- the long division when they do not settle
__device__ __forceinline__ uint64_t quantize64(u128 thr, u128 W) {
    if (W == 0) return 0;
    if (thr >= W) return ~0ULL;
    const double dw = u128_to_double(W);
    const double est = u128_to_double(thr) / dw * 18446744073709551616.0;
    uint64_t q = est >= 18446744073709549568.0 ? ~0ULL : (uint64_t)est;
    int64_t hi;
    u128 lo;
    quantize_rem(thr, W, q, hi, lo);
    // the remainder is a few thousand W at most: its quotient by W in
    // doubles, from its magnitude (the two halves of a negative one would
    // cancel in a double)
    double rem;
    if (hi < 0) {
        const u128 nlo = ~lo + 1;
        const uint64_t nhi = ~(uint64_t)hi + (nlo == 0 ? 1u : 0u);
        rem = -((double)nhi * 340282366920938463463374607431768211456.0 + u128_to_double(nlo));
    } else {
        rem = (double)hi * 340282366920938463463374607431768211456.0 + u128_to_double(lo);
    }
    const double delta = rem / dw;
    if (delta > -1e6 && delta < 1e6) {
        const int64_t step = (int64_t)floor(delta);
        if (step < 0) q = (uint64_t)(-step) > q ? 0 : q - (uint64_t)(-step);
        else q = (uint64_t)step > ~q ? ~0ULL : q + (uint64_t)step;
        quantize_rem(thr, W, q, hi, lo);
        for (int it = 0; it < 4; ++it) {
            if (hi < 0) {   // remainder below 0: one W too many
                --q;
                const u128 nlo = lo + W;
                hi += nlo < lo ? 1 : 0;
                lo = nlo;
            } else if (hi > 0 || lo >= W) {   // at least W left
                ++q;
                const u128 nlo = lo - W;
                hi -= nlo > lo ? 1 : 0;
                lo = nlo;
            } else {
                return q;
            }
        }
    }
    return quantize64_long(thr, W);
}

// ---- the split into levels (per table): heavy iff w_v >= ceil(W / 2^split)
struct LevelTask {
    const u128 *w;
    uint32_t *perm;
    SeedAgg *agg;          // per chunk: nh (heavies) and E (their weight), then their exclusive offsets
    int which;
};
struct LevelTasks {
    LevelTask t[3];
};

__device__ __forceinline__ u128 heavy_cut(u128 W, int split) {
    u128 c = W >> split;
    if ((c << split) != W) c += 1;
    return c;
}

// per-chunk count and weight of the heavy vertices (and the overflow check
// of the whole table: w_v n must fit 128 bits)
__global__ void __launch_bounds__(kSeedThreads) k_level_count(uint32_t n, const DevTotals *tot, LevelTasks tasks,
                                                             int split, uint32_t *flags) {
    const LevelTask &T = tasks.t[blockIdx.y];
    const u128 W = tot->gamma[T.which];
    if (blockIdx.x == 0 && threadIdx.x == 0 && n > 1 && W > (~(u128)0) / n) atomicOr(flags, kErrOverflow);
    if (W == 0) return;
    const u128 cut = heavy_cut(W, split);
    const uint64_t base = (uint64_t)blockIdx.x * kSeedChunk;
    // each thread's count and weight over its rounds, then one block sum
    uint32_t nh = 0;
    u128 E = 0;
    for (int r = 0; r < kSeedRounds; ++r) {
        const uint64_t j = base + (uint64_t)r * kSeedThreads + threadIdx.x;
        if (j < n) {
            const u128 w = T.w[j];
            if (w >= cut) {
                ++nh;
                E += w;
            }
        }
    }
    __shared__ uint32_t s_h[kSeedThreads / kWarp];
    __shared__ u128 s_E[kSeedThreads / kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nh += __shfl_down_sync(0xffffffffu, nh, d);
    E = warp_sum128(E);
    if (lane == 0) { s_h[warp] = nh; s_E[warp] = E; }
    __syncthreads();
    if (threadIdx.x == 0) {
        SeedAgg acc;
        acc.nl = 0;
        acc.nh = 0;
        acc.D = 0;
        acc.E = 0;
        for (int k = 0; k < kSeedThreads / kWarp; ++k) { acc.nh += s_h[k]; acc.E += s_E[k]; }
        T.agg[blockIdx.x] = acc;
    }
}

// exclusive offsets of the chunks (one block per table) and the level record
__global__ void __launch_bounds__(kSeedThreads) k_level_offsets(uint32_t chunks, DevTotals *tot, LevelTasks tasks) {
    const LevelTask &T = tasks.t[blockIdx.x];
    const u128 W = tot->gamma[T.which];
    SeedLevel &L = tot->level[T.which];
    if (W == 0) {
        if (threadIdx.x == 0) { L.nh = 0; L.tl = 0; L.WH = 0; L.WL = 0; }
        return;
    }
    __shared__ uint32_t run_h;
    __shared__ u128 run_E;
    __shared__ uint32_t sh[kSeedThreads];
    __shared__ u128 sE[kSeedThreads];
    if (threadIdx.x == 0) { run_h = 0; run_E = 0; }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < chunks; b0 += kSeedThreads) {
        const uint32_t b = b0 + threadIdx.x;
        uint32_t h = 0;
        u128 E = 0;
        if (b < chunks) { h = T.agg[b].nh; E = T.agg[b].E; }
        sh[threadIdx.x] = h;
        sE[threadIdx.x] = E;
        __syncthreads();
        for (int d = 1; d < kSeedThreads; d <<= 1) {   // inclusive scan (Hillis-Steele)
            uint32_t h2 = 0;
            u128 E2 = 0;
            if ((int)threadIdx.x >= d) { h2 = sh[threadIdx.x - d]; E2 = sE[threadIdx.x - d]; }
            __syncthreads();
            sh[threadIdx.x] += h2;
            sE[threadIdx.x] += E2;
            __syncthreads();
        }
        if (b < chunks) {
            T.agg[b].nh = run_h + sh[threadIdx.x] - h;
            T.agg[b].E = run_E + sE[threadIdx.x] - E;
        }
        __syncthreads();
        if (threadIdx.x == kSeedThreads - 1) { run_h += sh[threadIdx.x]; run_E += sE[threadIdx.x]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        L.nh = run_h;
        L.WH = run_E;
        L.WL = W - run_E;
        L.tl = run_h ? quantize64(W - run_E, W) : 0;
    }
}

// column order: every heavy vertex at its rank among the heavies, every light
// one at nh + its rank among the lights (a table of total 0: the identity)
__global__ void __launch_bounds__(kSeedThreads) k_level_place(uint32_t n, const DevTotals *tot, LevelTasks tasks,
                                                             int split) {
    const LevelTask &T = tasks.t[blockIdx.y];
    const u128 W = tot->gamma[T.which];
    const uint64_t base = (uint64_t)blockIdx.x * kSeedChunk;
    if (W == 0) {
        for (int r = 0; r < kSeedRounds; ++r) {
            const uint64_t j = base + (uint64_t)r * kSeedThreads + threadIdx.x;
            if (j < n) T.perm[j] = (uint32_t)j;
        }
        return;
    }
    const u128 cut = heavy_cut(W, split);
    const uint32_t nh = tot->level[T.which].nh;
    uint32_t before = T.agg[blockIdx.x].nh;   // heavies in earlier chunks
    __shared__ uint32_t s_w[2][kSeedThreads / kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < kSeedRounds; ++r) {
        const uint64_t j = base + (uint64_t)r * kSeedThreads + threadIdx.x;
        const bool heavy = j < n && T.w[j] >= cut;
        // rank among the round's heavies: a ballot per warp, the warps'
        // counts through shared memory (double-buffered: one barrier a round)
        const uint32_t b = __ballot_sync(0xffffffffu, heavy);
        if (lane == 0) s_w[r & 1][warp] = __popc(b);
        __syncthreads();
        uint32_t xh = __popc(b & ((1u << lane) - 1u)), total = 0;
        for (int k = 0; k < kSeedThreads / kWarp; ++k) {
            const uint32_t c = s_w[r & 1][k];
            if (k < warp) xh += c;
            total += c;
        }
        if (j < n) {
            const uint32_t hb = before + xh;   // heavies before j
            T.perm[heavy ? hb : nh + ((uint32_t)j - hb)] = (uint32_t)j;
        }
        before += total;
    }
}

// ---- the alias table of each level, in four phases (closed form of the sweep)
// phase 1: per-chunk aggregates
__global__ void __launch_bounds__(kSeedThreads) k_seed_count(uint32_t n, const DevTotals *tot, SeedTasks tasks,
                                                            uint32_t *flags) {
    const SeedTask &T = tasks.t[blockIdx.y];
    const u128 W = task_total(T, tot);
    // one level: the overflow check of the table (w_v n must fit 128 bits) is here
    if (flags && blockIdx.x == 0 && threadIdx.x == 0 && n > 1 && W > (~(u128)0) / n) atomicOr(flags, kErrOverflow);
    if (W == 0) return;
    const uint32_t m = task_items(T, tot, n), b0 = task_base(T, tot);
    const uint64_t base = (uint64_t)blockIdx.x * kSeedChunk;
    // each thread's counts and deficit/excess sums, then one block sum
    uint32_t cl = 0, ch = 0;
    u128 sD = 0, sE = 0;
    for (int r = 0; r < kSeedRounds; ++r) {
        bool light, heavy;
        u128 D, E;
        seed_item(T, base + (uint64_t)r * kSeedThreads + threadIdx.x, m, b0, W, light, heavy, D, E);
        cl += light;
        ch += heavy;
        sD += D;
        sE += E;
    }
    uint32_t xl, xh;
    u128 xD, xE;
    SeedAgg t;
    block_scan_counts(cl, ch, sD, sE, xl, xh, xD, xE, t);
    if (threadIdx.x == 0) T.agg[blockIdx.x] = t;
}

// phase 2: exclusive scan of the chunk aggregates (one block per level)
__global__ void __launch_bounds__(kSeedThreads) k_seed_offsets(uint32_t chunks, const DevTotals *tot,
                                                              SeedTasks tasks) {
    const SeedTask &T = tasks.t[blockIdx.x];
    if (T.level == 2 && threadIdx.x == 0) {   // one level: the record says so (no heavy vertex)
        SeedLevel &L = const_cast<DevTotals *>(tot)->level[T.which];
        L.nh = 0;
        L.tl = 0;
        L.WH = 0;
        L.WL = tot->gamma[T.which];
    }
    if (task_total(T, tot) == 0) {
        if (threadIdx.x == 0) { T.split->nl = 0; T.split->nh = 0; T.split->total = 0; }
        return;
    }
    __shared__ SeedAgg run;
    if (threadIdx.x == 0) { run.nl = run.nh = 0; run.D = run.E = 0; }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < chunks; b0 += kSeedThreads) {
        const uint32_t b = b0 + threadIdx.x;
        SeedAgg a;
        a.nl = a.nh = 0;
        a.D = a.E = 0;
        if (b < chunks) a = T.agg[b];
        // inclusive scan of the four fields through shared memory (Hillis-Steele)
        __shared__ uint32_t sl[kSeedThreads], sh[kSeedThreads];
        __shared__ u128 sD[kSeedThreads], sE[kSeedThreads];
        sl[threadIdx.x] = a.nl; sh[threadIdx.x] = a.nh; sD[threadIdx.x] = a.D; sE[threadIdx.x] = a.E;
        __syncthreads();
        for (int d = 1; d < kSeedThreads; d <<= 1) {
            uint32_t l2 = 0, h2 = 0;
            u128 D2 = 0, E2 = 0;
            if ((int)threadIdx.x >= d) {
                l2 = sl[threadIdx.x - d]; h2 = sh[threadIdx.x - d]; D2 = sD[threadIdx.x - d]; E2 = sE[threadIdx.x - d];
            }
            __syncthreads();
            sl[threadIdx.x] += l2; sh[threadIdx.x] += h2; sD[threadIdx.x] += D2; sE[threadIdx.x] += E2;
            __syncthreads();
        }
        if (b < chunks) {
            SeedAgg ex;
            ex.nl = run.nl + sl[threadIdx.x] - a.nl;
            ex.nh = run.nh + sh[threadIdx.x] - a.nh;
            ex.D = run.D + sD[threadIdx.x] - a.D;
            ex.E = run.E + sE[threadIdx.x] - a.E;
            T.agg[b] = ex;   // now the chunk's exclusive offsets
        }
        __syncthreads();
        if (threadIdx.x == kSeedThreads - 1) {
            run.nl += sl[threadIdx.x]; run.nh += sh[threadIdx.x]; run.D += sD[threadIdx.x]; run.E += sE[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        T.split->nl = run.nl;
        T.split->nh = run.nh;
        T.split->total = run.E;
    }
}

// phase 3: place every item at its split position with its prefix
__global__ void __launch_bounds__(kSeedThreads) k_seed_place(uint32_t n, const DevTotals *tot, SeedTasks tasks) {
    const SeedTask &T = tasks.t[blockIdx.y];
    const u128 W = task_total(T, tot);
    if (W == 0) return;
    const uint32_t m = task_items(T, tot, n), b0 = task_base(T, tot);
    // thread t takes kSeedRounds consecutive items of the chunk: its counts
    // and sums, one block scan of them, then the items again in order
    const uint64_t first = (uint64_t)blockIdx.x * kSeedChunk + (uint64_t)threadIdx.x * kSeedRounds;
    uint32_t cl = 0, ch = 0;
    u128 sD = 0, sE = 0;
    for (int r = 0; r < kSeedRounds; ++r) {
        bool light, heavy;
        u128 D, E;
        seed_item(T, first + r, m, b0, W, light, heavy, D, E);
        cl += light;
        ch += heavy;
        sD += D;
        sE += E;
    }
    uint32_t xl, xh;
    u128 xD, xE;
    SeedAgg t;
    block_scan_counts(cl, ch, sD, sE, xl, xh, xD, xE, t);
    const SeedAgg off = T.agg[blockIdx.x];
    uint32_t rl = off.nl + xl, rh = off.nh + xh;
    u128 A = off.D + xD, P = off.E + xE;
    for (int r = 0; r < kSeedRounds; ++r) {
        const uint64_t j = first + r;
        bool light, heavy;
        u128 D, E;
        seed_item(T, j, m, b0, W, light, heavy, D, E);
        if (light) {
            T.idx[rl] = (uint32_t)j;
            T.pre[rl] = A;                                 // exclusive A_i
            ++rl;
            A += D;
        } else if (heavy) {
            P += E;
            T.idx[m - 1 - rh] = (uint32_t)j;
            T.pre[m - 1 - rh] = P;                         // inclusive P_k
            ++rh;
        }
    }
}

// phase 4: thresholds and aliases, one thread per position of the split
// order; records {T lo, T hi, alias, self} + the alias's vertex record at the
// item's column
__global__ void k_seed_fill(uint32_t n, const DevTotals *tot, SeedTasks tasks) {
    const SeedTask &T = tasks.t[blockIdx.y];
    const u128 W = task_total(T, tot);
    const uint32_t m = task_items(T, tot, n), b0 = task_base(T, tot);
    const uint32_t *idx = T.idx;
    const u128 *pre = T.pre;
    const uint32_t nl = T.split->nl, nh = T.split->nh;
    const u128 Ptot = T.split->total;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
        if (W == 0) {   // a level without weight is never drawn
            const uint32_t v = task_vertex(T, b0 + (uint32_t)p);
            T.seed[2 * (uint64_t)(b0 + p)] = make_uint4(0u, 0u, v, v);
            T.seed[2 * (uint64_t)(b0 + p) + 1] = T.vrec[v];
            continue;
        }
        const uint32_t j = idx[p];
        u128 thr;
        uint32_t alias;
        if (p < nl) {
            const u128 A = pre[p];
            uint32_t lo = 0, len = nh;
            while (len > 0) {
                uint32_t half = len >> 1;
                if (pre[m - 1 - (lo + half)] < A) { lo += half + 1; len -= half + 1; } else { len = half; }
            }
            thr = T.w[task_vertex(T, b0 + j)] * (u128)m;
            alias = idx[m - 1 - lo];
        } else {
            const uint32_t k = (uint32_t)(m - 1 - p);
            const u128 Pk = pre[p];
            if (Pk < Ptot) {
                uint32_t lo = 0, len = nl;
                while (len > 0) {
                    uint32_t half = len >> 1;
                    if (pre[lo + half] <= Pk) { lo += half + 1; len -= half + 1; } else { len = half; }
                }
                const u128 Ai = lo < nl ? pre[lo] : Ptot;
                thr = W + Pk - Ai;
                alias = idx[m - 1 - (k + 1)];
            } else {
                thr = W;
                alias = j;
            }
        }
        const uint64_t Tq = quantize64(thr, W);
        const uint32_t av = task_vertex(T, b0 + alias), sv = task_vertex(T, b0 + j);
        T.seed[2 * (uint64_t)(b0 + j)] = make_uint4((uint32_t)Tq, (uint32_t)(Tq >> 32), av, sv);
        T.seed[2 * (uint64_t)(b0 + j) + 1] = T.vrec[av];
    }
}

// ---- hub adjacency (behind the edge filter)
constexpr uint32_t kHubBins = 65536;    // degree histogram, degrees >= 65535 in the last bin
constexpr uint32_t kHubSmallBins = 2048;  // counted in shared memory first
constexpr uint32_t kHubWarpWords = 16;    // rank-table entries (32 vertices each) per warp
constexpr uint32_t kHubBlockWarps = 8;

__global__ void __launch_bounds__(256) k_hub_hist(uint32_t n, const uint4 *__restrict__ vert, uint32_t *hist) {
    __shared__ uint32_t sh[kHubSmallBins];
    for (uint32_t b = threadIdx.x; b < kHubSmallBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t d = vert[v].y;
        if (d < kHubSmallBins) {
            if (d) atomicAdd(sh + d, 1u);
        } else {
            atomicAdd(hist + (d < kHubBins - 1 ? d : kHubBins - 1), 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kHubSmallBins; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, sh[b]);
}

// the smallest degree D >= 1 with at most `hubs` vertices of degree >= D
// (kHubBins when even the last bin holds more): one block of 1,024 threads,
// 64 bins each (read as 16 independent 16-byte loads), a suffix scan of the
// threads' totals; only the thread whose bins hold the crossing walks them
__global__ void __launch_bounds__(1024) k_hub_cut(const uint32_t *hist, uint32_t hubs, uint32_t *cut) {
    __shared__ uint32_t suf[1024];
    __shared__ uint32_t best;
    const uint32_t t = threadIdx.x, b0 = t * 64;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist + b0);
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint4 x = h4[q];
        s += x.x + x.y + x.z + x.w;
    }
    suf[t] = s;
    if (t == 0) best = kHubBins;
    __syncthreads();
    for (uint32_t d = 1; d < 1024; d <<= 1) {   // inclusive suffix scan (Hillis-Steele)
        const uint32_t x = t + d < 1024 ? suf[t + d] : 0;
        __syncthreads();
        suf[t] += x;
        __syncthreads();
    }
    const uint32_t above = suf[t] - s;   // vertices with degree in higher threads' bins
    uint32_t mine = kHubBins;
    if (suf[t] <= hubs) {                 // every bin of this thread qualifies
        mine = b0 >= 1 ? b0 : 1u;
    } else if (above <= hubs) {           // the crossing lies in this thread's bins
        uint32_t run = above;
        for (int b = (int)b0 + 63; b >= (int)b0; --b) {
            run += hist[b];
            if (run > hubs) break;
            if (b >= 1) mine = (uint32_t)b;
        }
    }
    atomicMin(&best, mine);
    __syncthreads();
    if (t == 0) *cut = best;
}

// rank-table bits: warp w of the grid takes entries [w kHubWarpWords, +kHubWarpWords),
// a ballot of deg >= D per 32 vertices; its hub count goes to warps[w]
__global__ void __launch_bounds__(256) k_hub_words(uint32_t n, const uint4 *__restrict__ vert, const uint32_t *cut,
                                                   uint2 *rank, uint32_t words, uint32_t *warps) {
    const uint32_t D = *cut, lane = threadIdx.x & 31;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t e0 = w * kHubWarpWords;
    uint32_t count = 0;
    for (uint32_t e = e0; e < e0 + kHubWarpWords && e < words; ++e) {
        const uint64_t v = (uint64_t)e * 32 + lane;
        const bool hub = D < kHubBins && v < n && vert[v].y >= D;
        const uint32_t bits = __ballot_sync(0xffffffffu, hub);
        if (lane == 0) rank[e].y = bits;
        count += __popc(bits);
    }
    if (lane == 0 && e0 < words) warps[w] = count;
}

// exclusive scan of the warps' hub counts (one block of 1,024, tile by tile);
// total -> *count
__global__ void __launch_bounds__(1024) k_hub_offsets(uint32_t nwarps, uint32_t *warps, uint32_t *count) {
    __shared__ uint32_t sh[1024];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nwarps; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < nwarps ? warps[i] : 0u;
        sh[threadIdx.x] = x;
        __syncthreads();
        for (uint32_t d = 1; d < 1024; d <<= 1) {   // inclusive prefix (Hillis-Steele)
            const uint32_t y = threadIdx.x >= d ? sh[threadIdx.x - d] : 0u;
            __syncthreads();
            sh[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nwarps) warps[i] = carry + sh[threadIdx.x] - x;
        const uint32_t total = sh[1023];
        __syncthreads();
        carry += total;
    }
    if (threadIdx.x == 0) *count = carry;
}

// rank-table prefixes and the hub list (ascending ids), warp by warp from
// the scanned counts; list entries past `hubs` (the table's capacity) are
// never written, as the cut keeps the hubs at or below it
__global__ void __launch_bounds__(256) k_hub_place(uint2 *rank, uint32_t words, const uint32_t *warps,
                                                   uint32_t *list, uint32_t hubs) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t e0 = w * kHubWarpWords;
    if (e0 >= words) return;
    uint32_t run = warps[w];
    for (uint32_t e = e0; e < e0 + kHubWarpWords && e < words; ++e) {
        const uint32_t bits = rank[e].y;
        if (lane == 0) rank[e].x = run;
        if (bits >> lane & 1u) {
            const uint32_t i = run + __popc(bits & ((1u << lane) - 1u));
            if (i < hubs) list[i] = e * 32 + lane;
        }
        run += __popc(bits);
    }
}

// a block per hub i: bit i H + j for every hub j in N_(hub i)
__global__ void __launch_bounds__(256) k_hub_bits(const uint32_t *list, const uint32_t *count, uint32_t hubs,
                                                  const uint4 *__restrict__ vert, const uint32_t *__restrict__ col,
                                                  const uint2 *rank, uint32_t *bits) {
    const uint32_t nh = *count;
    for (uint32_t i = blockIdx.x; i < nh && i < hubs; i += gridDim.x) {
        const uint4 r = vert[list[i]];
        for (uint32_t k = threadIdx.x; k < r.y; k += blockDim.x) {
            const uint32_t x = col[r.x + k];
            const uint32_t j = hub_index(rank[x >> 5], x);
            if (j != kNoHub) {
                const uint64_t bit = (uint64_t)i * hubs + j;
                atomicOr(bits + (bit >> 5), 1u << (bit & 31));
            }
        }
    }
}

}  // namespace

// ------------------------------------------------------------- launches ---
int table_blocks(uint32_t n) {
    const int sms = current_sms();
    const uint64_t warps_needed = (uint64_t)n;
    uint64_t blocks = (warps_needed + (kTableThreads / kWarp) - 1) / (kTableThreads / kWarp);
    const uint64_t cap = (uint64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

cudaError_t launch_vertices(const void *row_ptr, int is64, uint32_t n, uint64_t nnz, uint4 *vert, uint32_t *flags,
                            cudaStream_t s) {
    const int threads = 256;
    uint64_t blocks = ((uint64_t)n + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    if (is64)
        k_vertices<uint64_t><<<(unsigned)blocks, threads, 0, s>>>(static_cast<const uint64_t *>(row_ptr), n, nnz,
                                                                   vert, flags);
    else
        k_vertices<uint32_t><<<(unsigned)blocks, threads, 0, s>>>(static_cast<const uint32_t *>(row_ptr), n, nnz,
                                                                   vert, flags);
    return cudaGetLastError();
}

static unsigned long_blocks(uint32_t n);
int slot_partial_rows(uint32_t n) { return table_blocks(n); }   // k_vertex_weights' rows

static unsigned long_blocks(uint32_t n) {
    const int sms = current_sms();
    const uint64_t cap = (uint64_t)sms * 4, chunks = ((uint64_t)n + kLongThreads - 1) / kLongThreads;
    return (unsigned)(chunks < cap ? (chunks ? chunks : 1) : cap);
}

static unsigned flat_blocks(uint64_t items) {
    const int sms = current_sms();
    uint64_t b = (items + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

cudaError_t launch_slots(uint32_t n, uint64_t nnz, const uint32_t *col, uint4 *vert, uint4 *slot, uint32_t *acc,
                         uint32_t *owner, uint64_t *sq, u128 *gam0, u128 *gam1, u128 *gam2, u128 *partials,
                         int blocks, uint32_t *flags, cudaStream_t s, const AuxStreams *aux) {
    k_owner<<<blocks, kTableThreads, 0, s>>>(n, vert, owner);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nnz) {
        k_slot_weights<<<flat_blocks(nnz), 256, 0, s>>>(n, nnz, col, vert, owner, slot, acc, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the twin pass touches none of what the list scans write, and the short
    // and long list scans touch different lists and rows: all three run side
    // by side on the auxiliary streams when there are some
    const bool forked = aux && aux->fork(s) == cudaSuccess;
    if (aux && !forked) cudaGetLastError();
    cudaStream_t ts = forked ? aux->a[0] : s, ls = forked ? aux->a[1] : s;
    if (nnz) k_twin<<<flat_blocks(nnz), 256, 0, ts>>>(n, nnz, vert, col, owner, slot, flags);
    cudaError_t et = cudaGetLastError();
    k_slots_long<<<long_blocks(n), kLongThreads, 0, ls>>>(n, vert, acc, sq, gam2);
    cudaError_t el = cudaGetLastError();
    k_slots<<<blocks, kTableThreads, 0, s>>>(n, vert, acc, sq, gam2);
    e = cudaGetLastError();
    if (forked) {
        const cudaError_t ej = aux->join(s);
        if (e == cudaSuccess) e = ej;
    }
    if (e == cudaSuccess && et == cudaSuccess && el == cudaSuccess) {
        k_vertex_weights<<<blocks, kTableThreads, 0, s>>>(n, vert, gam0, gam1, gam2, partials);
        e = cudaGetLastError();
    }
    return e != cudaSuccess ? e : (et != cudaSuccess ? et : el);
}

cudaError_t launch_totals(const u128 *partials, int blocks, DevTotals *tot, cudaStream_t s) {
    k_totals<<<1, kTotalsThreads, 0, s>>>(partials, blocks, tot);
    return cudaGetLastError();
}

cudaError_t launch_edge_hash(uint64_t nnz, const uint32_t *col, const uint32_t *owner, unsigned long long *table,
                             uint32_t mask, uint32_t shift, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_edge_hash<<<flat_blocks(nnz), 256, 0, s>>>(nnz, col, owner, table, mask, shift);
    return cudaGetLastError();
}

cudaError_t launch_edge_filter(uint64_t nnz, const uint32_t *col, const uint32_t *owner, uint32_t *filter,
                               uint32_t shift, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_edge_filter<<<flat_blocks(nnz), 256, 0, s>>>(nnz, col, owner, filter, shift);
    return cudaGetLastError();
}

static uint64_t hub_words(uint32_t n) { return ((uint64_t)n + 31) / 32; }
static uint64_t hub_warps(uint32_t n) { return (hub_words(n) + kHubWarpWords - 1) / kHubWarpWords; }

uint64_t hub_bytes(uint32_t n) {
    const uint64_t h = hub_capacity(n);
    auto up = [](uint64_t b) { return (b + 255) & ~(uint64_t)255; };
    return up((hub_words(n) + 1) * 8) + up((h * h + 31) / 32 * 4) + up(h * 4) + up((uint64_t)kHubBins * 4) +
           up(hub_warps(n) * 4 + 4) + up(8);
}

cudaError_t launch_hub_tables(uint32_t n, const uint4 *vert, const uint32_t *col, void *mem, uint2 **rank_out,
                              uint32_t **bits_out, uint32_t **list_out, cudaStream_t s) {
    const uint32_t H = hub_capacity(n);
    const uint64_t words = hub_words(n), nwarps = hub_warps(n), bwords = ((uint64_t)H * H + 31) / 32;
    uint8_t *p = static_cast<uint8_t *>(mem);
    auto take = [&](uint64_t bytes) {
        uint8_t *r = p;
        p += (bytes + 255) & ~(uint64_t)255;
        return r;
    };
    uint2 *rank = reinterpret_cast<uint2 *>(take((words + 1) * 8));
    uint32_t *bits = reinterpret_cast<uint32_t *>(take(bwords * 4));
    uint32_t *list = reinterpret_cast<uint32_t *>(take((uint64_t)H * 4));
    uint32_t *hist = reinterpret_cast<uint32_t *>(take((uint64_t)kHubBins * 4));
    uint32_t *warps = reinterpret_cast<uint32_t *>(take(nwarps * 4 + 4));
    uint32_t *cnt = reinterpret_cast<uint32_t *>(take(8));   // [0] hubs, [1] the degree cut
    cudaError_t e = cudaMemsetAsync(rank, 0, (words + 1) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(list, 0xFF, (uint64_t)H * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, bwords * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, (uint64_t)kHubBins * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 8, s);
    if (e != cudaSuccess) return e;
    if (n) {
        const unsigned vb = (unsigned)std::min<uint64_t>(((uint64_t)n + 255) / 256, 1024);
        k_hub_hist<<<vb, 256, 0, s>>>(n, vert, hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_hub_cut<<<1, 1024, 0, s>>>(hist, H, cnt + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const unsigned wb = (unsigned)((nwarps + kHubBlockWarps - 1) / kHubBlockWarps);
        k_hub_words<<<wb, 32 * kHubBlockWarps, 0, s>>>(n, vert, cnt + 1, rank, (uint32_t)words, warps);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_hub_offsets<<<1, 1024, 0, s>>>((uint32_t)nwarps, warps, cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_hub_place<<<wb, 32 * kHubBlockWarps, 0, s>>>(rank, (uint32_t)words, warps, list, H);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_hub_bits<<<H, 256, 0, s>>>(list, cnt, H, vert, col, rank, bits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    *rank_out = rank;
    *bits_out = bits;
    *list_out = list;
    return cudaSuccess;
}

cudaError_t launch_sigma_alias(uint32_t n, uint64_t nnz, const uint4 *vert, const uint32_t *acc, const uint32_t *owner,
                               uint4 *slot, uint32_t *scratch_idx, uint64_t *scratch_pre, cudaStream_t s,
                               const AuxStreams *aux, int long_stream) {
    // the short and the long lists are built side by side (long lists on
    // aux->a[long_stream], forked from s by the caller); the fill waits for both
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaSuccess;
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_relaxed)) {
        e = cudaFuncSetAttribute(k_sigma_alias_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmemBytes);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_relaxed);
    }
    const unsigned chunks = (unsigned)(((uint64_t)n + kSigmaChunk - 1) / kSigmaChunk);
    cudaStream_t ls = aux ? aux->a[long_stream] : s;
    k_sigma_alias_long<<<chunks ? chunks : 1, kLongThreads, kLongSmemBytes, ls>>>(n, vert, acc, slot, scratch_idx,
                                                                                   scratch_pre);
    cudaError_t el = cudaGetLastError();
    k_sigma_alias<<<table_blocks(n), kTableThreads, 0, s>>>(n, vert, acc, slot);
    e = cudaGetLastError();
    if (aux) {
        const cudaError_t ew = aux->wait_for(s, long_stream);
        if (el == cudaSuccess) el = ew;
    }
    if (e != cudaSuccess) return e;
    if (el != cudaSuccess) return el;
    k_slot_alias_fill<<<flat_blocks(nnz), 256, 0, s>>>(nnz, vert, owner, slot);
    return cudaGetLastError();
}

uint64_t seed_scratch_bytes(uint32_t n) {
    const uint64_t chunks = ((uint64_t)n + kSeedChunk - 1) / kSeedChunk;
    // per table: the column order and the split's chunk aggregates; per level:
    // the split order, its prefixes, its totals and chunk aggregates
    const uint64_t table = (uint64_t)n * 4 + 256 + chunks * sizeof(SeedAgg) + 256;
    const uint64_t level = (uint64_t)n * 4 + 256 + (uint64_t)n * 16 + 256 + sizeof(SeedSplit) + 256 +
                           chunks * sizeof(SeedAgg) + 256;
    return 3 * (table + 2 * level);
}

cudaError_t launch_seed_alias(uint32_t n, DevTotals *tot, int ntables, const int *which, u128 *const *w,
                              uint4 *const *seed, const uint4 *const *vrec, void *scratch, uint32_t *flags, int split,
                              cudaStream_t s) {
    if (ntables < 1 || ntables > 3 || split < 0 || split > 64) return cudaErrorInvalidValue;
    const bool one_level = split == 64;   // one table over all vertices, in id order
    const uint32_t chunks = (uint32_t)(((uint64_t)n + kSeedChunk - 1) / kSeedChunk);
    LevelTasks lt = {};
    SeedTasks tasks = {};
    uint8_t *p = static_cast<uint8_t *>(scratch);
    auto take = [&](uint64_t bytes) {
        uint8_t *r = p;
        p += (bytes + 255) & ~(uint64_t)255;
        return r;
    };
    const int per = one_level ? 1 : 2;   // tasks per table
    for (int t = 0; t < ntables; ++t) {
        LevelTask &L = lt.t[t];
        L.w = w[t];
        L.which = which[t];
        L.perm = one_level ? nullptr : reinterpret_cast<uint32_t *>(take((uint64_t)n * 4));
        L.agg = one_level ? nullptr : reinterpret_cast<SeedAgg *>(take((uint64_t)chunks * sizeof(SeedAgg)));
        for (int level = 0; level < per; ++level) {
            SeedTask &T = tasks.t[per * t + level];
            T.w = w[t];
            T.seed = seed[t];
            T.vrec = vrec[t];
            T.perm = L.perm;
            T.level = one_level ? 2 : level;
            T.which = which[t];
            T.idx = reinterpret_cast<uint32_t *>(take((uint64_t)n * 4));
            T.pre = reinterpret_cast<u128 *>(take((uint64_t)n * 16));
            T.split = reinterpret_cast<SeedSplit *>(take(sizeof(SeedSplit)));
            T.agg = reinterpret_cast<SeedAgg *>(take((uint64_t)chunks * sizeof(SeedAgg)));
        }
    }
    const int nt = per * ntables;
    cudaError_t e = cudaSuccess;
    if (!one_level) {
        k_level_count<<<dim3(chunks, ntables), kSeedThreads, 0, s>>>(n, tot, lt, split, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_level_offsets<<<ntables, kSeedThreads, 0, s>>>(chunks, tot, lt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_level_place<<<dim3(chunks, ntables), kSeedThreads, 0, s>>>(n, tot, lt, split);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_seed_count<<<dim3(chunks, nt), kSeedThreads, 0, s>>>(n, tot, tasks, one_level ? flags : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_seed_offsets<<<nt, kSeedThreads, 0, s>>>(chunks, tot, tasks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_seed_place<<<dim3(chunks, nt), kSeedThreads, 0, s>>>(n, tot, tasks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int threads = 256;
    uint64_t blocks = ((uint64_t)n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_seed_fill<<<dim3((unsigned)blocks, nt), threads, 0, s>>>(n, tot, tasks);
    return cudaGetLastError();
}

}  // namespace moss
