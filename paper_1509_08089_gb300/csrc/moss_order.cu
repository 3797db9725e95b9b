// moss_order.cu -- optional degree ordering of a graph at load.
//
// The samplers reach a vertex about in proportion to its degree (the vertex
// draws of Sec. 4.1.3 and 5.1.4 are weighted by degree polynomials, the list
// draws land on a neighbour per edge), so on a heavy-tailed graph with random
// ids the records they read are scattered: each hot vertex record, slot
// record and list shares its cache lines with cold ones.  Loading in degree
// order renumbers the vertices by a degree key, highest first, before any
// table is built, so the hot records sit together and the tables the samples
// touch occupy fewer lines of L2 and HBM.  The renumbered graph is isomorphic
// to the input and every quantity of Sec. 2 and Table 1 is invariant under
// relabelling; per-sample records are mapped back to input ids.
//
// Key.  key(d) = d for d < 16, else 16 + 4 (L - 5) + the two bits below the
// leading one of d (L = bit length of d): quarter-octave classes, 128 keys
// for 32-bit degrees.  Internal order: key descending, input id ascending.
// Inside one key the input order is kept, so a renumbered list is the input
// list (ascending ids) stably partitioned by its entries' keys, highest key
// first: sorted by internal id without a comparison sort.
//
// Kernels.
//   k_order_count   a block per chunk of 8192 vertices counts the vertices
//                   and sums the degrees of each key (shared atomics), with
//                   the row_ptr checks of the vertex pass.
//   k_order_offsets one block scans the key-major count and degree arrays
//                   (key slot 0 = the highest key): each (key, chunk) cell
//                   becomes its first internal id and first CSR offset.
//   k_order_place   the same chunks again, 1024 vertices per warp in rounds
//                   of 32: each warp's cells first, then per round the rank
//                   among equal-key lanes (match_any) and the degree prefix
//                   over them; writes order, the renumbered row offsets and,
//                   per input vertex, its new id and key slot.
//   k_order_lists   in internal order, so the renumbered lists are written
//                   in order (written scattered by list, in input order, the
//                   pass took 2.35 ms against 1.93 on the 34M-edge graph):
//                   the lists of degree 32 or more a warp each: up to 128
//                   entries ranked in registers (four a lane, one pass),
//                   longer lists by a count over the 128 key slots and a
//                   placing pass in input order; the rest by tiles of 32,
//                   G lanes per list (G a power of two <= 32, the tile's
//                   longest), by rank counting on the renumbered ids.
#include "../../include/moss.h"
#include "moss_internal.cuh"
#include "moss_order.cuh"

namespace moss {

namespace {

constexpr int kOrderKeys = 128;
constexpr int kOrderThreads = 256;
constexpr int kOrderWarps = kOrderThreads / 32;
constexpr int kOrderRounds = 32;   // rounds of 32 vertices per warp and chunk
constexpr uint32_t kOrderChunk = (uint32_t)kOrderWarps * kOrderRounds * 32;   // 8192 vertices
constexpr int kScanThreads = 1024;
constexpr uint32_t kFull = 0xffffffffu;

// 127 - key(d): slot 0 holds the highest degrees
__device__ __forceinline__ uint32_t order_slot(uint32_t d) {
    uint32_t key = d;
    if (d >= 16) {
        const uint32_t L = 32u - (uint32_t)__clz(d);
        key = 16u + 4u * (L - 5u) + ((d >> (L - 3u)) & 3u);
    }
    return (uint32_t)(kOrderKeys - 1) - key;
}

// offset and degree of input vertex v; a row that breaks the row_ptr rules
// (the checks of the vertex pass) is empty and sets kErrRowPtr
template <typename IdxT>
__device__ __forceinline__ uint32_t input_row(const IdxT *rp, uint64_t v, uint32_t n, uint64_t nnz, uint64_t &off,
                                              uint32_t &err) {
    const uint64_t a = rp[v], b = rp[v + 1];
    if (b < a || b > nnz || (v == 0 && a != 0) || (v + 1 == n && b != nnz)) {
        err |= kErrRowPtr;
        off = 0;
        return 0;
    }
    off = a;
    return (uint32_t)(b - a);
}

template <typename IdxT>
__global__ void __launch_bounds__(kOrderThreads) k_order_count(const IdxT *rp, uint32_t n, uint64_t nnz,
                                                               uint32_t chunks, uint32_t *cnt, uint32_t *dsum,
                                                               uint32_t *flags) {
    __shared__ uint32_t s_c[kOrderKeys], s_d[kOrderKeys];
    for (int k = threadIdx.x; k < kOrderKeys; k += blockDim.x) s_c[k] = s_d[k] = 0;
    __syncthreads();
    uint32_t err = 0;
    const uint64_t v0 = (uint64_t)blockIdx.x * kOrderChunk;
    for (uint32_t i = threadIdx.x; i < kOrderChunk; i += blockDim.x) {
        const uint64_t v = v0 + i;
        if (v >= n) break;
        uint64_t off;
        const uint32_t d = input_row(rp, v, n, nnz, off, err);
        const uint32_t sl = order_slot(d);
        atomicAdd(&s_c[sl], 1u);
        atomicAdd(&s_d[sl], d);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kOrderKeys; k += blockDim.x) {
        cnt[(uint64_t)k * chunks + blockIdx.x] = s_c[k];
        dsum[(uint64_t)k * chunks + blockIdx.x] = s_d[k];
    }
    if (err) atomicOr(flags, err);
}

// exclusive scans of cnt and dsum (entries cells each), one block: each warp
// a contiguous range of whole rounds of 32 cells, summed, then rescanned
// round by round from its offset (lane-strided, coalesced loads)
__global__ void __launch_bounds__(kScanThreads) k_order_offsets(uint32_t *cnt, uint32_t *dsum, uint64_t entries) {
    constexpr int kW = kScanThreads / 32;
    __shared__ uint32_t s_a[kW], s_b[kW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t rounds = (entries + 31) / 32, per = (rounds + kW - 1) / kW;
    const uint64_t lo = (uint64_t)warp * per * 32;
    const uint64_t hi = lo + per * 32 < entries ? lo + per * 32 : entries;
    uint32_t a = 0, b = 0;
    for (uint64_t i = lo + lane; i < hi; i += 32) {
        a += cnt[i];
        b += dsum[i];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_xor_sync(kFull, a, d);
        b += __shfl_xor_sync(kFull, b, d);
    }
    if (lane == 0) {
        s_a[warp] = a;
        s_b[warp] = b;
    }
    __syncthreads();
    uint32_t ca = 0, cb = 0;   // the warp's first prefix
    for (int w = 0; w < warp; ++w) {
        ca += s_a[w];
        cb += s_b[w];
    }
    for (uint64_t r = lo; r < hi; r += 32) {
        const uint64_t i = r + lane;
        const uint32_t x = i < hi ? cnt[i] : 0u, y = i < hi ? dsum[i] : 0u;
        uint32_t ix = x, iy = y;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t tx = __shfl_up_sync(kFull, ix, d), ty = __shfl_up_sync(kFull, iy, d);
            if (lane >= d) {
                ix += tx;
                iy += ty;
            }
        }
        if (i < hi) {
            cnt[i] = ca + ix - x;
            dsum[i] = cb + iy - y;
        }
        ca += __shfl_sync(kFull, ix, 31);
        cb += __shfl_sync(kFull, iy, 31);
    }
}

template <typename IdxT>
__global__ void __launch_bounds__(kOrderThreads) k_order_place(const IdxT *rp, uint32_t n, uint64_t nnz,
                                                               uint32_t chunks, const uint32_t *cnt,
                                                               const uint32_t *dsum, uint32_t *order, uint32_t *inv,
                                                               uint8_t *slot_of, uint32_t *rp_out) {
    __shared__ uint32_t s_c[kOrderWarps][kOrderKeys], s_d[kOrderWarps][kOrderKeys];
    for (int k = threadIdx.x; k < kOrderWarps * kOrderKeys; k += blockDim.x) {
        (&s_c[0][0])[k] = 0;
        (&s_d[0][0])[k] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t w0 = (uint64_t)blockIdx.x * kOrderChunk + (uint64_t)warp * (kOrderRounds * 32);
    uint32_t err = 0;   // reported by k_order_count
    for (int r = 0; r < kOrderRounds; ++r) {
        const uint64_t v = w0 + (uint64_t)r * 32 + lane;
        if (v < n) {
            uint64_t off;
            const uint32_t d = input_row(rp, v, n, nnz, off, err);
            const uint32_t sl = order_slot(d);
            atomicAdd(&s_c[warp][sl], 1u);
            atomicAdd(&s_d[warp][sl], d);
        }
    }
    __syncthreads();
    // each warp's first internal id and first offset per key slot
    for (int k = threadIdx.x; k < kOrderKeys; k += blockDim.x) {
        uint32_t rc = cnt[(uint64_t)k * chunks + blockIdx.x], rd = dsum[(uint64_t)k * chunks + blockIdx.x];
        for (int w = 0; w < kOrderWarps; ++w) {
            const uint32_t tc = s_c[w][k], td = s_d[w][k];
            s_c[w][k] = rc;
            s_d[w][k] = rd;
            rc += tc;
            rd += td;
        }
    }
    __syncthreads();
    const uint32_t below = (1u << lane) - 1u;
    for (int r = 0; r < kOrderRounds; ++r) {
        const uint64_t v = w0 + (uint64_t)r * 32 + lane;
        const bool valid = v < n;
        uint32_t d = 0;
        if (valid) {
            uint64_t off;
            d = input_row(rp, v, n, nnz, off, err);
        }
        const uint32_t sl = valid ? order_slot(d) : (uint32_t)kOrderKeys + lane;   // lanes past n: own group
        const uint32_t m = __match_any_sync(kFull, sl);
        uint32_t dpre = 0, dtot = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint32_t dj = __shfl_sync(kFull, d, j);
            if (m >> j & 1u) {
                dtot += dj;
                if (j < lane) dpre += dj;
            }
        }
        uint32_t pos = 0, eoff = 0;
        if (valid) {
            pos = s_c[warp][sl] + __popc(m & below);
            eoff = s_d[warp][sl] + dpre;
        }
        __syncwarp();
        if (valid && (m & below) == 0) {
            s_c[warp][sl] += __popc(m);
            s_d[warp][sl] += dtot;
        }
        __syncwarp();
        if (valid) {
            if (pos < n) {
                order[pos] = (uint32_t)v;
                rp_out[pos] = eoff;
            }
            inv[v] = pos;
            slot_of[v] = (uint8_t)sl;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rp_out[n] = (uint32_t)nnz;
}

// One renumbered list on the whole warp: its d input entries at col_in[a..],
// written at col_out[o..] in internal-id order; up to 128 entries by rank
// counting (one entry a lane, or up to four in registers), longer lists by
// key counts (h: the warp's 128 counters).
__device__ __forceinline__ void list_on_warp(uint32_t d, uint64_t a, uint64_t o, uint32_t n, uint64_t nnz,
                                             const uint32_t *__restrict__ col_in, const uint32_t *__restrict__ inv,
                                             const uint8_t *__restrict__ slot_of, uint32_t *col_out, uint32_t *h,
                                             int lane, uint32_t &err) {
    const uint32_t below = (1u << lane) - 1u;
    if (d <= 32) {
        uint32_t u = 0, x = 0xffffffffu;
        if ((uint32_t)lane < d) {
            u = col_in[a + lane];
            if (u < n) {
                x = inv[u];
            } else {
                err |= kErrRange;
                x = n;   // out of range again: the slot pass rejects it too
            }
        }
        const uint32_t up = __shfl_up_sync(kFull, u, 1);
        if (lane > 0 && (uint32_t)lane < d && up >= u) err |= kErrOrder;
        uint32_t rank = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint32_t xj = __shfl_sync(kFull, x, j);
            rank += ((uint32_t)j < d && xj < x) ? 1u : 0u;
        }
        if ((uint32_t)lane < d && o + rank < nnz) col_out[o + rank] = x;
        return;
    }
    if (d <= 4 * 32) {   // up to four entries a lane, ranked against all d in registers
        const int rounds = (int)((d + 31) / 32);
        uint32_t u[4], x[4], rank[4];
        uint32_t last = 0;   // the entry before this round's first
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t idx = (uint32_t)(r * 32 + lane);
            u[r] = 0;
            x[r] = 0xffffffffu;
            rank[r] = 0;
            if (r < rounds) {
                if (idx < d) {
                    u[r] = col_in[a + idx];
                    if (u[r] < n) {
                        x[r] = inv[u[r]];
                    } else {
                        err |= kErrRange;
                        x[r] = n;
                    }
                }
                const uint32_t up = __shfl_up_sync(kFull, u[r], 1);
                const uint32_t prev = lane ? up : last;
                if (idx < d && idx > 0 && prev >= u[r]) err |= kErrOrder;
                last = __shfl_sync(kFull, u[r], 31);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (q >= rounds) break;
            for (int j = 0; j < 32; ++j) {
                const uint32_t xs = __shfl_sync(kFull, x[q], j);
                const bool in = (uint32_t)(q * 32 + j) < d;
#pragma unroll
                for (int r = 0; r < 4; ++r) rank[r] += (in && xs < x[r]) ? 1u : 0u;
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t idx = (uint32_t)(r * 32 + lane);
            if (idx < d && o + rank[r] < nnz) col_out[o + rank[r]] = x[r];
        }
        return;
    }
    for (int k = lane; k < kOrderKeys; k += 32) h[k] = 0;
    __syncwarp();
    uint32_t last = 0;   // the entry before this round's first
    for (uint32_t base = 0; base < d; base += 32) {
        const uint32_t idx = base + lane;
        uint32_t u = 0;
        if (idx < d) {
            u = col_in[a + idx];
            if (u < n)
                atomicAdd(&h[slot_of[u]], 1u);
            else
                err |= kErrRange;
        }
        const uint32_t up = __shfl_up_sync(kFull, u, 1);
        const uint32_t prev = lane ? up : last;
        if (idx < d && idx > 0 && prev >= u) err |= kErrOrder;
        last = __shfl_sync(kFull, u, 31);
    }
    __syncwarp();
    {   // exclusive scan of the 128 counts, 4 per lane
        const uint32_t c0 = h[4 * lane], c1 = h[4 * lane + 1], c2 = h[4 * lane + 2], c3 = h[4 * lane + 3];
        const uint32_t sum = c0 + c1 + c2 + c3;
        uint32_t incl = sum;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, dd);
            if (lane >= dd) incl += t;
        }
        const uint32_t e = incl - sum;
        h[4 * lane] = e;
        h[4 * lane + 1] = e + c0;
        h[4 * lane + 2] = e + c0 + c1;
        h[4 * lane + 3] = e + c0 + c1 + c2;
    }
    __syncwarp();
    for (uint32_t base = 0; base < d; base += 32) {
        const uint32_t idx = base + lane;
        uint32_t sl = (uint32_t)kOrderKeys + lane, x = 0;
        if (idx < d) {
            const uint32_t u = col_in[a + idx];
            if (u < n) {
                sl = slot_of[u];
                x = inv[u];
            }
        }
        const bool live = sl < (uint32_t)kOrderKeys;
        const uint32_t m = __match_any_sync(kFull, sl);
        const uint32_t pos = live ? h[sl] + __popc(m & below) : 0u;
        __syncwarp();
        if (live && (m & below) == 0) h[sl] += __popc(m);
        __syncwarp();
        if (live && o + pos < nnz) col_out[o + pos] = x;
    }
    __syncwarp();
}

// The internal vertices below *nlong (key >= 20: degree 32 or more, the
// front of the order) take a warp each, grid-stride, so the hubs spread
// over the warps.  The rest go by tiles of 32 consecutive internal vertices
// (their lists are written one after another): when none of a tile's lists
// is longer than G (a power of two <= 32), each group of G lanes takes one
// list, 32 / G lists a round; otherwise (not met: the tail's keys are below
// 20) the warp takes the lists one by one.
constexpr int kLongKeySlot = kOrderKeys - 1 - 19;   // first slot of the keys below 20

template <typename IdxT>
__global__ void __launch_bounds__(kOrderThreads, 8) k_order_lists(const IdxT *rp, uint32_t n, uint64_t nnz,
                                                               const uint32_t *__restrict__ order,
                                                               const uint32_t *__restrict__ rp_out,
                                                               const uint32_t *__restrict__ col_in,
                                                               const uint32_t *__restrict__ inv,
                                                               const uint8_t *__restrict__ slot_of, uint32_t *col_out,
                                                               const uint32_t *nlong_p, uint32_t *flags) {
    __shared__ uint32_t s_h[kOrderWarps][kOrderKeys];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *h = s_h[warp];
    uint32_t err = 0, ignored = 0;
    const uint64_t w0 = (uint64_t)blockIdx.x * kOrderWarps + warp, nw = (uint64_t)gridDim.x * kOrderWarps;
    const uint32_t nlong = *nlong_p < n ? *nlong_p : n;
    for (uint64_t i = w0; i < nlong; i += nw) {
        uint64_t a;
        const uint32_t d = input_row(rp, order[i], n, nnz, a, ignored);
        list_on_warp(d, a, rp_out[i], n, nnz, col_in, inv, slot_of, col_out, h, lane, err);
    }
    const uint64_t tiles = ((uint64_t)(n - nlong) + 31) / 32;
    for (uint64_t t = w0; t < tiles; t += nw) {
        const uint64_t i0 = nlong + t * 32, il = i0 + lane;
        uint32_t dl = 0, ol = 0;
        uint64_t al = 0;
        if (il < n) {
            dl = input_row(rp, order[il], n, nnz, al, ignored);   // row faults: reported by k_order_count
            ol = rp_out[il];
        }
        const uint32_t dmax = __reduce_max_sync(kFull, dl);
        if (dmax > 32) {
            for (int j = 0; j < 32; ++j) {
                const uint32_t d = __shfl_sync(kFull, dl, j), o = __shfl_sync(kFull, ol, j);
                const uint64_t a = __shfl_sync(kFull, al, j);
                list_on_warp(d, a, o, n, nnz, col_in, inv, slot_of, col_out, h, lane, err);   // d = 0 past n
            }
            continue;
        }
        int G = 1;
        while ((uint32_t)G < dmax) G <<= 1;
        const int per = 32 / G, g = lane / G, k = lane % G;
        for (int r = 0; r < G; ++r) {
            const int j = r * per + g;   // this group's list in the tile
            const uint32_t d = __shfl_sync(kFull, dl, j), o = __shfl_sync(kFull, ol, j);
            const uint64_t a = __shfl_sync(kFull, al, j);
            uint32_t u = 0, x = 0xffffffffu;
            if ((uint32_t)k < d) {
                u = col_in[a + k];
                if (u < n) {
                    x = inv[u];
                } else {
                    err |= kErrRange;
                    x = n;
                }
            }
            const uint32_t up = __shfl_up_sync(kFull, u, 1, G);
            if (k > 0 && (uint32_t)k < d && up >= u) err |= kErrOrder;
            uint32_t rank = 0;
            for (int q = 0; q < G; ++q) {
                const uint32_t xq = __shfl_sync(kFull, x, q, G);
                rank += ((uint32_t)q < d && xq < x) ? 1u : 0u;
            }
            if ((uint32_t)k < d && (uint64_t)o + rank < nnz) col_out[(uint64_t)o + rank] = x;
        }
    }
    if (err) atomicOr(flags, err);
}

__global__ void k_map_records(uint32_t *verts, uint64_t count, int words, const uint32_t *__restrict__ order,
                              uint32_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count * 5;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = verts[i];
        if ((int)(i % 5) < words && x < n) verts[i] = order[x];
    }
}

struct OrderScratch {
    uint32_t *inv, *rp, *cnt, *dsum;
    uint8_t *slot_of;
    uint32_t chunks;
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

OrderScratch carve(uint32_t n, void *base, uint64_t *bytes) {
    OrderScratch o{};
    o.chunks = (uint32_t)(((uint64_t)n + kOrderChunk - 1) / kOrderChunk);
    const uint64_t cells = (uint64_t)kOrderKeys * o.chunks;
    uint64_t off = 0;
    auto take = [&](uint64_t b) {
        const uint64_t at = off;
        off = align256(off + b);
        return base ? static_cast<uint8_t *>(base) + at : nullptr;
    };
    o.inv = reinterpret_cast<uint32_t *>(take((uint64_t)n * 4));
    o.rp = reinterpret_cast<uint32_t *>(take(((uint64_t)n + 1) * 4));
    o.cnt = reinterpret_cast<uint32_t *>(take(cells * 4));
    o.dsum = reinterpret_cast<uint32_t *>(take(cells * 4));
    o.slot_of = take(n);
    if (bytes) *bytes = off;
    return o;
}

template <typename IdxT>
cudaError_t order_with(const IdxT *rp, const uint32_t *col_in, uint32_t n, uint64_t nnz, uint32_t *order,
                       uint32_t *col_out, const OrderScratch &o, uint32_t *flags, cudaStream_t s) {
    k_order_count<IdxT><<<o.chunks, kOrderThreads, 0, s>>>(rp, n, nnz, o.chunks, o.cnt, o.dsum, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_order_offsets<<<1, kScanThreads, 0, s>>>(o.cnt, o.dsum, (uint64_t)kOrderKeys * o.chunks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_order_place<IdxT><<<o.chunks, kOrderThreads, 0, s>>>(rp, n, nnz, o.chunks, o.cnt, o.dsum, order, o.inv,
                                                           o.slot_of, o.rp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nnz == 0) return cudaSuccess;
    uint64_t blocks = ((uint64_t)n + kOrderWarps - 1) / kOrderWarps;
    const uint64_t cap = (uint64_t)current_sms() * 8;
    if (blocks > cap) blocks = cap;
    // after the scan, cell (first slot of the keys below 20, chunk 0) holds
    // the number of vertices of key 20 and up
    k_order_lists<IdxT><<<(unsigned)blocks, kOrderThreads, 0, s>>>(
        rp, n, nnz, order, o.rp, col_in, o.inv, o.slot_of, col_out, o.cnt + (uint64_t)kLongKeySlot * o.chunks, flags);
    return cudaGetLastError();
}

}  // namespace

uint64_t order_scratch_bytes(uint32_t n) {
    uint64_t b = 0;
    carve(n, nullptr, &b);
    return b;
}

cudaError_t launch_degree_order(const void *row_ptr, int is64, const uint32_t *col_in, uint32_t n, uint64_t nnz,
                                uint32_t *order, uint32_t *col_out, void *scratch, uint32_t **rp_out,
                                uint32_t *flags, cudaStream_t s) {
    const OrderScratch o = carve(n, scratch, nullptr);
    *rp_out = o.rp;
    if (is64)
        return order_with(static_cast<const uint64_t *>(row_ptr), col_in, n, nnz, order, col_out, o, flags, s);
    return order_with(static_cast<const uint32_t *>(row_ptr), col_in, n, nnz, order, col_out, o, flags, s);
}

cudaError_t launch_map_records(uint32_t *verts, uint64_t count, int words, const uint32_t *order, uint32_t n,
                               cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    uint64_t blocks = (count * 5 + 255) / 256;
    const uint64_t cap = (uint64_t)current_sms() * 16;
    if (blocks > cap) blocks = cap;
    k_map_records<<<(unsigned)blocks, 256, 0, s>>>(verts, count, words, order, n);
    return cudaGetLastError();
}

}  // namespace moss
