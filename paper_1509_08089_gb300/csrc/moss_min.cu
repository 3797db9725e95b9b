// moss_min.cu -- the MOSS-4Min tables (Sec. 4.2) on the device.
//
// The total order of Sec. 3.2 puts x above y when d_x > d_y, or d_x = d_y and
// x > y; the 64-bit key (d_x << 32) | x orders vertices exactly that way.
// N_{u,v} = {x in N_u : x above v}, d_{u,v} = |N_{u,v}|.  Every list N_v is
// stored sorted by that key, highest first (rlist), so N_{v,u} is its first
// d_{v,u} entries and d_{v,u} is the position of u in it:
//   * lists of at most 128 entries: a warp per list, each entry's rank is the
//     count of keys above its own;
//   * lists of at most kTile entries: a block per list, bitonic sort in
//     shared memory, each key's list position moving with it;
//   * longer lists: a block per list sorts tiles of kTile keys in shared
//     memory, then merges runs pairwise in global memory, each key (with its
//     position) placed by one binary search in the partner run (keys are
//     distinct).
// Then per slot (v -> u): u, d_u, off_u, d_{v,u} and d_{u,v} (the rank of the
// twin slot); per list: Gamma-check_v = sum_u d_{v,u} d_{u,v} and the alias
// table of sigma-check^(v) (eq. 3) -- the parallel closed form of the sweep
// used for sigma^(v) in moss_tables.cu, here in 128-bit arithmetic since
// q_j = w_j d_v can exceed 2^64; the exact total Gamma-check; and the vertex
// alias table of pi-check through the seed-table kernels.
#include <atomic>

#include "moss_alias.cuh"
#include "moss_internal.cuh"

namespace moss {

namespace {

constexpr int kWarp = 32;
constexpr uint32_t kTile = 4096;      // keys sorted per shared-memory pass (32 KB)
constexpr int kSortThreads = 512;
constexpr int kListThreads = 256;
constexpr uint32_t kWarpKeys = 4;     // k_rank_warp: lists up to 128 entries
constexpr uint32_t kLongList = 256;   // longer lists: k_min_alias_long, a block per list

__device__ __forceinline__ uint64_t order_key(uint32_t x, uint32_t dx) { return ((uint64_t)dx << 32) | x; }

// lists of at most kWarpKeys * 32 entries: lane l holds entries l, l + 32, ...;
// an entry's rank is the number of keys above its own, counted against every
// key of the list broadcast by shuffles
__global__ void __launch_bounds__(kListThreads) k_rank_warp(uint32_t n, const uint4 *__restrict__ vert,
                                                           const uint32_t *__restrict__ col, uint2 *rlist,
                                                           uint32_t *rank) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (uint64_t v = (uint64_t)blockIdx.x * wpb + warp; v < n; v += (uint64_t)gridDim.x * wpb) {
        const uint4 vr = vert[v];
        const uint32_t o = vr.x, d = vr.y;
        if (d == 0 || d > kWarpKeys * (uint32_t)kWarp) continue;   // warp-uniform
        const int rounds = (int)((d + kWarp - 1) / kWarp);
        uint32_t x[kWarpKeys], dx[kWarpKeys], r[kWarpKeys];
        uint64_t key[kWarpKeys];
#pragma unroll
        for (int k = 0; k < kWarpKeys; ++k) {
            const uint32_t i = k * kWarp + lane;
            x[k] = dx[k] = r[k] = 0;
            key[k] = 0;                               // below every real key (d_x >= 1)
            if (i < d) {
                x[k] = col[o + i];
                dx[k] = vert[x[k]].y;
                key[k] = order_key(x[k], dx[k]);
            }
        }
#pragma unroll
        for (int kk = 0; kk < kWarpKeys; ++kk) {
            if (kk >= rounds) break;                  // warp-uniform
            const int m = min((int)d - kk * kWarp, kWarp);
            for (int j = 0; j < m; ++j) {
                const uint64_t other = __shfl_sync(0xffffffffu, key[kk], j);
#pragma unroll
                for (int k = 0; k < kWarpKeys; ++k)
                    if (k < rounds) r[k] += other > key[k];   // warp-uniform
            }
        }
#pragma unroll
        for (int k = 0; k < kWarpKeys; ++k) {
            const uint32_t i = k * kWarp + lane;
            if (i < d) {
                rlist[o + r[k]] = make_uint2(x[k], dx[k]);
                rank[o + i] = r[k];
            }
        }
    }
}

__device__ __forceinline__ uint32_t pow2_at_least(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// keys of col[o + base, o + base + len) into k[0, P), zero padded (zero sorts
// last), with each key's position in the list in id[]
__device__ void load_keys(const uint4 *vert, const uint32_t *col, uint32_t o, uint32_t base, uint32_t len,
                          uint32_t P, uint64_t *k, uint16_t *id) {
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        uint64_t key = 0;
        if (i < len) {
            const uint32_t x = col[o + base + i];
            key = order_key(x, vert[x].y);
        }
        k[i] = key;
        id[i] = (uint16_t)i;
    }
    __syncthreads();
}

// block-wide bitonic sort of k[0, P), P a power of two, highest first; id[]
// moves with its key
__device__ void bitonic_desc(uint64_t *k, uint16_t *id, uint32_t P) {
    for (uint32_t size = 2; size <= P; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const uint32_t i = 2 * t - (t & (stride - 1)), j = i + stride;
                const uint64_t a = k[i], b = k[j];
                const bool down = (i & size) == 0;   // this run ends highest first
                if ((a < b) == down) {
                    k[i] = b;
                    k[j] = a;
                    const uint16_t t0 = id[i];
                    id[i] = id[j];
                    id[j] = t0;
                }
            }
            __syncthreads();
        }
}

// a block per 32 vertex records (the scheduler spreads the lists).  A list
// of at most kCountList entries ranks each key by counting the keys above it
// (every thread reads the same key at a time: shared-memory broadcasts, no
// barrier per step); a longer one sorts keys and positions together
// (bitonic, a barrier per stage).
constexpr uint32_t kCountList = 1024;

__global__ void __launch_bounds__(kSortThreads) k_rank_block(uint32_t n, const uint4 *__restrict__ vert,
                                                            const uint32_t *__restrict__ col, uint2 *rlist,
                                                            uint32_t *rank) {
    __shared__ uint64_t k[kTile];
    __shared__ uint16_t id[kTile];
    for_each_vertex<kSortThreads, kWarp>(
        n, vert, [](uint4 vr) { return vr.y > kWarpKeys * (uint32_t)kWarp && vr.y <= kTile; },
        [&](uint32_t v) {
            const uint4 vr = vert[v];
            const uint32_t o = vr.x, d = vr.y;
            if (d <= kCountList) {
                for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
                    const uint32_t x = col[o + i];
                    k[i] = order_key(x, vert[x].y);
                }
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
                    const uint64_t key = k[i];
                    uint32_t r = 0;
                    for (uint32_t j = 0; j < d; ++j) r += k[j] > key;
                    rlist[o + r] = make_uint2((uint32_t)key, (uint32_t)(key >> 32));
                    rank[o + i] = r;
                }
                __syncthreads();   // k is refilled for the next list
                return;
            }
            const uint32_t P = pow2_at_least(d);
            load_keys(vert, col, o, 0, d, P, k, id);
            bitonic_desc(k, id, P);
            for (uint32_t q = threadIdx.x; q < d; q += blockDim.x) {
                const uint64_t key = k[q];
                rlist[o + q] = make_uint2((uint32_t)key, (uint32_t)(key >> 32));
                rank[o + id[q]] = q;
            }
            __syncthreads();   // k and id are refilled for the next list
        });
}

// lists longer than kTile: tiles sorted in shared memory into a[], then runs
// of length L merged pairwise between a[] and b[] until one run is left
__global__ void __launch_bounds__(kSortThreads) k_rank_long(uint32_t n, const uint4 *__restrict__ vert,
                                                           const uint32_t *__restrict__ col, uint64_t *a,
                                                           uint64_t *b, uint32_t *ia, uint32_t *ib, uint2 *rlist,
                                                           uint32_t *rank) {
    __shared__ uint64_t k[kTile];
    __shared__ uint16_t id[kTile];
    for_each_vertex<kSortThreads>(n, vert, [](uint4 vr) { return vr.y > kTile; }, [&](uint32_t v) {
        const uint4 vr = vert[v];
        const uint32_t o = vr.x, d = vr.y;
        for (uint32_t base = 0; base < d; base += kTile) {
            const uint32_t len = min(kTile, d - base);
            const uint32_t P = pow2_at_least(len);
            load_keys(vert, col, o, base, len, P, k, id);
            bitonic_desc(k, id, P);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
                a[(uint64_t)o + base + i] = k[i];
                ia[(uint64_t)o + base + i] = base + id[i];
            }
            __syncthreads();
        }
        uint64_t *src = a, *dst = b;
        uint32_t *isrc = ia, *idst = ib;
        for (uint64_t L = kTile; L < d; L <<= 1) {
            for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
                const uint64_t run = i / L, start = run * L;
                const uint64_t ps = (run ^ 1) * L;               // the partner run
                const uint64_t ms = (run & ~1ull) * L;           // where the pair's merge starts
                const uint64_t key = src[(uint64_t)o + i];
                // partner keys above key (the partner run is sorted highest first)
                uint64_t lo = ps, len = ps < d ? min(ps + L, (uint64_t)d) - ps : 0;
                while (len > 0) {
                    const uint64_t half = len >> 1;
                    if (src[(uint64_t)o + lo + half] > key) {
                        lo += half + 1;
                        len -= half + 1;
                    } else {
                        len = half;
                    }
                }
                const uint64_t above = ps < d ? lo - ps : 0;
                dst[(uint64_t)o + ms + (i - start) + above] = key;
                idst[(uint64_t)o + ms + (i - start) + above] = isrc[(uint64_t)o + i];
            }
            __syncthreads();
            uint64_t *t = src;
            src = dst;
            dst = t;
            uint32_t *it = isrc;
            isrc = idst;
            idst = it;
        }
        for (uint32_t q = threadIdx.x; q < d; q += blockDim.x) {
            const uint64_t key = src[(uint64_t)o + q];
            rlist[o + q] = make_uint2((uint32_t)key, (uint32_t)(key >> 32));
            rank[o + isrc[(uint64_t)o + q]] = q;
        }
        __syncthreads();
    });
}

// per slot p (v -> u): {0, 0, 0, u} and {off_u, d_u, d_{v,u}, d_{u,v}}
__global__ void k_min_slots(uint64_t nnz, const uint4 *__restrict__ vert, const uint32_t *__restrict__ col,
                            const uint4 *__restrict__ slot, const uint32_t *__restrict__ rank, uint4 *mslot) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = col[p];
        const uint4 ur = vert[u];
        const uint32_t twin = slot_twin(reinterpret_cast<const uint32_t *>(slot), p);
        mslot[2 * p] = make_uint4(0u, 0u, 0u, u);
        mslot[2 * p + 1] = make_uint4(ur.x, ur.y, rank[p], rank[(uint64_t)ur.x + twin]);
    }
}

// (a read-only load: the alias passes write only the first half of each record)
__device__ __forceinline__ uint64_t min_weight(const uint4 *mslot, uint64_t p) {
    const uint4 r = __ldg(mslot + 2 * p + 1);
    return (uint64_t)r.z * r.w;   // d_{v,u} d_{u,v}
}

// threshold and alias position into the first half of a slot record
__device__ __forceinline__ void set_min_alias(uint32_t *m32, uint64_t p, uint64_t thr, uint32_t alias) {
    *reinterpret_cast<uint2 *>(m32 + 8 * p) = make_uint2((uint32_t)thr, (uint32_t)(thr >> 32));
    m32[8 * p + 2] = alias;
}

// warp per list: Gamma-check_v, mvert, and the alias table of sigma-check^(v)
// over capacity W = Gamma-check_v.  Lights (q_j = w_j d < W) carry the deficit
// W - q_j, heavies the excess q_j - W, both in list order; with A_i the
// exclusive prefix of the light deficits and P_k the inclusive prefix of the
// heavy excesses: light i keeps q_i and aliases heavy min{k : P_k >= A_i};
// heavy k keeps W + P_k - A_{i'} (i' = min{i : A_i > P_k}) and aliases heavy
// k+1, or keeps W when P_k is the total.  The split (idx, pre) of the list
// being built lives in the warp's share of shared memory; the prefixes are
// 64-bit when d W fits (every list short enough for this kernel with W below
// 2^56), else 128-bit.
template <typename T>
__device__ __forceinline__ T warp_scan_any(T v, int lane);
template <>
__device__ __forceinline__ uint64_t warp_scan_any<uint64_t>(uint64_t v, int lane) {
    return warp_incl_scan64(v, lane);
}
template <>
__device__ __forceinline__ u128 warp_scan_any<u128>(u128 v, int lane) {
    return warp_incl_scan128(v, lane);
}
__device__ __forceinline__ uint64_t shfl_idx_any(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ u128 shfl_idx_any(u128 v, int src) { return shfl_idx_u128(v, src); }

// alias table of sigma-check^(v) for the list at o of d <= kLongList entries
// with total W > 0, one warp; pre holds kLongList T, idx kLongList positions
template <typename T>
__device__ void warp_min_alias(const uint4 *mslot, uint32_t *m32, uint32_t o, uint32_t d, uint64_t W, T *pre,
                               uint32_t *idx) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    // pass 1: lights to the front, heavies to the back, with their prefixes
    uint32_t nl = 0, nh = 0;
    T Arun = 0, Prun = 0;
    for (uint32_t base = 0; base < d; base += kWarp) {
        const uint32_t j = base + lane;
        const bool valid = j < d;
        const T q = valid ? (T)min_weight(mslot, (uint64_t)o + j) * (T)d : (T)0;
        const bool light = valid && q < W;
        const uint32_t lmask = __ballot_sync(0xffffffffu, light);
        const uint32_t hmask = __ballot_sync(0xffffffffu, valid && !light);
        const T D = light ? (T)W - q : (T)0;
        const T E = valid && !light ? q - (T)W : (T)0;
        const T Dincl = warp_scan_any<T>(D, lane);
        const T Eincl = warp_scan_any<T>(E, lane);
        if (light) {
            const uint32_t r = nl + __popc(lmask & below);
            idx[r] = j;
            pre[r] = Arun + Dincl - D;          // exclusive A_i
        } else if (valid) {
            const uint32_t r = nh + __popc(hmask & below);
            idx[d - 1 - r] = j;
            pre[d - 1 - r] = Prun + Eincl;      // inclusive P_k
        }
        nl += __popc(lmask);
        nh += __popc(hmask);
        Arun += shfl_idx_any(Dincl, 31);
        Prun += shfl_idx_any(Eincl, 31);
    }
    __syncwarp();
    const T Ptot = Prun;   // == Arun
    const uint64_t ob = o;
    // pass 2: each lane merges a contiguous run of lights, then of heavies
    {
        const uint32_t cl = (nl + kWarp - 1) / kWarp;
        const uint32_t i0 = lane * cl, i1 = min(nl, i0 + cl);
        if (i0 < i1) {
            const T A0 = pre[i0];
            uint32_t k = 0, len = nh;   // first heavy with P_k >= A
            while (len > 0) {
                const uint32_t half = len >> 1;
                if (pre[d - 1 - (k + half)] < A0) {
                    k += half + 1;
                    len -= half + 1;
                } else {
                    len = half;
                }
            }
            for (uint32_t i = i0; i < i1; ++i) {
                const T A = pre[i];
                while (pre[d - 1 - k] < A) ++k;
                const uint32_t j = idx[i];
                const uint64_t thr = min_weight(mslot, ob + j) * (uint64_t)d;   // q_j < W < 2^64
                set_min_alias(m32, ob + j, thr, idx[d - 1 - k]);
            }
        }
    }
    {
        const uint32_t ch = (nh + kWarp - 1) / kWarp;
        const uint32_t k0 = lane * ch, k1 = min(nh, k0 + ch);
        if (k0 < k1) {
            const T P0 = pre[d - 1 - k0];
            uint32_t i = 0, len = nl;   // first light with A_i > P_k
            while (len > 0) {
                const uint32_t half = len >> 1;
                if (pre[i + half] <= P0) {
                    i += half + 1;
                    len -= half + 1;
                } else {
                    len = half;
                }
            }
            for (uint32_t k = k0; k < k1; ++k) {
                const T Pk = pre[d - 1 - k];
                while (i < nl && pre[i] <= Pk) ++i;
                const uint32_t j = idx[d - 1 - k];
                uint64_t thr;
                uint32_t alias;
                if (Pk < Ptot) {
                    const T Ai = i < nl ? pre[i] : Ptot;
                    thr = (uint64_t)((T)W + Pk - Ai);
                    alias = idx[d - 1 - (k + 1)];
                } else {
                    thr = W;
                    alias = j;
                }
                set_min_alias(m32, ob + j, thr, alias);
            }
        }
    }
}

__global__ void __launch_bounds__(kListThreads) k_min_alias(uint32_t n, const uint4 *__restrict__ vert, uint4 *mslot,
                                                           uint4 *mvert, u128 *gmin, u128 *partials) {
    __shared__ u128 s_pre[kListThreads / kWarp][kLongList];
    __shared__ uint32_t s_idx[kListThreads / kWarp][kLongList];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    uint32_t *m32 = reinterpret_cast<uint32_t *>(mslot);
    u128 total = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * wpb + warp; v < n; v += (uint64_t)gridDim.x * wpb) {
        const uint4 vr = vert[v];
        const uint32_t o = vr.x, d = vr.y;
        uint64_t W = 0;
        for (uint32_t j = lane; j < d; j += kWarp) W += min_weight(mslot, (uint64_t)o + j);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) W += __shfl_down_sync(0xffffffffu, W, s);
        W = __shfl_sync(0xffffffffu, W, 0);
        if (lane == 0) {
            mvert[v] = make_uint4(o, d, (uint32_t)W, (uint32_t)(W >> 32));
            gmin[v] = W;
            total += W;
        }
        if (d == 0 || (d > kLongList && W != 0)) continue;
        if (W == 0) {   // never drawn: keep every column
            for (uint32_t j = lane; j < d; j += kWarp) set_min_alias(m32, (uint64_t)o + j, 0, j);
            continue;
        }
        if (W < (1ull << 56))   // q = w d <= W kLongList < 2^64
            warp_min_alias<uint64_t>(mslot, m32, o, d, W, reinterpret_cast<uint64_t *>(s_pre[warp]), s_idx[warp]);
        else
            warp_min_alias<u128>(mslot, m32, o, d, W, s_pre[warp], s_idx[warp]);
        __syncwarp();
    }
    // block share of Gamma-check (lane 0 of each warp holds its warp's)
    __shared__ u128 sh[kListThreads / kWarp];
    if (lane == 0) sh[warp] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 s = 0;
        for (int w = 0; w < wpb; ++w) s += sh[w];
        partials[blockIdx.x] = s;
    }
}

// the alias tables of lists longer than kLongList, a block per list; each
// block forms Gamma-check_v itself (the same integer sum k_min_alias writes
// into mvert), so the two kernels may run side by side.  A block per kWarp
// vertex records (the scheduler spreads the long lists); the split of a list
// of at most kMinSmemList entries in dynamic shared memory, of a longer one in
// its range of the global scratch (idx, pre)
constexpr uint32_t kMinSmemList = 2048;
constexpr size_t kMinSmemBytes = (size_t)kMinSmemList * (sizeof(u128) + sizeof(uint32_t));

__global__ void __launch_bounds__(kListThreads) k_min_alias_long(uint32_t n, const uint4 *__restrict__ vert,
                                                                uint4 *mslot, uint32_t *idx, u128 *pre) {
    extern __shared__ u128 s_split[];   // kMinSmemList prefixes, then kMinSmemList positions
    __shared__ uint64_t s_w[kListThreads / kWarp];
    uint32_t *m32 = reinterpret_cast<uint32_t *>(mslot);
    for_each_vertex<kListThreads, kWarp>(
        n, vert, [](uint4 vr) { return vr.y > kLongList; },
        [&](uint32_t v) {
            const uint4 vr = vert[v];
            const uint32_t o = vr.x, d = vr.y;
            uint64_t W = 0;
            for (uint32_t j = threadIdx.x; j < d; j += kListThreads) W += min_weight(mslot, (uint64_t)o + j);
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) W += __shfl_down_sync(0xffffffffu, W, sft);
            if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = W;
            __syncthreads();
            W = 0;
            for (int w = 0; w < kListThreads / kWarp; ++w) W += s_w[w];
            __syncthreads();   // s_w is refilled for the next list
            if (W == 0) return;   // block-uniform: k_min_alias keeps every column
            const bool fits = d <= kMinSmemList;
            block_alias<u128, kListThreads>(
                d, (u128)W, [&](uint32_t j) { return (u128)min_weight(mslot, (uint64_t)o + j); },
                fits ? reinterpret_cast<uint32_t *>(s_split + kMinSmemList) : idx + o, fits ? s_split : pre + o,
                [&](uint32_t j, u128 thr, uint32_t alias) { set_min_alias(m32, (uint64_t)o + j, (uint64_t)thr, alias); });
        });
}

__global__ void k_min_total(const u128 *partials, int blocks, DevTotals *tot) {
    const int lane = threadIdx.x;   // one warp
    u128 s = 0;
    for (int b = lane; b < blocks; b += kWarp) s += partials[b];
    s = warp_sum128(s);
    if (lane == 0) tot->gamma[3] = s;
}

unsigned grid_for(uint64_t items, int per_block, int cap_per_sm) {
    const int sms = current_sms();
    uint64_t b = (items + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)sms * cap_per_sm;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

struct MinScratch {
    uint32_t *rank;   // nnz, then reused as the alias split order
    uint64_t *a, *b;  // nnz each (long-list merges), then reused as u128 prefixes
    uint32_t *ia, *ib;  // nnz each: list positions of the keys in a, b
    u128 *partials;
    void *seed;       // vertex alias scratch
    uint64_t bytes;
};

// per slot p of a list with Gamma-check_v < 2^32: the pick record (layout in
// moss_internal.cuh) from p's mslot record and its alias position's
__global__ void k_min_pick(uint64_t nnz, const uint32_t *__restrict__ owner, const uint4 *__restrict__ mvert,
                           const uint4 *__restrict__ mslot, uint4 *mpick) {
    constexpr uint32_t kNarrow = 0xffffu;   // fields below this fit a half word
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 mv = mvert[owner[p]];
        const uint4 a0 = mslot[2 * p], a1 = mslot[2 * p + 1];
        const uint64_t ap = (uint64_t)mv.x + a0.z;
        const uint4 b0 = mslot[2 * ap], b1 = mslot[2 * ap + 1];
        const bool fits = mv.w == 0 && a1.y < kNarrow && a1.z < kNarrow && a1.w < kNarrow && b1.y < kNarrow &&
                          b1.z < kNarrow && b1.w < kNarrow;
        mpick[2 * p] = make_uint4(a0.x, a0.w, a1.x, a1.z | a1.w << 16);
        mpick[2 * p + 1] = make_uint4(b0.w, b1.x, b1.z | b1.w << 16, fits ? (a1.y | b1.y << 16) : kSlotHub);
    }
}

MinScratch carve(void *base, uint32_t n, uint64_t nnz) {
    MinScratch m{};
    uint8_t *p = static_cast<uint8_t *>(base);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        off = (off + 255) & ~255ULL;
        uint8_t *r = p ? p + off : nullptr;
        off += bytes ? bytes : 1;
        return r;
    };
    const unsigned alias_blocks = grid_for((uint64_t)n, kListThreads / kWarp, 8);
    m.rank = reinterpret_cast<uint32_t *>(take(nnz * 4));
    m.a = reinterpret_cast<uint64_t *>(take(nnz * 16));
    m.b = m.a ? m.a + nnz : nullptr;
    m.ia = reinterpret_cast<uint32_t *>(take(nnz * 8));
    m.ib = m.ia ? m.ia + nnz : nullptr;
    m.partials = reinterpret_cast<u128 *>(take((uint64_t)alias_blocks * 16));
    m.seed = take(seed_scratch_bytes(n));
    m.bytes = off;
    return m;
}

}  // namespace

uint64_t min_scratch_bytes(uint32_t n, uint64_t nnz) { return carve(nullptr, n, nnz).bytes; }

cudaError_t launch_min_tables(uint32_t n, uint64_t nnz, const uint4 *vert, const uint32_t *col,
                              const uint32_t *owner, const uint4 *slot, uint4 *mvert, uint4 *mslot, uint4 *mpick,
                              uint2 *rlist, u128 *gmin, uint4 *seed_min, DevTotals *tot, void *scratch,
                              uint32_t *flags, int split, cudaStream_t s, const AuxStreams *aux) {
    // With helper streams h0, h1 (aux->a[3], a[4]): the three sort tiers side
    // by side (disjoint lists), then the slot records on s; the short-list
    // alias tables, the total and the vertex table on s, beside the long-list
    // alias tables and (once the short ones are done) the pick records on h0.
    const MinScratch m = carve(scratch, n, nnz);
    cudaStream_t h0 = aux ? aux->a[3] : s, h1 = aux ? aux->a[4] : s;
    cudaError_t e = cudaSuccess, eh = cudaSuccess;
    auto fork = [&](int k) {   // h0 (and h1) wait for what is queued on s
        if (!aux) return;
        if (e == cudaSuccess) e = cudaEventRecord(aux->sub_fork, s);
        for (int i = 0; i < k && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(aux->a[3 + i], aux->sub_fork, 0);
    };
    auto join = [&](int k) {   // s waits for h0 (and h1); done even after an error
        if (!aux) return;
        for (int i = 0; i < k; ++i) {
            cudaError_t ei = cudaEventRecord(aux->sub_done[i], aux->a[3 + i]);
            if (ei == cudaSuccess) ei = cudaStreamWaitEvent(s, aux->sub_done[i], 0);
            if (e == cudaSuccess) e = ei;
        }
    };
    if (nnz) {
        fork(2);
        if (e == cudaSuccess) {
            const unsigned chunks = (unsigned)(((uint64_t)n + kWarp - 1) / kWarp);
            k_rank_block<<<chunks, kSortThreads, 0, h0>>>(n, vert, col, rlist, m.rank);
            eh = cudaGetLastError();
            k_rank_long<<<grid_for((uint64_t)n, kSortThreads, 1), kSortThreads, 0, h1>>>(n, vert, col, m.a, m.b, m.ia,
                                                                                        m.ib, rlist, m.rank);
            if (eh == cudaSuccess) eh = cudaGetLastError();
            k_rank_warp<<<grid_for((uint64_t)n, kListThreads / kWarp, 8), kListThreads, 0, s>>>(n, vert, col, rlist,
                                                                                                 m.rank);
            e = cudaGetLastError();
        }
        join(2);
        if (e == cudaSuccess) e = eh;
        if (e != cudaSuccess) return e;
        k_min_slots<<<grid_for(nnz, 256, 16), 256, 0, s>>>(nnz, vert, col, slot, m.rank, mslot);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_relaxed)) {
        e = cudaFuncSetAttribute(k_min_alias_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMinSmemBytes);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_relaxed);
    }
    const unsigned ab = grid_for((uint64_t)n, kListThreads / kWarp, 8);
    fork(1);
    if (e != cudaSuccess) return e;
    // the rank array is dead now: the long-list kernel reuses it (split order) with a[] (prefixes)
    const unsigned chunks = (unsigned)(((uint64_t)n + kWarp - 1) / kWarp);
    k_min_alias_long<<<chunks, kListThreads, kMinSmemBytes, h0>>>(n, vert, mslot, m.rank, reinterpret_cast<u128 *>(m.a));
    eh = cudaGetLastError();
    k_min_alias<<<ab, kListThreads, 0, s>>>(n, vert, mslot, mvert, gmin, m.partials);
    e = cudaGetLastError();
    if (aux && e == cudaSuccess) {   // the pick records need both alias passes and mvert
        e = cudaEventRecord(aux->sub_mid, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h0, aux->sub_mid, 0);
    }
    if (e == cudaSuccess && eh == cudaSuccess && nnz) {
        k_min_pick<<<grid_for(nnz, 256, 16), 256, 0, h0>>>(nnz, owner, mvert, mslot, mpick);
        eh = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_min_total<<<1, kWarp, 0, s>>>(m.partials, (int)ab, tot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int which[1] = {3};
        u128 *w[1] = {gmin};
        uint4 *sd[1] = {seed_min};
        const uint4 *vr[1] = {mvert};
        e = launch_seed_alias(n, tot, 1, which, w, sd, vr, m.seed, flags, split, s);
    }
    join(1);
    return e != cudaSuccess ? e : eh;
}

}  // namespace moss
