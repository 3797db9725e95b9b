// moss_alias.cuh -- block-cooperative alias table of one long neighbour list.
//
// The closed form of moss_tables.cu (header comment there): q_j = w_j d,
// capacity W = sum w; lights (q_j < W) carry the deficit W - q_j, heavies the
// excess q_j - W, both in list order; with A_i the exclusive prefix of the
// light deficits and P_k the inclusive prefix of the heavy excesses, light i
// keeps q_i and aliases the first heavy k with P_k >= A_i; heavy k keeps
// W + P_k - A_{i'} (i' the first light with A_{i'} > P_k) and aliases heavy
// k+1, or keeps W when P_k is the total.  The warp-per-list kernels leave a
// hub's list to one warp, whose sequential merge then bounds the whole
// launch; here a block of NT threads shares one list: block scans split it,
// and each thread merges a run of about d / NT entries.
#pragma once

#include "moss_internal.cuh"

namespace moss {

template <typename T>
__device__ __forceinline__ T shfl_up_any(T v, int d);
template <>
__device__ __forceinline__ uint32_t shfl_up_any<uint32_t>(uint32_t v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
template <>
__device__ __forceinline__ uint64_t shfl_up_any<uint64_t>(uint64_t v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
template <>
__device__ __forceinline__ u128 shfl_up_any<u128>(u128 v, int d) {
    return shfl_up_u128(v, d);
}

// inclusive scan over the block (blockDim.x == NT); total receives the block
// sum.  smem holds NT / 32 entries; every thread of the block must call it.
template <typename T, int NT>
__device__ __forceinline__ T block_incl_scan(T v, T &total, T *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T t = shfl_up_any<T>(v, d);
        if (lane >= d) v += t;
    }
    if (lane == 31) smem[warp] = v;
    __syncthreads();
    T off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const T s = smem[w];
        if (w < warp) off += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return off + v;
}

// Inclusive scans over the block of three values at once (one pair of
// barriers): c, D and E become their inclusive prefixes, tc, tD and tE the
// block sums.  Every thread of the block must call it.
template <typename T, int NT>
__device__ __forceinline__ void block_scan3(uint64_t &c, T &D, T &E, uint64_t &tc, T &tD, T &tE) {
    __shared__ uint64_t s_c[NT / 32];
    __shared__ T s_D[NT / 32], s_E[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const uint64_t c1 = shfl_up_any<uint64_t>(c, k);
        const T D1 = shfl_up_any<T>(D, k), E1 = shfl_up_any<T>(E, k);
        if (lane >= k) {
            c += c1;
            D += D1;
            E += E1;
        }
    }
    if (lane == 31) {
        s_c[warp] = c;
        s_D[warp] = D;
        s_E[warp] = E;
    }
    __syncthreads();
    uint64_t oc = 0, ac = 0;
    T oD = 0, aD = 0, oE = 0, aE = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint64_t x = s_c[w];
        const T y = s_D[w], z = s_E[w];
        if (w < warp) {
            oc += x;
            oD += y;
            oE += z;
        }
        ac += x;
        aD += y;
        aE += z;
    }
    __syncthreads();
    c += oc;
    D += oD;
    E += oE;
    tc = ac;
    tD = aD;
    tE = aE;
}

// Alias table of the list of d entries with weights weight(j) (d * w_j and W
// must fit T) and capacity W > 0; idx (d uint32) and pre (d T) are scratch;
// store(j, thr, alias) receives each entry's threshold (<= W) and alias
// position.  Every thread of the block must call it.
template <typename T, int NT, typename Weight, typename Store>
__device__ void block_alias(uint32_t d, T W, Weight weight, uint32_t *idx, T *pre, Store store) {
    const int tid = threadIdx.x;
    uint32_t nl = 0, nh = 0;
    T Arun = 0, Prun = 0;
    for (uint32_t base = 0; base < d; base += NT) {
        const uint32_t j = base + tid;
        const bool valid = j < d;
        const T q = valid ? (T)weight(j) * (T)d : (T)0;
        const bool light = valid && q < W, heavy = valid && !light;
        const T D = light ? W - q : (T)0, E = heavy ? q - W : (T)0;
        // light and heavy counts packed in one 64-bit lane (low, high word)
        uint64_t ic = light ? 1ull : (heavy ? 1ull << 32 : 0ull), tc;
        T iD = D, iE = E, tD, tE;
        block_scan3<T, NT>(ic, iD, iE, tc, tD, tE);
        const uint32_t il = (uint32_t)ic, ih = (uint32_t)(ic >> 32);
        const uint32_t tl = (uint32_t)tc, th = (uint32_t)(tc >> 32);
        if (light) {
            const uint32_t r = nl + il - 1;
            idx[r] = j;
            pre[r] = Arun + iD - D;          // exclusive A_i
        } else if (heavy) {
            const uint32_t r = nh + ih - 1;
            idx[d - 1 - r] = j;
            pre[d - 1 - r] = Prun + iE;      // inclusive P_k
        }
        nl += tl;
        nh += th;
        Arun += tD;
        Prun += tE;
    }
    __syncthreads();   // the split is visible to the whole block
    const T Ptot = Prun;
    {
        const uint32_t cl = (nl + NT - 1) / NT;
        const uint32_t i0 = tid * cl, i1 = min(nl, i0 + cl);
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
                store(j, (T)weight(j) * (T)d, idx[d - 1 - k]);
            }
        }
    }
    {
        const uint32_t ch = (nh + NT - 1) / NT;
        const uint32_t k0 = tid * ch, k1 = min(nh, k0 + ch);
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
                if (Pk < Ptot) {
                    const T Ai = i < nl ? pre[i] : Ptot;
                    store(j, W + Pk - Ai, idx[d - 1 - (k + 1)]);
                } else {
                    store(j, W, j);
                }
            }
        }
    }
    __syncthreads();   // idx / pre are reused by the block's next list
}

// Calls body(v) for every vertex v < n whose record passes pred, one vertex at
// a time for the whole block (body is block-cooperative).  Blocks take chunks
// of CH <= NT vertices and test a chunk's records in parallel, so a block
// touches n / gridDim records rather than one by one; a small CH spreads
// frequent qualifying vertices over more blocks.  Chunk c holds the vertices
// c + j C (j < CH, C = ceil(n / CH) chunks): vertices that are close in id
// fall into different chunks, so a graph whose long lists sit together (one
// loaded in degree order) still spreads them over the blocks.
template <int NT, int CH = NT, typename Pred, typename Body>
__device__ void for_each_vertex(uint32_t n, const uint4 *rec, Pred pred, Body body) {
    static_assert(CH <= NT, "chunk larger than the block");
    __shared__ uint32_t found[CH];
    __shared__ uint32_t nfound;
    const uint64_t chunks = ((uint64_t)n + CH - 1) / CH;
    for (uint64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        if (threadIdx.x == 0) nfound = 0;
        __syncthreads();
        const uint64_t v = c + (uint64_t)threadIdx.x * chunks;
        if (threadIdx.x < CH && v < n && pred(rec[v])) found[atomicAdd(&nfound, 1u)] = (uint32_t)v;
        __syncthreads();
        const uint32_t cnt = nfound;
        for (uint32_t k = 0; k < cnt; ++k) body(found[k]);
        __syncthreads();
    }
}

}  // namespace moss
