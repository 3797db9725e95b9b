// moss_sample.cu -- the sampling loop of MOSS-4 (Algorithm 1), MOSS-4Min
// (Algorithm 2), T-5 (Algorithm 3) and Path-5 (Algorithm 4) on the device.
//
// One thread draws one sample at a time (grid-stride over sample ids), so
// every sample is an independent chain of dependent gathers:
//   random words -> vertex alias record (32 B, with the alias's vertex record;
//   vert[v] (16 B) only when the column keeps the draw) -> sigma
//   record(s) of N_v (32 B each, carrying the picked neighbour's list and
//   twin) -> uniform list picks (4 B) -> the unknown pairs, probed together
//   (hashed edge set, or lock-step binary searches) -> edge mask -> class
//   through a shared-memory table.
// Counts are aggregated per warp with __match_any_sync into shared-memory
// histograms and leave the block as one row of per-block partials; a second
// kernel adds the rows in a fixed order.  No global atomics.
//
// Word schedule (x_i = word i of the sample, output (4 s + method) 16 + i + 1
// of SplitMix64 seeded with seed, or Philox4x32-10 block i / 2; sample_words2
// in moss_internal.cuh):
//   MOSS-4 : x0,x1 vertex draw (column, threshold), x6 its level; x2,x3 sigma
//            draw of u; x4 w; x5 r.
//   T-5    : x0,x1 vertex draw, x7 its level; x2,x3 sigma of u; x4 w; x5 r;
//            x6 t.
//   MOSS-4Min: x0,x1 vertex draw (pi-check), x6 its level; x2,x3 sigma-check
//            draw of u; x4 w (uniform in N_{v,u}); x5 r (uniform in N_{u,v}).
//   Path-5 : x0,x1 vertex draw, x14 its level; x2 r; x3 t; attempts a = 0,1 use
//            x(4+4a)..x(7+4a) for two independent sigma draws (u, w), kept
//            when the positions differ (sigma_u sigma_w / (1 - sum sigma^2)
//            is exactly tau_u mu_w of Sec. 5.1.2); if both collide, x12 draws
//            u from tau^(v) and x13 draws w from mu^(v,u) with the interval of
//            u removed from ACC (Sec. 5.1.4).
// RandomVertex(N_v - X) (Sec. 4.1.3) takes the j-th admissible position,
// skipping the excluded positions of X in list order.
#include <algorithm>
#include <atomic>

#include "moss_internal.cuh"

namespace moss {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLut = 1024;
// hub-pair bits behind the filter, per method (MOSS-4, T-5, Path-5, MOSS-4Min):
// measured on the 34M-edge graph against the same build without them, 5e8
// samples per call, T-5 -7.5%, Path-5 -16%, MOSS-4Min -27%, MOSS-4 +0.8% (its
// three probes hold few hub pairs)
constexpr bool kHubProbes[kMethods] = {false, true, true, true};

__device__ uint8_t g_lut4[64];
__device__ uint8_t g_lut5[1024];
__device__ uint8_t g_lutc[4096];   // c(s) of MOSS-4Min by (edge mask << 6 | order bits)

__device__ __forceinline__ uint4 ld4(const uint4 *p) { return __ldg(p); }
__device__ __forceinline__ uint2 ld2(const uint2 *p) { return __ldg(p); }
__device__ __forceinline__ uint32_t ld1(const uint32_t *p) { return __ldg(p); }

// Probe modes of the sampler instances: kPmPlain (list search, or the hashed
// edge set with one-level vertex tables), kPmFilter (the edge filter in front
// of the set: L2 hints and hub-pair bits) and kPmStream (the set with
// two-level vertex tables, which fit the L1: the scattered loads of lists,
// slot records and buckets skip L1 allocation, so the heavy level's records,
// read evict-last, stay there and those draws cost no L2 request).
constexpr int kPmPlain = 0, kPmFilter = 1, kPmStream = 2;
constexpr uint32_t kStreamHeavy = 4096;   // heavy columns (32 B each) that kPmStream keeps in L1

// a vertex record without L1 allocation
__device__ __forceinline__ uint4 ld4_na(const uint4 *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

// a list entry (neighbour id) in mode PM
template <int PM>
__device__ __forceinline__ uint32_t ldc(const uint32_t *p) {
    if (PM != kPmStream) return __ldg(p);
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

struct Pick {
    uint32_t pos;   // position in N_v
    uint32_t id;    // the vertex
    uint32_t twin;  // position of v in N_id
    uint32_t off;   // N_id = col[off .. off + deg)
    uint32_t deg;
};

// one 32-byte sector in a single 256-bit load (32-byte aligned)
struct alignas(32) Sector {
    uint4 lo, hi;
};
__device__ __forceinline__ Sector ld8(const uint4 *p) {
    Sector r;
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r.lo.x), "=r"(r.lo.y), "=r"(r.lo.z), "=r"(r.lo.w), "=r"(r.hi.x), "=r"(r.hi.y), "=r"(r.hi.z),
          "=r"(r.hi.w)
        : "l"(p));
    return r;
}

// The same load without L1 allocation (scattered records in kPmStream)
__device__ __forceinline__ Sector ld8_na(const uint4 *p) {
    Sector r;
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r.lo.x), "=r"(r.lo.y), "=r"(r.lo.z), "=r"(r.lo.w), "=r"(r.hi.x), "=r"(r.hi.y), "=r"(r.hi.z),
          "=r"(r.hi.w)
        : "l"(p));
    return r;
}

// ... and kept in L1 as long as possible (heavy-level vertex records in kPmStream)
__device__ __forceinline__ Sector ld8_keep(const uint4 *p) {
    Sector r;
    asm("ld.global.nc.L1::evict_last.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r.lo.x), "=r"(r.lo.y), "=r"(r.lo.z), "=r"(r.lo.w), "=r"(r.hi.x), "=r"(r.hi.y), "=r"(r.hi.z),
          "=r"(r.hi.w)
        : "l"(p));
    return r;
}

// The same load marked evict-first in L2, for the per-slot records (sigma
// slot records, MOSS-4Min pick records): they are the largest and least
// densely used tables of a sampler, so with the working set at the size of
// the L2 they are the ones to give up first, which keeps the denser edge
// hash, neighbour lists and vertex alias records resident.
__device__ __forceinline__ Sector ld8_first(const uint4 *p) {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    Sector r;
    asm("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
        : "=r"(r.lo.x), "=r"(r.lo.y), "=r"(r.lo.z), "=r"(r.lo.w), "=r"(r.hi.x), "=r"(r.hi.y), "=r"(r.hi.z),
          "=r"(r.hi.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ Sector ld8_first_na(const uint4 *p) {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    Sector r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
        : "=r"(r.lo.x), "=r"(r.lo.y), "=r"(r.lo.z), "=r"(r.lo.w), "=r"(r.hi.x), "=r"(r.hi.y), "=r"(r.hi.z),
          "=r"(r.hi.w)
        : "l"(p), "l"(pol));
    return r;
}

// a scattered 32-byte record (bucket, MOSS-4Min slot record) in mode PM
template <int PM>
__device__ __forceinline__ Sector ld8s(const uint4 *p) {
    return PM == kPmFilter ? ld8_first(p) : (PM == kPmStream ? ld8_na(p) : ld8(p));
}
// a per-slot record (sigma slot, MOSS-4Min pick) in mode PM: evict-first in L2
template <int PM>
__device__ __forceinline__ Sector ld8p(const uint4 *p) {
    return PM == kPmStream ? ld8_first_na(p) : ld8_first(p);
}

struct VertexPick {
    uint32_t v;
    uint4 rec;      // v's vertex record (vert, or mvert for MOSS-4Min)
};

// WeightRandomVertex(V, .) through a vertex alias table whose 32-byte column
// records carry the alias's vertex record: one load, plus the column's own
// record only when the column keeps the draw.  The table has two levels: the
// level word picks the light one (columns nh..n-1) when it is below the
// level's bound, else the heavy one (columns 0..nh-1: the few vertices that
// carry almost all the weight, a table small enough to stay cached).  Behind
// the edge filter a light record is read evict-first, since that table is as
// large as the L2 and drawn uniformly, so a line is rarely read twice; in
// kPmStream a heavy record is kept in L1.
// The level word (word lw of the sample) is generated only for a table with
// a heavy level (uniform across the launch).
template <int PM, int RNG>
__device__ __forceinline__ VertexPick draw_vertex(const DevGraph &g, int l, const uint4 *vrec, uint64_t seed,
                                                  uint64_t s, uint32_t lw, uint64_t xc, uint64_t xt) {
    const uint32_t nh = g.nheavy[l];
    bool light = true;
    if (nh != 0) light = sample_word<RNG>(seed, (uint32_t)l, s, lw) < g.tlight[l];
    const uint32_t c = (light ? nh : 0u) + (uint32_t)word_index(xc, light ? g.n - nh : nh);
    const uint4 *rec = g.seed[l] + 2 * (uint64_t)c;
    const Sector r = PM == kPmFilter ? (light ? ld8_first(rec) : ld8(rec))
                                     : (PM == kPmStream ? (light ? ld8_na(rec) : ld8_keep(rec)) : ld8(rec));
    // {T lo, T hi, alias, self} {alias's record}
    const uint64_t T = ((uint64_t)r.lo.y << 32) | r.lo.x;
    if (xt < T) return VertexPick{r.lo.w, PM == kPmStream && light ? ld4_na(vrec + r.lo.w) : ld4(vrec + r.lo.w)};
    return VertexPick{r.lo.z, r.hi};
}

// The neighbour half of a slot record (col, nb, off): a neighbour with 2^16
// or more neighbours keeps its twin in off and its list in vert[].
__device__ __forceinline__ Pick unpack_pick(const uint4 *vert, uint32_t pos, uint32_t id, uint32_t nb, uint32_t off) {
    if (nb != kSlotHub) return Pick{pos, id, nb & (kSlotDegLimit - 1), off, nb >> 16};
    const uint4 r = ld4(vert + id);
    return Pick{pos, id, off, r.x, r.y};
}

// WeightRandomVertex(N_v, sigma^(v)) through the list's alias table: one
// 32-byte slot record holds the column's pick and its alias's, each with the
// picked neighbour's list and twin
template <int PM>
__device__ __forceinline__ Pick draw_sigma(const uint4 *slot, const uint4 *vert, uint32_t ov, uint32_t dv, uint32_t Sv,
                                           uint64_t xc, uint64_t xt) {
    const uint32_t j = (uint32_t)word_index(xc, dv);
    const Sector rec = ld8p<PM>(slot + 2 * (uint64_t)(ov + j));   // {col, nb, thr, alias} {off, alias col, nb, off}
    const bool keep = word_index(xt, Sv) < rec.lo.z;
    return unpack_pick(vert, keep ? j : rec.lo.w, keep ? rec.lo.x : rec.hi.y, keep ? rec.lo.y : rec.hi.z,
                       keep ? rec.hi.x : rec.hi.w);
}

// the pick of position p of N_v from its own half of the slot record
__device__ __forceinline__ Pick slot_pick(const uint4 *slot, const uint4 *vert, uint32_t ov, uint32_t p) {
    const Sector rec = ld8(slot + 2 * (uint64_t)(ov + p));
    return unpack_pick(vert, p, rec.lo.x, rec.lo.y, rec.hi.x);
}

__device__ __forceinline__ uint32_t skip1(uint32_t j, uint32_t e) { return j < e ? j : j + 1; }

__device__ __forceinline__ uint32_t skip2(uint32_t j, uint32_t e1, uint32_t e2) {
    const uint32_t lo = min(e1, e2), hi = max(e1, e2);
    j += (j >= lo);
    j += (j >= hi);
    return j;
}

// Membership tests (a_p, b_p) in E for P pairs, advanced in lock step so the
// P searches of a sample overlap in memory.  Each pair searches the shorter
// of the two sorted lists.  Returns bit p set when the pair is an edge.
template <int P>
__device__ __forceinline__ uint32_t probe_pairs(const uint32_t *col, const uint4 (&ra)[P], const uint4 (&rb)[P],
                                                const uint32_t (&a)[P], const uint32_t (&b)[P]) {
    uint32_t lo[P], len[P], key[P];
    uint32_t found = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const bool use_a = ra[p].y <= rb[p].y;
        lo[p] = use_a ? ra[p].x : rb[p].x;
        len[p] = use_a ? ra[p].y : rb[p].y;
        key[p] = use_a ? b[p] : a[p];
    }
    bool any = true;
    while (any) {
        any = false;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (len[p] > 0) {
                const uint32_t half = len[p] >> 1;
                const uint32_t val = ld1(col + lo[p] + half);
                if (val == key[p]) {
                    found |= 1u << p;
                    len[p] = 0;
                } else if (val < key[p]) {
                    lo[p] += half + 1;
                    len[p] -= half + 1;
                } else {
                    len[p] = half;
                }
                any |= len[p] > 0;
            }
        }
    }
    return found;
}

// Membership tests through the hashed edge set: one 32-byte bucket load per
// pair in the common case, all P loads issued together.  kPmFilter (behind
// the filter): the filter rules out most pairs; the set is far larger than the
// L2 and a bucket is rarely read twice, so buckets are read evict-first,
// which keeps the filter, lists and hub slot records resident.  With HUB,
// the ends' rank-table entries come first (one 8-byte load per vertex, all
// together), and a pair of two hubs is answered by one bit of the hubs'
// adjacency bitmap, loaded beside the other pairs' filter words.
template <int P, int PM, bool HUB>
__device__ __forceinline__ uint32_t probe_hash(const DevGraph &g, const uint32_t (&a)[P], const uint32_t (&b)[P]) {
    uint32_t bk[P];
    uint32_t found = 0, pending = (1u << P) - 1u;
    if (g.filter) {   // warp-uniform: only pairs the filter cannot rule out go to the set
        uint32_t hubpair = 0, bit[P];
        if (PM == kPmFilter && HUB && g.hub_rank) {   // warp-uniform
            uint2 ea[P], eb[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                ea[p] = ld2(g.hub_rank + (a[p] >> 5));
                eb[p] = ld2(g.hub_rank + (b[p] >> 5));
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const uint32_t ia = hub_index(ea[p], a[p]), ib = hub_index(eb[p], b[p]);
                bit[p] = ia * g.hubs + ib;
                if (ia != kNoHub && ib != kNoHub) hubpair |= 1u << p;
            }
        }
        uint32_t word[P];
#pragma unroll
        for (int p = 0; p < P; ++p)
            word[p] = ld1(hubpair >> p & 1u ? g.hub_bits + (bit[p] >> 5)
                                             : g.filter + (filter_hash(edge_key(a[p], b[p])) >> g.filter_shift));
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (hubpair >> p & 1u) {
                found |= (word[p] >> (bit[p] & 31u) & 1u) << p;
                pending &= ~(1u << p);
            } else {
                const uint32_t m = filter_mask(filter_hash(edge_key(a[p], b[p])));
                if ((word[p] & m) != m) pending &= ~(1u << p);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) bk[p] = edge_bucket(edge_key(a[p], b[p]), g.hash_shift);
    for (uint32_t it = 0; pending != 0 && it <= g.hash_mask; ++it) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (pending >> p & 1u) {
                const Sector e = ld8s<PM>(g.hash + 2 * (uint64_t)bk[p]);
                const uint64_t key = edge_key(a[p], b[p]);
                const uint32_t lo = (uint32_t)key, hi = (uint32_t)(key >> 32);
                const bool hit = (e.lo.x == lo && e.lo.y == hi) || (e.lo.z == lo && e.lo.w == hi) ||
                                 (e.hi.x == lo && e.hi.y == hi) || (e.hi.z == lo && e.hi.w == hi);
                if (hit) {
                    found |= 1u << p;
                    pending &= ~(1u << p);
                } else if (e.hi.z == 0xffffffffu && e.hi.w == 0xffffffffu) {   // last slot empty
                    pending &= ~(1u << p);
                } else {
                    bk[p] = (bk[p] + 1) & g.hash_mask;
                }
            }
        }
    }
    return found;
}

struct Sample {
    uint32_t v[5];
    int cls;
};

template <int RNG, bool HASH, int PM = kPmPlain>
__device__ __forceinline__ Sample sample_moss4(const DevGraph &g, const uint8_t *lut, uint64_t seed, uint64_t s) {
    Sample out;
    const Words2 x01 = sample_words2<RNG>(seed, 0, s, 0);
    const VertexPick pv = draw_vertex<PM, RNG>(g, 0, g.vert, seed, s, 6, x01.x[0], x01.x[1]);   // x6: level
    const uint32_t v = pv.v;
    const uint4 vr = pv.rec;
    const Words2 x23 = sample_words2<RNG>(seed, 0, s, 1);
    const Pick pu = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x23.x[0], x23.x[1]);
    const Words2 x45 = sample_words2<RNG>(seed, 0, s, 2);
    const uint32_t jw = skip1((uint32_t)word_index(x45.x[0], vr.y - 1), pu.pos);
    const uint32_t w = ldc<PM>(g.col + vr.x + jw);
    const uint32_t jr = skip1((uint32_t)word_index(x45.x[1], pu.deg - 1), pu.twin);
    const uint32_t r = ldc<PM>(g.col + pu.off + jr);
    out.v[0] = v; out.v[1] = pu.id; out.v[2] = w; out.v[3] = r; out.v[4] = 0;
    if (r == pu.id || r == w) {
        out.cls = 0;
        return out;
    }
    // unknown pairs: v-r, u-w, w-r
    const uint32_t A[3] = {v, pu.id, w}, B[3] = {r, w, r};
    uint32_t f;
    if (HASH) {
        f = probe_hash<3, PM, kHubProbes[0]>(g, A, B);
    } else {
        const uint4 ur = make_uint4(pu.off, pu.deg, 0u, 0u), wr = ld4(g.vert + w), rr = ld4(g.vert + r);
        const uint4 ra[3] = {vr, ur, wr}, rb[3] = {rr, wr, rr};
        f = probe_pairs<3>(g.col, ra, rb, A, B);
    }
    // pair bits (0,1)(0,2)(0,3)(1,2)(1,3)(2,3); known: v-u, v-w, u-r
    const uint32_t mask = 0x1u | 0x2u | ((f & 1u) << 2) | (((f >> 1) & 1u) << 3) | 0x10u | (((f >> 2) & 1u) << 5);
    out.cls = lut[mask];
    return out;
}

template <int RNG, bool HASH, int PM = kPmPlain>
__device__ __forceinline__ Sample sample_t5(const DevGraph &g, const uint8_t *lut, uint64_t seed, uint64_t s) {
    Sample out;
    const Words2 x01 = sample_words2<RNG>(seed, 1, s, 0);
    const VertexPick pv = draw_vertex<PM, RNG>(g, 1, g.vert, seed, s, 7, x01.x[0], x01.x[1]);   // x7: level
    const uint32_t v = pv.v;
    const uint4 vr = pv.rec;
    const Words2 x23 = sample_words2<RNG>(seed, 1, s, 1);
    const Pick pu = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x23.x[0], x23.x[1]);
    const Words2 x45 = sample_words2<RNG>(seed, 1, s, 2);
    const uint32_t jw = skip1((uint32_t)word_index(x45.x[0], vr.y - 1), pu.pos);
    const uint32_t jr = skip2((uint32_t)word_index(x45.x[1], vr.y - 2), pu.pos, jw);
    const uint32_t w = ldc<PM>(g.col + vr.x + jw);
    const uint32_t r = ldc<PM>(g.col + vr.x + jr);
    const uint32_t jt = skip1((uint32_t)word_index(sample_word<RNG>(seed, 1, s, 6), pu.deg - 1), pu.twin);
    const uint32_t t = ldc<PM>(g.col + pu.off + jt);
    out.v[0] = v; out.v[1] = pu.id; out.v[2] = w; out.v[3] = r; out.v[4] = t;
    if (t == w || t == r) {
        out.cls = 0;
        return out;
    }
    // unknown pairs: u-w, u-r, w-r, v-t, w-t, r-t
    const uint32_t A[6] = {pu.id, pu.id, w, v, w, r}, B[6] = {w, r, r, t, t, t};
    uint32_t f;
    if (HASH) {
        f = probe_hash<6, PM, kHubProbes[1]>(g, A, B);
    } else {
        const uint4 ur = make_uint4(pu.off, pu.deg, 0u, 0u);
        const uint4 wr = ld4(g.vert + w), rr = ld4(g.vert + r), tr = ld4(g.vert + t);
        const uint4 ra[6] = {ur, ur, wr, vr, wr, rr}, rb[6] = {wr, rr, rr, tr, tr, tr};
        f = probe_pairs<6>(g.col, ra, rb, A, B);
    }
    // pair bits (0,1)(0,2)(0,3)(0,4)(1,2)(1,3)(1,4)(2,3)(2,4)(3,4)
    // known: v-u (0), v-w (1), v-r (2), u-t (6)
    uint32_t mask = 0x1u | 0x2u | 0x4u | 0x40u;
    mask |= ((f >> 0) & 1u) << 4;   // u-w
    mask |= ((f >> 1) & 1u) << 5;   // u-r
    mask |= ((f >> 2) & 1u) << 7;   // w-r
    mask |= ((f >> 3) & 1u) << 3;   // v-t
    mask |= ((f >> 4) & 1u) << 8;   // w-t
    mask |= ((f >> 5) & 1u) << 9;   // r-t
    out.cls = lut[mask];
    return out;
}

// ------------------------------------------------------------- MOSS-4Min --

// order bits of the four roles for the c(s) table: bit b set when the first
// role of pair b ((0,1),(0,2),(0,3),(1,2),(1,3),(2,3)) is above the second;
// key[] holds the order keys (d_x << 32) | x
__device__ __forceinline__ uint32_t order_bits(const uint64_t (&key)[4]) {
    return (uint32_t)(key[0] > key[1]) | (uint32_t)(key[0] > key[2]) << 1 | (uint32_t)(key[0] > key[3]) << 2 |
           (uint32_t)(key[1] > key[2]) << 3 | (uint32_t)(key[1] > key[3]) << 4 | (uint32_t)(key[2] > key[3]) << 5;
}

// count slot of a MOSS-4Min hit: 4-cycles 0..3, diamonds 4..9, 4-cliques
// 10..21 by c; kSlots (not counted) for collisions and the other classes
__device__ __forceinline__ int min_slot(int cls, uint32_t c) {
    if (cls == 3 && c >= 1 && c <= 4) return (int)c - 1;
    if (cls == 5 && c >= 1 && c <= 6) return 4 + (int)c - 1;
    if (cls == 6 && c >= 1 && c <= 12) return 10 + (int)c - 1;
    return kSlots;
}

template <int RNG, bool HASH, int PM = kPmPlain>
__device__ __forceinline__ Sample sample_min(const DevGraph &g, const uint8_t *lut, const uint8_t *lutc, uint64_t seed,
                                             uint64_t s) {
    Sample out;
    const Words2 x01 = sample_words2<RNG>(seed, 3, s, 0);
    const VertexPick pv = draw_vertex<PM, RNG>(g, 3, g.mvert, seed, s, 6, x01.x[0], x01.x[1]);   // x6: level
    const uint32_t v = pv.v;
    const uint4 mv = pv.rec;                           // {off, d_v, Gamma-check_v}
    const uint64_t Gv = ((uint64_t)mv.w << 32) | mv.z;
    // WeightRandomVertex(N_v, sigma-check^(v)): from a list with
    // Gamma-check_v < 2^32, one pick record carries the draw and both
    // possible picks; otherwise (or when a field overflows 16 bits) the slot
    // record, and the alias position's when the column does not keep the draw
    const Words2 x23 = sample_words2<RNG>(seed, 3, s, 1);
    const uint32_t j = (uint32_t)word_index(x23.x[0], mv.y);
    const uint64_t y = word_index(x23.x[1], Gv);
    uint4 sb;   // {off_u, d_u, d_{v,u}, d_{u,v}}
    uint32_t u;
    Sector pk;
    pk.hi.w = kSlotHub;
    if (mv.w == 0) pk = ld8p<PM>(g.mpick + 2 * (uint64_t)(mv.x + j));
    if (pk.hi.w != kSlotHub) {
        const bool keep = y < pk.lo.x;
        const uint32_t dd = keep ? pk.lo.w : pk.hi.z;
        u = keep ? pk.lo.y : pk.hi.x;
        sb = make_uint4(keep ? pk.lo.z : pk.hi.y, keep ? (pk.hi.w & 0xffffu) : (pk.hi.w >> 16), dd & 0xffffu,
                        dd >> 16);
    } else {
        Sector ms = ld8s<PM == kPmFilter ? kPmPlain : PM>(g.mslot + 2 * (uint64_t)(mv.x + j));
        if (!(y < (((uint64_t)ms.lo.y << 32) | ms.lo.x)))
            ms = ld8s<PM == kPmFilter ? kPmPlain : PM>(g.mslot + 2 * (uint64_t)(mv.x + ms.lo.z));
        sb = ms.hi;
        u = ms.lo.w;
    }
    const Words2 x45 = sample_words2<RNG>(seed, 3, s, 2);
    const uint2 we = ld2(g.rlist + mv.x + (uint32_t)word_index(x45.x[0], sb.z));   // w in N_{v,u}
    const uint2 re = ld2(g.rlist + sb.x + (uint32_t)word_index(x45.x[1], sb.w));   // r in N_{u,v}
    const uint32_t w = we.x, r = re.x;
    out.v[0] = v; out.v[1] = u; out.v[2] = w; out.v[3] = r; out.v[4] = 0;
    if (r == u || r == w) {
        out.cls = 0;
        return out;
    }
    // unknown pairs: v-r, u-w, w-r
    const uint32_t A[3] = {v, u, w}, B[3] = {r, w, r};
    uint32_t f;
    if (HASH) {
        f = probe_hash<3, PM, kHubProbes[3]>(g, A, B);
    } else {
        const uint4 vr = make_uint4(mv.x, mv.y, 0u, 0u), ur = make_uint4(sb.x, sb.y, 0u, 0u);
        const uint4 wr = ld4(g.vert + w), rr = ld4(g.vert + r);
        const uint4 ra[3] = {vr, ur, wr}, rb[3] = {rr, wr, rr};
        f = probe_pairs<3>(g.col, ra, rb, A, B);
    }
    // known: v-u, v-w, u-r
    const uint32_t mask = 0x1u | 0x2u | ((f & 1u) << 2) | (((f >> 1) & 1u) << 3) | 0x10u | (((f >> 2) & 1u) << 5);
    out.cls = lut[mask];
    // c(s) from the table (zero for the classes MOSS-4Min does not count)
    const uint64_t key[4] = {((uint64_t)mv.y << 32) | v, ((uint64_t)sb.y << 32) | u, ((uint64_t)we.y << 32) | w,
                             ((uint64_t)re.y << 32) | r};
    out.v[4] = lutc[mask << 6 | order_bits(key)];
    return out;
}

// Path-5 fallback: u from tau^(v), w from mu^(v,u) (Sec. 5.1.4).  The
// prefix of the tau weights w_i (S - w_i), w_i = d_x - 1, is S ACC[p] - sq[p],
// so u is the last position whose prefix is <= y, found by binary search
// (the same position a scan of the running sum gives); w by the search of
// ACC with u's interval removed.
__device__ __noinline__ void path5_fallback(const uint32_t *acc, const uint64_t *sq, uint32_t v, uint4 vr,
                                            uint64_t x12, uint64_t x13, uint32_t &iu, uint32_t &iw) {
    const uint32_t o = vr.x, d = vr.y, S = vr.z;
    const uint32_t wl = S - ld1(acc + o + d - 1);
    const uint64_t Q = __ldg(sq + o + d - 1) + (uint64_t)wl * wl;
    const uint64_t G = (uint64_t)S * S - Q;
    const uint64_t y = word_index(x12, G);
    {
        uint32_t lo = 0, len = d;   // first p with prefix(p) > y
        while (len > 0) {
            const uint32_t half = len >> 1, p = lo + half;
            const uint64_t f = (uint64_t)S * ld1(acc + o + p) - __ldg(sq + o + p);
            if (f <= y) {
                lo = p + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        iu = lo - 1;
    }
    const uint32_t au = ld1(acc + o + iu);
    const uint32_t wu = (iu + 1 < d ? ld1(acc + o + iu + 1) : S) - au;
    uint64_t y2 = word_index(x13, (uint64_t)(S - wu));
    if (y2 >= au) y2 += wu;
    // last i with ACC[i] <= y2
    uint32_t lo = 0, len = d;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if ((uint64_t)ld1(acc + o + lo + half) <= y2) { lo += half + 1; len -= half + 1; } else { len = half; }
    }
    iw = lo - 1;
}

// Path-5 in stages, so that the rare paths do not set the register budget
// of the common one: STAGE 0 takes the first attempt and returns kDeferred
// when it collides (the main launch); STAGE 1 the second attempt of such a
// sample, again kDeferred when it collides; STAGE 2 the fallback of a sample
// whose two attempts collided; STAGE 3 all three in turn.  The draws depend
// only on the sample id, so the stages give the sample the same result as
// STAGE 3.
constexpr int kDeferred = 254;

template <int RNG, bool HASH, int STAGE, int PM = kPmPlain>
__device__ __forceinline__ Sample sample_path5(const DevGraph &g, const uint8_t *lut, uint64_t seed, uint64_t s) {
    Sample out;
    const Words2 x01 = sample_words2<RNG>(seed, 2, s, 0);
    const VertexPick pv = draw_vertex<PM, RNG>(g, 2, g.vert, seed, s, 14, x01.x[0], x01.x[1]);   // x14: level
    const uint32_t v = pv.v;
    const uint4 vr = pv.rec;
    Pick pu, pw;
    bool collide = true;
    if (STAGE == 0 || STAGE == 3) {
        const Words2 x45 = sample_words2<RNG>(seed, 2, s, 2);
        const Words2 x67 = sample_words2<RNG>(seed, 2, s, 3);
        pu = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x45.x[0], x45.x[1]);
        pw = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x67.x[0], x67.x[1]);
        collide = pu.pos == pw.pos;
        if (STAGE == 0 && collide) {
            out.cls = kDeferred;
            return out;
        }
    }
    if (STAGE == 1 || (STAGE == 3 && collide)) {
        const Words2 x89 = sample_words2<RNG>(seed, 2, s, 4);
        const Words2 x1011 = sample_words2<RNG>(seed, 2, s, 5);
        pu = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x89.x[0], x89.x[1]);
        pw = draw_sigma<PM>(g.slot, g.vert, vr.x, vr.y, vr.z, x1011.x[0], x1011.x[1]);
        collide = pu.pos == pw.pos;
        if (STAGE == 1 && collide) {
            out.cls = kDeferred;
            return out;
        }
    }
    if (STAGE == 2 || (STAGE == 3 && collide)) {
        const Words2 x1213 = sample_words2<RNG>(seed, 2, s, 6);
        uint32_t iu, iw;
        path5_fallback(g.acc, g.sq, v, vr, x1213.x[0], x1213.x[1], iu, iw);
        pu = slot_pick(g.slot, g.vert, vr.x, iu);
        pw = slot_pick(g.slot, g.vert, vr.x, iw);
    }
    const uint32_t u = pu.id, w = pw.id;
    const Words2 x23 = sample_words2<RNG>(seed, 2, s, 1);
    const uint32_t r = ldc<PM>(g.col + pu.off + skip1((uint32_t)word_index(x23.x[0], pu.deg - 1), pu.twin));
    const uint32_t t = ldc<PM>(g.col + pw.off + skip1((uint32_t)word_index(x23.x[1], pw.deg - 1), pw.twin));
    out.v[0] = v; out.v[1] = u; out.v[2] = w; out.v[3] = r; out.v[4] = t;
    if (t == u || r == w || t == r) {
        out.cls = 0;
        return out;
    }
    // unknown pairs: v-r, v-t, u-w, u-t, w-r, r-t
    const uint32_t A[6] = {v, v, u, u, w, r}, B[6] = {r, t, w, t, r, t};
    uint32_t f;
    if (HASH) {
        f = probe_hash<6, PM, kHubProbes[2]>(g, A, B);
    } else {
        const uint4 ur = make_uint4(pu.off, pu.deg, 0u, 0u), wr = make_uint4(pw.off, pw.deg, 0u, 0u);
        const uint4 rr = ld4(g.vert + r), tr = ld4(g.vert + t);
        const uint4 ra[6] = {vr, vr, ur, ur, wr, rr}, rb[6] = {rr, tr, wr, tr, rr, tr};
        f = probe_pairs<6>(g.col, ra, rb, A, B);
    }
    // known: v-u (0), v-w (1), u-r (5), w-t (8)
    uint32_t mask = 0x1u | 0x2u | 0x20u | 0x100u;
    mask |= ((f >> 0) & 1u) << 2;   // v-r
    mask |= ((f >> 1) & 1u) << 3;   // v-t
    mask |= ((f >> 2) & 1u) << 4;   // u-w
    mask |= ((f >> 3) & 1u) << 6;   // u-t
    mask |= ((f >> 4) & 1u) << 7;   // w-r
    mask |= ((f >> 5) & 1u) << 9;   // r-t
    out.cls = lut[mask];
    return out;
}

// Resident blocks per SM each sampler is compiled for: the loop is bound by
// memory latency, so more warps in flight help until register spills cost
// more than they hide (measured: 6 blocks of 256 threads for every main
// sampler; Path-5 reaches it only with its second attempt and fallback
// deferred).  The second-attempt launch runs 5 blocks, the fallback launch 4.
// Under Philox words the samplers and the redraw stages hold the generator's
// state beside their records and would spill at those register budgets, so
// they are compiled for one block fewer (4 for the redraws); the grid of a
// main launch follows each instance's occupancy.
template <int METHOD, int RNG>
constexpr int min_blocks() { return RNG == kRngPhilox ? 5 : 6; }
template <int STAGE>
constexpr int defer_min_blocks() { return STAGE == 1 ? 5 : 4; }
template <int STAGE, int RNG>
constexpr int defer_bound_blocks() { return RNG == kRngPhilox ? 4 : defer_min_blocks<STAGE>(); }

template <int METHOD, bool RECORD, bool HASH, int PM, int RNG>
__global__ void __launch_bounds__(kThreads, min_blocks<METHOD, RNG>()) k_sample(DevGraph g, uint64_t first, uint64_t count, uint64_t seed,
                                                     uint64_t *partials, uint8_t *classes, uint32_t *verts) {
    __shared__ uint8_t lut[kLut];
    __shared__ uint8_t lutc[METHOD == 3 ? 4096 : 1];
    __shared__ uint32_t hist[kWarps][kSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *src = (METHOD == 0 || METHOD == 3) ? g_lut4 : g_lut5;
    const int lut_n = (METHOD == 0 || METHOD == 3) ? 64 : 1024;
    for (int i = threadIdx.x; i < lut_n; i += kThreads) lut[i] = src[i];
    if (METHOD == 3)
        for (int i = threadIdx.x; i < 4096; i += kThreads) lutc[i] = g_lutc[i];
    for (int i = threadIdx.x; i < kWarps * kSlots; i += kThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    // warp-uniform loop: every lane of a warp runs the same trip count
    const uint64_t warp_base = ((uint64_t)blockIdx.x * kThreads) + (uint64_t)warp * 32;
    for (uint64_t base = warp_base; base < count; base += stride) {
        const uint64_t i = base + lane;
        int cls = kSlots;  // no sample (tail)
        bool deferred = false;
        if (i < count) {
            const uint64_t s = first + i;
            Sample sm;
            if (METHOD == 0) sm = sample_moss4<RNG, HASH, PM>(g, lut, seed, s);
            else if (METHOD == 1) sm = sample_t5<RNG, HASH, PM>(g, lut, seed, s);
            else if (METHOD == 2) sm = sample_path5<RNG, HASH, 0, PM>(g, lut, seed, s);
            else sm = sample_min<RNG, HASH, PM>(g, lut, lutc, seed, s);
            deferred = METHOD == 2 && sm.cls == kDeferred;
            if (!deferred) {
                cls = METHOD == 3 ? min_slot(sm.cls, sm.v[4]) : sm.cls;
                if (RECORD) {
                    classes[i] = (uint8_t)sm.cls;
                    if (verts) {
#pragma unroll
                        for (int k = 0; k < 5; ++k) verts[5 * i + k] = sm.v[k];
                    }
                }
            }
        }
        if (METHOD == 2) {   // one bitmap word per 32 sample ids, written by the warp that drew them
            // (streaming store: the word is read once, by the next launch, and
            // should not push the tables out of L2 meanwhile)
            const uint32_t bits = __ballot_sync(0xffffffffu, deferred);
            if (lane == 0) __stcs(g.defer + (base >> 5), bits);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, cls);
        if (cls < kSlots && lane == __ffs(peers) - 1) atomicAdd(&hist[warp][cls], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < kSlots) {
        uint64_t sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += hist[w][threadIdx.x];
        partials[(uint64_t)blockIdx.x * kSlots + threadIdx.x] = sum;
    }
}

// The Path-5 samples a launch deferred, redrawn by the next stage (STAGE 1:
// second attempt, re-deferring the samples that collide again; STAGE 2:
// fallback).  A warp takes windows of 32 bitmap words (grid-stride); it
// appends each window's flagged ids to a list in shared memory (a warp scan
// of the words' popcounts places them) and draws from the list 32 at a time,
// one per lane, keeping fewer than 32 ids over to its next window, so every
// round but the warp's last runs with all lanes busy however sparse the
// flags.  STAGE 1 clears the words it reads and sets the bits of re-deferred
// samples again (plain stores: a window's words belong to one warp).  Counts
// are aggregated as in k_sample into this launch's partial rows; STAGE 2,
// launched with no more blocks than STAGE 1, adds into STAGE 1's rows.
constexpr uint32_t kDeferList = 1024 + 32;   // a window's ids plus the carry-over

template <bool RECORD, bool HASH, int STAGE, int PM, int RNG>
__global__ void __launch_bounds__(kThreads, defer_bound_blocks<STAGE, RNG>())
    k_sample_deferred(DevGraph g, uint64_t first, uint64_t count, uint64_t seed, uint64_t *partials,
                      uint8_t *classes, uint32_t *verts) {
    static_assert(STAGE == 1 || STAGE == 2, "deferred stages are 1 and 2");
    __shared__ uint8_t lut[kLut];
    __shared__ uint32_t hist[kWarps][kSlots];
    __shared__ uint32_t list[kWarps][kDeferList];   // ids relative to the chunk's first
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kLut; i += kThreads) lut[i] = g_lut5[i];
    for (int i = threadIdx.x; i < kWarps * kSlots; i += kThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const uint64_t words = (count + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * kWarps * 32;
    uint32_t *lst = list[warp];
    // draws lst[k0 + lane] for lane < cnt (warp-uniform arguments)
    auto round = [&](uint32_t k0, uint32_t cnt) {
        int cls = kSlots;
        bool again = false;
        uint64_t i = 0;
        if ((uint32_t)lane < cnt) {
            i = lst[k0 + lane];   // < count: only drawn ids are flagged
            const Sample sm = sample_path5<RNG, HASH, STAGE, PM>(g, lut, seed, first + i);
            again = STAGE == 1 && sm.cls == kDeferred;
            if (!again) {
                cls = sm.cls;
                if (RECORD) {
                    classes[i] = (uint8_t)sm.cls;
                    if (verts) {
#pragma unroll
                        for (int k = 0; k < 5; ++k) verts[5 * i + k] = sm.v[k];
                    }
                }
            }
        }
        if (STAGE == 1 && __any_sync(0xffffffffu, again)) {
            // OR of the re-deferred bits per word; the first lane of each word stores it
            const uint64_t wi = again ? i >> 5 : ~0ull;
            const uint32_t bit = again ? 1u << (i & 31) : 0u;
            uint32_t bits = 0, first_lane = 32;
            for (int l = 0; l < 32; ++l) {
                const uint64_t wl = __shfl_sync(0xffffffffu, wi, l);
                const uint32_t bl = __shfl_sync(0xffffffffu, bit, l);
                if (wl == wi) {
                    bits |= bl;
                    first_lane = min(first_lane, (uint32_t)l);
                }
            }
            if (again && first_lane == (uint32_t)lane) g.defer[wi] |= bits;
            __syncwarp();
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, cls);
        if (cls < kSlots && lane == __ffs(peers) - 1) atomicAdd(&hist[warp][cls], (uint32_t)__popc(peers));
    };
    uint32_t n = 0;   // ids waiting in the list (warp-uniform, < 32 between windows)
    for (uint64_t w0 = ((uint64_t)blockIdx.x * kWarps + warp) * 32; w0 < words; w0 += stride) {
        const uint64_t w = w0 + lane;
        uint32_t bits = w < words ? __ldcs(g.defer + w) : 0u;
        if (STAGE == 1 && bits) g.defer[w] = 0u;   // re-deferred ids are set again by round()
        const uint32_t c = __popc(bits);
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t at = n + incl - c;
        while (bits) {
            lst[at++] = (uint32_t)(w * 32 + __ffs(bits) - 1);
            bits &= bits - 1;
        }
        n += total;
        __syncwarp();
        uint32_t done = 0;
        for (; n - done >= 32; done += 32) round(done, 32);
        if (done) {   // move the remainder (< 32 ids) to the front
            const uint32_t rem = n - done;
            const uint32_t x = (uint32_t)lane < rem ? lst[done + lane] : 0u;
            __syncwarp();
            if ((uint32_t)lane < rem) lst[lane] = x;
            __syncwarp();
            n = rem;
        }
    }
    if (n) round(0, n);
    __syncthreads();
    if (threadIdx.x < kSlots) {
        uint64_t sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += hist[w][threadIdx.x];
        uint64_t *row = partials + (uint64_t)blockIdx.x * kSlots + threadIdx.x;
        *row = STAGE == 1 ? sum : *row + sum;
    }
}

// one warp per class slot: lanes stride over the block rows, then a warp sum
// ---------------------------------------------------------------- batches --
// Many requests on many graphs in one persistent launch.  Warps take tiles
// (fixed-size runs of sample ids of one task) from a global counter -- one
// atomic per tile, none per sample -- and write each tile's class counts to
// the tile's own row, so a task's counts are the sum of its rows whatever
// warp ran which tile, and equal the counts of a solo launch of the task.
constexpr int kBatchBlocks = 4;   // resident blocks per SM (Path-5 bound)

// the count slot of sample s of a method: its class, or for MOSS-4Min its
// (class, c) slot
// (plain loads for every graph: a second, streaming body per method in the
// persistent batch kernel cost 12% on the 512-graph batch)
template <bool HASH, int RNG>
__device__ __forceinline__ int sample_any(const DevGraph &g, const uint8_t *lut4, const uint8_t *lut5,
                                          const uint8_t *lutc, uint32_t method, uint64_t seed, uint64_t s) {
    if (method == 0) return sample_moss4<RNG, HASH>(g, lut4, seed, s).cls;
    if (method == 1) return sample_t5<RNG, HASH>(g, lut5, seed, s).cls;
    if (method == 3) {
        const Sample sm = sample_min<RNG, HASH>(g, lut4, lutc, seed, s);
        return min_slot(sm.cls, sm.v[4]);
    }
    return sample_path5<RNG, HASH, 3>(g, lut5, seed, s).cls;
}

// Persistent sampler over a batch: warps take tiles of `tile_samples` ids of
// one task from a device counter.  THREADS per block is a tuning choice (the
// resident threads per SM stay the same: THREADS x blocks = 1,024).  RNGS:
// the generators the batch's graphs use (kBatchSplitMix, kBatchPhilox, or
// kBatchBoth: chosen per tile), so a single-generator batch carries one
// sampler body.  With tile_cycles non-null the first lane of a warp records
// each tile's duration in SM clock cycles (the autotuner's per-graph cost of
// a probe strategy).
template <int THREADS, int RNGS>
__global__ void __launch_bounds__(THREADS, kBatchBlocks * kThreads / THREADS)
    k_sample_batch(const DevGraph *graphs, const BatchTask *tasks, int ntasks, uint64_t ntiles, uint32_t tile_samples,
                   unsigned long long *next_tile, uint32_t *tile_counts, unsigned long long *tile_cycles) {
    constexpr int kW = THREADS / 32;
    __shared__ uint8_t lut4[64];
    __shared__ uint8_t lut5[kLut];
    __shared__ uint8_t lutc[4096];
    __shared__ uint32_t hist[kW][kSlots];
    __shared__ DevGraph gsh[kW];
    static_assert(sizeof(DevGraph) % 4 == 0 && sizeof(DevGraph) / 4 <= 64, "graph descriptor staging");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 64; i += THREADS) lut4[i] = g_lut4[i];
    for (int i = threadIdx.x; i < kLut; i += THREADS) lut5[i] = g_lut5[i];
    for (int i = threadIdx.x; i < 4096; i += THREADS) lutc[i] = g_lutc[i];
    __syncthreads();
    for (;;) {
        const long long c0 = clock64();
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_tile, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        // the task of tile t: the last task whose first tile is <= t
        int lo = 0, len = ntasks;
        while (len > 0) {
            const int half = len >> 1;
            if (tasks[lo + half].tile0 <= t) { lo += half + 1; len -= half + 1; } else { len = half; }
        }
        const BatchTask tk = tasks[lo - 1];
        for (int wd = lane; wd < (int)(sizeof(DevGraph) / 4); wd += 32)
            reinterpret_cast<uint32_t *>(&gsh[warp])[wd] = reinterpret_cast<const uint32_t *>(graphs + tk.graph)[wd];
        if (lane < kSlots) hist[warp][lane] = 0;
        __syncwarp();
        const DevGraph &g = gsh[warp];
        const uint64_t f = tk.first + (t - tk.tile0) * tile_samples;
        const uint64_t left = tk.first + tk.count - f;
        const uint32_t cnt = (uint32_t)(left < tile_samples ? left : tile_samples);
        const bool hashed = g.hash != nullptr;
        // warp-uniform: a tile belongs to one graph
        const bool philox = RNGS == kBatchPhilox || (RNGS == kBatchBoth && g.rng == kRngPhilox);
        for (uint32_t base = 0; base < cnt; base += 32) {
            const uint32_t i = base + lane;
            int cls = kSlots;
            if (i < cnt) {
                if (philox)
                    cls = hashed ? sample_any<true, kRngPhilox>(g, lut4, lut5, lutc, tk.method, tk.seed, f + i)
                                 : sample_any<false, kRngPhilox>(g, lut4, lut5, lutc, tk.method, tk.seed, f + i);
                else
                    cls = hashed ? sample_any<true, kRngSplitMix>(g, lut4, lut5, lutc, tk.method, tk.seed, f + i)
                                 : sample_any<false, kRngSplitMix>(g, lut4, lut5, lutc, tk.method, tk.seed, f + i);
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, cls);
            if (cls < kSlots && lane == __ffs(peers) - 1) atomicAdd(&hist[warp][cls], (uint32_t)__popc(peers));
        }
        __syncwarp();
        if (lane < kSlots) tile_counts[t * kSlots + lane] = hist[warp][lane];
        if (tile_cycles && lane == 0) tile_cycles[t] = (unsigned long long)(clock64() - c0);
        __syncwarp();
    }
}

// block per task, warp per class slot: sum the task's tile rows
__global__ void k_batch_reduce(const BatchTask *tasks, uint32_t tile_samples, const uint32_t *tile_counts,
                               uint64_t *task_counts) {
    const BatchTask tk = tasks[blockIdx.x];
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t nt = (tk.count + tile_samples - 1) / tile_samples;
    uint64_t s = 0;
    for (uint64_t j = lane; j < nt; j += 32) s += tile_counts[(tk.tile0 + j) * kSlots + c];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) task_counts[(uint64_t)blockIdx.x * kSlots + c] = s;
}

// accumulate: add to out (later chunks of one count) instead of overwriting
// One block of 32 x kSlots threads: thread t adds slot t % kSlots of every
// 32nd row from row t / kSlots (consecutive threads read consecutive words),
// then 32 partial sums per slot are added in shared memory.
__global__ void k_reduce(const uint64_t *partials, int blocks, uint64_t *out, int accumulate) {
    __shared__ uint64_t part[32][kSlots];
    const int c = threadIdx.x % kSlots, r0 = threadIdx.x / kSlots;
    uint64_t s = 0;
    for (int b = r0; b < blocks; b += 32) s += partials[(uint64_t)b * kSlots + c];
    part[r0][c] = s;
    __syncthreads();
    if (threadIdx.x < kSlots) {
        uint64_t t = 0;
        for (int r = 0; r < 32; ++r) t += part[r][threadIdx.x];
        out[threadIdx.x] = accumulate ? out[threadIdx.x] + t : t;
    }
}

// the probe variant of a launch: 0 list search, 1 hashed set, 2 filter in
// front of it, 3 hashed set with two-level vertex tables (kPmStream)
int probe_variant(int method, const DevGraph &g) {
    if (!g.hash) return 0;
    if (g.filter) return 2;
    return g.nheavy[method] != 0 && g.nheavy[method] <= kStreamHeavy ? 3 : 1;
}

template <int M, bool R, int RNG>
cudaError_t launch_one_rng(const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed, uint64_t *partials,
                           int blocks, uint8_t *classes, uint32_t *verts, cudaStream_t s) {
    switch (probe_variant(M, g)) {
        case 2:
            k_sample<M, R, true, kPmFilter, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        case 3:
            k_sample<M, R, true, kPmStream, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        case 1:
            k_sample<M, R, true, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        default:
            k_sample<M, R, false, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
    }
    return cudaGetLastError();
}

template <int M, bool R>
cudaError_t launch_one(const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed, uint64_t *partials,
                       int blocks, uint8_t *classes, uint32_t *verts, cudaStream_t s) {
    if (g.rng == kRngPhilox)
        return launch_one_rng<M, R, kRngPhilox>(g, first, count, seed, partials, blocks, classes, verts, s);
    return launch_one_rng<M, R, kRngSplitMix>(g, first, count, seed, partials, blocks, classes, verts, s);
}

}  // namespace

void upload_luts(const uint8_t *lut4, const uint8_t *lut5, const uint8_t *lutc) {
    cudaMemcpyToSymbol(g_lut4, lut4, 64);
    cudaMemcpyToSymbol(g_lut5, lut5, 1024);
    cudaMemcpyToSymbol(g_lutc, lutc, 4096);
}

// resident blocks per SM of each sampler variant (probe 0 search, 1 hash, 2
// filter, 3 hash with two-level tables; + 4 under Philox words) on each
// device, 0 until queried
constexpr int kProbeVariants = 4;
constexpr int kVariants = 2 * kProbeVariants;
std::atomic<int> g_sample_per_sm[64][kMethods][kVariants];

template <int M, int RNG>
cudaError_t occupancy_probe(int *per) {
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], k_sample<M, false, false, kPmPlain, RNG>, kThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], k_sample<M, false, true, kPmPlain, RNG>, kThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], k_sample<M, false, true, kPmFilter, RNG>, kThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[3], k_sample<M, false, true, kPmStream, RNG>, kThreads, 0);
    return e;
}

template <int M>
cudaError_t occupancy_all(int (&per)[kVariants]) {
    cudaError_t e = occupancy_probe<M, kRngSplitMix>(per);
    if (e == cudaSuccess) e = occupancy_probe<M, kRngPhilox>(per + kProbeVariants);
    return e;
}

// resident blocks per SM of a variant (at least 1)
int sample_per_sm(int method, int device, int variant) {
    const bool cached = device >= 0 && device < 64 && method >= 0 && method < kMethods;
    if (cached) {
        const int c = g_sample_per_sm[device][method][variant].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int per[kVariants] = {1, 1, 1, 1, 1, 1, 1, 1};
    cudaError_t e;
    if (method == 0) e = occupancy_all<0>(per);
    else if (method == 1) e = occupancy_all<1>(per);
    else if (method == 2) e = occupancy_all<2>(per);
    else e = occupancy_all<3>(per);
    for (int v = 0; v < kVariants; ++v) {
        if (e != cudaSuccess || per[v] < 1) per[v] = 1;
        if (cached && e == cudaSuccess) g_sample_per_sm[device][method][v].store(per[v], std::memory_order_relaxed);
    }
    return per[variant];
}

int sample_blocks(int method, int device) {
    int per = 1;
    for (int v = 0; v < kVariants; ++v) per = std::max(per, sample_per_sm(method, device, v));
    return device_sms(device) * per;   // the most any variant launches
}

int sample_launch_blocks(int method, int device, const DevGraph &g) {
    return device_sms(device) *
           sample_per_sm(method, device, probe_variant(method, g) + (g.rng == kRngPhilox ? kProbeVariants : 0));
}

namespace {

cudaError_t launch_sample(int method, const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed,
                          uint64_t *partials, int blocks, uint8_t *classes, uint32_t *verts, cudaStream_t s) {
    const bool rec = classes != nullptr;
    switch (method * 2 + (rec ? 1 : 0)) {
        case 0: return launch_one<0, false>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 1: return launch_one<0, true>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 2: return launch_one<1, false>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 3: return launch_one<1, true>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 4: return launch_one<2, false>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 5: return launch_one<2, true>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 6: return launch_one<3, false>(g, first, count, seed, partials, blocks, classes, verts, s);
        case 7: return launch_one<3, true>(g, first, count, seed, partials, blocks, classes, verts, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int STAGE, int RNG>
cudaError_t launch_deferred_rng(const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed, uint64_t *partials,
                                int blocks, uint8_t *classes, uint32_t *verts, cudaStream_t s) {
    const bool rec = classes != nullptr;
    switch (probe_variant(2, g)) {
        case 2:
            if (rec) k_sample_deferred<true, true, STAGE, kPmFilter, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            else k_sample_deferred<false, true, STAGE, kPmFilter, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        case 3:
            if (rec) k_sample_deferred<true, true, STAGE, kPmStream, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            else k_sample_deferred<false, true, STAGE, kPmStream, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        case 1:
            if (rec) k_sample_deferred<true, true, STAGE, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            else k_sample_deferred<false, true, STAGE, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            break;
        default:
            if (rec) k_sample_deferred<true, false, STAGE, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
            else k_sample_deferred<false, false, STAGE, kPmPlain, RNG><<<blocks, kThreads, 0, s>>>(g, first, count, seed, partials, classes, verts);
    }
    return cudaGetLastError();
}

template <int STAGE>
cudaError_t launch_deferred(const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed, uint64_t *partials,
                            int blocks, uint8_t *classes, uint32_t *verts, cudaStream_t s) {
    if (g.rng == kRngPhilox)
        return launch_deferred_rng<STAGE, kRngPhilox>(g, first, count, seed, partials, blocks, classes, verts, s);
    return launch_deferred_rng<STAGE, kRngSplitMix>(g, first, count, seed, partials, blocks, classes, verts, s);
}

// blocks of a deferred stage: its resident blocks per SM times the SMs
int defer_blocks(int device, int stage) {
    return device_sms(device) * (stage == 1 ? defer_min_blocks<1>() : defer_min_blocks<2>());
}

}  // namespace

int sample_rows(int method, int device) {
    return sample_blocks(method, device) + (method == 2 ? defer_blocks(device, 1) : 0);
}

cudaError_t launch_counts(int method, const DevGraph &g, uint64_t first, uint64_t count, uint64_t seed,
                          uint64_t *partials, uint8_t *classes, uint32_t *verts, uint64_t *counts_dev,
                          cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int blocks = sample_launch_blocks(method, dev, g);
    cudaError_t e;
    if (method != 2) {
        if ((e = launch_sample(method, g, first, count, seed, partials, blocks, classes, verts, s)) != cudaSuccess)
            return e;
        k_reduce<<<1, 32 * kSlots, 0, s>>>(partials, blocks, counts_dev, 0);
        return cudaGetLastError();
    }
    // the fallback stage adds into the first rows of the second-attempt stage
    const int d1 = defer_blocks(dev, 1), d2 = min(defer_blocks(dev, 2), d1);
    for (uint64_t c0 = 0; c0 < count; c0 += kDeferChunk) {
        const uint64_t len = count - c0 < kDeferChunk ? count - c0 : kDeferChunk;
        uint8_t *cl = classes ? classes + c0 : nullptr;
        uint32_t *vt = verts ? verts + 5 * c0 : nullptr;
        uint64_t *drows = partials + (uint64_t)blocks * kSlots;
        if ((e = launch_sample(2, g, first + c0, len, seed, partials, blocks, cl, vt, s)) != cudaSuccess) return e;
        if ((e = launch_deferred<1>(g, first + c0, len, seed, drows, d1, cl, vt, s)) != cudaSuccess) return e;
        if ((e = launch_deferred<2>(g, first + c0, len, seed, drows, d2, cl, vt, s)) != cudaSuccess) return e;
        k_reduce<<<1, 32 * kSlots, 0, s>>>(partials, blocks + d1, counts_dev, c0 > 0 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int T>
int max_per_sm_rngs(int rngs) {
    int per = 0;
    cudaError_t e;
    if (rngs == kBatchSplitMix) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sample_batch<T, kBatchSplitMix>, T, 0);
    else if (rngs == kBatchPhilox) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sample_batch<T, kBatchPhilox>, T, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sample_batch<T, kBatchBoth>, T, 0);
    return e == cudaSuccess && per > 0 ? per : 1;
}

int batch_max_per_sm(int threads, int rngs) {
    if (threads == 128) return max_per_sm_rngs<128>(rngs);
    if (threads == 512) return max_per_sm_rngs<512>(rngs);
    return max_per_sm_rngs<256>(rngs);
}

int batch_blocks(int device, int threads, int per_sm, int rngs) {
    const int max = batch_max_per_sm(threads, rngs);
    const int per = per_sm <= 0 || per_sm > max ? max : per_sm;
    return device_sms(device) * per;
}

template <int T, int R>
void launch_batch_kernel(const DevGraph *graphs, const BatchTask *tasks, int ntasks, uint64_t ntiles,
                         uint32_t tile_samples, unsigned long long *next_tile, uint32_t *tile_counts, int blocks,
                         unsigned long long *tile_cycles, cudaStream_t s) {
    k_sample_batch<T, R><<<blocks, T, 0, s>>>(graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts,
                                              tile_cycles);
}

template <int T>
void launch_batch_rngs(int rngs, const DevGraph *graphs, const BatchTask *tasks, int ntasks, uint64_t ntiles,
                       uint32_t tile_samples, unsigned long long *next_tile, uint32_t *tile_counts, int blocks,
                       unsigned long long *tile_cycles, cudaStream_t s) {
    if (rngs == kBatchSplitMix)
        launch_batch_kernel<T, kBatchSplitMix>(graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts,
                                               blocks, tile_cycles, s);
    else if (rngs == kBatchPhilox)
        launch_batch_kernel<T, kBatchPhilox>(graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts,
                                             blocks, tile_cycles, s);
    else
        launch_batch_kernel<T, kBatchBoth>(graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts,
                                           blocks, tile_cycles, s);
}

cudaError_t launch_sample_batch(const DevGraph *graphs, const BatchTask *tasks, int ntasks, uint64_t ntiles,
                                uint32_t tile_samples, unsigned long long *next_tile, uint32_t *tile_counts,
                                int threads, int blocks, unsigned long long *tile_cycles, int rngs, cudaStream_t s) {
    if (ntasks <= 0 || ntiles == 0) return cudaSuccess;
    if (threads == 128)
        launch_batch_rngs<128>(rngs, graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts, blocks,
                               tile_cycles, s);
    else if (threads == 512)
        launch_batch_rngs<512>(rngs, graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts, blocks,
                               tile_cycles, s);
    else
        launch_batch_rngs<256>(rngs, graphs, tasks, ntasks, ntiles, tile_samples, next_tile, tile_counts, blocks,
                               tile_cycles, s);
    return cudaGetLastError();
}

cudaError_t launch_batch_reduce(const BatchTask *tasks, int ntasks, uint32_t tile_samples,
                                const uint32_t *tile_counts, uint64_t *task_counts, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    k_batch_reduce<<<ntasks, 32 * kSlots, 0, s>>>(tasks, tile_samples, tile_counts, task_counts);
    return cudaGetLastError();
}

}  // namespace moss
