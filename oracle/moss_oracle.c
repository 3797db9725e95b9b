/*
 * moss_oracle.c -- plain, slow CPU oracle of the Moss sampling path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares
 * no code with the CUDA library: everything here (weights, alias tables, the
 * SplitMix64 generator, sampling, classification, enumeration) is written out
 * independently, sequentially and without any blocking or fusion.
 *
 * Paper: P. Wang, J. Tao, J. Zhao, X. Guan, "Moss: A Scalable Tool for
 * Efficiently Sampling and Counting 4- and 5-Node Graphlets" (arXiv 1509.08089).
 *
 *  - vertex weights Gamma_v (Sec. 4.1.1), Gamma^(1)_v (Sec. 5.1.1),
 *    Gamma^(2)_v (Sec. 5.1.2), Lambda_3 (eq. 2), Lambda_4 (Sec. 5.1.3),
 *    the totals of Table 1;
 *  - WeightRandomVertex (Sec. 4.1.3) realised with alias tables built by a
 *    sequential sweep (Walker/Vose alias method, sweeping variant) in exact
 *    integer arithmetic; over V, on graphs of 2^14 vertices or more, in two
 *    levels: the heavy vertices (w_v 2^t >= W, t = 12, from 2^20 vertices
 *    20, unless chosen) and the light ones each get an alias table, and a
 *    separate word picks the level with probability floor(W_light 2^64 / W)
 *    / 2^64 for the light one;
 *  - RandomVertex(N_v - X) (Sec. 4.1.3): a uniform index over the d_v - |X|
 *    admissible positions, skipping the excluded positions in list order;
 *  - MOSS-4 (Algorithm 1), T-5 (Algorithm 3), Path-5 (Algorithm 4);
 *  - the motif class of a CIS from the counts of spanning subgraphs
 *    isomorphic to M_1^(4)/M_2^(4) (Sec. 4.1.2) or M_3^(5)/M_1^(5)/M_2^(5)
 *    (Table 2);
 *  - ESU enumeration (Wernicke 2006, cited in the paper's introduction) of
 *    every connected induced k-subgraph, for exact ground truth.
 *
 * RNG: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), used in counter form: word i (0 <= i < 16) of
 * sample s of method tag t under seed k is output number (4 s + t) 16 + i + 1
 * of the generator seeded with k, i.e. mix(k + ((4 s + t) 16 + i + 1) gamma).
 * The paper draws uniform choices without fixing a generator.  The second
 * generator is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011): words 2b and 2b+1 of sample s of
 * method tag t under seed k are the four 32-bit outputs of block
 * (s mod 2^32, s div 2^32, t, b) under the key (k mod 2^32, k div 2^32),
 * low half first: x_2b = out0 + 2^32 out1, x_2b+1 = out2 + 2^32 out3.
 * Word schedule (x_i = word i):
 *   MOSS-4 : x0,x1 seed draw (column, threshold), x6 its level; x2,x3 sigma
 *            draw of u; x4 w; x5 r.
 *   T-5    : x0,x1 seed, x7 its level; x2,x3 sigma of u; x4 w; x5 r; x6 t.
 *   Path-5 : x0,x1 seed, x14 its level; x2 r; x3 t; attempt a in {0,1}: x(4+4a),x(5+4a)
 *            sigma draw of u, x(6+4a),x(7+4a) sigma draw of w, accepted when
 *            the two positions differ; if both attempts collide, x12 draws u
 *            from tau^(v) and x13 draws w from mu^(v,u) by the prefix-sum
 *            method of Sec. 5.1.4.
 * Index from a word: floor(x * m / 2^64).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* WeightRandomVertex(V, .) in two levels: columns [0, nh) form the alias
 * table of the heavy vertices (ascending ids), columns [nh, n) that of the
 * light ones; each column keeps its own vertex with probability T / 2^64 and
 * else gives its alias. */
typedef struct {
    uint32_t nh;        /* heavy vertices */
    uint64_t TL;        /* the light level is drawn iff the level word < TL */
    uint32_t *self;     /* vertex of each column */
    u128 *thr;          /* threshold in units where a column holds its level's total */
    uint64_t *T;        /* floor(thr 2^64 / level total), saturated */
    uint32_t *alias;    /* alias vertex of each column */
} vtab;

enum { M_MOSS4 = 0, M_T5 = 1, M_P5 = 2 };

/* -------------------------------------------------------- SplitMix64 ---- */
/* Output number k >= 1 of SplitMix64 seeded with seed: the state advances by
 * the Weyl increment gamma = 0x9E3779B97F4A7C15 before each output, and the
 * output is the state through the mixing function (xor-shift 30, multiply by
 * 0xBF58476D1CE4E5B9, xor-shift 27, multiply by 0x94D049BB133111EB,
 * xor-shift 31), all modulo 2^64. */
uint64_t oracle_splitmix(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Philox4x32-10: ten rounds on the counter (c0, c1, c2, c3) under the key
 * (k0, k1).  A round takes the two 64-bit products p = 0xD2511F53 c0 and
 * q = 0xCD9E8D57 c2 and makes the counter (hi(q) ^ c1 ^ k0, lo(q),
 * hi(p) ^ c3 ^ k1, lo(p)); between rounds the key grows by the Weyl
 * increments (0x9E3779B9, 0xBB67AE85) modulo 2^32. */
void oracle_philox4x32(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p = (uint64_t)0xD2511F53u * c0;
        uint64_t q = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(q >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)q;
        uint32_t n2 = (uint32_t)(p >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint64_t index_of(uint64_t x, uint64_t m) { return (uint64_t)(((u128)x * m) >> 64); }

/* ------------------------------------------------------------ context ---- */
typedef struct {
    uint32_t n;
    uint64_t nnz;
    uint64_t *off;      /* n+1 */
    uint32_t *col;      /* nnz, each list sorted */
    uint64_t *deg;      /* d_v */
    uint64_t *S, *Q;    /* sum (d_x-1), sum (d_x-1)^2 over x in N_v */
    u128 *gam[3];       /* Gamma_v, Gamma^(1)_v, Gamma^(2)_v */
    u128 tot[3];        /* Gamma, Gamma^(1), Gamma^(2) */
    u128 lam3, lam4;
    /* two-level vertex tables over V, one per weight */
    int vsplit;         /* heavy vertices: w_v 2^vsplit >= W */
    int vsplit_min;     /* the same for the MOSS-4Min table (Gamma-check) */
    vtab vt[3];
    /* sigma alias tables over each N_v (weights d_x - 1), local positions */
    uint64_t *gthr;
    uint32_t *galias;
    uint64_t *acc;      /* ACC_sigma^(v)[i] exclusive prefix (Sec. 4.1.3) */
    /* MOSS-4Min (Sec. 4.2), built on request by oracle_build_min */
    int has_min;
    uint32_t *rlist;    /* N_v ordered by the total order, highest first */
    uint64_t *rank;     /* slot (v->u): d_{v,u} = |{x in N_v : x > u}| */
    u128 *gmin;         /* Gamma-check_v = sum_{x in N_v} d_{v,x} d_{x,v} */
    u128 tmin;          /* Gamma-check */
    vtab mvt;           /* vertex table of Gamma-check */
    uint64_t *cthr;     /* per-list alias tables of sigma-check (eq. 3) */
    uint32_t *calias;
} ctx;

/* ---------------------------------------------------- alias (sweep) ---- */
/* Alias table for m items with weights w[] (exact integers).  With
 * q_j = w_j m and total W = sum w, every column holds W: item j keeps
 * thr_j of its column and the rest W - thr_j belongs to alias_j.  Items with
 * q_j < W ("light") are filled in index order from the current "heavy" item
 * (q_j >= W, index order); a heavy item whose residue drops below W is filled
 * from the next heavy item.  Zero weights are light with thr 0 and are never
 * an alias.  thr is in [0, W]. */
static int alias_sweep(uint64_t m, const u128 *w, u128 *thr, uint32_t *alias) {
    u128 W = 0;
    for (uint64_t j = 0; j < m; j++) W += w[j];
    if (W == 0) {
        for (uint64_t j = 0; j < m; j++) { thr[j] = 0; alias[j] = (uint32_t)j; }
        return 0;
    }
    uint64_t *L = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint64_t *H = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    if (!L || !H) { free(L); free(H); return -1; }
    uint64_t nl = 0, nh = 0;
    for (uint64_t j = 0; j < m; j++) {
        if (w[j] * m < W) L[nl++] = j; else H[nh++] = j;
    }
    uint64_t h = 0;
    u128 r = w[H[0]] * m;                      /* residue of the current heavy item */
    for (uint64_t i = 0; i < nl; i++) {
        uint64_t j = L[i];
        thr[j] = w[j] * m;
        alias[j] = (uint32_t)H[h];
        r -= W - w[j] * m;
        while (r < W && h + 1 < nh) {          /* the heavy item turned light */
            thr[H[h]] = r;
            alias[H[h]] = (uint32_t)H[h + 1];
            h++;
            r = w[H[h]] * m - (W - thr[H[h - 1]]);
        }
    }
    for (; h < nh; h++) { thr[H[h]] = W; alias[H[h]] = (uint32_t)H[h]; }
    free(L);
    free(H);
    return 0;
}

/* floor(thr 2^64 / W) for thr <= W, saturated to 2^64-1 (binary long division) */
static uint64_t quantize(u128 thr, u128 W) {
    if (W == 0) return 0;
    if (thr >= W) return UINT64_MAX;
    uint64_t q = 0;
    u128 r = thr;
    for (int i = 0; i < 64; i++) {
        int carry = (int)(r >> 127);
        r <<= 1;
        q <<= 1;
        if (carry || r >= W) { r -= W; q |= 1; }
    }
    return q;
}

static void vtab_free(vtab *t) {
    free(t->self); free(t->thr); free(t->T); free(t->alias);
    t->self = NULL; t->thr = NULL; t->T = NULL; t->alias = NULL;
}

/* The two-level table of weights w[0..n) with total W: heavy iff
 * w_v >= ceil(W / 2^split) (so at most 2^split of them); each level's table
 * is the sweep over its vertices in ascending id order; the light level is
 * drawn iff the level word < floor(W_L 2^64 / W).  split = 64: no heavy
 * level, one table over all vertices.  W = 0: never drawn. */
static int vtab_build(vtab *t, uint32_t n, const u128 *w, u128 W, int split) {
    uint64_t n1 = n ? n : 1;
    t->self = (uint32_t *)malloc(sizeof(uint32_t) * n1);
    t->thr = (u128 *)malloc(sizeof(u128) * n1);
    t->T = (uint64_t *)malloc(sizeof(uint64_t) * n1);
    t->alias = (uint32_t *)malloc(sizeof(uint32_t) * n1);
    u128 *sw = (u128 *)malloc(sizeof(u128) * n1);
    u128 *st = (u128 *)malloc(sizeof(u128) * n1);
    uint32_t *sa = (uint32_t *)malloc(sizeof(uint32_t) * n1);
    if (!t->self || !t->thr || !t->T || !t->alias || !sw || !st || !sa) {
        free(sw); free(st); free(sa);
        vtab_free(t);
        return -1;
    }
    t->nh = 0;
    t->TL = 0;
    if (W == 0) {
        for (uint32_t v = 0; v < n; v++) { t->self[v] = v; t->thr[v] = 0; t->T[v] = 0; t->alias[v] = v; }
        free(sw); free(st); free(sa);
        return 0;
    }
    const int one_level = split >= 64;
    u128 cut = one_level ? 0 : W >> split;
    if (!one_level && (cut << split) != W) cut += 1;   /* ceil(W / 2^split) */
    uint32_t k = 0;
    u128 WH = 0;
    for (uint32_t v = 0; v < n; v++)
        if (!one_level && w[v] >= cut) { t->self[k++] = v; WH += w[v]; }
    t->nh = k;
    for (uint32_t v = 0; v < n; v++)
        if (one_level || w[v] < cut) t->self[k++] = v;
    const u128 WL = W - WH;
    for (int level = 0; level < 2; level++) {
        const uint32_t c0 = level == 0 ? 0 : t->nh, m = level == 0 ? t->nh : n - t->nh;
        const u128 Wl = level == 0 ? WH : WL;
        for (uint32_t i = 0; i < m; i++) sw[i] = w[t->self[c0 + i]];
        if (alias_sweep(m, sw, st, sa)) { free(sw); free(st); free(sa); vtab_free(t); return -1; }
        for (uint32_t i = 0; i < m; i++) {
            t->thr[c0 + i] = st[i];
            t->T[c0 + i] = quantize(st[i], Wl);
            t->alias[c0 + i] = t->self[c0 + sa[i]];
        }
    }
    t->TL = t->nh == 0 ? 0 : quantize(WL, W);
    free(sw); free(st); free(sa);
    return 0;
}

/* WeightRandomVertex with a two-level table: level word xl, column word xc,
 * threshold word xt */
static uint32_t vtab_draw(const vtab *t, uint32_t n, uint64_t xl, uint64_t xc, uint64_t xt) {
    const int light = t->nh == 0 || xl < t->TL;
    const uint64_t m = light ? n - t->nh : t->nh;
    const uint64_t col = (light ? t->nh : 0) + index_of(xc, m);
    return xt < t->T[col] ? t->self[col] : t->alias[col];
}

/* standalone entry for tests: weights as lo/hi u64 pairs */
int oracle_alias_build(uint64_t m, const uint64_t *w_lohi, uint64_t *thr_lohi, uint32_t *alias) {
    u128 *w = (u128 *)malloc(sizeof(u128) * (m ? m : 1));
    u128 *t = (u128 *)malloc(sizeof(u128) * (m ? m : 1));
    if (!w || !t) { free(w); free(t); return -1; }
    for (uint64_t j = 0; j < m; j++) w[j] = ((u128)w_lohi[2 * j + 1] << 64) | w_lohi[2 * j];
    int rc = alias_sweep(m, w, t, alias);
    for (uint64_t j = 0; j < m; j++) { thr_lohi[2 * j] = (uint64_t)t[j]; thr_lohi[2 * j + 1] = (uint64_t)(t[j] >> 64); }
    free(w);
    free(t);
    return rc;
}

/* ------------------------------------------------------ construction ---- */
void oracle_free(ctx *c) {
    if (!c) return;
    free(c->off); free(c->col); free(c->deg); free(c->S); free(c->Q);
    for (int l = 0; l < 3; l++) { free(c->gam[l]); vtab_free(&c->vt[l]); }
    free(c->gthr); free(c->galias); free(c->acc);
    free(c->rlist); free(c->rank); free(c->gmin); vtab_free(&c->mvt);
    free(c->cthr); free(c->calias);
    free(c);
}

static u128 choose(uint64_t d, int k) {
    if (d < (uint64_t)k) return 0;
    u128 r = 1;
    for (int i = 0; i < k; i++) r = r * (u128)(d - (uint64_t)i) / (u128)(i + 1);
    return r;
}

/* vsplit: heavy vertices of the vertex tables have w_v 2^vsplit >= W (0..63;
 * 64: one level) */
ctx *oracle_new_split(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int vsplit) {
    if (vsplit < 0 || vsplit > 64) return NULL;
    ctx *c = (ctx *)calloc(1, sizeof(ctx));
    if (!c) return NULL;
    c->n = n;
    c->vsplit = vsplit;
    c->vsplit_min = vsplit;
    c->nnz = row_ptr[n];
    uint64_t nnz1 = c->nnz ? c->nnz : 1;
    c->off = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    c->col = (uint32_t *)malloc(sizeof(uint32_t) * nnz1);
    c->deg = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    c->S = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    c->Q = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    c->gthr = (uint64_t *)malloc(sizeof(uint64_t) * nnz1);
    c->galias = (uint32_t *)malloc(sizeof(uint32_t) * nnz1);
    c->acc = (uint64_t *)malloc(sizeof(uint64_t) * nnz1);
    if (!c->off || !c->col || !c->deg || !c->S || !c->Q || !c->gthr || !c->galias || !c->acc) { oracle_free(c); return NULL; }
    memcpy(c->off, row_ptr, sizeof(uint64_t) * (n + 1));
    if (c->nnz) memcpy(c->col, col, sizeof(uint32_t) * c->nnz);
    for (uint32_t v = 0; v < n; v++) c->deg[v] = c->off[v + 1] - c->off[v];

    /* Initialization (Sec. 4.1.3): S_v, Q_v, then the three vertex weights */
    for (uint32_t v = 0; v < n; v++) {
        for (uint64_t p = c->off[v]; p < c->off[v + 1]; p++) {
            uint64_t dx = c->deg[c->col[p]];
            c->S[v] += dx - 1;
            c->Q[v] += (dx - 1) * (dx - 1);
        }
    }
    for (int l = 0; l < 3; l++) {
        c->gam[l] = (u128 *)malloc(sizeof(u128) * (n ? n : 1));
        if (!c->gam[l]) { oracle_free(c); return NULL; }
    }
    for (uint32_t v = 0; v < n; v++) {
        uint64_t d = c->deg[v];
        u128 S = c->S[v];
        /* Gamma_v = (d_v - 1) sum_{x in N_v} (d_x - 1)              (Sec. 4.1.1) */
        c->gam[0][v] = d >= 1 ? (u128)(d - 1) * S : 0;
        /* Gamma^(1)_v = (d_v - 1)(d_v - 2) sum (d_x - 1)            (Sec. 5.1.1) */
        c->gam[1][v] = d >= 2 ? (u128)(d - 1) * (u128)(d - 2) * S : 0;
        /* Gamma^(2)_v = (sum (d_x - 1))^2 - sum (d_x - 1)^2         (Sec. 5.1.2) */
        c->gam[2][v] = S * S - (u128)c->Q[v];
        for (int l = 0; l < 3; l++) c->tot[l] += c->gam[l][v];
        c->lam3 += choose(d, 3);   /* Lambda_3 = sum C(d_v, 3)  (eq. 2)      */
        c->lam4 += choose(d, 4);   /* Lambda_4 = sum C(d_v, 4)  (Sec. 5.1.3) */
    }
    /* WeightRandomVertex(V, pi), (V, rho^(1)), (V, rho^(2)) tables */
    for (int l = 0; l < 3; l++)
        if (vtab_build(&c->vt[l], n, c->gam[l], c->tot[l], c->vsplit)) { oracle_free(c); return NULL; }
    /* WeightRandomVertex(N_v, sigma^(v)) tables and ACC_sigma^(v) */
    u128 *w = (u128 *)malloc(sizeof(u128) * nnz1), *t = (u128 *)malloc(sizeof(u128) * nnz1);
    if (!w || !t) { free(w); free(t); oracle_free(c); return NULL; }
    for (uint32_t v = 0; v < n; v++) {
        uint64_t o = c->off[v], d = c->deg[v];
        uint64_t run = 0;
        for (uint64_t i = 0; i < d; i++) {
            w[i] = c->deg[c->col[o + i]] - 1;
            c->acc[o + i] = run;
            run += (uint64_t)w[i];
        }
        if (alias_sweep(d, w, t, c->galias + o)) { free(w); free(t); oracle_free(c); return NULL; }
        for (uint64_t i = 0; i < d; i++) c->gthr[o + i] = (uint64_t)t[i];
    }
    free(w);
    free(t);
    return c;
}

/* the default splits: two levels with split 20 from 2^20 vertices, with
 * split 12 from 2^14, else one level; the MOSS-4Min table two levels with
 * split 20 from 2^20 vertices, else one */
ctx *oracle_new(uint32_t n, const uint64_t *row_ptr, const uint32_t *col) {
    ctx *c = oracle_new_split(n, row_ptr, col, n >= (1u << 20) ? 20 : (n >= (1u << 14) ? 12 : 64));
    if (c) c->vsplit_min = n >= (1u << 20) ? 20 : 64;
    return c;
}

/* the split of the MOSS-4Min vertex table, before oracle_build_min (0..64) */
int oracle_set_min_split(ctx *c, int vsplit) {
    if (vsplit < 0 || vsplit > 64) return -1;
    c->vsplit_min = vsplit;
    return 0;
}

/* --------------------------------------------------------- accessors ---- */
static void put128(uint64_t *dst, u128 x) { dst[0] = (uint64_t)x; dst[1] = (uint64_t)(x >> 64); }

/* out[10] = lo/hi of Gamma, Gamma^(1), Gamma^(2), Lambda_3, Lambda_4 */
void oracle_totals(const ctx *c, uint64_t *out) {
    put128(out + 0, c->tot[0]);
    put128(out + 2, c->tot[1]);
    put128(out + 4, c->tot[2]);
    put128(out + 6, c->lam3);
    put128(out + 8, c->lam4);
}

void oracle_vertex(const ctx *c, uint64_t *deg, uint64_t *S, uint64_t *Q, uint64_t *gam_lohi /* 3*2n */) {
    for (uint32_t v = 0; v < c->n; v++) {
        deg[v] = c->deg[v];
        S[v] = c->S[v];
        Q[v] = c->Q[v];
        for (int l = 0; l < 3; l++) put128(gam_lohi + (uint64_t)l * 2 * c->n + 2 * (uint64_t)v, c->gam[l][v]);
    }
}

/* the two-level vertex table of weight l (0..2; 3: Gamma-check), column order */
void oracle_vertex_table(const ctx *c, int l, uint32_t *nh, uint64_t *TL, uint32_t *self, uint64_t *thr_lohi,
                         uint64_t *T, uint32_t *alias) {
    const vtab *t = l == 3 ? &c->mvt : &c->vt[l];
    *nh = t->nh;
    *TL = t->TL;
    for (uint32_t v = 0; v < c->n; v++) {
        self[v] = t->self[v];
        put128(thr_lohi + 2 * (uint64_t)v, t->thr[v]);
        T[v] = t->T[v];
        alias[v] = t->alias[v];
    }
}

void oracle_sigma_table(const ctx *c, uint64_t *thr, uint32_t *alias, uint64_t *acc) {
    for (uint64_t p = 0; p < c->nnz; p++) { thr[p] = c->gthr[p]; alias[p] = c->galias[p]; acc[p] = c->acc[p]; }
}

/* --------------------------------------------------- graph primitives ---- */
/* (a, b) in E: binary search of b in the sorted list N_a */
static int is_edge(const ctx *c, uint32_t a, uint32_t b) {
    uint64_t lo = c->off[a], hi = c->off[a + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (c->col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < c->off[a + 1] && c->col[lo] == b;
}

/* POS_{a,b}: the position of b in N_a (Sec. 4.1.3); b must be a neighbour */
static uint64_t pos_of(const ctx *c, uint32_t a, uint32_t b) {
    uint64_t lo = c->off[a], hi = c->off[a + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (c->col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo - c->off[a];
}

/* ----------------------------------------------------- classification ---- */
/* Table 2 of the paper: (phi^(1), phi^(2), phi^(3)) of M_1^(5)..M_21^(5). */
static const int PHI5[21][3] = {
    {0, 1, 0}, {0, 0, 1}, {1, 0, 0}, {1, 2, 0}, {2, 2, 0}, {0, 5, 0}, {2, 1, 0},
    {2, 0, 1}, {4, 4, 0}, {4, 7, 0}, {5, 2, 1}, {4, 4, 1}, {6, 6, 0}, {10, 10, 1},
    {9, 6, 1}, {12, 6, 2}, {10, 14, 0}, {20, 24, 1}, {20, 18, 2}, {36, 36, 3}, {60, 60, 5}};
/* Sec. 4.1.2: (phi^(1), phi^(2)) of M_1^(4)..M_6^(4). */
static const int PHI4[6][2] = {{1, 0}, {0, 1}, {4, 0}, {2, 1}, {6, 2}, {12, 4}};

static int uf_find(int *p, int x) { while (p[x] != x) x = p[x]; return x; }

/* Class of the graph on k vertices whose pair (i,j), i<j, listed in the order
 * (0,1),(0,2),...,(k-2,k-1), is an edge iff its bit of mask is set.  The
 * spanning subgraphs with k-1 edges are enumerated; each is a tree when it is
 * connected, and its type follows from its degree sequence.  Returns the
 * class 1..6 / 1..21, or 0 when the graph is not connected. */
int oracle_classify(int k, uint32_t mask) {
    int pa[10], pb[10], np = 0;
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++) { pa[np] = i; pb[np] = j; np++; }
    int cnt_path = 0, cnt_star = 0, cnt_fork = 0, connected = 0;
    for (uint32_t sub = 0; sub < (1u << np); sub++) {
        if ((sub & mask) != sub) continue;
        if (__builtin_popcount(sub) != k - 1) continue;
        int deg[5] = {0, 0, 0, 0, 0}, par[5] = {0, 1, 2, 3, 4}, comps = k;
        for (int e = 0; e < np; e++) {
            if (!(sub >> e & 1)) continue;
            deg[pa[e]]++;
            deg[pb[e]]++;
            int x = uf_find(par, pa[e]), y = uf_find(par, pb[e]);
            if (x != y) { par[x] = y; comps--; }
        }
        if (comps != 1) continue;           /* not a spanning tree */
        connected = 1;
        int maxd = 0, n2 = 0;
        for (int i = 0; i < k; i++) { if (deg[i] > maxd) maxd = deg[i]; if (deg[i] == 2) n2++; }
        if (maxd == 2) cnt_path++;                    /* P4 / P5 */
        else if (maxd == k - 1) cnt_star++;           /* 3-star / 4-star */
        else if (k == 5 && maxd == 3 && n2 == 1) cnt_fork++; /* fork M_3^(5) */
    }
    if (!connected) return 0;
    if (k == 4) {
        for (int i = 0; i < 6; i++) if (PHI4[i][0] == cnt_path && PHI4[i][1] == cnt_star) return i + 1;
    } else {
        for (int i = 0; i < 21; i++)
            if (PHI5[i][0] == cnt_fork && PHI5[i][1] == cnt_path && PHI5[i][2] == cnt_star) return i + 1;
    }
    return -1; /* unreachable for a connected graph */
}

static int classify_vertices(const ctx *c, int k, const uint32_t *x) {
    uint32_t mask = 0;
    int bit = 0;
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++, bit++)
            if (is_edge(c, x[i], x[j])) mask |= 1u << bit;
    return oracle_classify(k, mask);
}

/* ----------------------------------------------------------- sampling ---- */
/* WeightRandomVertex(V, .) with the vertex table of weight l */
static uint32_t draw_seed(const ctx *c, int l, uint64_t xl, uint64_t xc, uint64_t xt) {
    return vtab_draw(&c->vt[l], c->n, xl, xc, xt);
}

/* WeightRandomVertex(N_v, sigma^(v)): returns the position in N_v */
static uint64_t draw_sigma(const ctx *c, uint32_t v, uint64_t xc, uint64_t xt) {
    uint64_t o = c->off[v];
    uint64_t j = index_of(xc, c->deg[v]);
    uint64_t y = index_of(xt, c->S[v]);
    return y < c->gthr[o + j] ? j : c->galias[o + j];
}

/* RandomVertex(N_v - {positions e1 < e2 ...}): the j-th admissible position */
static uint64_t skip1(uint64_t j, uint64_t e) { return j < e ? j : j + 1; }
static uint64_t skip2(uint64_t j, uint64_t e1, uint64_t e2) {
    uint64_t lo = e1 < e2 ? e1 : e2, hi = e1 < e2 ? e2 : e1;
    if (j >= lo) j++;
    if (j >= hi) j++;
    return j;
}

/* Path-5 (Sec. 5.1.2): the pair (u, w) with probability tau_u mu_w, given as
 * positions.  Up to two attempts draw u and w independently from sigma^(v)
 * and keep the pair when u != w; because sigma_u sigma_w / (1 - sum sigma^2)
 * equals tau_u mu_w, each accepted attempt has the paper's law.  When both
 * attempts collide, u is drawn from tau^(v) and then w from mu^(v,u) with the
 * ACC array and the interval of u removed (Sec. 5.1.4), which has that same
 * law; the mixture is therefore exact. */
static void draw_pair(const ctx *c, uint32_t v, const uint64_t *x, uint64_t *pu, uint64_t *pw) {
    for (int a = 0; a < 2; a++) {
        uint64_t iu = draw_sigma(c, v, x[4 + 4 * a], x[5 + 4 * a]);
        uint64_t iw = draw_sigma(c, v, x[6 + 4 * a], x[7 + 4 * a]);
        if (iu != iw) { *pu = iu; *pw = iw; return; }
    }
    uint64_t o = c->off[v], d = c->deg[v], S = c->S[v];
    /* u from tau^(v): weight (d_u - 1)(S_v - (d_u - 1)), total Gamma^(2)_v */
    u128 G = c->gam[2][v];
    uint64_t y = index_of(x[12], (uint64_t)G);
    u128 run = 0;
    uint64_t iu = 0;
    for (uint64_t i = 0; i < d; i++) {
        uint64_t wi = c->deg[c->col[o + i]] - 1;
        u128 tw = (u128)wi * (S - wi);
        if ((u128)y < run + tw) { iu = i; break; }
        run += tw;
    }
    /* w from mu^(v,u): rnd over [0, S_v) minus the interval of u */
    uint64_t wu = c->deg[c->col[o + iu]] - 1;
    uint64_t y2 = index_of(x[13], S - wu);
    if (y2 >= c->acc[o + iu]) y2 += wu;
    uint64_t iw = 0;
    for (uint64_t i = 0; i < d; i++)
        if (c->acc[o + i] <= y2) iw = i;   /* last i with ACC[i] <= rnd */
    *pu = iu;
    *pw = iw;
}

/* One sample from explicit words x[0..13].  Writes the k vertices in role
 * order (v,u,w,r[,t]) and returns the class (0 = collision, no CIS). */
static int sample_one(const ctx *c, int method, const uint64_t *x, uint32_t *out) {
    if (method == M_MOSS4) {
        /* Algorithm 1 */
        uint32_t v = draw_seed(c, 0, x[6], x[0], x[1]);
        uint64_t ov = c->off[v], dv = c->deg[v];
        uint64_t iu = draw_sigma(c, v, x[2], x[3]);
        uint32_t u = c->col[ov + iu];
        uint32_t w = c->col[ov + skip1(index_of(x[4], dv - 1), iu)];
        uint64_t ou = c->off[u], du = c->deg[u];
        uint32_t r = c->col[ou + skip1(index_of(x[5], du - 1), pos_of(c, u, v))];
        out[0] = v; out[1] = u; out[2] = w; out[3] = r; out[4] = 0;
        if (r == u || r == w) return 0;
        return classify_vertices(c, 4, out);
    }
    if (method == M_T5) {
        /* Algorithm 3 */
        uint32_t v = draw_seed(c, 1, x[7], x[0], x[1]);
        uint64_t ov = c->off[v], dv = c->deg[v];
        uint64_t iu = draw_sigma(c, v, x[2], x[3]);
        uint32_t u = c->col[ov + iu];
        uint64_t iw = skip1(index_of(x[4], dv - 1), iu);
        uint32_t w = c->col[ov + iw];
        uint32_t r = c->col[ov + skip2(index_of(x[5], dv - 2), iu, iw)];
        uint64_t ou = c->off[u], du = c->deg[u];
        uint32_t t = c->col[ou + skip1(index_of(x[6], du - 1), pos_of(c, u, v))];
        out[0] = v; out[1] = u; out[2] = w; out[3] = r; out[4] = t;
        if (t == w || t == r) return 0;
        return classify_vertices(c, 5, out);
    }
    /* Algorithm 4 */
    uint32_t v = draw_seed(c, 2, x[14], x[0], x[1]);
    uint64_t ov = c->off[v];
    uint64_t iu, iw;
    draw_pair(c, v, x, &iu, &iw);
    uint32_t u = c->col[ov + iu], w = c->col[ov + iw];
    uint32_t r = c->col[c->off[u] + skip1(index_of(x[2], c->deg[u] - 1), pos_of(c, u, v))];
    uint32_t t = c->col[c->off[w] + skip1(index_of(x[3], c->deg[w] - 1), pos_of(c, w, v))];
    out[0] = v; out[1] = u; out[2] = w; out[3] = r; out[4] = t;
    if (t == u || r == w || t == r) return 0;
    return classify_vertices(c, 5, out);
}

/* validity of a method on this graph: its total weight must be positive */
static int method_ok(const ctx *c, int method) {
    if (method == 3) return c->has_min && c->tmin != 0;
    if (method < 0 || method > 2) return 0;
    return c->tot[method] != 0;
}

static int sample_min(const ctx *c, const uint64_t *x, uint32_t *out, int *cp);
static int min_slot(int cls, int cp);

/* One sample from explicit words.  Method 3 (MOSS-4Min) puts c(s) in verts[4]. */
int oracle_sample_words(const ctx *c, int method, const uint64_t *words, uint32_t *verts, int *cls) {
    if (!method_ok(c, method)) return -1;
    if (method == 3) {
        int cp;
        *cls = sample_min(c, words, verts, &cp);
    } else {
        *cls = sample_one(c, method, words, verts);
    }
    return 0;
}

/* words of sample s under a generator: SplitMix64 (rng 0), x[i] = output
 * (4 s + tag) 16 + i + 1 of SplitMix64(seed); Philox4x32-10 (rng 1), x[2b],
 * x[2b+1] from block (s lo, s hi, tag, b) under the key (seed lo, seed hi) */
static void sample_words(int rng, int method, uint64_t seed, uint64_t s, uint64_t *x) {
    if (rng == 1) {
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (uint32_t b = 0; b < 8; b++) {
            const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)method, b};
            uint32_t o[4];
            oracle_philox4x32(ctr, key, o);
            x[2 * b] = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            x[2 * b + 1] = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
        }
        return;
    }
    for (uint64_t i = 0; i < 16; i++) x[i] = oracle_splitmix(seed, (4 * s + (uint64_t)method) * 16 + i + 1);
}

/* the words x[0..15] of sample s of a method under a generator (for tests) */
void oracle_words(int rng, int method, uint64_t seed, uint64_t s, uint64_t *x) { sample_words(rng, method, seed, s, x); }

/* Run samples s in [first, first+count) of one method, words from generator
 * rng (0 SplitMix64, 1 Philox4x32-10): counts[0] collisions,
 * counts[i] class i; for MOSS-4Min (method 3) counts[min_slot(class, c)]
 * instead.  classes/verts (nullable) receive per-sample records. */
int oracle_run_rng(const ctx *c, int method, int rng, uint64_t seed, uint64_t first, uint64_t count,
                   uint64_t *counts, uint8_t *classes, uint32_t *verts) {
    for (int i = 0; i < 22; i++) counts[i] = 0;
    if (!method_ok(c, method)) return -1;
    uint64_t x[16];
    uint32_t vv[5];
    for (uint64_t k = 0; k < count; k++) {
        sample_words(rng, method, seed, first + k, x);
        int cls;
        if (method == 3) {
            /* Algorithm 2: counts by (class, c(s)) slot */
            int cp;
            cls = sample_min(c, x, vv, &cp);
            int sl = min_slot(cls, cp);
            if (sl >= 0) counts[sl]++;
        } else {
            cls = sample_one(c, method, x, vv);
            if (cls < 0) return -2;
            counts[cls]++;
        }
        if (classes) classes[k] = (uint8_t)cls;
        if (verts) memcpy(verts + 5 * k, vv, sizeof(vv));
    }
    return 0;
}

/* oracle_run_rng with SplitMix64 words */
int oracle_run(const ctx *c, int method, uint64_t seed, uint64_t first, uint64_t count,
               uint64_t *counts, uint8_t *classes, uint32_t *verts) {
    return oracle_run_rng(c, method, 0, seed, first, count, counts, classes, verts);
}

/* --------------------------------------------------------- MOSS-4Min ---- */
/* The total order of Sec. 3.2: a > b iff d_a > d_b, or d_a = d_b and a > b. */
static int order_gt(const ctx *c, uint32_t a, uint32_t b) {
    return c->deg[a] > c->deg[b] || (c->deg[a] == c->deg[b] && a > b);
}

static uint64_t order_key(const ctx *c, uint32_t x) { return (c->deg[x] << 32) | x; }

static int cmp_desc_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x < y) - (x > y);
}

/* Tables of Sec. 4.2: the ordered lists, d_{v,u}, Gamma-check and the alias
 * tables of the vertex distribution pi-check and of sigma-check^(v) (eq. 3). */
int oracle_build_min(ctx *c) {
    if (c->has_min) return 0;
    uint64_t nnz1 = c->nnz ? c->nnz : 1, n1 = c->n ? c->n : 1;
    c->rlist = (uint32_t *)malloc(sizeof(uint32_t) * nnz1);
    c->rank = (uint64_t *)malloc(sizeof(uint64_t) * nnz1);
    c->gmin = (u128 *)calloc(n1, sizeof(u128));
    c->cthr = (uint64_t *)malloc(sizeof(uint64_t) * nnz1);
    c->calias = (uint32_t *)malloc(sizeof(uint32_t) * nnz1);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * nnz1);
    if (!c->rlist || !c->rank || !c->gmin || !c->cthr || !c->calias || !keys) {
        free(keys);
        return -1;
    }
    /* ordered lists; d_{v,u} is u's position in the ordered N_v */
    for (uint32_t v = 0; v < c->n; v++) {
        uint64_t o = c->off[v], d = c->deg[v];
        for (uint64_t i = 0; i < d; i++) keys[o + i] = order_key(c, c->col[o + i]);
        qsort(keys + o, d, sizeof(uint64_t), cmp_desc_u64);
        for (uint64_t i = 0; i < d; i++) c->rlist[o + i] = (uint32_t)keys[o + i];
        for (uint64_t i = 0; i < d; i++) {
            uint64_t k = order_key(c, c->col[o + i]);
            uint64_t lo = 0, hi = d;          /* position of k in the descending keys */
            while (lo < hi) {
                uint64_t mid = (lo + hi) / 2;
                if (keys[o + mid] > k) lo = mid + 1; else hi = mid;
            }
            c->rank[o + i] = lo;
        }
    }
    /* Gamma-check_v and the sigma-check weights d_{v,u} d_{u,v} */
    u128 *w = (u128 *)malloc(sizeof(u128) * nnz1), *t = (u128 *)malloc(sizeof(u128) * nnz1);
    if (!w || !t) { free(keys); free(w); free(t); return -1; }
    c->tmin = 0;
    for (uint32_t v = 0; v < c->n; v++) {
        uint64_t o = c->off[v], d = c->deg[v];
        for (uint64_t i = 0; i < d; i++) {
            uint32_t u = c->col[o + i];
            uint64_t dvu = c->rank[o + i];
            uint64_t duv = c->rank[c->off[u] + pos_of(c, u, v)];
            w[i] = (u128)dvu * duv;
            c->gmin[v] += w[i];
        }
        c->tmin += c->gmin[v];
        if (alias_sweep(d, w, t, c->calias + o)) { free(keys); free(w); free(t); return -1; }
        for (uint64_t i = 0; i < d; i++) c->cthr[o + i] = (uint64_t)t[i];
    }
    if (vtab_build(&c->mvt, c->n, c->gmin, c->tmin, c->vsplit_min)) { free(keys); free(w); free(t); return -1; }
    free(keys);
    free(w);
    free(t);
    c->has_min = 1;
    return 0;
}

/* c(s): the 3-paths p0-p1-p2-p3 of the CIS whose ends satisfy p0 > p2 and
 * p3 > p1 -- the paths MOSS-4Min can draw, each from both of its orientations,
 * so the CIS is drawn with probability 2 c(s) / Gamma-check.  Vertices in role
 * order, mask over the pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3). */
static int centered_paths(const ctx *c, const uint32_t *x, uint32_t mask) {
    int pair[4][4];
    int b = 0;
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++, b++) pair[i][j] = pair[j][i] = (mask >> b) & 1;
    int count = 0;
    int p[4];
    for (p[0] = 0; p[0] < 4; p[0]++)
        for (p[1] = 0; p[1] < 4; p[1]++)
            for (p[2] = 0; p[2] < 4; p[2]++)
                for (p[3] = 0; p[3] < 4; p[3]++) {
                    if (p[0] == p[1] || p[0] == p[2] || p[0] == p[3] || p[1] == p[2] || p[1] == p[3] ||
                        p[2] == p[3])
                        continue;
                    if (!pair[p[0]][p[1]] || !pair[p[1]][p[2]] || !pair[p[2]][p[3]]) continue;
                    if (order_gt(c, x[p[0]], x[p[2]]) && order_gt(c, x[p[3]], x[p[1]])) count++;
                }
    return count / 2;
}

/* count slot of (class, c): C4 c=1..4 -> 0..3, diamond c=1..6 -> 4..9,
 * K4 c=1..12 -> 10..21; other outcomes are not counted (-1) */
static int min_slot(int cls, int cp) {
    if (cls == 3 && cp >= 1 && cp <= 4) return cp - 1;
    if (cls == 5 && cp >= 1 && cp <= 6) return 4 + cp - 1;
    if (cls == 6 && cp >= 1 && cp <= 12) return 10 + cp - 1;
    return -1;
}

/* Algorithm 2 from explicit words: x0,x1 vertex draw (x6 its level), x2,x3
 * sigma-check draw of u, x4 w (uniform in N_{v,u}), x5 r (uniform in
 * N_{u,v}).  Returns the class (0 = collision) and *cp = c(s) for classes 3,
 * 5, 6 (else 0). */
static int sample_min(const ctx *c, const uint64_t *x, uint32_t *out, int *cp) {
    uint32_t v = vtab_draw(&c->mvt, c->n, x[6], x[0], x[1]);
    uint64_t ov = c->off[v];
    uint64_t j = index_of(x[2], c->deg[v]);
    uint64_t y = index_of(x[3], (uint64_t)c->gmin[v]);
    uint64_t iu = y < c->cthr[ov + j] ? j : c->calias[ov + j];
    uint32_t u = c->col[ov + iu];
    uint64_t dvu = c->rank[ov + iu];                       /* |N_{v,u}| */
    uint64_t duv = c->rank[c->off[u] + pos_of(c, u, v)];    /* |N_{u,v}| */
    uint32_t w = c->rlist[ov + index_of(x[4], dvu)];
    uint32_t r = c->rlist[c->off[u] + index_of(x[5], duv)];
    out[0] = v; out[1] = u; out[2] = w; out[3] = r; out[4] = 0;
    *cp = 0;
    if (r == u || r == w) return 0;
    uint32_t mask = 0;
    int bit = 0;
    for (int i = 0; i < 4; i++)
        for (int k = i + 1; k < 4; k++, bit++)
            if (is_edge(c, out[i], out[k])) mask |= 1u << bit;
    int cls = oracle_classify(4, mask);
    if (cls == 3 || cls == 5 || cls == 6) *cp = centered_paths(c, out, mask);
    out[4] = (uint32_t)*cp;
    return cls;
}

int oracle_min_words(const ctx *c, const uint64_t *words, uint32_t *verts, int *cls, int *cp) {
    if (!c->has_min || c->tmin == 0) return -1;
    *cls = sample_min(c, words, verts, cp);
    return 0;
}

/* out[2] = Gamma-check lo/hi */
void oracle_min_total(const ctx *c, uint64_t *out) { put128(out, c->tmin); }

void oracle_min_tables(const ctx *c, uint32_t *rlist, uint64_t *rank, uint64_t *cthr, uint32_t *calias,
                       uint64_t *gmin_lohi) {
    for (uint64_t p = 0; p < c->nnz; p++) {
        rlist[p] = c->rlist[p];
        rank[p] = c->rank[p];
        cthr[p] = c->cthr[p];
        calias[p] = c->calias[p];
    }
    for (uint32_t v = 0; v < c->n; v++) {
        put128(gmin_lohi + 2 * (uint64_t)v, c->gmin[v]);
    }
}

/* --------------------------------------------------------------- ESU ---- */
/* Wernicke's ESU: every connected induced k-subgraph is produced once, grown
 * from its smallest vertex through exclusive neighbourhoods. */
typedef struct { const ctx *c; int k; uint64_t *counts; } esu_state;

static int in_set(const uint32_t *s, int m, uint32_t x) {
    for (int i = 0; i < m; i++) if (s[i] == x) return 1;
    return 0;
}

static void esu_extend(esu_state *st, uint32_t *sub, int ns, uint32_t *ext, uint64_t next, uint32_t root) {
    if (ns == st->k) {
        st->counts[classify_vertices(st->c, st->k, sub)]++;
        return;
    }
    const ctx *c = st->c;
    uint64_t ne = next;
    while (ne > 0) {
        uint32_t w = ext[--ne];
        /* new extension = rest of ext + exclusive neighbours of w that exceed root */
        uint64_t cap = ne + c->deg[w];
        uint32_t *ext2 = (uint32_t *)malloc(sizeof(uint32_t) * (cap ? cap : 1));
        uint64_t n2 = ne;
        memcpy(ext2, ext, sizeof(uint32_t) * ne);
        for (uint64_t p = c->off[w]; p < c->off[w + 1]; p++) {
            uint32_t u = c->col[p];
            if (u <= root || in_set(sub, ns, u) || in_set(ext, ne, u) || u == w) continue;
            int adj = 0;
            for (int i = 0; i < ns && !adj; i++) adj = is_edge(c, sub[i], u);
            if (!adj && !in_set(ext2, n2, u)) ext2[n2++] = u;
        }
        sub[ns] = w;
        esu_extend(st, sub, ns + 1, ext2, n2, root);
        free(ext2);
    }
}

/* exact counts of connected induced k-subgraphs by class (counts[1..]) */
int oracle_esu(const ctx *c, int k, uint64_t *counts) {
    for (int i = 0; i < 22; i++) counts[i] = 0;
    if (k != 4 && k != 5) return -1;
    esu_state st = {c, k, counts};
    uint32_t sub[5];
    for (uint32_t v = 0; v < c->n; v++) {
        uint64_t d = c->deg[v];
        uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (d ? d : 1));
        uint64_t ne = 0;
        for (uint64_t p = c->off[v]; p < c->off[v + 1]; p++) if (c->col[p] > v) ext[ne++] = c->col[p];
        sub[0] = v;
        esu_extend(&st, sub, 1, ext, ne, v);
        free(ext);
    }
    return 0;
}
