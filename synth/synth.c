/*
 * synth.c -- seeded synthetic graph generators shared by the oracle, the
 * tests and the benchmark.  This file holds no part of the sampling method:
 * it only produces simple undirected graphs as sorted CSR arrays.
 *
 * Generators
 *   Chung-Lu   expected-degree random graph, p_ij = min(1, w_i w_j / sum(w)),
 *              drawn with the O(n + m) skipping method of Miller and Hagberg
 *              ("Efficient generation of networks with given expected degrees",
 *              WAW 2011).  Weights follow a truncated power law
 *              w_i = c (i + i0)^(-1/(gamma-1)), i = 0..n-1, with c fixed by the
 *              maximum weight (w_0 = d_max) and i0 solved for the mean degree.
 *   RGG        2-D random geometric graph on the unit torus, radius
 *              r = sqrt(dbar / (pi n)).
 * Both relabel vertices with a seeded random permutation (Fisher-Yates) so
 * that hubs are not clustered at small ids, then emit a sorted, symmetric CSR
 * with no self-loops and no duplicate edges.
 *
 * Portability: the x86 container and the Arm GPU host must produce the same
 * graph for the same seed.  All randomness is integer (splitmix64) and the few
 * transcendental functions are evaluated by the series below using only
 * IEEE +, -, *, / (build with -ffp-contract=off so no FMA is formed).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG ---- */
typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *g) {
    /* splitmix64 (Steele, Lea, Flood 2014 / Vigna) */
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in the open interval (0, 1) */
static double sm64_open01(sm64 *g) {
    return ((double)(sm64_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, m) by rejection (exact) */
static uint64_t sm64_below(sm64 *g, uint64_t m) {
    uint64_t lim = (UINT64_MAX / m) * m;
    uint64_t x;
    do { x = sm64_next(g); } while (x >= lim);
    return x % m;
}

/* ------------------------------------------------- portable log / exp ---- */
static const double LN2 = 0.69314718055994530942;

/* split x > 0 into m in [sqrt(1/2), sqrt(2)) and integer e with x = m 2^e */
static double split_pow2(double x, int *e) {
    int k = 0;
    while (x >= 2.0) { x *= 0.5; k++; }
    while (x < 1.0) { x *= 2.0; k--; }
    if (x > 1.4142135623730951) { x *= 0.5; k++; }
    *e = k;
    return x;
}

/* natural log: log(m) = 2 atanh((m-1)/(m+1)), odd power series */
static double p_log(double x) {
    int e;
    double m = split_pow2(x, &e);
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s, term = s, sum = 0.0;
    for (int k = 0; k < 14; k++) {
        sum = sum + term / (double)(2 * k + 1);
        term = term * s2;
    }
    return 2.0 * sum + (double)e * LN2;
}

/* exp by range reduction x = k ln2 + r, |r| <= ln2/2, Taylor series for e^r */
static double p_exp(double x) {
    double kf = x / LN2;
    long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
    double r = x - (double)k * LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 24; i++) {
        term = term * r / (double)i;
        sum = sum + term;
    }
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}

static double p_pow(double a, double b) { return p_exp(b * p_log(a)); }

/* --------------------------------------------------------- edge list ---- */
typedef struct { uint32_t *a, *b; uint64_t m, cap; } edges;

static int edges_push(edges *E, uint32_t a, uint32_t b) {
    if (E->m == E->cap) {
        uint64_t nc = E->cap ? E->cap * 2 : 1024;
        uint32_t *na = (uint32_t *)realloc(E->a, nc * sizeof(uint32_t));
        if (!na) return -1;
        E->a = na;
        uint32_t *nb = (uint32_t *)realloc(E->b, nc * sizeof(uint32_t));
        if (!nb) return -1;
        E->b = nb;
        E->cap = nc;
    }
    E->a[E->m] = a;
    E->b[E->m] = b;
    E->m++;
    return 0;
}

static void edges_free(edges *E) { free(E->a); free(E->b); memset(E, 0, sizeof(*E)); }

/* ------------------------------------------------------ Chung-Lu ---- */
/* mean of w_i = dmax (i0 / (i + i0))^alpha over i = 0..n-1.  The first terms
 * are summed exactly and the tail by the Euler-Maclaurin integral with its
 * first two corrections; the result only fixes the generator's parameter. */
static double cl_mean(uint32_t n, double alpha, double dmax, double i0) {
    const uint32_t head = n < 20000 ? n : 20000;
    double sum = 0.0;
    for (uint32_t i = 0; i < head; i++) sum += p_pow((double)i + i0, -alpha);
    if (head < n) {
        double a = (double)head + i0, b = (double)(n - 1) + i0;
        double integral;
        if (alpha == 1.0) integral = p_log(b) - p_log(a);
        else integral = (p_pow(b, 1.0 - alpha) - p_pow(a, 1.0 - alpha)) / (1.0 - alpha);
        double fa = p_pow(a, -alpha), fb = p_pow(b, -alpha);
        double dfa = -alpha * p_pow(a, -alpha - 1.0), dfb = -alpha * p_pow(b, -alpha - 1.0);
        sum += integral + 0.5 * (fa + fb) + (dfb - dfa) / 12.0;
    }
    return dmax * p_pow(i0, alpha) * sum / (double)n;
}

/* Solve i0 for the requested mean degree; fill w[] (descending). */
static int cl_weights(uint32_t n, double gamma, double dbar, double dmax, double *w) {
    double alpha = 1.0 / (gamma - 1.0);
    if (!(gamma > 1.0) || !(dbar > 0.0) || !(dmax >= dbar)) return -1;
    double lo = -30.0, hi = 40.0; /* bisection on log(i0) */
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (cl_mean(n, alpha, dmax, p_exp(mid)) < dbar) lo = mid; else hi = mid;
    }
    double i0 = p_exp(0.5 * (lo + hi));
    for (uint32_t i = 0; i < n; i++) w[i] = dmax * p_pow(i0 / ((double)i + i0), alpha);
    return 0;
}

/* Miller-Hagberg: for each u, jump over runs of non-edges with geometric
 * skips drawn against the current upper bound p, then thin by q/p. */
static int cl_edges(uint32_t n, const double *w, sm64 *g, edges *E) {
    double S = 0.0;
    for (uint32_t i = 0; i < n; i++) S += w[i];
    for (uint32_t u = 0; u + 1 < n; u++) {
        uint64_t v = (uint64_t)u + 1;
        double p = w[u] * w[v] / S;
        if (p > 1.0) p = 1.0;
        while (v < n && p > 0.0) {
            if (p != 1.0) {
                double r = sm64_open01(g);
                double skip = p_log(r) / p_log(1.0 - p);
                if (skip >= (double)n) break;
                v += (uint64_t)skip;
            }
            if (v < n) {
                double q = w[u] * w[v] / S;
                if (q > 1.0) q = 1.0;
                double r = sm64_open01(g);
                if (r < q / p && edges_push(E, u, (uint32_t)v)) return -1;
                p = q;
                v++;
            }
        }
    }
    return 0;
}

/* --------------------------------------------------------- RGG ---- */
static int rgg_edges(uint32_t n, double dbar, sm64 *g, edges *E) {
    const double PI = 3.14159265358979323846;
    double r = p_exp(0.5 * p_log(dbar / (PI * (double)n)));
    if (r >= 0.5) r = 0.5;
    uint32_t cells = (uint32_t)(1.0 / r);
    /* a 3x3 stencil needs at least 3 cells per side; below that one cell
     * holding every point is scanned (small graphs only) */
    if (cells < 3) cells = 1;
    if (cells > 4096) cells = 4096;
    double *x = (double *)malloc(sizeof(double) * n), *y = (double *)malloc(sizeof(double) * n);
    uint32_t *cell_of = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint64_t nc = (uint64_t)cells * cells;
    uint32_t *start = (uint32_t *)calloc(nc + 1, sizeof(uint32_t));
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n);
    int rc = 0;
    if (!x || !y || !cell_of || !start || !order) { rc = -1; goto out; }
    for (uint32_t i = 0; i < n; i++) {
        x[i] = sm64_open01(g);
        y[i] = sm64_open01(g);
        uint32_t cx = (uint32_t)(x[i] * cells), cy = (uint32_t)(y[i] * cells);
        if (cx >= cells) cx = cells - 1;
        if (cy >= cells) cy = cells - 1;
        cell_of[i] = cy * cells + cx;
        start[cell_of[i] + 1]++;
    }
    for (uint64_t c = 0; c < nc; c++) start[c + 1] += start[c];
    {
        uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * nc);
        if (!fill) { rc = -1; goto out; }
        memcpy(fill, start, sizeof(uint32_t) * nc);
        for (uint32_t i = 0; i < n; i++) order[fill[cell_of[i]]++] = i;
        free(fill);
    }
    double r2 = r * r;
    for (uint32_t i = 0; i < n; i++) {
        int32_t cx = (int32_t)(cell_of[i] % cells), cy = (int32_t)(cell_of[i] / cells);
        for (int dy = -1; dy <= 1; dy++) {
            for (int dx = -1; dx <= 1; dx++) {
                if (cells == 1 && (dx != 0 || dy != 0)) continue;
                int32_t tx = ((cx + dx) % (int32_t)cells + (int32_t)cells) % (int32_t)cells;
                int32_t ty = ((cy + dy) % (int32_t)cells + (int32_t)cells) % (int32_t)cells;
                uint32_t c = (uint32_t)ty * cells + (uint32_t)tx;
                for (uint32_t k = start[c]; k < start[c + 1]; k++) {
                    uint32_t j = order[k];
                    if (j <= i) continue;
                    double ddx = x[i] - x[j], ddy = y[i] - y[j];
                    if (ddx > 0.5) ddx -= 1.0;
                    if (ddx < -0.5) ddx += 1.0;
                    if (ddy > 0.5) ddy -= 1.0;
                    if (ddy < -0.5) ddy += 1.0;
                    if (ddx * ddx + ddy * ddy <= r2 && edges_push(E, i, j)) { rc = -1; goto out; }
                }
            }
        }
    }
out:
    free(x); free(y); free(cell_of); free(start); free(order);
    return rc;
}

/* ------------------------------------------------------ CSR output ---- */
static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* relabel with a seeded permutation and build sorted symmetric CSR */
static int to_csr(uint32_t n, edges *E, sm64 *g, int relabel, uint64_t **row_ptr, uint32_t **col) {
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint64_t *rp = (uint64_t *)calloc((uint64_t)n + 1, sizeof(uint64_t));
    uint32_t *cl = (uint32_t *)malloc(sizeof(uint32_t) * (E->m ? 2 * E->m : 1));
    if (!perm || !rp || !cl) { free(perm); free(rp); free(cl); return -1; }
    for (uint32_t i = 0; i < n; i++) perm[i] = i;
    if (relabel)
        for (uint32_t i = n; i > 1; i--) {
            uint32_t j = (uint32_t)sm64_below(g, i);
            uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
        }
    for (uint64_t e = 0; e < E->m; e++) {
        rp[perm[E->a[e]] + 1]++;
        rp[perm[E->b[e]] + 1]++;
    }
    for (uint32_t i = 0; i < n; i++) rp[i + 1] += rp[i];
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!fill) { free(perm); free(rp); free(cl); return -1; }
    memcpy(fill, rp, sizeof(uint64_t) * n);
    for (uint64_t e = 0; e < E->m; e++) {
        uint32_t a = perm[E->a[e]], b = perm[E->b[e]];
        cl[fill[a]++] = b;
        cl[fill[b]++] = a;
    }
    for (uint32_t i = 0; i < n; i++)
        qsort(cl + rp[i], (size_t)(rp[i + 1] - rp[i]), sizeof(uint32_t), cmp_u32);
    free(fill);
    free(perm);
    *row_ptr = rp;
    *col = cl;
    return 0;
}

/* --------------------------------------------------------- exported ---- */
/* kind 0: Chung-Lu(gamma, dbar, dmax); kind 1: RGG(dbar).
 * On success *row_ptr has n+1 entries, *col has row_ptr[n] entries; release
 * both with synth_free. */
int synth_generate(int kind, uint32_t n, double gamma, double dbar, double dmax,
                   uint64_t seed, int relabel, uint64_t **row_ptr, uint32_t **col) {
    sm64 g = {seed * 0x2545F4914F6CDD1DULL + 0x1234567ULL};
    edges E = {0};
    int rc = 0;
    *row_ptr = NULL;
    *col = NULL;
    if (n == 0) return -1;
    if (kind == 0) {
        double *w = (double *)malloc(sizeof(double) * n);
        if (!w) return -1;
        rc = cl_weights(n, gamma, dbar, dmax, w);
        if (!rc) rc = cl_edges(n, w, &g, &E);
        free(w);
    } else if (kind == 1) {
        rc = rgg_edges(n, dbar, &g, &E);
    } else {
        rc = -1;
    }
    if (!rc) rc = to_csr(n, &E, &g, relabel, row_ptr, col);
    edges_free(&E);
    return rc;
}

void synth_free(void *p) { free(p); }

/* exported for the portability tests of the series above */
double synth_log(double x) { return p_log(x); }
double synth_exp(double x) { return p_exp(x); }
