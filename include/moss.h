/*
 * moss.h -- C ABI of the GB300 Moss motif sampler (libmoss.so).
 *
 * Estimates the frequencies of the 6 connected induced 4-node subgraph
 * classes (M_1^(4)..M_6^(4)) and the 21 5-node classes (M_1^(5)..M_21^(5))
 * of an undirected simple graph, with the unbiased sampling estimators and
 * closed-form variances of
 *   P. Wang, J. Tao, J. Zhao, X. Guan, "Moss: A Scalable Tool for Efficiently
 *   Sampling and Counting 4- and 5-Node Graphlets", arXiv 1509.08089:
 *     MOSS-4  (Sec. 4.1, Algorithm 1, Theorems 2-3),
 *     MOSS-5  = T-5 (Algorithm 3, Theorems 6-7) + Path-5 (Algorithm 4,
 *               Theorems 8-9) + the mix estimator (Sec. 5.1.3, Theorem 10),
 *     MOSS-4Min (Sec. 4.2, Algorithm 2, Theorem 5) and its mix with MOSS-4
 *               (Theorem 1), with the per-CIS sampling probability
 *               2 c(s) / Gamma-check described at MOSS_METHOD_MOSS4MIN.
 * Every step runs as CUDA kernels on one GPU (sm_103a).  The only data that
 * crosses to the host during sampling is the final result.
 *
 * Conventions
 *   - Every function returns an int status: MOSS_OK (0) or a negative
 *     MOSS_E* code.  No exception crosses the ABI.  moss_last_error_detail()
 *     returns a thread-local description of the last failure on the calling
 *     thread.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.  All work of a call is enqueued on that
 *     stream.  Calls documented as synchronous return after the stream has
 *     drained the work of the call.
 *   - The library never frees or retains caller memory.  Graph objects own
 *     their device memory and release it in moss_graph_free.
 *   - A moss_graph may be used by one host thread at a time.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) in counter
 * form.  Word i (0 <= i < 16) of sample s of method t under seed k is output
 * number (4 s + t) 16 + i + 1 of SplitMix64 seeded with k; t = 0 (MOSS-4),
 * 1 (T-5), 2 (Path-5), 3 (MOSS-4Min).  The
 * counts of a sample range are therefore independent of launch shape, stream
 * and device count, and shards [a,b) + [b,c) add up to [a,c) exactly.
 */
#ifndef MOSS_H
#define MOSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define MOSS_OK          0
#define MOSS_EINVAL     -1  /* bad argument (null pointer, k not 4/5, ...)   */
#define MOSS_ENOMEM     -2  /* device or host allocation failed             */
#define MOSS_ECUDA      -3  /* a CUDA runtime call failed                   */
#define MOSS_EGRAPH     -4  /* CSR is not a sorted symmetric simple graph   */
#define MOSS_EOVERFLOW  -5  /* a size or an exact total exceeds its range   */
#define MOSS_ESTATE     -6  /* tables for the requested k were not built    */
#define MOSS_EBUSY      -7  /* a request did not finish before a timeout     */

#define MOSS_METHOD_MOSS4  0   /* Algorithm 1 */
#define MOSS_METHOD_T5     1   /* Algorithm 3 */
#define MOSS_METHOD_PATH5  2   /* Algorithm 4 */
/* Algorithm 2 (Sec. 4.2).  v from pi-check (weight Gamma-check_v =
 * sum_{x in N_v} d_{v,x} d_{x,v}), u from sigma-check^(v) (eq. 3), w uniform
 * in N_{v,u}, r uniform in N_{u,v}, where N_{u,v} holds the neighbours of u
 * above v in the total order of Sec. 3.2 (higher degree, ties by the larger
 * id) and d_{u,v} = |N_{u,v}|.  Every admissible (v, u, w, r) has probability
 * 1 / Gamma-check, so a CIS s is drawn with probability 2 c(s) / Gamma-check,
 * c(s) being the number of 3-paths p0-p1-p2-p3 of s with p0 above p2 and p3
 * above p1.  c(s) is 1 for a 4-cycle and 3 for a 4-clique (Theorem 4), but
 * 1, 2 or 3 for a diamond (Theorem 4 states 1), so the counts of this method
 * are kept per (class, c) slot: 4-cycles with c = 1..4 in slots 0..3,
 * diamonds with c = 1..6 in slots 4..9, 4-cliques with c = 1..12 in slots
 * 10..21; collisions (r = w) and the other classes are not counted.  Word
 * schedule: x0,x1 vertex draw, x2,x3 sigma-check draw, x4 w, x5 r. */
#define MOSS_METHOD_MOSS4MIN 3

#define MOSS_NCLASS_SLOTS 22   /* [0] = collisions, [1..21] = classes */

/* How the induced-edge tests of CIS() (Algorithms 1, 3, 4) are answered:
 * SEARCH: binary search in the shorter sorted neighbour list (O(log d) loads);
 * HASH: one lookup in a hashed set of all edges (one 16-byte bucket load in
 * the common case);
 * FILTER: the hashed set behind a blocked Bloom filter of about 8 bits per
 * edge (3 bits of one 32-bit word per edge, no false negatives): a pair the
 * filter rejects is a non-edge without touching the set, so on a graph whose
 * set does not fit the L2 cache most probes stay in L2;
 * AUTO (default): FILTER when the set exceeds 64 MiB, else HASH, decided by
 * moss_build_tables.  All give identical results. */
#define MOSS_PROBE_SEARCH  0
#define MOSS_PROBE_HASH    1
#define MOSS_PROBE_FILTER  2
#define MOSS_PROBE_AUTO    3

typedef struct moss_graph moss_graph;

/* Exact totals of Table 1 (as 128-bit lo/hi pairs and as doubles). */
typedef struct {
    uint32_t n;                 /* vertices                                 */
    uint64_t nnz;               /* directed CSR slots = 2 |E|               */
    uint32_t d_max;             /* maximum degree                           */
    uint64_t gamma[4][2];       /* Gamma, Gamma^(1), Gamma^(2), Gamma-check  */
                                /* (0 until the MOSS-4Min tables are built): {lo, hi} */
    uint64_t lambda3[2];        /* Lambda_3 = sum C(d_v,3): {lo, hi}         */
    uint64_t lambda4[2];        /* Lambda_4 = sum C(d_v,4): {lo, hi}         */
    double gamma_d[4], lambda3_d, lambda4_d;
} moss_stats;

/* Result of one estimate.  Index i of est/var is class M_i (1-based); index
 * 0 is unused.  For k = 4 only indices 1..6 are meaningful. */
typedef struct {
    int k;                      /* 4 or 5                                   */
    int n_classes;              /* 6 or 21                                  */
    uint64_t K[2];              /* samples drawn: k=4 {K, 0} (with MOSS-4Min  */
                                /* {K, K-check}); k=5 {K1, K2}                */
    uint64_t hits[2][MOSS_NCLASS_SLOTS]; /* [sub-method][0 = collisions, i];  */
                                /* MOSS-4Min: its (class, c) slots           */
    double est[MOSS_NCLASS_SLOTS];       /* estimate of n_i / eta_i          */
    double var[MOSS_NCLASS_SLOTS];       /* plug-in variance of est[i]       */
    double lambda[2][MOSS_NCLASS_SLOTS]; /* weight of each sub-method in est */
                                /* (k=5: T-5 / Path-5; mix: MOSS-4 / 4Min)   */
    double triangles;           /* k=4: triangle count implied by the r = w collisions */
    double triangles_var;
    double conc[MOSS_NCLASS_SLOTS];      /* concentration est[i] / sum_j est[j] (Sec. 6.3) */
} moss_result;

/* Load an undirected graph given as CSR and run the initialization pass
 * (Sec. 4.1.3): exact per-vertex weights Gamma_v, Gamma^(1)_v, Gamma^(2)_v
 * (Sec. 4.1.1, 5.1.1, 5.1.2), the totals of Table 1 and the ACC prefix arrays.
 *   row_ptr : n+1 offsets, uint64 when row_ptr_is_64 != 0 else uint32;
 *             row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col     : nnz vertex ids; each list N_v (Table 1) strictly increasing, no
 *             self loop, every (v,u) matched by (u,v).
 *   Both arrays may be host or device memory (detected); they are copied and
 *   may be released after the call.  device: CUDA ordinal the graph lives on.
 *   Limits: n < 2^32 - 1, nnz < 2^32.
 * Validates the graph on the device and returns MOSS_EGRAPH (with detail) if
 * any rule is broken.  Synchronous on stream.  *out receives a new graph that
 * the caller releases with moss_graph_free. */
int moss_graph_load_csr(const void *row_ptr, int row_ptr_is_64, const uint32_t *col,
                        uint32_t n, uint64_t nnz, int device, void *stream, moss_graph **out);

/* moss_graph_load_csr with a choice of internal vertex order.
 *   MOSS_ORDER_INPUT  : the input ids (moss_graph_load_csr).
 *   MOSS_ORDER_DEGREE : the vertices renumbered on the device before the
 *     initialization pass, by key(d_v) descending, then input id ascending;
 *     key(d) = d for d < 16, else 16 + 4 (L - 5) + ((d >> (L - 3)) & 3), L
 *     the bit length of d (quarter-octave classes).  Each list stays sorted
 *     in the new ids.  The samplers read records in proportion to degree
 *     (Sec. 4.1.3, 5.1.4), so grouping the heavy vertices puts the hot
 *     records of a heavy-tailed graph in fewer cache lines.
 * Estimates, counts and variances are those of the renumbered graph, which
 * is isomorphic to the input; every quantity of Sec. 2 and Table 1 is
 * invariant under relabelling, but the draws of a seed differ from those of
 * the input order.  moss_sample_records reports input ids; the tables of
 * moss_table_export hold internal ids, and MOSS_TABLE_ORDER gives the input
 * id of each internal vertex.  Input rules and errors as
 * moss_graph_load_csr; the renumbering needs about 9.2 n bytes of scratch
 * during the call (plus 4 nnz when col is not device memory of `device`) and
 * keeps 4 n bytes for the id map.
 * MOSS_EINVAL for another order. */
#define MOSS_ORDER_INPUT  0
#define MOSS_ORDER_DEGREE 1
int moss_graph_load_csr_order(const void *row_ptr, int row_ptr_is_64, const uint32_t *col,
                              uint32_t n, uint64_t nnz, int order, int device, void *stream,
                              moss_graph **out);

/* Sampling tables (Sec. 4.1.3 WeightRandomVertex, Sec. 5.1.4): the per-list
 * alias tables of sigma^(v) (eq. 1), the vertex alias tables of pi (k_mask
 * bit 4) and rho^(1), rho^(2) (k_mask bit 5) from the exact weights computed
 * at load, and the hashed edge set and its filter as the probe strategy
 * needs them.  k_mask: any
 * non-empty combination of (1<<4), (1<<5) and MOSS_TABLES_4MIN, which adds
 * the MOSS-4Min tables (Sec. 4.2): every N_v ordered by the total order,
 * d_{v,u} per slot, Gamma-check_v, the alias tables of sigma-check^(v)
 * (eq. 3) and of pi-check, and the exact total Gamma-check -- about
 * 40 bytes per CSR slot plus 48 per vertex, held until moss_graph_free.
 * MOSS_EOVERFLOW if a scaled total leaves 128 bits.  Synchronous on stream;
 * the tables of k_mask are rebuilt and only those stay usable. */
#define MOSS_TABLES_4MIN (1u << 6)
int moss_build_tables(moss_graph *g, unsigned k_mask, void *stream);

/* Select the probe strategy (MOSS_PROBE_*) for later samples.  Switching to
 * a strategy whose structures were not built (the hashed set, the filter)
 * requires moss_build_tables afterwards (MOSS_ESTATE until then). */
int moss_set_probe(moss_graph *g, int strategy);

/* Word generator of the graph's samples (every sampling call, batch and
 * server request on it); the paper draws uniformly without naming one.
 *   MOSS_RNG_SPLITMIX64 (default): word i (0 <= i < 16) of sample s of
 *     method t under seed k is output (4 s + t) 16 + i + 1 of SplitMix64
 *     (Steele, Lea, Flood, OOPSLA 2014) seeded with k.
 *   MOSS_RNG_PHILOX4X32: words 2b, 2b+1 are the outputs of Philox4x32-10
 *     (Salmon et al., SC 2011) for the counter (s mod 2^32, s div 2^32, t, b)
 *     under the key (k mod 2^32, k div 2^32), low output first.
 * Either is counter-based: a sample's draws depend on (seed, method, id)
 * alone, so counts do not depend on launch shape, stream or device count.
 * Changing it needs no table rebuild.  MOSS_EINVAL for another value;
 * moss_get_rng returns the current one (MOSS_EINVAL for NULL). */
#define MOSS_RNG_SPLITMIX64 0
#define MOSS_RNG_PHILOX4X32 1
int moss_set_rng(moss_graph *g, int rng);
int moss_get_rng(const moss_graph *g);

/* WeightRandomVertex(V, .) (Sec. 4.1.3) draws from an alias table per
 * weight, which on graphs of 2^14 vertices or more has two levels: the heavy
 * vertices, w_v 2^split >= W (at most 2^split of them, in ascending id
 * order), and the light ones; a separate word picks the light table with
 * probability floor(W_light 2^64 / W) / 2^64 (exact up to 2^-64, as every
 * threshold).  On power-law graphs a few hundred to a few thousand vertices
 * carry most of the weight, so most draws read a table small enough to stay
 * cached (in L1 on graphs whose edge set is probed without the filter).  The
 * level word is x6 for MOSS-4 and MOSS-4Min, x7 for T-5 and x14 for Path-5;
 * with one level it is not read.  moss_set_vertex_split (0..63, or
 * MOSS_VERTEX_ONE_LEVEL, for every table; the default is
 * MOSS_VERTEX_SPLIT_DEFAULT from 2^20 vertices, MOSS_VERTEX_SPLIT_MID from
 * 2^14, else one level -- for the MOSS-4Min table (Gamma-check) one level
 * below 2^20 vertices, where a heavy level measured slower) takes effect at
 * the next moss_build_tables
 * (sampling returns MOSS_ESTATE until then); moss_vertex_levels reports, for
 * weight which (0 Gamma, 1 Gamma^(1), 2 Gamma^(2), 3 Gamma-check), the
 * heavy count (0 with one level) and the light level's bound. */
#define MOSS_VERTEX_SPLIT_DEFAULT 20
#define MOSS_VERTEX_SPLIT_MID 12
#define MOSS_VERTEX_ONE_LEVEL 64
int moss_set_vertex_split(moss_graph *g, int split);
int moss_vertex_levels(const moss_graph *g, int which, uint32_t *nheavy, uint64_t *tlight);

/* Sample-and-estimate.  k = 4: MOSS-4 with K = budget.  k = 5: T-5 with
 * K1 = floor(budget/2) and Path-5 with K2 = budget - K1 (K1 = K2, Sec. 5.1.5).
 * A sub-method whose total weight is 0 draws nothing (its classes cannot
 * occur and are estimated as exactly 0).  Sample ids are 0..K-1 per
 * sub-method.  out is caller-owned host memory.  Synchronous on stream. */
int moss_sample_estimate(moss_graph *g, int k, uint64_t budget, uint64_t seed, void *stream,
                         moss_result *out);

/* Counts of samples first..first+count-1 of one method: counts_dev (device,
 * 22 uint64) receives [0] = collisions (no CIS) and [i] = samples of class i
 * (MOSS_METHOD_MOSS4MIN: its (class, c) slots).  Asynchronous on stream.
 * Shards of a sample range sum exactly. */
int moss_sample_counts(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed,
                       void *stream, uint64_t *counts_dev);

/* moss_sample_counts without any device allocation.  The paper has no
 * counterpart: this serves callers that may not allocate device memory while
 * they run -- a service that reserves its whole memory budget at start-up, a
 * latency-bound loop that cannot take the device synchronisation an
 * allocation or free may cause, or an embedding whose allocator belongs to
 * another framework.  Same arguments and result as moss_sample_counts (the
 * graph and counts_dev are allocated by the caller beforehand); the per-block
 * partial counts live in one fixed device array of 360,448 bytes (2048 rows of
 * 22 uint64) that every GPU loading the library holds until exit.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress), so
 * make it before any stream capture; the address is kept for the life of the
 * process, so after a cudaDeviceReset of that device the entry point must not
 * be called again.  Calls share the array: calls whose work
 * overlaps on the GPU race and must be ordered by the caller.  MOSS_EOVERFLOW
 * if the device needs more than 2048 blocks.  Asynchronous on stream. */
int moss_sample_counts_noalloc(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed,
                               void *stream, uint64_t *counts_dev);

/* Per-sample records of samples first..first+count-1 (for verification):
 * classes_dev (device, count uint8: 0 = collision, else class) and, when not
 * NULL, verts_dev (device, 5*count uint32: v,u,w,r,t in draw order, as input
 * ids; t = 0 for MOSS-4; MOSS-4Min: v,u,w,r,c(s), c(s) = 0 outside classes
 * 3, 5, 6).
 * Asynchronous on stream. */
int moss_sample_records(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed,
                        void *stream, uint8_t *classes_dev, uint32_t *verts_dev);

/* Estimators and variances from counts gathered elsewhere (e.g. summed over
 * shards): K[2] and hits[2][22] as in moss_result.  The arithmetic runs on
 * the device in FP64.  Synchronous on stream. */
int moss_finalize(moss_graph *g, int k, const uint64_t *K, const uint64_t *hits, void *stream,
                  moss_result *out);

/* MOSS-4 with K = budget and MOSS-4Min with K-check = budget_min (sample ids
 * 0.. of each, same seed), mixed class by class (Theorem 1): requires the
 * tables of (1<<4) | MOSS_TABLES_4MIN.  Classes 3, 5, 6 have both estimates
 * n-hat_i (Theorem 2) and n-check_i = Gamma-check / (2 K-check) sum_c
 * m_{i,c} / c (each hit weighted by its inverse probability); Var(n-check_i)
 * is (S_i - n_i^2) / K-check with S_i = sum_s 1/P(s) = n_i Gamma-check h_i / 2,
 * h_i the mean of 1/c(s) over the class, estimated from the hits as
 * sum_c m_{i,c}/c^2 / sum_c m_{i,c}/c (1, 1, 1/3 for classes 3, 5, 6 when
 * there is none).  Both variances use the plug-in n_i = (K n-hat_i +
 * K-check n-check_i) / (K + K-check); the weights are lambda = V_other /
 * (V_1 + V_2) and the mixed variance V_1 V_2 / (V_1 + V_2).  Classes 1 and 4
 * come from MOSS-4 alone, n_2 from eq. (2).  Result: k = 4, K = {K, K-check},
 * hits[0] MOSS-4 counts, hits[1] MOSS-4Min slots, lambda[0] / lambda[1]
 * the weights.  Synchronous on stream. */
int moss_sample_estimate_min(moss_graph *g, uint64_t budget, uint64_t budget_min, uint64_t seed, void *stream,
                             moss_result *out);

/* The estimate above from counts gathered elsewhere: K[2] = {K, K-check},
 * hits[2][22] = {MOSS-4 counts, MOSS-4Min slots}.  cov_host (nullable, 22 x 22
 * doubles, host) receives the covariance matrix: -n_i n_j sum_l a_i a_j / K_l
 * between classes (a = the weights, a sample lands in one class), the
 * variances on the diagonal, the row of class 2 from eq. (2).  Synchronous on
 * stream. */
int moss_finalize_min(moss_graph *g, const uint64_t *K, const uint64_t *hits, void *stream, double *cov_host,
                      moss_result *out);

/* ----------------------------------------------------------------- batches
 * Many sample-and-estimate requests, on many loaded graphs, in one persistent
 * launch.  Each request (graph, k, budget, seed) is exactly one
 * moss_sample_estimate (MOSS-4, Sec. 4.1; MOSS-5 with K1 = floor(B/2),
 * K2 = B - K1, Sec. 5.1) and yields the same counts and estimates; the batch
 * only changes how the work is scheduled: every sub-method's sample ids are
 * cut into tiles that one kernel drains from a device counter, per-tile
 * counts are summed per request in tile order, and the finalize runs per
 * request on the device.  The launch sequence is captured into a CUDA graph
 * on the batch's own stream and replayed until the request list or the tile
 * size changes.  Graphs must stay alive, built and unchanged while they are
 * in a batch. */
typedef struct moss_batch moss_batch;
int moss_batch_create(int device, moss_batch **out);
/* Append a request; *index (nullable) receives its position in the results. */
int moss_batch_add(moss_batch *b, moss_graph *g, int k, uint64_t budget, uint64_t seed, int *index);
/* Append a MOSS-4 + MOSS-4Min request (the mix of Sec. 4.2, Theorem 1):
 * budget MOSS-4 samples and budget_min MOSS-4Min samples, finalized as
 * moss_sample_estimate_min is, whose result it equals.  The graph needs the
 * k = 4 tables and MOSS_TABLES_4MIN (MOSS_ESTATE otherwise). */
int moss_batch_add_min(moss_batch *b, moss_graph *g, uint64_t budget, uint64_t budget_min, uint64_t seed,
                       int *index);
int moss_batch_size(const moss_batch *b);
int moss_batch_clear(moss_batch *b);
/* Samples per tile (32 .. 2^30; default 8192). */
int moss_batch_set_tile(moss_batch *b, uint32_t tile_samples);
uint32_t moss_batch_tile(const moss_batch *b);
/* Run every request: results[i] (caller-owned host array of moss_batch_size
 * entries) receives request i.  Ordered after prior work on `stream`;
 * synchronous. */
int moss_batch_run(moss_batch *b, void *stream, moss_result *results);
/* Launch shape of the persistent sampler: threads per block (128, 256 or
 * 512; the resident threads per SM stay 1,024) and resident blocks per SM
 * (0: as many as fit, the default). */
int moss_batch_set_launch(moss_batch *b, int threads_per_block, int blocks_per_sm);
/* Probe strategy (MOSS_PROBE_*) the batch uses for graph g, overriding the
 * graph's own (MOSS_PROBE_AUTO removes the override); MOSS_ESTATE when the
 * graph lacks the tables the strategy needs.  Counts do not depend on it. */
int moss_batch_set_graph_probe(moss_batch *b, const moss_graph *g, int strategy);
typedef struct {
    uint32_t tile_samples;     /* samples per tile: one warp's unit of work      */
    int threads_per_block;     /* 128, 256 or 512                                 */
    int blocks_per_sm;         /* resident blocks of the persistent launch per SM */
    int tuned;                 /* 1 once moss_batch_tune has run                   */
    int graphs;                /* distinct graphs of the batch (when tuned)        */
    int graphs_search;         /* graphs given list-search probes                  */
    int graphs_hash;           /* graphs given the hashed edge set                 */
    int graphs_filter;         /* graphs given the filtered edge set               */
    double run_s;              /* host time of one run under the chosen settings   */
} moss_batch_tuning;
/* Choose the batch's launch settings by measurement, then keep them:
 * (1) each graph's probe strategy, from the SM cycles per sample of its
 * tiles in one run with every graph on list search, one on the hashed set
 * and one on the filtered set (each where its tables exist); (2) the tile
 * size among 1,024 .. 65,536 samples; (3) the block shape among 128, 256 and
 * 512 threads at 1/2, 3/4 and all of the resident blocks that fit; (4) the
 * tile size again under that shape.  *chosen (nullable) receives the tile.
 * Every setting leaves each request's result unchanged. */
int moss_batch_tune(moss_batch *b, void *stream, uint32_t *chosen);
/* The settings in force (and what the last tuning chose). */
int moss_batch_get_tuning(const moss_batch *b, moss_batch_tuning *out);
void moss_batch_free(moss_batch *b);

/* ----------------------------------------------------------------- serving
 * A continuous-batching server over resident graphs.  Requests (graph, k,
 * and either a budget or a target relative standard error) may be submitted
 * from any thread.  A scheduler thread admits them into at most max_active
 * slots while at least reserve_bytes of device memory stay free, and runs
 * ticks: one persistent launch over the next chunk of sample ids of every
 * active request, about tick_samples samples shared fairly, so requests that
 * arrive while a tick runs are sampled in the next one.  A result equals
 * moss_sample_estimate(graph, k, final budget, seed) exactly, alone or in any
 * mix.  With a target eps instead of a budget, the first pilot_samples set
 * the budget: for each class with at least 10 pilot hits, hit fraction f,
 * the samples at which the relative standard error of Theorems 3, 7, 9
 * (sqrt((1/f - 1)/K)) reaches eps, the largest over classes (doubled at k=5,
 * K1 = K2), clamped to [min_budget, max_budget]. */
typedef struct {
    int max_active;            /* requests sampled concurrently (slots)           */
    uint64_t tick_samples;     /* samples per launch over all active requests    */
    uint32_t tile_samples;     /* tile of the persistent launch                   */
    uint64_t pilot_samples;    /* first chunk of a target-error request           */
    uint64_t min_budget;       /* clamp of a budget derived from a target         */
    uint64_t max_budget;
    uint64_t reserve_bytes;    /* admission keeps this much device memory free    */
} moss_server_config;

typedef struct {
    uint64_t budget;           /* samples the request used                         */
    double latency_s;          /* submit to result                                 */
    double queue_s;            /* submit to admission                              */
    uint64_t ticks;            /* launches the request took part in                */
} moss_request_stats;

typedef struct {
    uint64_t ticks, samples, completed, pending, active;
    double busy_s;             /* time inside launches                             */
    double span_s;             /* first submit to last completion                  */
} moss_server_info;

typedef struct moss_server moss_server;
void moss_server_default_config(moss_server_config *cfg);
int moss_server_create(int device, const moss_server_config *cfg /* nullable */, moss_server **out);
/* Register a graph built for k = 4 and 5 (before the first request). */
int moss_server_add_graph(moss_server *s, moss_graph *g, int *graph_id);
/* budget > 0: fixed budget; budget == 0: derive it from target_rse. */
int moss_server_submit(moss_server *s, int graph_id, int k, uint64_t budget, double target_rse, uint64_t seed,
                       uint64_t *request_id);
/* Submit a MOSS-4 + MOSS-4Min request with explicit budgets (budget MOSS-4,
 * budget_min MOSS-4Min samples); its result equals moss_sample_estimate_min
 * on the same graph and seed.  The graph needs the k = 4 tables and
 * MOSS_TABLES_4MIN (MOSS_ESTATE otherwise). */
int moss_server_submit_min(moss_server *s, int graph_id, uint64_t budget, uint64_t budget_min, uint64_t seed,
                           uint64_t *request_id);
/* A MOSS-4 + MOSS-4Min request with a target relative standard error in
 * (0, 1): a pilot of pilot_samples (split evenly) sets the total budget B by
 * moss_budget_for_target_min, and the request then draws K = floor(B/2)
 * MOSS-4 and K-check = B - K MOSS-4Min samples; its result equals
 * moss_sample_estimate_min(graph, K, K-check, seed). */
int moss_server_submit_min_target(moss_server *s, int graph_id, double target_rse, uint64_t seed,
                                  uint64_t *request_id);
/* Block until the request finishes (MOSS_EBUSY after timeout_s); out and
 * stats are nullable.  A request can be waited for once. */
int moss_server_wait(moss_server *s, uint64_t request_id, double timeout_s, moss_result *out,
                     moss_request_stats *stats);
int moss_server_stats(moss_server *s, moss_server_info *out);
/* Stops the scheduler (unfinished requests are abandoned) and frees it. */
void moss_server_free(moss_server *s);
/* The budget rule above, from pilot counts K[2], hits[2][22] (host only). */
uint64_t moss_budget_for_target(int k, const uint64_t *K, const uint64_t *hits, double target,
                                uint64_t min_budget, uint64_t max_budget);
/* The budget rule of MOSS-4 + MOSS-4Min requests (host only), from pilot
 * counts K = {K, K-check} and hits[0] (MOSS-4 classes), hits[1] (MOSS-4Min
 * (class, c) slots).  For each class with at least 10 pilot hits in a
 * source, that source's relative variance per sample: 1/f - 1 for MOSS-4
 * (Theorem 3, f the hit fraction) and K-check b / a^2 - 1 for MOSS-4Min
 * (Theorem 5 with per-CIS probabilities; a = sum_c m_c / c, b = sum_c m_c /
 * c^2); a class seen by both takes their Theorem 1 combination r1 r2 /
 * (r1 + r2).  Since the request draws K = K-check = B / 2, B = 2 r / eps^2,
 * the largest over classes, clamped to [min_budget, max_budget]. */
uint64_t moss_budget_for_target_min(const uint64_t *K, const uint64_t *hits, double target, uint64_t min_budget,
                                    uint64_t max_budget);

/* The covariance matrix of the estimates of moss_finalize's inputs: cov_host
 * (22 x 22 doubles, row-major, host) receives Cov(est_i, est_j) for classes
 * 1..n_classes -- -n_i n_j / K between sampled MOSS-4 classes (proof of
 * Theorem 3), Theorem 10's covariances for MOSS-5 -- with the plug-in values
 * of the variances, the variances on the diagonal, and the row of class 2
 * (n_2, eta_2) from its identity (eq. 2, Sec. 5.1.3).  out (nullable)
 * receives the result as moss_finalize would.  Synchronous on stream. */
int moss_covariance(moss_graph *g, int k, const uint64_t *K, const uint64_t *hits, void *stream, double *cov_host,
                    moss_result *out);

/* Exact totals (requires moss_build_tables for the gamma entries). */
int moss_graph_stats(const moss_graph *g, moss_stats *out);

/* Copy one internal table to host memory (verification and debugging).
 *   MOSS_TABLE_VERT   n x {uint32 off, deg, S_v, 0}
 *   MOSS_TABLE_SLOT   nnz x {uint32 col, nb, sigma threshold, sigma
 *                            alias (position in N_v), off, then col, nb and
 *                            off of the alias position}: for the neighbour
 *                            x = col with twin = position of v in N_x,
 *                            nb = twin | d_x << 16 and off = offset of N_x
 *                            when d_x < 2^16, else nb = 0xFFFFFFFF and
 *                            off = twin
 *   MOSS_TABLE_ACC    nnz x uint32 ACC_sigma^(v) exclusive prefix (Sec. 4.1.3)
 *   MOSS_TABLE_SEED0+l n x {uint64 threshold T, uint32 alias vertex,
 *                      uint32 own vertex, then the alias's MOSS_TABLE_VERT
 *                      record} (32 bytes), l = 0 pi, 1 rho^(1), 2 rho^(2);
 *                      one column per vertex in id order, or with two
 *                      levels (moss_vertex_levels) the nh heavy vertices'
 *                      columns first, then the light ones', each level an
 *                      alias table of its own over its columns in
 *                      ascending id order
 *   MOSS_TABLE_GAMMA0+l n x {uint64 lo, hi} vertex weight of table l
 * and, after a build with MOSS_TABLES_4MIN (Sec. 4.2):
 *   MOSS_TABLE_MIN_SEED  n x {uint64 threshold T, uint32 alias vertex, uint32
 *                        own vertex, then the alias's MOSS_TABLE_MIN_VERT
 *                        record} of pi-check, columns as MOSS_TABLE_SEED0
 *   MOSS_TABLE_MIN_GAMMA n x {uint64 lo, hi} Gamma-check_v
 *   MOSS_TABLE_MIN_VERT  n x {uint32 off, deg, Gamma-check_v lo, hi}
 *   MOSS_TABLE_MIN_SLOT  nnz x {uint64 sigma-check threshold, uint32 alias
 *                        (position in N_v), u, off_u, d_u, d_{v,u}, d_{u,v}}
 *   MOSS_TABLE_MIN_LIST  nnz x {uint32 x, d_x}: each N_v highest first
 *   MOSS_TABLE_MIN_PICK  nnz x {uint32 threshold, u, off_u, d_{v,u} |
 *                        d_{u,v} << 16, then the alias position's u, off_u,
 *                        d_{v,u} | d_{u,v} << 16, and d_u | alias's d_u << 16}
 *                        -- meaningful where Gamma-check_v < 2^32 and every
 *                        field fits 16 bits; otherwise the last word is
 *                        0xFFFFFFFF
 * and, after a build under MOSS_PROBE_FILTER (or AUTO choosing it):
 *   MOSS_TABLE_FILTER    W x uint32 filter words, W the largest power of two
 *                        <= nnz / 8 (at least 1)
 *   MOSS_TABLE_HUB_LIST  H x uint32: the hubs -- every vertex of degree >= D,
 *                        D the smallest degree >= 1 with at most H such
 *                        vertices, H = min(8192, max(16, n / 16)) -- in
 *                        ascending id order (hub i is the i-th),
 *                        0xFFFFFFFF past the last
 *   MOSS_TABLE_HUB_BITS  ceil(H^2 / 32) x uint32: bit i H + j (word / 32, bit
 *                        % 32) set iff hubs i and j are adjacent; edge probes
 *                        between two hubs are answered from these bits
 * and always:
 *   MOSS_TABLE_ORDER     n x uint32: the input id of each internal vertex
 *                        (the identity under MOSS_ORDER_INPUT)
 * bytes must equal the table size.  Synchronous. */
#define MOSS_TABLE_VERT   0
#define MOSS_TABLE_SLOT   1
#define MOSS_TABLE_ACC    2
#define MOSS_TABLE_SEED0  3
#define MOSS_TABLE_GAMMA0 6
#define MOSS_TABLE_MIN_SEED  9
#define MOSS_TABLE_MIN_GAMMA 10
#define MOSS_TABLE_MIN_VERT  11
#define MOSS_TABLE_MIN_SLOT  12
#define MOSS_TABLE_MIN_LIST  13
#define MOSS_TABLE_FILTER    14
#define MOSS_TABLE_MIN_PICK  15
#define MOSS_TABLE_HUB_LIST  16
#define MOSS_TABLE_HUB_BITS  17
#define MOSS_TABLE_ORDER     18
int moss_table_export(const moss_graph *g, int table, void *host_dst, uint64_t bytes);

void moss_graph_free(moss_graph *g);

/* The library's classification tables (host only, no GPU needed; any
 * pointer may be NULL): class4[64] and class5[1024] map an edge mask over
 * the sampled roles (pair bits (0,1),(0,2),...) to its class M_i (Sec. 4.1.2,
 * Table 2; 0 when disconnected); centred[4096] holds c(s) of MOSS-4Min
 * (Sec. 4.2: the 3-paths p0-p1-p2-p3 with p0 above p2 and p3 above p1, each
 * once) at index mask << 6 | order, order bit b set when the first role of
 * pair b is above the second, and 0 for classes other than 4-cycle, diamond
 * and 4-clique. */
int moss_class_tables(uint8_t *class4, uint8_t *class5, uint8_t *centred);

/* Measurement helper, not a step of the method.  Every sampler step reads
 * one 32-byte sector at an address no other lane shares (Sec. 4.1.3: alias
 * draws, uniform list picks and adjacency probes at random positions), so
 * the samplers are bounded by the rate of independent random sector reads,
 * not by streaming bandwidth.  This call allocates a zeroed device buffer of
 * `bytes` (a positive multiple of 32) on `device`, reads 2^28 sectors of it
 * at uniform random positions from a full persistent grid (four independent
 * 256-bit loads in flight per thread) after one warm-up launch of the same
 * length, and writes the sectors per second of the timed launch (CUDA
 * events on `stream`, NULL = default stream) to *sectors_per_s.  A buffer
 * smaller than L2 measures the L2 random-read ceiling, one far larger the
 * HBM one.  Synchronous; frees its buffer before returning.  Errors:
 * MOSS_EINVAL (NULL output, bad size or device), MOSS_ENOMEM, MOSS_ECUDA. */
int moss_gather_rate(uint64_t bytes, int device, void *stream, double *sectors_per_s);

const char *moss_strerror(int status);
const char *moss_last_error_detail(void);
const char *moss_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MOSS_H */
