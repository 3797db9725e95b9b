// moss_capi.cu -- the C ABI (include/moss.h): argument checking, device
// memory, stream ordering and error reporting around the kernels of
// moss_tables.cu, moss_sample.cu and moss_finalize.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>

#include "../../include/moss.h"
#include "moss_internal.cuh"
#include "moss_order.cuh"

using namespace moss;

// ---------------------------------------------------------------- errors --
namespace {

thread_local char g_detail[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? MOSS_ENOMEM : MOSS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MOSS_CUDA(call, what)                       \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ------------------------------------------------------ class lookup table --
// The class of each edge mask.  Pair (i,j), i<j, in the order
// (0,1),(0,2),...,(k-2,k-1) is an edge when its bit is set.  A connected
// graph is identified by how many spanning 3-paths and 3-stars (k = 4,
// Sec. 4.1.2) or forks, 5-paths and 4-stars (k = 5, Table 2) it contains:
// paths are counted as vertex orders along edges (halved), stars as vertices
// adjacent to all others, forks as ordered (centre, middle, end) triples whose
// remaining two vertices hang on the centre.
const int kTable4[6][2] = {{1, 0}, {0, 1}, {4, 0}, {2, 1}, {6, 2}, {12, 4}};
const int kTable2[21][3] = {{0, 1, 0},  {0, 0, 1},  {1, 0, 0},   {1, 2, 0},   {2, 2, 0},   {0, 5, 0},   {2, 1, 0},
                            {2, 0, 1},  {4, 4, 0},  {4, 7, 0},   {5, 2, 1},   {4, 4, 1},   {6, 6, 0},   {10, 10, 1},
                            {9, 6, 1},  {12, 6, 2}, {10, 14, 0}, {20, 24, 1}, {20, 18, 2}, {36, 36, 3}, {60, 60, 5}};

int mask_class(int k, uint32_t mask) {
    bool adj[5][5] = {};
    int b = 0;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j, ++b)
            if (mask >> b & 1u) adj[i][j] = adj[j][i] = true;
    // connectivity by repeated relaxation from vertex 0
    bool seen[5] = {true, false, false, false, false};
    for (int it = 0; it < k; ++it)
        for (int i = 0; i < k; ++i)
            if (seen[i])
                for (int j = 0; j < k; ++j)
                    if (adj[i][j]) seen[j] = true;
    for (int i = 0; i < k; ++i)
        if (!seen[i]) return 0;
    // Hamiltonian paths: vertex orders with consecutive edges, each path twice
    int perm[5] = {0, 1, 2, 3, 4};
    int orders = 0;
    // iterate all permutations of perm[0..k)
    int c[5] = {0, 0, 0, 0, 0};
    auto path_ok = [&](const int *p) {
        for (int i = 0; i + 1 < k; ++i)
            if (!adj[p[i]][p[i + 1]]) return false;
        return true;
    };
    orders += path_ok(perm);
    for (int i = 1; i < k;) {  // Heap's algorithm
        if (c[i] < i) {
            int a = (i % 2 == 0) ? 0 : c[i];
            int t = perm[a]; perm[a] = perm[i]; perm[i] = t;
            orders += path_ok(perm);
            ++c[i];
            i = 1;
        } else {
            c[i] = 0;
            ++i;
        }
    }
    const int paths = orders / 2;
    int stars = 0;
    for (int i = 0; i < k; ++i) {
        int d = 0;
        for (int j = 0; j < k; ++j) d += adj[i][j];
        if (d == k - 1) ++stars;
    }
    if (k == 4) {
        for (int i = 0; i < 6; ++i)
            if (kTable4[i][0] == paths && kTable4[i][1] == stars) return i + 1;
        return -1;
    }
    int forks = 0;
    for (int ce = 0; ce < 5; ++ce)
        for (int mid = 0; mid < 5; ++mid) {
            if (mid == ce || !adj[ce][mid]) continue;
            for (int end = 0; end < 5; ++end) {
                if (end == ce || end == mid || !adj[mid][end]) continue;
                bool ok = true;
                for (int x = 0; x < 5; ++x)
                    if (x != ce && x != mid && x != end && !adj[ce][x]) ok = false;
                forks += ok;
            }
        }
    for (int i = 0; i < 21; ++i)
        if (kTable2[i][0] == forks && kTable2[i][1] == paths && kTable2[i][2] == stars) return i + 1;
    return -1;
}

// c(s) of Sec. 4.2 for a 4-vertex CIS with edge mask `mask` over the roles
// 0..3 (pair bits (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)) whose vertices are
// ordered by `above`: bit b set when the first vertex of pair b is above the
// second in the total order.  Counts the 3-paths p0-p1-p2-p3 with p0 above p2
// and p3 above p1, each unordered path once (the orientation whose end roles
// satisfy p0 < p3).
int centred_paths_of(uint32_t mask, uint32_t above) {
    auto bit = [](int a, int b) { return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5); };   // a < b
    auto edge = [&](int a, int b) { return (mask >> (a < b ? bit(a, b) : bit(b, a)) & 1u) != 0; };
    auto over = [&](int a, int b) { return a < b ? (above >> bit(a, b) & 1u) != 0 : (above >> bit(b, a) & 1u) == 0; };
    int c = 0;
    for (int e0 = 0; e0 < 4; ++e0)
        for (int e3 = e0 + 1; e3 < 4; ++e3) {
            int mid[2], k = 0;
            for (int x = 0; x < 4; ++x)
                if (x != e0 && x != e3) mid[k++] = x;
            for (int o = 0; o < 2; ++o) {
                const int p1 = mid[o], p2 = mid[1 - o];
                if (edge(e0, p1) && edge(p1, p2) && edge(p2, e3) && over(e0, p2) && over(e3, p1)) ++c;
            }
        }
    return c;
}

std::atomic<int> g_sms[64];   // SM counts, 0 until queried

std::mutex g_lut_mutex;
bool g_lut_ready[64] = {};
uint8_t g_lut4_h[64], g_lut5_h[1024], g_lutc_h[4096];
bool g_lut_built = false;

// the host copies of the tables (callers hold g_lut_mutex)
void build_host_luts() {
    if (!g_lut_built) {
        for (uint32_t m = 0; m < 64; ++m) g_lut4_h[m] = (uint8_t)mask_class(4, m);
        for (uint32_t m = 0; m < 1024; ++m) g_lut5_h[m] = (uint8_t)mask_class(5, m);
        for (uint32_t i = 0; i < 4096; ++i) {   // counted classes only: 4-cycle, diamond, 4-clique
            const int cls = g_lut4_h[i >> 6];
            g_lutc_h[i] = (uint8_t)(cls == 3 || cls == 5 || cls == 6 ? centred_paths_of(i >> 6, i & 63u) : 0);
        }
        g_lut_built = true;
    }
}

int ensure_luts(int device) {
    std::lock_guard<std::mutex> lk(g_lut_mutex);
    build_host_luts();
    if (device < 0 || device >= 64) return fail(MOSS_EINVAL, "device ordinal %d out of range", device);
    if (!g_lut_ready[device]) {
        upload_luts(g_lut4_h, g_lut5_h, g_lutc_h);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "uploading class tables");
        g_lut_ready[device] = true;
    }
    return MOSS_OK;
}

}  // namespace

// ------------------------------------------------------------ graph object --
struct moss_graph {
    int device = 0;
    uint32_t n = 0;
    uint64_t nnz = 0;
    uint4 *vert = nullptr;
    uint32_t *col = nullptr;
    uint4 *slot = nullptr;
    uint32_t *acc = nullptr;
    uint32_t *owner = nullptr;   // vertex of each CSR slot (flat per-slot passes)
    uint64_t *sq = nullptr;      // prefix of (d_x - 1)^2 within each list
    u128 *gam[kMethods] = {nullptr, nullptr, nullptr, nullptr};    // [3]: Gamma-check_v (min arena)
    uint4 *seed[kMethods] = {nullptr, nullptr, nullptr, nullptr};
    uint4 *mvert = nullptr;      // MOSS-4Min tables, in min_arena
    uint4 *mslot = nullptr;
    uint4 *mpick = nullptr;
    uint2 *rlist = nullptr;
    void *min_arena = nullptr;
    DevTotals *tot = nullptr;
    DevTotals tot_h{};
    unsigned built = 0;          // bit l: vertex table l; bit 3: sigma tables; bit 4: edge hash; bit 5: MOSS-4Min
    uint64_t *partials = nullptr;
    int partial_rows = 0;
    uint64_t *counts = nullptr;  // 2 x 22
    moss_result *res_dev = nullptr;
    double *cov_dev = nullptr;   // 22 x 22 covariance matrix
    uint32_t *flags = nullptr;   // device status: [0] error bits, [1] matched twins
    uint32_t *defer = nullptr;   // Path-5 deferral bitmap (kDeferChunk bits)
    void *arena = nullptr;       // every device array above lives in this one allocation
    int probe = MOSS_PROBE_AUTO; // membership tests (MOSS_PROBE_*), as requested
    int rng = MOSS_RNG_SPLITMIX64;   // word generator of the samples (MOSS_RNG_*)
    int vsplit = MOSS_VERTEX_ONE_LEVEL;   // heavy level of the vertex tables: w_v 2^vsplit >= W (set at load)
    int vsplit_min = MOSS_VERTEX_ONE_LEVEL;   // the same for the MOSS-4Min table
    unsigned long long *hash = nullptr;  // kBucketKeys keys per bucket
    uint64_t hash_buckets = 0;
    uint32_t *filter = nullptr;  // Bloom filter in front of the hash
    uint64_t filter_words = 0;
    void *hub_mem = nullptr;     // hub adjacency behind the filter: rank table, bitmap, hub list
    uint2 *hub_rank = nullptr;
    uint32_t *hub_bits = nullptr;
    uint32_t *hub_list = nullptr;
    uint32_t *order = nullptr;   // input id of each internal vertex (MOSS_ORDER_DEGREE), else null
    moss_result res_host{};      // host staging of the result
    uint32_t flags_host[2] = {0, 0};
};

namespace {

void release(moss_graph *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    // ordered on the legacy default stream, i.e. after the work of blocking streams
    if (g->arena) cudaFreeAsync(g->arena, 0);
    if (g->hash) cudaFreeAsync(g->hash, 0);
    if (g->filter) cudaFreeAsync(g->filter, 0);
    if (g->hub_mem) cudaFreeAsync(g->hub_mem, 0);
    if (g->min_arena) cudaFreeAsync(g->min_arena, 0);
    delete g;
}

// buckets of the hashed edge set: the next power of two >= nnz / 2, so at
// least 4 slots per undirected edge (nnz / 2 edges, kBucketKeys slots each)
uint64_t hash_buckets_for(uint64_t nnz) {
    uint64_t b = 2;
    while (b < (nnz + 1) / 2) b <<= 1;
    return b;
}

// words of the edge filter: the largest power of two <= nnz / 8 (4 to 8 bits per edge)
uint64_t filter_words_for(uint64_t nnz) {
    uint64_t w = 1;
    while (w * 2 <= nnz / 8) w <<= 1;
    return w;
}

int effective_probe(const moss_graph *g) {
    if (g->probe != MOSS_PROBE_AUTO) return g->probe;
    return hash_buckets_for(g->nnz) * 8 * kBucketKeys > (64ull << 20) ? MOSS_PROBE_FILTER : MOSS_PROBE_HASH;
}

DevGraph view_with(const moss_graph *g, int eff) {
    DevGraph d;
    d.vert = g->vert;
    d.col = g->col;
    d.slot = g->slot;
    d.acc = g->acc;
    d.sq = g->sq;
    for (int l = 0; l < kMethods; ++l) d.seed[l] = g->seed[l];
    d.mvert = g->mvert;
    d.mslot = g->mslot;
    d.mpick = g->mpick;
    d.rlist = g->rlist;
    d.defer = g->defer;
    d.n = g->n;
    d.rng = g->rng == MOSS_RNG_PHILOX4X32 ? kRngPhilox : kRngSplitMix;
    for (int l = 0; l < kMethods; ++l) {
        d.nheavy[l] = g->tot_h.level[l].nh;
        d.tlight[l] = g->tot_h.level[l].tl;
    }
    const bool use_hash = eff != MOSS_PROBE_SEARCH && (g->built >> 4 & 1u);
    const bool use_filter = eff == MOSS_PROBE_FILTER && (g->built >> 6 & 1u);
    d.hash = use_hash ? reinterpret_cast<const uint4 *>(g->hash) : nullptr;
    d.filter = use_hash && use_filter ? g->filter : nullptr;
    const bool hubs = use_hash && use_filter && g->hub_bits;
    d.hub_rank = hubs ? g->hub_rank : nullptr;
    d.hub_bits = hubs ? g->hub_bits : nullptr;
    d.hubs = hub_capacity(g->n);
    uint32_t lg = 0;
    while ((1ULL << lg) < g->hash_buckets) ++lg;
    d.hash_mask = use_hash ? (uint32_t)(g->hash_buckets - 1) : 0;
    d.hash_shift = 64 - lg;
    uint32_t lf = 0;
    while ((1ULL << lf) < g->filter_words) ++lf;
    d.filter_shift = 64 - lf;
    return d;
}

DevGraph view(const moss_graph *g) { return view_with(g, effective_probe(g)); }

void describe_flags(uint32_t f, char *buf, size_t len) {
    buf[0] = 0;
    const char *names[] = {"row_ptr not monotone or wrong ends", "neighbour id >= n", "self loop",
                           "list not strictly increasing", "edge without its reverse", "total out of range"};
    for (int b = 0; b < 6; ++b)
        if (f >> b & 1u) {
            size_t u = strlen(buf);
            snprintf(buf + u, len - u, "%s%s", u ? "; " : "", names[b]);
        }
}

// A stream-ordered memory pool per device, owned by the library, that keeps
// freed memory for reuse (so repeated load/build/free cycles do not return to
// the driver).
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[64];
bool g_pool_ok[64] = {};

cudaError_t pool_alloc(int device, void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mutex);
        if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
        if (!g_pool_ok[device]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            cudaError_t e = cudaMemPoolCreate(&g_pool[device], &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = ~0ULL;
            e = cudaMemPoolSetAttribute(g_pool[device], cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            g_pool_ok[device] = true;
        }
        pool = g_pool[device];
    }
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s);
}

// Carves 256-byte aligned arrays out of one allocation (first pass: size).
struct Carver {
    uint8_t *base = nullptr;
    size_t off = 0;
    template <typename T>
    T *take(uint64_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += (size_t)(count ? count : 1) * sizeof(T);
        return p;
    }
};

int read_flags(moss_graph *g, cudaStream_t s) {
    MOSS_CUDA(cudaMemcpyAsync(g->flags_host, g->flags, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s),
              "reading status");
    MOSS_CUDA(cudaStreamSynchronize(s), "synchronising stream");
    return MOSS_OK;
}

bool method_ready(const moss_graph *g, int method) {
    const int eff = effective_probe(g);
    const bool probes = eff == MOSS_PROBE_SEARCH ||
                        ((g->built >> 4 & 1u) && (eff != MOSS_PROBE_FILTER || (g->built >> 6 & 1u)));
    if (method == MOSS_METHOD_MOSS4MIN) return (g->built >> 5 & 1u) && probes;
    return (g->built >> 3 & 1u) && (g->built >> method & 1u) && probes;
}

}  // namespace

extern "C" {

int moss_class_tables(uint8_t *class4, uint8_t *class5, uint8_t *centred) {
    std::lock_guard<std::mutex> lk(g_lut_mutex);
    build_host_luts();
    if (class4) memcpy(class4, g_lut4_h, sizeof(g_lut4_h));
    if (class5) memcpy(class5, g_lut5_h, sizeof(g_lut5_h));
    if (centred) memcpy(centred, g_lutc_h, sizeof(g_lutc_h));
    return MOSS_OK;
}

const char *moss_version(void) { return "moss-gb300 0.1 (sm_103a)"; }

const char *moss_last_error_detail(void) { return g_detail; }

const char *moss_strerror(int status) {
    switch (status) {
        case MOSS_OK: return "ok";
        case MOSS_EINVAL: return "invalid argument";
        case MOSS_ENOMEM: return "out of memory";
        case MOSS_ECUDA: return "CUDA error";
        case MOSS_EGRAPH: return "invalid graph";
        case MOSS_EOVERFLOW: return "value out of range";
        case MOSS_ESTATE: return "tables not built";
        case MOSS_EBUSY: return "not finished";
        default: return "unknown status";
    }
}

int moss_graph_load_csr(const void *row_ptr, int row_ptr_is_64, const uint32_t *col, uint32_t n, uint64_t nnz,
                        int device, void *stream, moss_graph **out) {
    return moss_graph_load_csr_order(row_ptr, row_ptr_is_64, col, n, nnz, MOSS_ORDER_INPUT, device, stream, out);
}

int moss_graph_load_csr_order(const void *row_ptr, int row_ptr_is_64, const uint32_t *col, uint32_t n, uint64_t nnz,
                              int order, int device, void *stream, moss_graph **out) {
    if (!out) return fail(MOSS_EINVAL, "out is NULL");
    *out = nullptr;
    if (order != MOSS_ORDER_INPUT && order != MOSS_ORDER_DEGREE) return fail(MOSS_EINVAL, "order %d", order);
    const bool ordered = order == MOSS_ORDER_DEGREE;
    if (!row_ptr) return fail(MOSS_EINVAL, "row_ptr is NULL");
    if (nnz > 0 && !col) return fail(MOSS_EINVAL, "col is NULL with nnz > 0");
    if (n == 0) return fail(MOSS_EINVAL, "graph has no vertex");
    if (n == 0xFFFFFFFFu) return fail(MOSS_EOVERFLOW, "n must be below 2^32 - 1");
    if (nnz >= (1ULL << 32)) return fail(MOSS_EOVERFLOW, "nnz = %llu must be below 2^32", (unsigned long long)nnz);
    if (nnz % 2) return fail(MOSS_EGRAPH, "nnz is odd: an undirected graph stores both directions");
    int ndev = 0;
    MOSS_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(MOSS_EINVAL, "device %d not present (%d devices)", device, ndev);
    DeviceGuard dg(device);
    int rc = ensure_luts(device);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    moss_graph *g = new (std::nothrow) moss_graph;
    if (!g) return fail(MOSS_ENOMEM, "host allocation");
    g->device = device;
    g->n = n;
    g->vsplit = n >= (1u << 20) ? MOSS_VERTEX_SPLIT_DEFAULT
                                : (n >= (1u << 14) ? MOSS_VERTEX_SPLIT_MID : MOSS_VERTEX_ONE_LEVEL);
    g->vsplit_min = n >= (1u << 20) ? MOSS_VERTEX_SPLIT_DEFAULT : MOSS_VERTEX_ONE_LEVEL;
    g->nnz = nnz;
    void *rp_dev = nullptr;
    void *oscratch = nullptr;   // renumbering scratch (released before return)
    const size_t rp_bytes = (size_t)(n + 1ULL) * (row_ptr_is_64 ? 8 : 4);
    cudaError_t e = cudaSuccess;
    int blocks = table_blocks(n);
    int prow = 0;
    for (int m = 0; m < kMethods; ++m) {
        int b = sample_rows(m, device);
        prow = b > prow ? b : prow;
    }
    g->partial_rows = prow;
#define STEP(call, what)                          \
    do {                                          \
        e = (call);                               \
        if (e != cudaSuccess) {                   \
            rc = cuda_fail(e, what);              \
            goto fail_out;                        \
        }                                         \
    } while (0)
    {
        Carver c;
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                STEP(pool_alloc(device, &g->arena, c.off, s), "allocating graph memory");
                c.base = static_cast<uint8_t *>(g->arena);
                c.off = 0;
            }
            g->vert = c.take<uint4>(n);
            g->col = c.take<uint32_t>(nnz);
            g->slot = c.take<uint4>(2 * nnz);
            g->acc = c.take<uint32_t>(nnz);
            g->owner = c.take<uint32_t>(nnz);
            g->sq = c.take<uint64_t>(nnz);
            for (int l = 0; l < 3; ++l) {
                g->gam[l] = c.take<u128>(n);
                g->seed[l] = c.take<uint4>(2 * (uint64_t)n);
            }
            g->tot = c.take<DevTotals>(1);
            g->partials = c.take<uint64_t>((uint64_t)prow * kSlots + (uint64_t)slot_partial_rows(n) * 6 * 2);
            g->counts = c.take<uint64_t>(2 * kSlots);
            g->res_dev = c.take<moss_result>(1);
            g->cov_dev = c.take<double>(kSlots * kSlots);
            g->flags = c.take<uint32_t>(2);
            g->defer = c.take<uint32_t>(kDeferChunk / 32);
            rp_dev = c.take<uint8_t>(rp_bytes);
            if (ordered) g->order = c.take<uint32_t>(n);
        }
    }
    STEP(cudaMemcpyAsync(rp_dev, row_ptr, rp_bytes, cudaMemcpyDefault, s), "copying row_ptr");
    STEP(cudaMemsetAsync(g->flags, 0, 2 * sizeof(uint32_t), s), "clearing status");
    if (ordered) {
        // the input lists are read in place when they are device memory of
        // this device, else copied beside the scratch first
        bool direct = false;
        if (nnz) {
            cudaPointerAttributes pa;
            if (cudaPointerGetAttributes(&pa, col) == cudaSuccess)
                direct = pa.type == cudaMemoryTypeDevice && pa.device == device;
            else
                cudaGetLastError();
        }
        const uint64_t ob = (order_scratch_bytes(n) + 255) & ~255ull;
        STEP(pool_alloc(device, &oscratch, ob + (direct ? 0 : nnz * sizeof(uint32_t)), s), "allocating order scratch");
        const uint32_t *src = col;
        if (nnz && !direct) {
            uint32_t *copy = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(oscratch) + ob);
            STEP(cudaMemcpyAsync(copy, col, nnz * sizeof(uint32_t), cudaMemcpyDefault, s), "copying col");
            src = copy;
        }
        uint32_t *rp_new = nullptr;
        STEP(launch_degree_order(rp_dev, row_ptr_is_64, src, n, nnz, g->order, g->col, oscratch, &rp_new, g->flags, s),
             "ordering kernels");
        STEP(launch_vertices(rp_new, 0, n, nnz, g->vert, g->flags, s), "vertex kernel");
        void *done = oscratch;
        oscratch = nullptr;
        STEP(cudaFreeAsync(done, s), "releasing order scratch");
    } else {
        if (nnz) STEP(cudaMemcpyAsync(g->col, col, nnz * sizeof(uint32_t), cudaMemcpyDefault, s), "copying col");
        STEP(launch_vertices(rp_dev, row_ptr_is_64, n, nnz, g->vert, g->flags, s), "vertex kernel");
    }
    {
        u128 *tp = reinterpret_cast<u128 *>(g->partials + (uint64_t)prow * kSlots);
        STEP(launch_slots(n, nnz, g->col, g->vert, g->slot, g->acc, g->owner, g->sq, g->gam[0], g->gam[1], g->gam[2],
                          tp, blocks, g->flags, s, aux_streams()),
             "slot kernels");
        STEP(launch_totals(tp, slot_partial_rows(n), g->tot, s), "totals kernel");
    }
    STEP(cudaMemcpyAsync(&g->tot_h, g->tot, sizeof(DevTotals), cudaMemcpyDeviceToHost, s), "reading totals");
    rc = read_flags(g, s);
    if (rc) goto fail_out;
    if (!g->flags_host[0] && g->flags_host[1] != nnz) g->flags_host[0] |= kErrAsym;
    if (g->flags_host[0]) {
        char buf[256];
        describe_flags(g->flags_host[0], buf, sizeof(buf));
        rc = fail(MOSS_EGRAPH, "invalid CSR: %s", buf);
        goto fail_out;
    }
#undef STEP
    *out = g;
    return MOSS_OK;
fail_out:
    if (oscratch) cudaFreeAsync(oscratch, s);
    release(g);
    return rc;
}

// The MOSS-4Min tables in their own allocation (made once per graph).
static int build_min_tables(moss_graph *g, cudaStream_t s, const AuxStreams *aux) {
    cudaError_t e;
    if (!g->min_arena) {
        Carver c;
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                if ((e = pool_alloc(g->device, &g->min_arena, c.off, s)) != cudaSuccess)
                    return cuda_fail(e, "allocating MOSS-4Min tables");
                c.base = static_cast<uint8_t *>(g->min_arena);
                c.off = 0;
            }
            g->mvert = c.take<uint4>(g->n);
            g->mslot = c.take<uint4>(2 * g->nnz);
            g->mpick = c.take<uint4>(2 * g->nnz);
            g->rlist = c.take<uint2>(g->nnz);
            g->gam[3] = c.take<u128>(g->n);
            g->seed[3] = c.take<uint4>(2 * (uint64_t)g->n);
        }
    }
    void *scratch = nullptr;
    if ((e = pool_alloc(g->device, &scratch, min_scratch_bytes(g->n, g->nnz), s)) != cudaSuccess)
        return cuda_fail(e, "allocating scratch");
    e = launch_min_tables(g->n, g->nnz, g->vert, g->col, g->owner, g->slot, g->mvert, g->mslot, g->mpick, g->rlist,
                          g->gam[3], g->seed[3], g->tot, scratch, g->flags, g->vsplit_min, s, aux);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "MOSS-4Min table kernels");
    return MOSS_OK;
}

int moss_build_tables(moss_graph *g, unsigned k_mask, void *stream) {
    if (!g) return fail(MOSS_EINVAL, "graph is NULL");
    if ((k_mask & ~((1u << 4) | (1u << 5) | MOSS_TABLES_4MIN)) || !k_mask)
        return fail(MOSS_EINVAL, "k_mask must combine (1<<4), (1<<5) and MOSS_TABLES_4MIN");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // independent chains on s and the caller thread's auxiliary streams (when
    // it has them), each with its own scratch: the per-list tables of short
    // lists on s and of long lists on the first auxiliary stream, the vertex
    // tables on the second, the edge hash (and filter) on the third -- or,
    // when the MOSS-4Min tables are built (the longest chain), those on the
    // third and the edge hash after the per-list tables on s
    const uint64_t sigma_bytes = ((g->nnz * 4 + 255) & ~255ULL) + ((g->nnz * 8 + 255) & ~255ULL);
    const uint64_t seed_bytes = seed_scratch_bytes(g->n);
    void *scratch = nullptr;
    int rc = MOSS_OK;
    cudaError_t e;
    g->built = 0;
    const int eff = effective_probe(g);
    const bool want_hash = eff != MOSS_PROBE_SEARCH, want_filter = eff == MOSS_PROBE_FILTER;
    const uint64_t buckets = hash_buckets_for(g->nnz), words = filter_words_for(g->nnz);
    if (want_hash && buckets > (1ULL << 32)) return fail(MOSS_EOVERFLOW, "edge hash above 2^32 buckets");
    // allocations first, on s, so that every chain may use them after the fork
    if (want_hash && g->hash && g->hash_buckets != buckets) {
        cudaFreeAsync(g->hash, s);
        g->hash = nullptr;
    }
    if (want_hash && !g->hash) {
        if ((e = pool_alloc(g->device, reinterpret_cast<void **>(&g->hash), buckets * 8 * kBucketKeys, s)) !=
            cudaSuccess)
            return cuda_fail(e, "allocating edge hash");
        g->hash_buckets = buckets;
    }
    if (want_filter && g->filter && g->filter_words != words) {
        cudaFreeAsync(g->filter, s);
        g->filter = nullptr;
    }
    if (want_filter && !g->filter) {
        if ((e = pool_alloc(g->device, reinterpret_cast<void **>(&g->filter), words * 4, s)) != cudaSuccess)
            return cuda_fail(e, "allocating edge filter");
        g->filter_words = words;
    }
    if (want_filter && !g->hub_mem) {
        if ((e = pool_alloc(g->device, &g->hub_mem, hub_bytes(g->n), s)) != cudaSuccess)
            return cuda_fail(e, "allocating hub adjacency");
    }
    if ((e = pool_alloc(g->device, &scratch, sigma_bytes + seed_bytes, s)) != cudaSuccess)
        return cuda_fail(e, "allocating scratch");
    uint32_t *idx = static_cast<uint32_t *>(scratch);
    uint64_t *pre = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(scratch) + ((g->nnz * 4 + 255) & ~255ULL));
    void *seed_scratch = static_cast<uint8_t *>(scratch) + sigma_bytes;
    e = cudaMemsetAsync(g->flags, 0, 2 * sizeof(uint32_t), s);
    const AuxStreams *aux = e == cudaSuccess ? aux_streams() : nullptr;
    if (aux && aux->fork(s) != cudaSuccess) {
        cudaGetLastError();
        aux = nullptr;
    }
    const bool want_min = (k_mask & MOSS_TABLES_4MIN) != 0;
    cudaStream_t sv = aux ? aux->a[1] : s, sm = aux ? aux->a[2] : s, sh = aux && !want_min ? aux->a[2] : s;
    // MOSS-4Min tables
    bool min_built = false;
    if (e == cudaSuccess && want_min) {
        rc = build_min_tables(g, sm, aux);
        min_built = rc == MOSS_OK;
    }
    // vertex alias tables
    int which[3], nt = 0;
    u128 *w[3];
    uint4 *seed[3];
    const uint4 *vrec[3] = {g->vert, g->vert, g->vert};
    for (int l = 0; l < 3; ++l) {
        const bool want = (l == 0 && (k_mask & (1u << 4))) || (l > 0 && (k_mask & (1u << 5)));
        if (want) {
            which[nt] = l;
            w[nt] = g->gam[l];
            seed[nt] = g->seed[l];
            ++nt;
        }
    }
    cudaError_t ev = cudaSuccess;
    if (e == cudaSuccess && nt > 0)
        ev = launch_seed_alias(g->n, g->tot, nt, which, w, seed, vrec, seed_scratch, g->flags, g->vsplit, sv);
    // per-list tables
    if (e == cudaSuccess)
        e = launch_sigma_alias(g->n, g->nnz, g->vert, g->acc, g->owner, g->slot, idx, pre, s, aux, 0);
    // edge hash and filter
    bool hashed = false, filtered = false;
    cudaError_t eh = cudaSuccess;
    if (e == cudaSuccess && want_hash) {
        uint32_t lg = 0;
        while ((1ULL << lg) < buckets) ++lg;
        eh = cudaMemsetAsync(g->hash, 0xFF, buckets * 8 * kBucketKeys, sh);
        if (eh == cudaSuccess)
            eh = launch_edge_hash(g->nnz, g->col, g->owner, g->hash, (uint32_t)(buckets - 1), 64 - lg, sh);
        hashed = eh == cudaSuccess;
    }
    if (e == cudaSuccess && eh == cudaSuccess && want_filter) {
        uint32_t lf = 0;
        while ((1ULL << lf) < words) ++lf;
        eh = cudaMemsetAsync(g->filter, 0, words * 4, sh);
        if (eh == cudaSuccess) eh = launch_edge_filter(g->nnz, g->col, g->owner, g->filter, 64 - lf, sh);
        if (eh == cudaSuccess) eh = launch_hub_tables(g->n, g->vert, g->col, g->hub_mem, &g->hub_rank, &g->hub_bits,
                                                       &g->hub_list, sh);
        filtered = eh == cudaSuccess;
    }
    if (aux) {
        const cudaError_t ej = aux->join(s);
        if (e == cudaSuccess) e = ej;
    }
    cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = eh != cudaSuccess ? eh : ev;
    if (e != cudaSuccess) return cuda_fail(e, "table kernels");
    if (rc) return rc;
    MOSS_CUDA(cudaMemcpyAsync(&g->tot_h, g->tot, sizeof(DevTotals), cudaMemcpyDeviceToHost, s), "reading totals");
    rc = read_flags(g, s);
    if (rc) return rc;
    if (g->flags_host[0] & kErrOverflow) return fail(MOSS_EOVERFLOW, "a vertex weight total times n exceeds 2^128");
    g->built = 1u << 3;
    if (k_mask & (1u << 4)) g->built |= 1u;
    if (k_mask & (1u << 5)) g->built |= 6u;
    if (hashed) g->built |= 1u << 4;
    if (min_built) g->built |= 1u << 5;
    if (filtered) g->built |= 1u << 6;
    return MOSS_OK;
}

int moss_set_probe(moss_graph *g, int strategy) {
    if (!g) return fail(MOSS_EINVAL, "graph is NULL");
    if (strategy < MOSS_PROBE_SEARCH || strategy > MOSS_PROBE_AUTO)
        return fail(MOSS_EINVAL, "unknown probe strategy %d", strategy);
    g->probe = strategy;
    return MOSS_OK;
}

int moss_set_rng(moss_graph *g, int rng) {
    if (!g) return fail(MOSS_EINVAL, "graph is NULL");
    if (rng != MOSS_RNG_SPLITMIX64 && rng != MOSS_RNG_PHILOX4X32) return fail(MOSS_EINVAL, "unknown generator %d", rng);
    g->rng = rng;
    return MOSS_OK;
}

int moss_get_rng(const moss_graph *g) { return g ? g->rng : MOSS_EINVAL; }

int moss_set_vertex_split(moss_graph *g, int split) {
    if (!g) return fail(MOSS_EINVAL, "graph is NULL");
    if (split < 0 || split > MOSS_VERTEX_ONE_LEVEL)
        return fail(MOSS_EINVAL, "vertex split %d outside 0..%d", split, MOSS_VERTEX_ONE_LEVEL);
    if (split != g->vsplit || split != g->vsplit_min) g->built &= ~0xFu & ~(1u << 5);   // rebuilt at the next build
    g->vsplit = split;
    g->vsplit_min = split;
    return MOSS_OK;
}

int moss_vertex_levels(const moss_graph *g, int which, uint32_t *nheavy, uint64_t *tlight) {
    if (!g || !nheavy || !tlight) return fail(MOSS_EINVAL, "NULL argument");
    if (which < 0 || which >= kMethods) return fail(MOSS_EINVAL, "which must be 0..3");
    *nheavy = g->tot_h.level[which].nh;
    *tlight = g->tot_h.level[which].tl;
    return MOSS_OK;
}

static int sample_into(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed, cudaStream_t s,
                       uint64_t *counts_dev, uint8_t *classes, uint32_t *verts) {
    if (method < 0 || method >= kMethods) return fail(MOSS_EINVAL, "method %d", method);
    if (!method_ready(g, method)) return fail(MOSS_ESTATE, "tables for method %d not built", method);
    if (count > 0 && g->tot_h.gamma[method] == 0)
        return fail(MOSS_EINVAL, "method %d has total weight 0 on this graph: no sample exists", method);
    if (first + count < first) return fail(MOSS_EOVERFLOW, "sample range wraps");
    const DevGraph dv = view(g);
    const int blocks = sample_launch_blocks(method, g->device, dv);
    // per-warp 32-bit counters: keep each launch below 2^31 samples per warp
    const uint64_t max_chunk = (uint64_t)blocks * 8 * (1ULL << 31);
    if (count == 0) {
        MOSS_CUDA(cudaMemsetAsync(counts_dev, 0, kSlots * sizeof(uint64_t), s), "clearing counts");
        return MOSS_OK;
    }
    if (count > max_chunk) return fail(MOSS_EOVERFLOW, "count above %llu per call", (unsigned long long)max_chunk);
    MOSS_CUDA(launch_counts(method, dv, first, count, seed, g->partials, classes, verts, counts_dev, s),
              "sample kernels");
    return MOSS_OK;
}

int moss_sample_counts(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed, void *stream,
                       uint64_t *counts_dev) {
    if (!g || !counts_dev) return fail(MOSS_EINVAL, "NULL argument");
    DeviceGuard dg(g->device);
    return sample_into(g, method, first, count, seed, static_cast<cudaStream_t>(stream), counts_dev, nullptr, nullptr);
}

int moss_sample_records(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed, void *stream,
                        uint8_t *classes_dev, uint32_t *verts_dev) {
    if (!g || !classes_dev) return fail(MOSS_EINVAL, "NULL argument");
    DeviceGuard dg(g->device);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = sample_into(g, method, first, count, seed, s, g->counts, classes_dev, verts_dev);
    if (rc || !g->order || !verts_dev) return rc;
    // vertex words of the records back to input ids (MOSS-4 and MOSS-4Min: the first four)
    MOSS_CUDA(launch_map_records(verts_dev, count, method == 1 || method == 2 ? 5 : 4, g->order, g->n, s),
              "record id map");
    return MOSS_OK;
}

static int finalize_from_device(moss_graph *g, int k, const uint64_t K[2], cudaStream_t s, moss_result *out) {
    FinalizeIn in;
    in.k = k;
    in.K[0] = K[0];
    in.K[1] = K[1];
    MOSS_CUDA(launch_finalize(in, g->counts, g->tot, g->res_dev, s), "finalize kernel");
    MOSS_CUDA(cudaMemcpyAsync(&g->res_host, g->res_dev, sizeof(moss_result), cudaMemcpyDeviceToHost, s), "reading result");
    MOSS_CUDA(cudaStreamSynchronize(s), "synchronising stream");
    memcpy(out, &g->res_host, sizeof(moss_result));
    return MOSS_OK;
}

int moss_sample_estimate(moss_graph *g, int k, uint64_t budget, uint64_t seed, void *stream, moss_result *out) {
    if (!g || !out) return fail(MOSS_EINVAL, "NULL argument");
    if (k != 4 && k != 5) return fail(MOSS_EINVAL, "k must be 4 or 5 (got %d)", k);
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t K[2] = {0, 0};
    int rc;
    if (k == 4) {
        if (!method_ready(g, 0)) return fail(MOSS_ESTATE, "tables for k=4 not built");
        K[0] = g->tot_h.gamma[0] ? budget : 0;
        MOSS_CUDA(cudaMemsetAsync(g->counts + kSlots, 0, kSlots * sizeof(uint64_t), s), "clearing counts");
        if ((rc = sample_into(g, 0, 0, K[0], seed, s, g->counts, nullptr, nullptr))) return rc;
    } else {
        if (!method_ready(g, 1) || !method_ready(g, 2)) return fail(MOSS_ESTATE, "tables for k=5 not built");
        K[0] = g->tot_h.gamma[1] ? budget / 2 : 0;
        K[1] = g->tot_h.gamma[2] ? budget - budget / 2 : 0;
        if ((rc = sample_into(g, 1, 0, K[0], seed, s, g->counts, nullptr, nullptr))) return rc;
        if ((rc = sample_into(g, 2, 0, K[1], seed, s, g->counts + kSlots, nullptr, nullptr))) return rc;
    }
    return finalize_from_device(g, k, K, s, out);
}

int moss_finalize(moss_graph *g, int k, const uint64_t *K, const uint64_t *hits, void *stream, moss_result *out) {
    if (!g || !K || !hits || !out) return fail(MOSS_EINVAL, "NULL argument");
    if (k != 4 && k != 5) return fail(MOSS_EINVAL, "k must be 4 or 5 (got %d)", k);
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MOSS_CUDA(cudaMemcpyAsync(g->counts, hits, 2 * kSlots * sizeof(uint64_t), cudaMemcpyDefault, s), "copying counts");
    uint64_t KK[2] = {K[0], k == 4 ? 0 : K[1]};
    return finalize_from_device(g, k, KK, s, out);
}

int moss_covariance(moss_graph *g, int k, const uint64_t *K, const uint64_t *hits, void *stream, double *cov_host,
                    moss_result *out) {
    if (!g || !K || !hits || !cov_host) return fail(MOSS_EINVAL, "NULL argument");
    if (k != 4 && k != 5) return fail(MOSS_EINVAL, "k must be 4 or 5 (got %d)", k);
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MOSS_CUDA(cudaMemcpyAsync(g->counts, hits, 2 * kSlots * sizeof(uint64_t), cudaMemcpyDefault, s), "copying counts");
    FinalizeIn in;
    in.k = k;
    in.K[0] = K[0];
    in.K[1] = k == 4 ? 0 : K[1];
    MOSS_CUDA(launch_covariance(in, g->counts, g->tot, g->res_dev, g->cov_dev, s), "covariance kernel");
    MOSS_CUDA(cudaMemcpyAsync(cov_host, g->cov_dev, kSlots * kSlots * sizeof(double), cudaMemcpyDeviceToHost, s),
              "reading covariance");
    MOSS_CUDA(cudaMemcpyAsync(&g->res_host, g->res_dev, sizeof(moss_result), cudaMemcpyDeviceToHost, s),
              "reading result");
    MOSS_CUDA(cudaStreamSynchronize(s), "synchronising stream");
    if (out) memcpy(out, &g->res_host, sizeof(moss_result));
    return MOSS_OK;
}

int moss_sample_estimate_min(moss_graph *g, uint64_t budget, uint64_t budget_min, uint64_t seed, void *stream,
                             moss_result *out) {
    if (!g || !out) return fail(MOSS_EINVAL, "NULL argument");
    if (!method_ready(g, MOSS_METHOD_MOSS4) || !method_ready(g, MOSS_METHOD_MOSS4MIN))
        return fail(MOSS_ESTATE, "tables for k=4 and MOSS-4Min not built");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FinalizeIn in;
    in.k = 4;
    in.mix = 1;
    in.K[0] = g->tot_h.gamma[0] ? budget : 0;
    in.K[1] = g->tot_h.gamma[3] ? budget_min : 0;
    int rc;
    if ((rc = sample_into(g, MOSS_METHOD_MOSS4, 0, in.K[0], seed, s, g->counts, nullptr, nullptr))) return rc;
    if ((rc = sample_into(g, MOSS_METHOD_MOSS4MIN, 0, in.K[1], seed, s, g->counts + kSlots, nullptr, nullptr)))
        return rc;
    MOSS_CUDA(launch_finalize(in, g->counts, g->tot, g->res_dev, s), "finalize kernel");
    MOSS_CUDA(cudaMemcpyAsync(&g->res_host, g->res_dev, sizeof(moss_result), cudaMemcpyDeviceToHost, s), "reading result");
    MOSS_CUDA(cudaStreamSynchronize(s), "synchronising stream");
    memcpy(out, &g->res_host, sizeof(moss_result));
    return MOSS_OK;
}

int moss_finalize_min(moss_graph *g, const uint64_t *K, const uint64_t *hits, void *stream, double *cov_host,
                      moss_result *out) {
    if (!g || !K || !hits || !out) return fail(MOSS_EINVAL, "NULL argument");
    if (!(g->built >> 5 & 1u)) return fail(MOSS_ESTATE, "MOSS-4Min tables not built (Gamma-check unknown)");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MOSS_CUDA(cudaMemcpyAsync(g->counts, hits, 2 * kSlots * sizeof(uint64_t), cudaMemcpyDefault, s), "copying counts");
    FinalizeIn in;
    in.k = 4;
    in.mix = 1;
    in.K[0] = K[0];
    in.K[1] = K[1];
    if (cov_host) {
        MOSS_CUDA(launch_covariance(in, g->counts, g->tot, g->res_dev, g->cov_dev, s), "covariance kernel");
        MOSS_CUDA(cudaMemcpyAsync(cov_host, g->cov_dev, kSlots * kSlots * sizeof(double), cudaMemcpyDeviceToHost, s),
                  "reading covariance");
    } else {
        MOSS_CUDA(launch_finalize(in, g->counts, g->tot, g->res_dev, s), "finalize kernel");
    }
    MOSS_CUDA(cudaMemcpyAsync(&g->res_host, g->res_dev, sizeof(moss_result), cudaMemcpyDeviceToHost, s),
              "reading result");
    MOSS_CUDA(cudaStreamSynchronize(s), "synchronising stream");
    memcpy(out, &g->res_host, sizeof(moss_result));
    return MOSS_OK;
}

int moss_graph_stats(const moss_graph *g, moss_stats *out) {
    if (!g || !out) return fail(MOSS_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = g->n;
    out->nnz = g->nnz;
    out->d_max = g->tot_h.d_max;
    auto put = [](uint64_t *dst, u128 x) {
        dst[0] = (uint64_t)x;
        dst[1] = (uint64_t)(x >> 64);
    };
    auto dbl = [](u128 x) { return (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x; };
    for (int l = 0; l < kMethods; ++l) {
        put(out->gamma[l], g->tot_h.gamma[l]);
        out->gamma_d[l] = dbl(g->tot_h.gamma[l]);
    }
    put(out->lambda3, g->tot_h.lambda3);
    put(out->lambda4, g->tot_h.lambda4);
    out->lambda3_d = dbl(g->tot_h.lambda3);
    out->lambda4_d = dbl(g->tot_h.lambda4);
    return MOSS_OK;
}

int moss_table_export(const moss_graph *g, int table, void *host_dst, uint64_t bytes) {
    if (!g || !host_dst) return fail(MOSS_EINVAL, "NULL argument");
    DeviceGuard dg(g->device);
    const void *src = nullptr;
    uint64_t need = 0;
    if (table == MOSS_TABLE_VERT) { src = g->vert; need = (uint64_t)g->n * 16; }
    else if (table == MOSS_TABLE_SLOT) { src = g->slot; need = g->nnz * 32; }
    else if (table == MOSS_TABLE_ACC) { src = g->acc; need = g->nnz * 4; }
    else if (table >= MOSS_TABLE_SEED0 && table < MOSS_TABLE_SEED0 + 3) {
        if (!(g->built >> (table - MOSS_TABLE_SEED0) & 1u)) return fail(MOSS_ESTATE, "vertex table not built");
        src = g->seed[table - MOSS_TABLE_SEED0];
        need = (uint64_t)g->n * 32;
    } else if (table >= MOSS_TABLE_GAMMA0 && table < MOSS_TABLE_GAMMA0 + 3) {
        src = g->gam[table - MOSS_TABLE_GAMMA0];
        need = (uint64_t)g->n * 16;
    } else if (table == MOSS_TABLE_FILTER) {
        if (!(g->built >> 6 & 1u)) return fail(MOSS_ESTATE, "edge filter not built");
        src = g->filter;
        need = g->filter_words * 4;
    } else if (table == MOSS_TABLE_HUB_LIST || table == MOSS_TABLE_HUB_BITS) {
        if (!(g->built >> 6 & 1u) || !g->hub_bits) return fail(MOSS_ESTATE, "hub adjacency not built");
        const uint64_t h = hub_capacity(g->n);
        src = table == MOSS_TABLE_HUB_LIST ? static_cast<const void *>(g->hub_list) : g->hub_bits;
        need = table == MOSS_TABLE_HUB_LIST ? h * 4 : (h * h + 31) / 32 * 4;
    } else if (table == MOSS_TABLE_ORDER) {
        need = (uint64_t)g->n * 4;
        if (bytes != need) return fail(MOSS_EINVAL, "table %d has %llu bytes, got %llu", table,
                                       (unsigned long long)need, (unsigned long long)bytes);
        if (!g->order) {   // input order: the identity
            uint32_t *dst = static_cast<uint32_t *>(host_dst);
            for (uint32_t i = 0; i < g->n; ++i) dst[i] = i;
            return MOSS_OK;
        }
        src = g->order;
    } else if ((table >= MOSS_TABLE_MIN_SEED && table <= MOSS_TABLE_MIN_LIST) || table == MOSS_TABLE_MIN_PICK) {
        if (!(g->built >> 5 & 1u)) return fail(MOSS_ESTATE, "MOSS-4Min tables not built");
        switch (table) {
            case MOSS_TABLE_MIN_SEED: src = g->seed[3]; need = (uint64_t)g->n * 32; break;
            case MOSS_TABLE_MIN_GAMMA: src = g->gam[3]; need = (uint64_t)g->n * 16; break;
            case MOSS_TABLE_MIN_VERT: src = g->mvert; need = (uint64_t)g->n * 16; break;
            case MOSS_TABLE_MIN_SLOT: src = g->mslot; need = g->nnz * 32; break;
            case MOSS_TABLE_MIN_PICK: src = g->mpick; need = g->nnz * 32; break;
            default: src = g->rlist; need = g->nnz * 8; break;
        }
    } else {
        return fail(MOSS_EINVAL, "unknown table %d", table);
    }
    if (table == MOSS_TABLE_SLOT && !(g->built >> 3 & 1u)) return fail(MOSS_ESTATE, "sigma tables not built");
    if (bytes != need) return fail(MOSS_EINVAL, "table %d has %llu bytes, got %llu", table, (unsigned long long)need,
                                   (unsigned long long)bytes);
    if (need) MOSS_CUDA(cudaMemcpy(host_dst, src, need, cudaMemcpyDeviceToHost), "copying table");
    return MOSS_OK;
}

void moss_graph_free(moss_graph *g) { release(g); }

}  // extern "C"

// ------------------------------------------- access for other translation units
namespace moss {

int device_sms(int device) {
    if (device < 0 || device >= 64) return 1;
    int v = g_sms[device].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v < 1) v = 1;
        g_sms[device].store(v, std::memory_order_relaxed);
    }
    return v;
}

int current_sms() {
    int dev = 0;
    cudaGetDevice(&dev);
    return device_sms(dev);
}

cudaError_t AuxStreams::fork(cudaStream_t s) const {
    cudaError_t e = cudaEventRecord(forked, s);
    for (int i = 0; i < kAuxOuter && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(a[i], forked, 0);
    return e;
}

cudaError_t AuxStreams::join(cudaStream_t s) const {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kAuxOuter; ++i) {
        cudaError_t ei = cudaEventRecord(done[i], a[i]);
        if (ei == cudaSuccess) ei = cudaStreamWaitEvent(s, done[i], 0);
        if (e == cudaSuccess) e = ei;
    }
    return e;
}

cudaError_t AuxStreams::wait_for(cudaStream_t s, int i) const {
    cudaError_t e = cudaEventRecord(mid, a[i]);
    return e == cudaSuccess ? cudaStreamWaitEvent(s, mid, 0) : e;
}

namespace {
// per host thread and device; released when the thread exits
struct AuxSet {
    AuxStreams dev[64];
    bool tried[64] = {};
    ~AuxSet() {
        for (auto &x : dev) {
            for (int i = 0; i < kAuxStreams; ++i) {
                if (x.a[i]) cudaStreamDestroy(x.a[i]);
                if (x.done[i]) cudaEventDestroy(x.done[i]);
            }
            if (x.forked) cudaEventDestroy(x.forked);
            if (x.mid) cudaEventDestroy(x.mid);
            if (x.sub_fork) cudaEventDestroy(x.sub_fork);
            if (x.sub_mid) cudaEventDestroy(x.sub_mid);
            for (auto ev : x.sub_done)
                if (ev) cudaEventDestroy(ev);
        }
    }
};
thread_local AuxSet t_aux;
}  // namespace

const AuxStreams *aux_streams() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
    AuxStreams &x = t_aux.dev[d];
    if (!t_aux.tried[d]) {
        t_aux.tried[d] = true;
        bool ok = cudaEventCreateWithFlags(&x.forked, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&x.mid, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&x.sub_fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&x.sub_mid, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&x.sub_done[0], cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&x.sub_done[1], cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kAuxStreams && ok; ++i)
            ok = cudaStreamCreateWithFlags(&x.a[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&x.done[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            x = AuxStreams{};   // stay on the caller's stream (handles created so far are dropped)
        }
    }
    return x.a[0] ? &x : nullptr;
}

int graph_view_for(const moss_graph *g, int strategy, DevGraph *out) {
    const bool hash = (g->built >> 4 & 1u) != 0, filter = (g->built >> 6 & 1u) != 0;
    if (strategy == MOSS_PROBE_AUTO) strategy = effective_probe(g);
    if (strategy == MOSS_PROBE_HASH && !hash) return set_error(MOSS_ESTATE, "hashed edge set not built");
    if (strategy == MOSS_PROBE_FILTER && !(hash && filter)) return set_error(MOSS_ESTATE, "edge filter not built");
    if (strategy < MOSS_PROBE_SEARCH || strategy > MOSS_PROBE_FILTER) return set_error(MOSS_EINVAL, "unknown probe strategy");
    *out = view_with(g, strategy);
    return MOSS_OK;
}

int graph_info(const moss_graph *g, GraphInfo *out) {
    out->view = view(g);
    out->tot = g->tot;
    out->device = g->device;
    out->built = g->built;
    for (int l = 0; l < kMethods; ++l) {
        out->total_nonzero[l] = g->tot_h.gamma[l] != 0;
        out->ready[l] = method_ready(g, l);
    }
    return MOSS_OK;
}

int set_error(int code, const char *detail) { return fail(code, "%s", detail); }

}  // namespace moss
