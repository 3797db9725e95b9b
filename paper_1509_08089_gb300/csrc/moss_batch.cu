// moss_batch.cu -- many sample-and-estimate requests, on many graphs, in one
// persistent launch.
//
// A batch is a list of requests (graph, k, budget, seed).  Each request
// becomes one task per sub-method (MOSS-4; T-5 and Path-5 with K1 =
// floor(B/2), K2 = B - K1 as in moss_sample_estimate; or MOSS-4 and
// MOSS-4Min with K and K-check as in moss_sample_estimate_min), each task a run
// of tiles of `tile` sample ids.  One persistent kernel drains the tile list
// through a device counter; per-tile counts are summed per task in tile order
// and finalized per request on the device.  Since every sample is keyed by
// its id, each request's counts equal those of its solo moss_sample_estimate.
//
// The launch sequence (counter reset, sampler, per-task sums, finalize,
// result copy) is captured once into a CUDA graph on the batch's own stream
// and replayed by later runs until the request list or a launch choice
// changes.  moss_batch_tune picks those choices by measurement: the probe
// strategy of each graph (list search, hashed set or filtered set, from the
// SM cycles its tiles take under each), the tile size (samples per warp task)
// and the block shape (threads per block, resident blocks per SM).  None of
// them changes a count: samples are keyed by id and every probe strategy
// answers the same membership questions.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/moss.h"
#include "moss_internal.cuh"

using namespace moss;

namespace {

struct Req {
    moss_graph *g;
    int k;
    uint64_t budget, seed;
    bool mix;              // MOSS-4 with MOSS-4Min (k = 4)
    uint64_t budget_min;   // K-check of the mix
};

template <typename T>
cudaError_t grow(T **p, size_t *cap, size_t need, cudaStream_t s) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFreeAsync(*p, s);
    *p = nullptr;
    size_t c = need < 64 ? 64 : need + need / 2;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), c * sizeof(T), s);
    if (e == cudaSuccess) *cap = c;
    return e;
}

}  // namespace

struct moss_batch {
    int device = 0;
    cudaStream_t stream = nullptr;     // the batch's own stream (capturable)
    cudaEvent_t ready = nullptr;
    std::vector<Req> reqs;
    uint32_t tile = 8192;
    int threads = 256;                 // threads per block of the persistent launch
    int per_sm = 0;                    // resident blocks per SM (0: as many as fit)
    int rngs = kBatchSplitMix;         // generators of the planned graphs (kBatch*)
    std::vector<std::pair<const moss_graph *, int>> probes;   // per-graph probe strategy overrides
    bool record = false;               // record per-tile SM cycles (tuning runs)
    bool dirty = true;                 // request list or a launch choice changed since the last capture
    moss_batch_tuning tuning{};
    // host copy of the current plan: tasks and the graph of each
    std::vector<BatchTask> plan_tasks;
    std::vector<const moss_graph *> plan_graphs;
    // device buffers
    DevGraph *d_graphs = nullptr;
    size_t cap_graphs = 0;
    BatchTask *d_tasks = nullptr;
    size_t cap_tasks = 0;
    BatchRequest *d_reqs = nullptr;
    size_t cap_reqs = 0;
    uint32_t *d_tiles = nullptr;
    size_t cap_tiles = 0;
    uint64_t *d_task_counts = nullptr;
    size_t cap_tc = 0;
    moss_result *d_results = nullptr;
    size_t cap_res = 0;
    unsigned long long *d_next = nullptr;
    unsigned long long *d_cycles = nullptr;
    size_t cap_cycles = 0;
    moss_result *h_results = nullptr;  // pinned
    size_t cap_hres = 0;
    // shape of the current plan
    int ntasks = 0;
    uint64_t ntiles = 0;
    int blocks = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t runs = 0;
};

namespace {

int plan(moss_batch *b) {
    cudaStream_t s = b->stream;
    const int nreq = (int)b->reqs.size();
    std::vector<DevGraph> graphs;
    std::vector<const moss_graph *> gkeys;
    std::vector<BatchTask> tasks;
    std::vector<BatchRequest> reqs(nreq);
    uint64_t tile0 = 0;
    for (int r = 0; r < nreq; ++r) {
        const Req &q = b->reqs[r];
        GraphInfo gi;
        graph_info(q.g, &gi);
        if (gi.device != b->device) return set_error(MOSS_EINVAL, "a graph of the batch lives on another device");
        int gidx = -1;
        for (size_t i = 0; i < gkeys.size(); ++i)
            if (gkeys[i] == q.g) gidx = (int)i;
        if (gidx < 0) {
            gidx = (int)graphs.size();
            DevGraph v = gi.view;
            for (auto &pr : b->probes)
                if (pr.first == q.g) {
                    int rc = graph_view_for(q.g, pr.second, &v);
                    if (rc) return rc;
                }
            graphs.push_back(v);
            gkeys.push_back(q.g);
        }
        BatchRequest &br = reqs[r];
        br.in.k = q.k;
        br.in.mix = q.mix ? 1 : 0;
        br.in.K[0] = br.in.K[1] = 0;
        br.tot = gi.tot;
        br.task[0] = br.task[1] = -1;
        int methods[2], nm = 0;
        uint64_t Ks[2];
        if (q.k == 4) {
            methods[nm] = 0;
            Ks[nm++] = gi.total_nonzero[0] ? q.budget : 0;
            if (q.mix) {
                methods[nm] = 3;
                Ks[nm++] = gi.total_nonzero[3] ? q.budget_min : 0;
            }
        } else {
            methods[nm] = 1;
            Ks[nm++] = gi.total_nonzero[1] ? q.budget / 2 : 0;
            methods[nm] = 2;
            Ks[nm++] = gi.total_nonzero[2] ? q.budget - q.budget / 2 : 0;
        }
        for (int j = 0; j < nm; ++j) {
            const int m = methods[j];
            if (!gi.ready[m]) return set_error(MOSS_ESTATE, "tables of a batched graph not built");
            br.in.K[j] = Ks[j];
            if (Ks[j] == 0) continue;
            BatchTask t;
            t.seed = q.seed;
            t.first = 0;
            t.count = Ks[j];
            t.tile0 = tile0;
            t.graph = (uint32_t)gidx;
            t.method = (uint32_t)m;
            br.task[j] = (int)tasks.size();
            tasks.push_back(t);
            tile0 += (Ks[j] + b->tile - 1) / b->tile;
        }
    }
    b->ntasks = (int)tasks.size();
    b->ntiles = tile0;
    b->plan_tasks = tasks;
    b->plan_graphs = gkeys;
    cudaError_t e = cudaSuccess;
    if (b->record) e = grow(&b->d_cycles, &b->cap_cycles, (size_t)b->ntiles + 1, s);
    if (e == cudaSuccess) e = grow(&b->d_graphs, &b->cap_graphs, graphs.size() + 1, s);
    if (e == cudaSuccess) e = grow(&b->d_tasks, &b->cap_tasks, tasks.size() + 1, s);
    if (e == cudaSuccess) e = grow(&b->d_reqs, &b->cap_reqs, reqs.size() + 1, s);
    if (e == cudaSuccess) e = grow(&b->d_tiles, &b->cap_tiles, (size_t)(b->ntiles + 1) * kSlots, s);
    if (e == cudaSuccess) e = grow(&b->d_task_counts, &b->cap_tc, (tasks.size() + 1) * kSlots, s);
    if (e == cudaSuccess) e = grow(&b->d_results, &b->cap_res, reqs.size() + 1, s);
    if (e != cudaSuccess) return set_error(MOSS_ENOMEM, "batch device buffers");
    if (b->cap_hres < reqs.size() + 1) {
        if (b->h_results) cudaFreeHost(b->h_results);
        b->h_results = nullptr;
        b->cap_hres = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&b->h_results), (reqs.size() + 1) * sizeof(moss_result)) !=
            cudaSuccess)
            return set_error(MOSS_ENOMEM, "batch pinned results");
        b->cap_hres = reqs.size() + 1;
    }
    if (!graphs.empty())
        e = cudaMemcpyAsync(b->d_graphs, graphs.data(), graphs.size() * sizeof(DevGraph), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !tasks.empty())
        e = cudaMemcpyAsync(b->d_tasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nreq)
        e = cudaMemcpyAsync(b->d_reqs, reqs.data(), reqs.size() * sizeof(BatchRequest), cudaMemcpyHostToDevice, s);
    // the host vectors die at return: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(MOSS_ECUDA, "uploading the batch plan");
    b->rngs = batch_rngs(graphs.data(), graphs.size());
    b->blocks = batch_blocks(b->device, b->threads, b->per_sm, b->rngs);
    return MOSS_OK;
}

// the launch sequence of one run, enqueued on the batch stream
cudaError_t enqueue(moss_batch *b) {
    cudaStream_t s = b->stream;
    const int nreq = (int)b->reqs.size();
    cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_sample_batch(b->d_graphs, b->d_tasks, b->ntasks, b->ntiles, b->tile, b->d_next, b->d_tiles,
                                b->threads, b->blocks, b->record ? b->d_cycles : nullptr, b->rngs, s);
    if (e == cudaSuccess) e = launch_batch_reduce(b->d_tasks, b->ntasks, b->tile, b->d_tiles, b->d_task_counts, s);
    if (e == cudaSuccess) e = launch_finalize_batch(b->d_reqs, nreq, b->d_task_counts, b->d_results, s);
    if (e == cudaSuccess && nreq)
        e = cudaMemcpyAsync(b->h_results, b->d_results, nreq * sizeof(moss_result), cudaMemcpyDeviceToHost, s);
    return e;
}

int capture(moss_batch *b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_error(MOSS_ECUDA, "beginning batch capture");
    cudaError_t e2 = enqueue(b);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (e2 != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return set_error(MOSS_ECUDA, "capturing the batch launch");
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return set_error(MOSS_ECUDA, "instantiating the batch graph");
    }
    b->dirty = false;
    return MOSS_OK;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int moss_batch_create(int device, moss_batch **out) {
    if (!out) return set_error(MOSS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return set_error(MOSS_ECUDA, "cudaGetDeviceCount failed");
    if (device < 0 || device >= ndev) return set_error(MOSS_EINVAL, "device not present");
    Guard dg(device);
    moss_batch *b = new (std::nothrow) moss_batch;
    if (!b) return set_error(MOSS_ENOMEM, "host allocation");
    b->device = device;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&b->d_next), sizeof(unsigned long long)) != cudaSuccess) {
        moss_batch_free(b);
        return set_error(MOSS_ECUDA, "creating the batch stream and counter");
    }
    *out = b;
    return MOSS_OK;
}

int moss_batch_add(moss_batch *b, moss_graph *g, int k, uint64_t budget, uint64_t seed, int *index) {
    if (!b || !g) return set_error(MOSS_EINVAL, "NULL argument");
    if (k != 4 && k != 5) return set_error(MOSS_EINVAL, "k must be 4 or 5");
    GraphInfo gi;
    graph_info(g, &gi);
    if (gi.device != b->device) return set_error(MOSS_EINVAL, "graph lives on another device than the batch");
    if (k == 4 ? !gi.ready[0] : !(gi.ready[1] && gi.ready[2]))
        return set_error(MOSS_ESTATE, "tables for this k are not built");
    b->reqs.push_back(Req{g, k, budget, seed, false, 0});
    if (index) *index = (int)b->reqs.size() - 1;
    b->dirty = true;
    return MOSS_OK;
}

int moss_batch_add_min(moss_batch *b, moss_graph *g, uint64_t budget, uint64_t budget_min, uint64_t seed, int *index) {
    if (!b || !g) return set_error(MOSS_EINVAL, "NULL argument");
    GraphInfo gi;
    graph_info(g, &gi);
    if (gi.device != b->device) return set_error(MOSS_EINVAL, "graph lives on another device than the batch");
    if (!gi.ready[0] || !gi.ready[3]) return set_error(MOSS_ESTATE, "MOSS-4 and MOSS-4Min tables are not built");
    b->reqs.push_back(Req{g, 4, budget, seed, true, budget_min});
    if (index) *index = (int)b->reqs.size() - 1;
    b->dirty = true;
    return MOSS_OK;
}

int moss_batch_size(const moss_batch *b) { return b ? (int)b->reqs.size() : 0; }

int moss_batch_clear(moss_batch *b) {
    if (!b) return set_error(MOSS_EINVAL, "NULL batch");
    b->reqs.clear();
    b->dirty = true;
    return MOSS_OK;
}

int moss_batch_set_tile(moss_batch *b, uint32_t tile_samples) {
    if (!b) return set_error(MOSS_EINVAL, "NULL batch");
    if (tile_samples < 32 || tile_samples > (1u << 30)) return set_error(MOSS_EINVAL, "tile size out of [32, 2^30]");
    if (tile_samples != b->tile) b->dirty = true;
    b->tile = tile_samples;
    return MOSS_OK;
}

uint32_t moss_batch_tile(const moss_batch *b) { return b ? b->tile : 0; }

int moss_batch_run(moss_batch *b, void *stream, moss_result *results) {
    if (!b || (!results && !b->reqs.empty())) return set_error(MOSS_EINVAL, "NULL argument");
    Guard dg(b->device);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    // order after the caller's prior work on its stream
    if (cudaEventRecord(b->ready, user) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ready, 0) != cudaSuccess)
        return set_error(MOSS_ECUDA, "ordering the batch after the caller's stream");
    if (b->reqs.empty()) return MOSS_OK;
    int rc;
    if (b->dirty) {
        if ((rc = plan(b))) return rc;
        if ((rc = capture(b))) return rc;
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return set_error(MOSS_ECUDA, "launching the batch graph");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(MOSS_ECUDA, "running the batch");
    memcpy(results, b->h_results, b->reqs.size() * sizeof(moss_result));
    ++b->runs;
    return MOSS_OK;
}

int moss_batch_set_launch(moss_batch *b, int threads_per_block, int blocks_per_sm) {
    if (!b) return set_error(MOSS_EINVAL, "NULL batch");
    if (threads_per_block != 128 && threads_per_block != 256 && threads_per_block != 512)
        return set_error(MOSS_EINVAL, "threads per block must be 128, 256 or 512");
    if (blocks_per_sm < 0) return set_error(MOSS_EINVAL, "blocks per SM must be >= 0 (0: as many as fit)");
    if (threads_per_block != b->threads || blocks_per_sm != b->per_sm) b->dirty = true;
    b->threads = threads_per_block;
    b->per_sm = blocks_per_sm;
    return MOSS_OK;
}

int moss_batch_set_graph_probe(moss_batch *b, const moss_graph *g, int strategy) {
    if (!b || !g) return set_error(MOSS_EINVAL, "NULL argument");
    DevGraph v;
    int rc = graph_view_for(g, strategy, &v);   // the tables the strategy needs must exist
    if (rc) return rc;
    for (size_t i = 0; i < b->probes.size(); ++i)
        if (b->probes[i].first == g) {
            b->probes.erase(b->probes.begin() + (long)i);
            break;
        }
    if (strategy != MOSS_PROBE_AUTO) b->probes.push_back({g, strategy});
    b->dirty = true;
    return MOSS_OK;
}

int moss_batch_get_tuning(const moss_batch *b, moss_batch_tuning *out) {
    if (!b || !out) return set_error(MOSS_EINVAL, "NULL argument");
    *out = b->tuning;
    out->tile_samples = b->tile;
    out->threads_per_block = b->threads;
    out->blocks_per_sm = b->per_sm > 0 ? b->per_sm : batch_max_per_sm(b->threads, b->rngs);
    return MOSS_OK;
}

namespace {

// host time of one run (the best of `reps` after a run that plans, captures
// and warms up)
int timed_runs(moss_batch *b, void *stream, std::vector<moss_result> &tmp, int reps, double *best) {
    int rc = moss_batch_run(b, stream, tmp.data());
    if (rc) return rc;
    *best = 1e300;
    for (int r = 0; r < reps; ++r) {
        auto t0 = std::chrono::steady_clock::now();
        if ((rc = moss_batch_run(b, stream, tmp.data()))) return rc;
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        *best = dt < *best ? dt : *best;
    }
    return MOSS_OK;
}

}  // namespace

int moss_batch_tune(moss_batch *b, void *stream, uint32_t *chosen) {
    if (!b) return set_error(MOSS_EINVAL, "NULL batch");
    if (b->reqs.empty()) return set_error(MOSS_EINVAL, "empty batch");
    Guard dg(b->device);
    std::vector<moss_result> tmp(b->reqs.size());
    int rc;
    // 1. probe strategy per graph: one run with every graph on each strategy
    //    it has tables for; a graph's cost under a strategy is the SM cycles
    //    of its tiles per sample
    std::vector<const moss_graph *> gs;
    for (const Req &q : b->reqs)
        if (std::find(gs.begin(), gs.end(), q.g) == gs.end()) gs.push_back(q.g);
    const int strategies[3] = {MOSS_PROBE_SEARCH, MOSS_PROBE_HASH, MOSS_PROBE_FILTER};
    std::vector<double> cost(gs.size() * 3, -1.0);
    const auto saved = b->probes;
    for (int si = 0; si < 3; ++si) {
        b->probes.clear();
        std::vector<bool> avail(gs.size(), false);
        for (size_t gi = 0; gi < gs.size(); ++gi) {
            DevGraph v;
            if (graph_view_for(gs[gi], strategies[si], &v) == MOSS_OK) {
                b->probes.push_back({gs[gi], strategies[si]});
                avail[gi] = true;
            }
        }
        b->record = true;
        b->dirty = true;
        double t;
        if ((rc = timed_runs(b, stream, tmp, 1, &t))) break;
        std::vector<unsigned long long> cyc(b->ntiles);
        if (b->ntiles && cudaMemcpy(cyc.data(), b->d_cycles, b->ntiles * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = set_error(MOSS_ECUDA, "reading tile cycles");
            break;
        }
        std::vector<double> c(gs.size(), 0.0), n(gs.size(), 0.0);
        for (const BatchTask &t : b->plan_tasks) {
            const moss_graph *g = b->plan_graphs[t.graph];
            const size_t gi = (size_t)(std::find(gs.begin(), gs.end(), g) - gs.begin());
            const uint64_t nt = (t.count + b->tile - 1) / b->tile;
            for (uint64_t j = 0; j < nt; ++j) c[gi] += (double)cyc[t.tile0 + j];
            n[gi] += (double)t.count;
        }
        for (size_t gi = 0; gi < gs.size(); ++gi)
            if (avail[gi] && n[gi] > 0) cost[gi * 3 + si] = c[gi] / n[gi];
    }
    b->record = false;
    b->dirty = true;
    if (rc) {
        b->probes = saved;
        return rc;
    }
    b->probes.clear();
    int per_strategy[3] = {0, 0, 0};
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        int best = -1;
        for (int si = 0; si < 3; ++si)
            if (cost[gi * 3 + si] >= 0 && (best < 0 || cost[gi * 3 + si] < cost[gi * 3 + best])) best = si;
        if (best < 0) {   // no tile of this graph ran (zero budgets): keep its own strategy
            continue;
        }
        b->probes.push_back({gs[gi], strategies[best]});
        ++per_strategy[best];
    }
    // 2. tile size, 3. block shape, 4. tile size again under that shape
    const uint32_t tiles[] = {1024, 4096, 16384, 65536};
    double best_t = 1e300;
    auto try_tiles = [&]() -> int {
        uint32_t best = b->tile;
        for (uint32_t c : tiles) {
            int r = moss_batch_set_tile(b, c);
            double t;
            if (r || (r = timed_runs(b, stream, tmp, 2, &t))) return r;
            if (t < best_t) {
                best_t = t;
                best = c;
            }
        }
        return moss_batch_set_tile(b, best);
    };
    if ((rc = try_tiles())) return rc;
    int best_threads = b->threads, best_per = b->per_sm;
    for (int th : {128, 256, 512}) {
        const int mx = batch_max_per_sm(th, b->rngs);
        int pers[3] = {mx, (3 * mx + 3) / 4, (mx + 1) / 2};
        for (int pi = 0; pi < 3; ++pi) {
            if (pi > 0 && pers[pi] == pers[pi - 1]) continue;
            if ((rc = moss_batch_set_launch(b, th, pers[pi]))) return rc;
            double t;
            if ((rc = timed_runs(b, stream, tmp, 2, &t))) return rc;
            if (t < best_t) {
                best_t = t;
                best_threads = th;
                best_per = pers[pi];
            }
        }
    }
    if ((rc = moss_batch_set_launch(b, best_threads, best_per))) return rc;
    if ((rc = try_tiles())) return rc;
    b->tuning.graphs = (int)gs.size();
    b->tuning.graphs_search = per_strategy[0];
    b->tuning.graphs_hash = per_strategy[1];
    b->tuning.graphs_filter = per_strategy[2];
    b->tuning.run_s = best_t;
    b->tuning.tuned = 1;
    if (chosen) *chosen = b->tile;
    return MOSS_OK;
}

void moss_batch_free(moss_batch *b) {
    if (!b) return;
    Guard dg(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    void *dev[] = {b->d_graphs, b->d_tasks, b->d_reqs, b->d_tiles, b->d_task_counts, b->d_results};
    for (void *p : dev)
        if (p) cudaFreeAsync(p, b->stream);
    if (b->d_cycles) cudaFreeAsync(b->d_cycles, b->stream);
    if (b->d_next) cudaFree(b->d_next);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->h_results) cudaFreeHost(b->h_results);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
