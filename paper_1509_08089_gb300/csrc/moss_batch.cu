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
// and replayed by later runs until the request list or the tile size
// changes.  moss_batch_tune times a few tile sizes and keeps the fastest.
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
    bool dirty = true;                 // request list or tile changed since the last capture
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
            graphs.push_back(gi.view);
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
    cudaError_t e = cudaSuccess;
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
    b->blocks = batch_blocks(b->device);
    return MOSS_OK;
}

// the launch sequence of one run, enqueued on the batch stream
cudaError_t enqueue(moss_batch *b) {
    cudaStream_t s = b->stream;
    const int nreq = (int)b->reqs.size();
    cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_sample_batch(b->d_graphs, b->d_tasks, b->ntasks, b->ntiles, b->tile, b->d_next, b->d_tiles,
                                b->blocks, s);
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

int moss_batch_tune(moss_batch *b, void *stream, uint32_t *chosen) {
    if (!b) return set_error(MOSS_EINVAL, "NULL batch");
    if (b->reqs.empty()) return set_error(MOSS_EINVAL, "empty batch");
    std::vector<moss_result> tmp(b->reqs.size());
    const uint32_t cands[] = {1024, 4096, 16384, 65536};
    uint32_t best = b->tile;
    double best_t = 1e300;
    for (uint32_t c : cands) {
        int rc = moss_batch_set_tile(b, c);
        if (rc) return rc;
        if ((rc = moss_batch_run(b, stream, tmp.data()))) return rc;  // plan + capture + warm
        double t = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            auto t0 = std::chrono::steady_clock::now();
            if ((rc = moss_batch_run(b, stream, tmp.data()))) return rc;
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            t = dt < t ? dt : t;
        }
        if (t < best_t) {
            best_t = t;
            best = c;
        }
    }
    int rc = moss_batch_set_tile(b, best);
    if (rc) return rc;
    if (chosen) *chosen = best;
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
    if (b->d_next) cudaFree(b->d_next);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->h_results) cudaFreeHost(b->h_results);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
