// moss_server.cu -- a continuous-batching request server over resident graphs.
//
// Requests (graph, k, budget or target relative error, seed) are submitted
// from any host thread.  A scheduler thread admits them into a bounded set of
// active slots (while enough device memory stays free) and runs ticks: each
// tick is one persistent launch of the batch sampler over the next chunk of
// sample ids of every active request, sized so the tick holds about
// `tick_samples` samples shared fairly between the requests.  Requests that
// arrive while a tick runs join the next one, so small requests finish in a
// tick or two while large ones keep streaming.  Under overload (samples
// for at least two more full ticks can be scheduled already) ticks are
// double-buffered: while tick N runs, the scheduler plans tick N+1 from what is
// already known (every request's next sample ids; a request still waiting
// for its pilot's counts sits one tick out) and queues it behind tick N, so
// the GPU does not idle while the host takes tick N's counts back.  Below
// that a queued tick would mostly hold back requests that arrive or finish
// their pilot meanwhile (adding a tick to their latency), so the next tick
// is planned after tick N returns.
// Requests that finish are finalized on a second stream, so their results
// do not wait behind a queued tick.  Counts are accumulated per
// request in exact integers; a finished request is finalized on the device
// (the same arithmetic as moss_sample_estimate).  Since every sample is keyed
// by its id, a served result equals moss_sample_estimate with the same final
// budget, alone or in any mix.
//
// Budget from a target: the first chunk (pilot_samples) is drawn as usual;
// its hit fraction f_i = m_i / K of each class with at least 10 hits gives
// the samples K = (1/f_i - 1) / eps^2 at which the relative standard error
// sqrt(Var)/n_i of Theorems 3, 7 and 9 (Var = n_i (1/p_i - n_i) / K, with
// p_i n_i = f_i) reaches eps; the request's budget is the largest such K over
// its classes (per sub-method, doubled for K1 = K2 at k = 5), clamped to
// [min_budget, max_budget] and to at least the pilot.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/moss.h"
#include "moss_internal.cuh"

using namespace moss;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SReq {
    uint64_t id = 0;
    int graph = 0, k = 4;
    bool mix = false;            // MOSS-4 with MOSS-4Min (k = 4, explicit budgets)
    double target = 0;
    uint64_t seed = 0;
    bool pilot = false;          // budget still to be derived from the first chunk
    uint64_t budget = 0;         // final budget once known
    uint64_t K[2] = {0, 0};      // samples of each sub-method (current goal)
    uint64_t next[2] = {0, 0};   // next sample id to schedule
    uint64_t done[2] = {0, 0};   // samples counted
    uint64_t hits[2][kSlots] = {};
    int state = 0;               // 0 pending, 1 active, 2 finished
    double t_arrive = 0, t_admit = 0, t_done = 0;
    uint64_t ticks = 0;
    moss_result result{};
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

// the buffers of one tick in flight
struct TickBuffers {
    BatchTask *d_tasks = nullptr;
    size_t cap_tasks = 0;
    uint32_t *d_tiles = nullptr;
    size_t cap_tiles = 0;
    uint64_t *d_task_counts = nullptr;
    size_t cap_tc = 0;
    uint64_t *h_task_counts = nullptr;   // pinned
    size_t cap_htc = 0;
    unsigned long long *d_next = nullptr;
    cudaEvent_t start = nullptr, end = nullptr;   // timed: the tick's span on the stream
    std::vector<BatchTask> tasks;
    std::vector<std::pair<uint64_t, int>> owner;   // (request id, sub-method slot) of each task
};

template <typename T>
cudaError_t grow_host(T **p, size_t *cap, size_t need) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    size_t c = need < 64 ? 64 : need + need / 2;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(p), c * sizeof(T));
    if (e == cudaSuccess) *cap = c;
    return e;
}

// sub-methods of a request: (method, budget share); the mix draws budget
// MOSS-4 and budget_min MOSS-4Min samples
int sub_methods(int k, bool mix, uint64_t budget, uint64_t budget_min, const bool nonzero[kMethods], int m[2],
                uint64_t K[2]) {
    if (mix) {
        m[0] = 0;
        m[1] = 3;
        K[0] = nonzero[0] ? budget : 0;
        K[1] = nonzero[3] ? budget_min : 0;
        return 2;
    }
    if (k == 4) {
        m[0] = 0;
        K[0] = nonzero[0] ? budget : 0;
        K[1] = 0;
        return 1;
    }
    m[0] = 1;
    m[1] = 2;
    K[0] = nonzero[1] ? budget / 2 : 0;
    K[1] = nonzero[2] ? budget - budget / 2 : 0;
    return 2;
}

}  // namespace

extern "C" uint64_t moss_budget_for_target(int k, const uint64_t *K, const uint64_t *hits, double target,
                                           uint64_t min_budget, uint64_t max_budget) {
    // largest K_i = (1/f_i - 1) / eps^2 over classes with >= 10 pilot hits
    double need = 0.0;
    const int nsub = k == 4 ? 1 : 2;
    for (int l = 0; l < nsub; ++l) {
        if (K[l] == 0) continue;
        for (int i = 1; i < kSlots; ++i) {
            const uint64_t m = hits[l * kSlots + i];
            if (m < 10) continue;
            const double f = (double)m / (double)K[l];
            double Ki = (1.0 / f - 1.0) / (target * target);
            if (k == 5) Ki *= 2.0;   // the budget is split K1 = K2
            need = Ki > need ? Ki : need;
        }
    }
    double b = std::ceil(need);
    if (b < (double)min_budget) b = (double)min_budget;
    if (b > (double)max_budget) b = (double)max_budget;
    return (uint64_t)b;
}

extern "C" uint64_t moss_budget_for_target_min(const uint64_t *K, const uint64_t *hits, double target,
                                               uint64_t min_budget, uint64_t max_budget) {
    // per-sample relative variance of each source's estimate of class i from
    // the pilot, then the Theorem 1 mix of the two; the mix draws K = K-check
    // = B / 2, so the relative variance r / (B / 2) reaches eps^2 at B = 2 r / eps^2
    static const int first_slot[7] = {-1, -1, -1, 0, -1, 4, 10};   // MOSS-4Min (class, c) slots
    static const int nslots[7] = {0, 0, 0, 4, 0, 6, 12};
    double need = 0.0;
    for (int i = 1; i <= 6; ++i) {
        if (i == 2) continue;   // the 3-star is never sampled: eq. (2) closes it
        double r1 = -1.0, r2 = -1.0;
        if (K[0] > 0 && hits[i] >= 10) r1 = (double)K[0] / (double)hits[i] - 1.0;   // Theorem 3: 1/f - 1
        if (K[1] > 0 && nslots[i] > 0) {
            double a = 0.0, b = 0.0, m = 0.0;
            for (int c = 1; c <= nslots[i]; ++c) {
                const double x = (double)hits[kSlots + first_slot[i] + c - 1];
                a += x / c;
                b += x / ((double)c * c);
                m += x;
            }
            // Theorem 5 with per-CIS probabilities: Gamma-check h / (2 n) - 1 = K-check b / a^2 - 1
            if (m >= 10) r2 = (double)K[1] * b / (a * a) - 1.0;
        }
        double r;
        if (r1 > 0 && r2 > 0) r = r1 * r2 / (r1 + r2);   // Theorem 1
        else if (r1 > 0) r = r1;
        else if (r2 > 0) r = r2;
        else continue;
        const double B = 2.0 * r / (target * target);
        need = B > need ? B : need;
    }
    double b = std::ceil(need);
    if (b < (double)min_budget) b = (double)min_budget;
    if (b > (double)max_budget) b = (double)max_budget;
    return (uint64_t)b;
}

struct moss_server {
    int device = 0;
    moss_server_config cfg{};
    std::vector<moss_graph *> graphs;
    std::vector<GraphInfo> ginfo;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> active;
    std::unordered_map<uint64_t, SReq> reqs;
    uint64_t next_id = 1;
    bool stop = false, started = false;
    std::thread worker;
    cudaStream_t stream = nullptr;      // ticks
    cudaStream_t fin_stream = nullptr;  // finalize of finished requests
    int status = MOSS_OK;          // sticky error of the scheduler
    // device / pinned buffers
    DevGraph *d_graphs = nullptr;
    size_t cap_graphs = 0;
    TickBuffers tick[2];           // two ticks in flight at most
    BatchRequest *d_breq = nullptr;
    size_t cap_breq = 0;
    uint64_t *d_totals = nullptr;
    size_t cap_tot = 0;
    moss_result *d_results = nullptr;
    size_t cap_res = 0;
    moss_result *h_results = nullptr;
    size_t cap_hres = 0;
    int blocks = 0;
    int rngs = kBatchSplitMix;     // generators of the server's graphs (kBatch*)
    bool graphs_uploaded = false;
    // statistics
    uint64_t ticks = 0, samples = 0, completed = 0;
    double busy_s = 0, first_submit = 0, last_done = 0;
    size_t free_bytes = 0;
};

namespace {

int fail_server(moss_server *s, int code, const char *what) {
    s->status = code;
    return set_error(code, what);
}

// queue one tick on the stream: sample the tasks of buffer set tb, sum them
// per task and copy the counts to tb's pinned host array; `end` records
// when they have arrived
int enqueue_tick(moss_server *s, TickBuffers &tb, uint64_t ntiles) {
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    if (!s->graphs_uploaded) {
        std::vector<DevGraph> gv;
        for (auto &gi : s->ginfo) gv.push_back(gi.view);
        e = grow(&s->d_graphs, &s->cap_graphs, gv.size() + 1, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_graphs, gv.data(), gv.size() * sizeof(DevGraph), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail_server(s, MOSS_ECUDA, "uploading server graphs");
        s->graphs_uploaded = true;
        s->rngs = batch_rngs(gv.data(), gv.size());
        s->blocks = batch_blocks(s->device, 256, 0, s->rngs);
    }
    const size_t nt = tb.tasks.size();
    if (e == cudaSuccess) e = grow(&tb.d_tasks, &tb.cap_tasks, nt + 1, st);
    if (e == cudaSuccess) e = grow(&tb.d_tiles, &tb.cap_tiles, (size_t)(ntiles + 1) * kSlots, st);
    if (e == cudaSuccess) e = grow(&tb.d_task_counts, &tb.cap_tc, (nt + 1) * kSlots, st);
    if (e == cudaSuccess) e = grow_host(&tb.h_task_counts, &tb.cap_htc, (nt + 1) * kSlots);
    if (e != cudaSuccess) return fail_server(s, MOSS_ENOMEM, "server tick buffers");
    // tb.tasks and tb.owner stay as they are until the tick is taken back
    e = cudaEventRecord(tb.start, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb.d_tasks, tb.tasks.data(), nt * sizeof(BatchTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.d_next, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = launch_sample_batch(s->d_graphs, tb.d_tasks, (int)nt, ntiles, s->cfg.tile_samples, tb.d_next, tb.d_tiles,
                                256, s->blocks, nullptr, s->rngs, st);
    if (e == cudaSuccess)
        e = launch_batch_reduce(tb.d_tasks, (int)nt, s->cfg.tile_samples, tb.d_tiles, tb.d_task_counts, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb.h_task_counts, tb.d_task_counts, nt * kSlots * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(tb.end, st);
    if (e != cudaSuccess) return fail_server(s, MOSS_ECUDA, "server tick");
    return MOSS_OK;
}

// finalize finished requests on the device (one thread each)
int finalize(moss_server *s, const std::vector<SReq *> &fin) {
    if (fin.empty()) return MOSS_OK;
    cudaStream_t st = s->fin_stream;
    const size_t n = fin.size();
    std::vector<BatchRequest> br(n);
    std::vector<uint64_t> tot(2 * n * kSlots);
    for (size_t i = 0; i < n; ++i) {
        const SReq &q = *fin[i];
        br[i].in.k = q.k;
        br[i].in.mix = q.mix ? 1 : 0;
        br[i].in.K[0] = q.K[0];
        br[i].in.K[1] = q.K[1];
        br[i].tot = s->ginfo[q.graph].tot;
        br[i].task[0] = (int)(2 * i);
        br[i].task[1] = (int)(2 * i + 1);
        memcpy(&tot[2 * i * kSlots], q.hits, sizeof(q.hits));
    }
    cudaError_t e = grow(&s->d_breq, &s->cap_breq, n + 1, st);
    if (e == cudaSuccess) e = grow(&s->d_totals, &s->cap_tot, 2 * n * kSlots + 1, st);
    if (e == cudaSuccess) e = grow(&s->d_results, &s->cap_res, n + 1, st);
    if (e == cudaSuccess) e = grow_host(&s->h_results, &s->cap_hres, n + 1);
    if (e != cudaSuccess) return fail_server(s, MOSS_ENOMEM, "server finalize buffers");
    e = cudaMemcpyAsync(s->d_breq, br.data(), n * sizeof(BatchRequest), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_totals, tot.data(), tot.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_finalize_batch(s->d_breq, (int)n, s->d_totals, s->d_results, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_results, s->d_results, n * sizeof(moss_result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_server(s, MOSS_ECUDA, "server finalize");
    for (size_t i = 0; i < n; ++i) fin[i]->result = s->h_results[i];
    return MOSS_OK;
}

void admit(moss_server *s, double t) {
    while (!s->pending.empty() && (int)s->active.size() < s->cfg.max_active) {
        if (s->cfg.reserve_bytes && s->free_bytes < s->cfg.reserve_bytes) break;  // keep HBM headroom
        const uint64_t id = s->pending.front();
        s->pending.pop_front();
        SReq &q = s->reqs[id];
        q.state = 1;
        q.t_admit = t;
        s->active.push_back(id);
    }
}

// plan the next tick into tb from the active requests (under the lock):
// the next fair-share chunk of every sub-method with ids left to schedule;
// returns the tick's tile count (0: nothing to run)
uint64_t plan_tick(moss_server *s, TickBuffers &tb) {
    tb.tasks.clear();
    tb.owner.clear();
    uint64_t ntiles = 0;
    const uint64_t tile = s->cfg.tile_samples;
    size_t open = 0;   // requests with ids left to schedule
    for (uint64_t id : s->active) {
        const SReq &q = s->reqs[id];
        if (q.next[0] < q.K[0] || q.next[1] < q.K[1]) ++open;
    }
    if (open == 0) return 0;
    uint64_t share = s->cfg.tick_samples / open;
    share = share < tile ? tile : share - share % tile;
    for (uint64_t id : s->active) {
        SReq &q = s->reqs[id];
        int m[2];
        uint64_t Kdummy[2];
        const int nsub = sub_methods(q.k, q.mix, 0, 0, s->ginfo[q.graph].total_nonzero, m, Kdummy);
        bool any = false;
        for (int j = 0; j < nsub; ++j) {
            if (q.next[j] >= q.K[j]) continue;
            const uint64_t c = std::min(share, q.K[j] - q.next[j]);
            BatchTask t;
            t.seed = q.seed;
            t.first = q.next[j];
            t.count = c;
            t.tile0 = ntiles;
            t.graph = (uint32_t)q.graph;
            t.method = (uint32_t)m[j];
            tb.tasks.push_back(t);
            tb.owner.push_back({id, j});
            ntiles += (c + tile - 1) / tile;
            q.next[j] += c;
            any = true;
        }
        if (any) ++q.ticks;
    }
    return ntiles;
}

// take a finished tick back: add its counts to its requests, set the budget
// of requests whose pilot it completed, and return the requests it finished
void take_tick(moss_server *s, TickBuffers &tb, std::vector<SReq *> &fin) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tb.start, tb.end);
    std::lock_guard<std::mutex> lk(s->mu);
    s->busy_s += ms * 1e-3;
    ++s->ticks;
    for (size_t i = 0; i < tb.tasks.size(); ++i) {
        SReq &q = s->reqs[tb.owner[i].first];
        const int j = tb.owner[i].second;
        for (int c = 0; c < kSlots; ++c) q.hits[j][c] += tb.h_task_counts[i * kSlots + c];
        q.done[j] += tb.tasks[i].count;
        s->samples += tb.tasks[i].count;
    }
    std::vector<uint64_t> still;
    for (uint64_t id : s->active) {
        SReq &q = s->reqs[id];
        const bool all = q.done[0] >= q.K[0] && q.done[1] >= q.K[1];
        if (!all) {
            still.push_back(id);
            continue;
        }
        if (q.pilot) {   // the pilot chunk sets the budget
            q.pilot = false;
            uint64_t b = q.mix ? moss_budget_for_target_min(q.K, &q.hits[0][0], q.target, s->cfg.min_budget,
                                                            s->cfg.max_budget)
                               : moss_budget_for_target(q.k, q.K, &q.hits[0][0], q.target, s->cfg.min_budget,
                                                        s->cfg.max_budget);
            const uint64_t pilot_total = q.K[0] + q.K[1];
            if (b < pilot_total) b = pilot_total;
            q.budget = b;
            int m[2];
            uint64_t K[2];
            sub_methods(q.k, q.mix, q.mix ? b / 2 : b, b - b / 2, s->ginfo[q.graph].total_nonzero, m, K);
            q.K[0] = K[0];
            q.K[1] = K[1];
            if (q.done[0] < q.K[0] || q.done[1] < q.K[1]) {
                still.push_back(id);
                continue;
            }
        }
        fin.push_back(&q);
    }
    s->active.swap(still);
}

void scheduler(moss_server *s) {
    cudaSetDevice(s->device);
    int queued[2] = {-1, -1};   // buffer sets of the ticks in flight, oldest first
    int nq = 0;
    for (;;) {
        // with a tick in flight, queue the next one now only under backlog
        bool ahead = nq == 0;
        if (nq == 1) {
            std::lock_guard<std::mutex> lk(s->mu);
            uint64_t left = 0;
            for (uint64_t id : s->active) {
                const SReq &q = s->reqs[id];
                left += (q.K[0] - q.next[0]) + (q.K[1] - q.next[1]);
            }
            ahead = left >= 2 * s->cfg.tick_samples;
        }
        // plan and queue a tick while a buffer set is free
        bool launched = false;
        if (ahead) {
            const int b = nq == 0 ? 0 : 1 - queued[0];
            uint64_t ntiles = 0;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                if (s->stop) break;   // shutting down: unfinished requests are abandoned
                if (s->cfg.reserve_bytes) {
                    size_t fr = 0, totb = 0;
                    if (cudaMemGetInfo(&fr, &totb) == cudaSuccess) s->free_bytes = fr;
                }
                admit(s, now_s());
                ntiles = plan_tick(s, s->tick[b]);
                if (ntiles == 0 && nq == 0) {   // nothing to run and nothing in flight
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                    continue;
                }
            }
            if (ntiles > 0) {
                if (enqueue_tick(s, s->tick[b], ntiles) != MOSS_OK) break;
                queued[nq++] = b;
                launched = true;
            }
        }
        // with two ticks queued, or nothing new to queue, take the oldest back
        if (nq == 2 || (!launched && nq > 0)) {
            TickBuffers &tb = s->tick[queued[0]];
            if (cudaEventSynchronize(tb.end) != cudaSuccess) {
                fail_server(s, MOSS_ECUDA, "server tick");
                break;
            }
            queued[0] = queued[1];
            --nq;
            std::vector<SReq *> fin;
            take_tick(s, tb, fin);
            if (finalize(s, fin) != MOSS_OK) break;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                const double t = now_s();
                for (SReq *q : fin) {
                    q->state = 2;
                    q->t_done = t;
                    ++s->completed;
                    s->last_done = t;
                }
            }
            if (!fin.empty()) s->cv_done.notify_all();
        }
    }
    if (s->stream) cudaStreamSynchronize(s->stream);   // no tick left running on the buffers
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_done.notify_all();
}

}  // namespace

extern "C" {

void moss_server_default_config(moss_server_config *c) {
    if (!c) return;
    c->max_active = 256;
    c->tick_samples = 50'000'000;
    c->tile_samples = 4096;
    c->pilot_samples = 20'000;
    c->min_budget = 10'000;
    c->max_budget = 10'000'000;
    c->reserve_bytes = 1ull << 30;
}

int moss_server_create(int device, const moss_server_config *cfg, moss_server **out) {
    if (!out) return set_error(MOSS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return set_error(MOSS_ECUDA, "cudaGetDeviceCount failed");
    if (device < 0 || device >= ndev) return set_error(MOSS_EINVAL, "device not present");
    moss_server *s = new (std::nothrow) moss_server;
    if (!s) return set_error(MOSS_ENOMEM, "host allocation");
    s->device = device;
    if (cfg) s->cfg = *cfg; else moss_server_default_config(&s->cfg);
    if (s->cfg.max_active < 1 || s->cfg.tile_samples < 32 || s->cfg.tick_samples < s->cfg.tile_samples ||
        s->cfg.min_budget < 1 || s->cfg.max_budget < s->cfg.min_budget) {
        delete s;
        return set_error(MOSS_EINVAL, "inconsistent server configuration");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->fin_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (TickBuffers &tb : s->tick)
        ok = ok && cudaMalloc(reinterpret_cast<void **>(&tb.d_next), sizeof(unsigned long long)) == cudaSuccess &&
             cudaEventCreate(&tb.start) == cudaSuccess && cudaEventCreate(&tb.end) == cudaSuccess;
    s->blocks = batch_blocks(device, 256, 0, kBatchSplitMix);
    if (prev >= 0) cudaSetDevice(prev);
    if (!ok) {
        moss_server_free(s);
        return set_error(MOSS_ECUDA, "creating the server stream");
    }
    *out = s;
    return MOSS_OK;
}

int moss_server_add_graph(moss_server *s, moss_graph *g, int *graph_id) {
    if (!s || !g) return set_error(MOSS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return set_error(MOSS_ESTATE, "graphs are added before the first request");
    GraphInfo gi;
    graph_info(g, &gi);
    if (gi.device != s->device) return set_error(MOSS_EINVAL, "graph lives on another device");
    if (!gi.ready[0] || !gi.ready[1] || !gi.ready[2])
        return set_error(MOSS_ESTATE, "server graphs need the tables of k = 4 and 5");
    s->graphs.push_back(g);
    s->ginfo.push_back(gi);
    if (graph_id) *graph_id = (int)s->graphs.size() - 1;
    return MOSS_OK;
}

int moss_server_submit(moss_server *s, int graph_id, int k, uint64_t budget, double target_rse, uint64_t seed,
                       uint64_t *request_id) {
    if (!s) return set_error(MOSS_EINVAL, "NULL server");
    if (k != 4 && k != 5) return set_error(MOSS_EINVAL, "k must be 4 or 5");
    if (budget == 0 && !(target_rse > 0.0 && target_rse < 1.0))
        return set_error(MOSS_EINVAL, "give a budget or a target relative error in (0, 1)");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->status != MOSS_OK) return set_error(s->status, "the server stopped after an error");
    if (graph_id < 0 || graph_id >= (int)s->graphs.size()) return set_error(MOSS_EINVAL, "unknown graph id");
    if (!s->started) {
        s->started = true;
        s->worker = std::thread(scheduler, s);
    }
    SReq q;
    q.id = s->next_id++;
    q.graph = graph_id;
    q.k = k;
    q.seed = seed;
    q.target = target_rse;
    q.t_arrive = now_s();
    if (s->first_submit == 0) s->first_submit = q.t_arrive;
    int m[2];
    if (budget) {
        q.budget = budget;
        sub_methods(k, false, budget, 0, s->ginfo[graph_id].total_nonzero, m, q.K);
    } else {
        q.pilot = true;
        sub_methods(k, false, s->cfg.pilot_samples, 0, s->ginfo[graph_id].total_nonzero, m, q.K);
    }
    const uint64_t id = q.id;
    s->reqs.emplace(id, q);
    s->pending.push_back(id);
    if (request_id) *request_id = id;
    lk.unlock();
    s->cv_work.notify_one();
    return MOSS_OK;
}

// a MOSS-4 + MOSS-4Min request: explicit budgets, or (target > 0) a pilot
// of pilot_samples split evenly whose counts set the budget
static int submit_min(moss_server *s, int graph_id, uint64_t budget, uint64_t budget_min, double target, uint64_t seed,
               uint64_t *request_id) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->status != MOSS_OK) return set_error(s->status, "the server stopped after an error");
    if (graph_id < 0 || graph_id >= (int)s->graphs.size()) return set_error(MOSS_EINVAL, "unknown graph id");
    if (!s->ginfo[graph_id].ready[0] || !s->ginfo[graph_id].ready[3])
        return set_error(MOSS_ESTATE, "MOSS-4 and MOSS-4Min tables of this graph are not built");
    if (!s->started) {
        s->started = true;
        s->worker = std::thread(scheduler, s);
    }
    SReq q;
    q.id = s->next_id++;
    q.graph = graph_id;
    q.k = 4;
    q.mix = true;
    q.seed = seed;
    q.target = target;
    q.t_arrive = now_s();
    if (s->first_submit == 0) s->first_submit = q.t_arrive;
    int m[2];
    if (target > 0.0) {   // pilot: the configured pilot samples, split evenly
        q.pilot = true;
        budget = s->cfg.pilot_samples / 2;
        budget_min = s->cfg.pilot_samples - budget;
    }
    q.budget = budget + budget_min;
    sub_methods(4, true, budget, budget_min, s->ginfo[graph_id].total_nonzero, m, q.K);
    const uint64_t id = q.id;
    s->reqs.emplace(id, q);
    s->pending.push_back(id);
    if (request_id) *request_id = id;
    lk.unlock();
    s->cv_work.notify_one();
    return MOSS_OK;
}

int moss_server_submit_min(moss_server *s, int graph_id, uint64_t budget, uint64_t budget_min, uint64_t seed,
                           uint64_t *request_id) {
    if (!s) return set_error(MOSS_EINVAL, "NULL server");
    if (budget == 0 && budget_min == 0) return set_error(MOSS_EINVAL, "give the MOSS-4 or MOSS-4Min budget");
    return submit_min(s, graph_id, budget, budget_min, 0.0, seed, request_id);
}

int moss_server_submit_min_target(moss_server *s, int graph_id, double target_rse, uint64_t seed,
                                  uint64_t *request_id) {
    if (!s) return set_error(MOSS_EINVAL, "NULL server");
    if (!(target_rse > 0.0 && target_rse < 1.0)) return set_error(MOSS_EINVAL, "target relative error must be in (0, 1)");
    return submit_min(s, graph_id, 0, 0, target_rse, seed, request_id);
}

int moss_server_wait(moss_server *s, uint64_t request_id, double timeout_s, moss_result *out,
                     moss_request_stats *stats) {
    if (!s) return set_error(MOSS_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return set_error(MOSS_EINVAL, "unknown request id");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (it->second.state != 2) {
        if (s->status != MOSS_OK) return set_error(s->status, "the server stopped after an error");
        if (s->stop) return set_error(MOSS_ESTATE, "the server is shutting down");
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state != 2)
            return set_error(MOSS_EBUSY, "request not finished before the timeout");
        it = s->reqs.find(request_id);
    }
    const SReq &q = it->second;
    if (out) *out = q.result;
    if (stats) {
        stats->budget = q.budget;
        stats->latency_s = q.t_done - q.t_arrive;
        stats->queue_s = q.t_admit - q.t_arrive;
        stats->ticks = q.ticks;
    }
    s->reqs.erase(it);
    return MOSS_OK;
}

int moss_server_stats(moss_server *s, moss_server_info *out) {
    if (!s || !out) return set_error(MOSS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->ticks = s->ticks;
    out->samples = s->samples;
    out->completed = s->completed;
    out->pending = s->pending.size();
    out->active = s->active.size();
    out->busy_s = s->busy_s;
    out->span_s = s->last_done > s->first_submit ? s->last_done - s->first_submit : 0.0;
    return MOSS_OK;
}

void moss_server_free(moss_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (s->fin_stream) {   // the finalize buffers live on the finalize stream
        void *fdev[] = {s->d_breq, s->d_totals, s->d_results};
        for (void *p : fdev)
            if (p) cudaFreeAsync(p, s->fin_stream);
        cudaStreamSynchronize(s->fin_stream);
    }
    if (s->stream) {
        if (s->d_graphs) cudaFreeAsync(s->d_graphs, s->stream);
        for (TickBuffers &tb : s->tick) {
            void *tdev[] = {tb.d_tasks, tb.d_tiles, tb.d_task_counts};
            for (void *p : tdev)
                if (p) cudaFreeAsync(p, s->stream);
        }
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
    }
    if (s->fin_stream) cudaStreamDestroy(s->fin_stream);
    for (TickBuffers &tb : s->tick) {
        if (tb.d_next) cudaFree(tb.d_next);
        if (tb.h_task_counts) cudaFreeHost(tb.h_task_counts);
        if (tb.start) cudaEventDestroy(tb.start);
        if (tb.end) cudaEventDestroy(tb.end);
    }
    if (s->h_results) cudaFreeHost(s->h_results);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
