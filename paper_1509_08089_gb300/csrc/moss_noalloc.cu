// moss_noalloc.cu -- moss_sample_counts_noalloc: sample counts without any
// device allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- a service that reserves its whole device-memory budget at start
// and forbids growth, a latency-critical loop that cannot afford the device
// synchronisation cudaMalloc/cudaFree may imply, or a host whose allocator
// is owned by another framework.  The ordinary moss_sample_counts uses
// per-block partial counts held by the graph object; this variant keeps
// them in one fixed array of this file instead, so the call itself touches
// no allocator (the graph, its tables and the output buffer are the caller's
// inputs and outputs, allocated earlier).
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot use the symbol as a device address, so the first call on each device
// looks up the array's device address with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should therefore come
// before any stream capture.  The cached address lives as long as the
// process: a cudaDeviceReset of the device makes it stale, so the entry point
// is not to be called again after one.  All calls share the one array: each call's
// sampling kernel overwrites every row it later reads, so nothing needs
// clearing, but calls whose kernels overlap on the GPU (different streams,
// no ordering between them) race on the array and must be serialised by the
// caller.
#include <mutex>

#include "../../include/moss.h"
#include "moss_internal.cuh"

namespace moss {

namespace {

constexpr int kNoAllocMaxBlocks = 2048;   // rows of 22 uint64 partial counts
constexpr size_t kNoAllocScratchBytes = (size_t)kNoAllocMaxBlocks * kSlots * sizeof(uint64_t);  // 360,448 B
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint64_t g_noalloc_partials[kNoAllocMaxBlocks * kSlots];
static_assert(sizeof(g_noalloc_partials) == kNoAllocScratchBytes, "the held scratch is the stated size");

std::mutex g_mutex;
uint64_t *g_scratch[kMaxDevices] = {};

// device address of the array on `device` (current), looked up once
int scratch_on(int device, uint64_t **out) {
    if (device < 0 || device >= kMaxDevices) return set_error(MOSS_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_scratch[device]) {
        uint64_t *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_partials);
        if (e != cudaSuccess || !p) return set_error(MOSS_ECUDA, "cudaGetSymbolAddress of the partial-count array failed");
        g_scratch[device] = p;
    }
    *out = g_scratch[device];
    return MOSS_OK;
}

}  // namespace

}  // namespace moss

using namespace moss;

extern "C" int moss_sample_counts_noalloc(moss_graph *g, int method, uint64_t first, uint64_t count, uint64_t seed,
                                          void *stream, uint64_t *counts_dev) {
    if (!g || !counts_dev) return set_error(MOSS_EINVAL, "NULL argument");
    if (method < 0 || method >= kMethods) return set_error(MOSS_EINVAL, "method must be 0, 1, 2 or 3");
    GraphInfo gi;
    graph_info(g, &gi);
    if (!gi.ready[method]) return set_error(MOSS_ESTATE, "tables for this method are not built");
    if (count > 0 && !gi.total_nonzero[method])
        return set_error(MOSS_EINVAL, "method has total weight 0 on this graph: no sample exists");
    if (first + count < first) return set_error(MOSS_EOVERFLOW, "sample range wraps");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != gi.device && cudaSetDevice(gi.device) != cudaSuccess)
        return set_error(MOSS_ECUDA, "cannot make the graph's device current");
    int rc = MOSS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *partials = nullptr;
    const int blocks = sample_launch_blocks(method, gi.device, gi.view);
    const uint64_t max_chunk = (uint64_t)blocks * 8 * (1ULL << 31);
    if (sample_rows(method, gi.device) > kNoAllocMaxBlocks) {
        rc = set_error(MOSS_EOVERFLOW, "this GPU needs more than 2048 blocks of partial counts, the fixed maximum");
    } else if (count > max_chunk) {
        rc = set_error(MOSS_EOVERFLOW, "count above the per-call maximum of 2^31 samples per warp");
    } else if ((rc = scratch_on(gi.device, &partials)) == MOSS_OK) {
        cudaError_t e;
        if (count == 0) {
            e = cudaMemsetAsync(counts_dev, 0, kSlots * sizeof(uint64_t), s);
        } else {
            e = launch_counts(method, gi.view, first, count, seed, partials, nullptr, nullptr, counts_dev, s);
        }
        if (e != cudaSuccess) rc = set_error(MOSS_ECUDA, cudaGetErrorString(e));
    }
    if (prev >= 0 && prev != gi.device) cudaSetDevice(prev);
    return rc;
}
