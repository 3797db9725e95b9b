// moss_measure.cu -- the random-gather ceiling the samplers are measured
// against (a measurement helper, not a step of the method).
//
// Every sampler step (seed alias record, sigma slot record, list picks, edge
// probes) is a read of one 32-byte sector at an address no neighbouring
// thread shares, so their throughput is bounded by how many independent
// random sectors per second the memory system serves, not by the streaming
// copy bandwidth: from a buffer that fits in L2 the bound is the L1-to-L2
// request rate, from one far larger than L2 it is the HBM random-access rate.
// k_gather reads sectors of a buffer of its own at uniform random positions
// (four independent 256-bit loads in flight per thread, a full persistent
// grid) and moss_gather_rate reports the sectors per second it sustained.
#include <cstdint>
#include <cstdio>

#include "moss.h"
#include "moss_internal.cuh"

namespace moss {
namespace {

constexpr int kGatherThreads = 256;
constexpr int kGatherBlocksPerSm = 8;
constexpr int kGatherInFlight = 4;               // independent loads per thread per round
constexpr uint64_t kGatherSectors = 1ull << 28;  // sectors read by the timed launch

__device__ uint32_t g_gather_sink;

__device__ __forceinline__ uint64_t gather_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// rounds rounds of kGatherInFlight loads per thread; sector indices are
// __umul64hi(h, nsec) < nsec, so every load lies inside the buffer
__global__ void __launch_bounds__(kGatherThreads) k_gather(const uint8_t *buf, uint64_t nsec, uint64_t rounds) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        uint32_t v[kGatherInFlight][8];
#pragma unroll
        for (int u = 0; u < kGatherInFlight; ++u) {
            const uint64_t h = gather_mix((tid * rounds + r) * kGatherInFlight + u + 1);
            const uint8_t *p = buf + __umul64hi(h, nsec) * 32;
            asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[u][0]), "=r"(v[u][1]), "=r"(v[u][2]), "=r"(v[u][3]), "=r"(v[u][4]),
                           "=r"(v[u][5]), "=r"(v[u][6]), "=r"(v[u][7])
                         : "l"(p));
        }
#pragma unroll
        for (int u = 0; u < kGatherInFlight; ++u) acc += v[u][0] ^ v[u][7];
    }
    if (acc == 0x9E3779B9u) g_gather_sink = acc;   // keeps the loads; the buffer is zero
}

}  // namespace
}  // namespace moss

extern "C" int moss_gather_rate(uint64_t bytes, int device, void *stream, double *sectors_per_s) {
    using namespace moss;
    if (!sectors_per_s) return set_error(MOSS_EINVAL, "sectors_per_s is NULL");
    *sectors_per_s = 0.0;
    if (bytes < 32 || bytes % 32 != 0) return set_error(MOSS_EINVAL, "bytes must be a positive multiple of 32");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_error(MOSS_EINVAL, "no such CUDA device");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return set_error(MOSS_ECUDA, "cudaSetDevice failed");
    const cudaStream_t s = (cudaStream_t)stream;
    int rc = MOSS_OK;
    char detail[160];
    uint8_t *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        const int blocks = device_sms(device) * kGatherBlocksPerSm;
        const uint64_t per_round = (uint64_t)blocks * kGatherThreads * kGatherInFlight;
        const uint64_t rounds = (kGatherSectors + per_round - 1) / per_round;
        const uint64_t nsec = bytes / 32;
        // a first launch of the same length brings an L2-sized buffer into L2
        k_gather<<<blocks, kGatherThreads, 0, s>>>(buf, nsec, rounds);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_gather<<<blocks, kGatherThreads, 0, s>>>(buf, nsec, rounds);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f) *sectors_per_s = (double)(per_round * rounds) / (ms * 1e-3);
    }
    if (e != cudaSuccess) {
        snprintf(detail, sizeof(detail), "gather measurement: %s", cudaGetErrorString(e));
        rc = set_error(e == cudaErrorMemoryAllocation ? MOSS_ENOMEM : MOSS_ECUDA, detail);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) {
        cudaStreamSynchronize(s);
        cudaFree(buf);
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
