// moss_order.cuh -- degree ordering of a graph at load (moss_order.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace moss {

// Scratch of launch_degree_order for n vertices (the input col is not part of it).
uint64_t order_scratch_bytes(uint32_t n);

// Renumbers the CSR (row_ptr: n+1 offsets, uint64 when is64, else uint32;
// col_in: nnz ids, device memory) in degree-key order and writes the
// renumbered lists to col_out (nnz) and order[i] = the input id of internal
// vertex i (n).  *rp_out receives the renumbered row offsets (n+1 uint32,
// inside scratch, valid until scratch is released).  Input faults go to
// flags[0] as the vertex and slot passes report them (kErr* bits): row_ptr
// (its bad rows become empty), an id >= n, a list not strictly increasing.
cudaError_t launch_degree_order(const void *row_ptr, int is64, const uint32_t *col_in, uint32_t n, uint64_t nnz,
                                uint32_t *order, uint32_t *col_out, void *scratch, uint32_t **rp_out,
                                uint32_t *flags, cudaStream_t s);

// Maps the vertex ids of count sample records (5 words each; the first
// `words` of them are vertex ids) from internal to input ids.
cudaError_t launch_map_records(uint32_t *verts, uint64_t count, int words, const uint32_t *order, uint32_t n,
                               cudaStream_t s);

}  // namespace moss
