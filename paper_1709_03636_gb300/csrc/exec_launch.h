// Host-side entry points of the CUDA executors (internal).
#pragma once

#include <cuda_runtime.h>

#include "device_program.h"

namespace qtc {

// Register cap of the shared-memory executor (CTAs of 128 threads: a CTA
// team, or up to four warp teams).  96 keeps the float warp kernels free of
// spills; it also caps residency at 65536 / (96 * 128) = 5 CTAs per SM.
constexpr int kExecMaxRegs = 96;
constexpr int kExecCtasPerSmByRegs = 65536 / (kExecMaxRegs * 128);

// dtype: 0 = complex double, otherwise complex float.
// mode: 0 = the whole CTA runs one network at a time; 1 = each warp of a CTA
// runs its own network from steps staged in shared memory; 2 = the same with
// steps streamed from global memory (step lists too long to stage).
cudaError_t smem_exec_configure(int dtype, int mode, size_t smem_bytes, size_t max_dynamic,
                                int block, int* blocks_per_sm);
cudaError_t smem_exec_launch(const ProgramDev& prog, int dtype, int mode, int grid, int block,
                             size_t smem_bytes, cudaStream_t stream);

// Graph executor (networks larger than one CTA's shared memory); one launch
// per wave.
// tc: the program has tensor-core GEMM tasks (GraphProgDev.tmem_cols > 0).
// hi_occ (complex64 without tensor cores): the instantiation capped for five
// CTAs per SM.
// tiles: the program has steps in tile form (the instantiation with tile code)
cudaError_t graph_exec_configure(int dtype, bool tc, bool hi_occ, bool tiles, size_t smem_bytes,
                                 size_t max_dynamic, int* blocks_per_sm);
cudaError_t graph_exec_launch(const GraphProgDev& prog, int dtype, bool hi_occ, bool tiles,
                              int grid, size_t smem_bytes, cudaStream_t stream);

}  // namespace qtc
