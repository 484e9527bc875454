// Host-side entry points of the CUDA executors (internal).
#pragma once

#include <cuda_runtime.h>

#include "device_program.h"

namespace qtc {

// dtype: 0 = complex double, otherwise complex float.
cudaError_t smem_exec_configure(int dtype, size_t smem_bytes, size_t max_dynamic, int block,
                                int* blocks_per_sm);
cudaError_t smem_exec_launch(const ProgramDev& prog, int dtype, int grid, int block,
                             size_t smem_bytes, cudaStream_t stream);

}  // namespace qtc
