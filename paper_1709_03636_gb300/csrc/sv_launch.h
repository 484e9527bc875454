// Host entry of the state-vector reference kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qtc {

// Evolves |+>^n through p QAOA layers in psi (2^n elements; dtype 0 = complex
// double, else complex float) and accumulates acc[0] = <C> and, when per_edge,
// acc[1 + i] = <Z_a Z_b> of edge i (acc: 1 + m doubles, cleared here).
// n <= 32, m <= 512.  *launches counts the kernels issued.
cudaError_t sv_qaoa_launch(int dtype, void* psi, int n, int m, const uint32_t* adj_dev,
                           const int2* edges_dev, const double* params_dev, int p,
                           double* acc_dev, int per_edge, cudaStream_t stream, int* launches);

}  // namespace qtc
