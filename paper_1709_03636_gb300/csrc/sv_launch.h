// Host entry of the state-vector reference kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace qtc {

// Tile bits of one state-vector pass (64 KB tiles): 12 for complex double
// (dtype 0), 13 for complex float.
int sv_tile_bits(int dtype);

// Pass layout for n qubits and tiles of at most tmax bits: pass 0 holds bits
// 0..len[0]-1; pass k > 0 mixes bits lo[k]..lo[k]+len[k]-1 and carries bits
// 0..rl[k]-1 along (rl[k] + len[k] = tmax).  Returns the pass count (arrays of
// 16).
int sv_passes(int n, int tmax, int* lo, int* len, int* rl);

// Cut edges inside a pass's tile for every tile index (tile bit j = vertex j,
// or for lo > 0: bits 0..rl-1 = vertices 0..rl-1, bit rl + i = vertex lo + i).
std::vector<uint16_t> sv_cut_table(const std::vector<uint32_t>& adj, int n, int lo, int len,
                                   int rl);

struct SvTables {
  const uint16_t* wcut_first;   // sv_cut_table of pass 0
  const uint16_t* wcut_last;    // sv_cut_table of the last pass (when there are several)
  void* scratch;                // p (m + 1) + p + 2 elements of 16 bytes: phase and rotation
                                // tables, the last layer's scale
};

// Evolves |+>^n through p QAOA layers in psi (2^n elements; dtype 0 = complex
// double, else complex float) and accumulates acc[0] = <C> and, when per_edge,
// acc[1 + i] = <Z_a Z_b> of edge i (acc: 1 + m doubles, cleared here).
// n <= 32, m <= 512.  *launches counts the kernels issued.
cudaError_t sv_qaoa_launch(int dtype, void* psi, int n, int m, const uint32_t* adj_dev,
                           const int2* edges_dev, const double* params_dev, int p,
                           const SvTables& tabs, double* acc_dev, int per_edge,
                           cudaStream_t stream, int* launches);

}  // namespace qtc
