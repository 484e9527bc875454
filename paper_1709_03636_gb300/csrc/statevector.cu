// Full-Hilbert-space reference on the GPU (the comparison method of Section 5:
// simulate the whole 2^n state).  QAOA Max-Cut of Section 4.1: |+>^n, then per
// layer the diagonal phase exp(-i gamma/2 sum_e z_a z_b) and exp(-i beta X) on
// every qubit; finally <C> = sum_x |psi_x|^2 cut(x) (Eqs. 9-10) and, on request,
// <Z_a Z_b> per edge.
//
// Layout: qubit q is bit q of the element index.  A pass moves tiles of 2^t
// elements through shared memory: pass 0 holds qubits 0..11 (contiguous
// tiles; the layer's phase is applied on load), every further pass holds
// qubits 0..3 (so each row of 16 elements is one 128-byte line) plus the next
// group of up to 8 qubits.  The mixer's 2x2 rotation is applied to every tile
// qubit in shared memory.  The last pass of the last layer accumulates
// |psi|^2 * cut(x) in FP64.
#include <cuda_runtime.h>

#include "exec_common.cuh"
#include "sv_launch.h"

namespace qtc {

constexpr int kSvThreads = 256;
constexpr int kSvMaxEdges = 512;

struct SvArgs {
  void* psi;
  int n, m;
  const uint32_t* adj;       // per qubit: bit mask of its neighbours (n <= 32)
  const int2* edges;         // m edges (a, b)
  const double* params;      // gammas (p), betas (p)
  int p, layer;
  int lo, len;               // pass: tile qubits are 0..3 and lo..lo+len-1 (pass 0: 0..len-1)
  int first;                 // 1: the state is |+>, do not read it
  int last;                  // 1: accumulate <C> (and per-edge) after this pass
  double* acc;               // [<C>, <ZZ> per edge]
  int per_edge;
};

// number of cut edges of basis state x
__device__ __forceinline__ int cut_of(uint32_t x, const uint32_t* adj, int n) {
  int c = 0;
  for (int a = 0; a < n; ++a)
    if ((x >> a) & 1u) c += __popc(adj[a] & ~x);
  return c;
}

template <typename T> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

template <typename T>
__global__ void __launch_bounds__(kSvThreads) sv_pass_kernel(const SvArgs args) {
  using R = typename RealOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ uint32_t s_adj[32];
  __shared__ double s_red[kSvThreads];
  __shared__ T s_phase[kSvMaxEdges + 1];
  const int n = args.n;
  if (threadIdx.x < n) s_adj[threadIdx.x] = args.adj[threadIdx.x];
  // tile bits: pass 0: 0..len-1; else 0..3 and lo..lo+len-1
  const bool pass0 = args.lo == 0;
  const int tbits = pass0 ? args.len : 4 + args.len;
  const uint32_t tsize = 1u << tbits;
  // fixed bits of this tile from blockIdx: every bit outside the tile bits
  uint64_t rest = blockIdx.x;
  auto global_index = [&](uint32_t t) -> uint64_t {
    if (pass0) return (rest << args.len) | t;
    const uint64_t low = t & 15u, mid = t >> 4;
    const uint64_t below = rest & ((1ull << (args.lo - 4)) - 1);  // bits 4..lo-1
    const uint64_t above = rest >> (args.lo - 4);                  // bits lo+len..
    return low | (below << 4) | (mid << args.lo) | (above << (args.lo + args.len));
  };
  const double gamma = args.params[args.layer];
  const double beta = args.params[args.p + args.layer];
  if (pass0)  // the layer's phase depends on x only through cut(x) in 0..m
    for (int c = threadIdx.x; c <= args.m; c += blockDim.x) {
      double sn, cs;
      sincos(-0.5 * gamma * (double)(args.m - 2 * c), &sn, &cs);
      s_phase[c] = from_d2<T>(make_double2(cs, sn));
    }
  __syncthreads();
  T* psi = reinterpret_cast<T*>(args.psi);
  const R amp0 = (R)exp2(-0.5 * n);
  for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) {
    const uint64_t x = global_index(t);
    T v;
    if (args.first) {
      v.x = amp0;
      v.y = 0;
    } else {
      v = psi[x];
    }
    if (pass0) {
      // the layer's phase exp(-i gamma/2 (m - 2 cut(x)))
      const T ph = s_phase[cut_of((uint32_t)x, s_adj, n)];
      const R re = v.x * ph.x - v.y * ph.y;
      v.y = v.x * ph.y + v.y * ph.x;
      v.x = re;
    }
    tile[t] = v;
  }
  __syncthreads();
  // exp(-i beta X) = [[c, -i s], [-i s, c]] on the pass's own qubits (qubits
  // 0..3 ride along in later passes only for coalescing)
  double sbd, cbd;
  sincos(beta, &sbd, &cbd);
  const R sb = (R)sbd, cb = (R)cbd;
  for (int k = pass0 ? 0 : 4; k < tbits; ++k) {
    const uint32_t bit = 1u << k;
    for (uint32_t j = threadIdx.x; j < tsize / 2; j += blockDim.x) {
      const uint32_t i0 = ((j & ~(bit - 1)) << 1) | (j & (bit - 1));
      const uint32_t i1 = i0 | bit;
      const T a = tile[i0], b = tile[i1];
      T a2, b2;
      a2.x = cb * a.x + sb * b.y;
      a2.y = cb * a.y - sb * b.x;
      b2.x = cb * b.x + sb * a.y;
      b2.y = cb * b.y - sb * a.x;
      tile[i0] = a2;
      tile[i1] = b2;
    }
    __syncthreads();
  }
  R part = 0;
  for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) {
    const uint64_t x = global_index(t);
    const T v = tile[t];
    psi[x] = v;
    if (args.last) part += (v.x * v.x + v.y * v.y) * (R)cut_of((uint32_t)x, s_adj, n);
  }
  if (!args.last) return;
  s_red[threadIdx.x] = (double)part;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) s_red[threadIdx.x] += s_red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&args.acc[0], s_red[0]);
}

// <Z_a Z_b> for edges [e0, e0 + 16): one pass over the state.
template <typename T>
__global__ void __launch_bounds__(kSvThreads) sv_edge_kernel(const SvArgs args, int e0) {
  __shared__ double s_red[16][kSvThreads / 32];
  const T* psi = reinterpret_cast<const T*>(args.psi);
  const int ne = min(16, args.m - e0);
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  int2 ed[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) ed[k] = k < ne ? args.edges[e0 + k] : make_int2(0, 0);
  const uint64_t total = 1ull << args.n;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const double2 d = to_d2(psi[x]);
    const double pr = d.x * d.x + d.y * d.y;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t diff = ((x >> ed[k].x) ^ (x >> ed[k].y)) & 1u;
      acc[k] += diff ? -pr : pr;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < ne) {
    double v = 0.0;
    for (int w = 0; w < kSvThreads / 32; ++w) v += s_red[threadIdx.x][w];
    atomicAdd(&args.acc[1 + e0 + threadIdx.x], v);
  }
}

int sv_passes(int n, int* lo, int* len) {
  // pass 0: qubits 0..min(n,12)-1; then groups of up to 8 qubits with 0..3
  int k = 0;
  lo[k] = 0;
  len[k] = n < 12 ? n : 12;
  ++k;
  for (int q = 12; q < n; q += 8) {
    lo[k] = q;
    len[k] = n - q < 8 ? n - q : 8;
    ++k;
  }
  return k;
}

cudaError_t sv_qaoa_launch(int dtype, void* psi, int n, int m, const uint32_t* adj_dev,
                           const int2* edges_dev, const double* params_dev, int p,
                           double* acc_dev, int per_edge, cudaStream_t stream, int* launches) {
  int lo[8], len[8];
  const int passes = sv_passes(n, lo, len);
  const size_t elem = dtype == 0 ? 16 : 8;
  *launches = 0;
  cudaError_t err = cudaMemsetAsync(acc_dev, 0, sizeof(double) * (1 + m), stream);
  if (err != cudaSuccess) return err;
  for (int layer = 0; layer < p; ++layer)
    for (int k = 0; k < passes; ++k) {
      SvArgs a{};
      a.psi = psi;
      a.n = n;
      a.m = m;
      a.adj = adj_dev;
      a.edges = edges_dev;
      a.params = params_dev;
      a.p = p;
      a.layer = layer;
      a.lo = lo[k];
      a.len = len[k];
      a.first = layer == 0 && k == 0;
      a.last = layer == p - 1 && k == passes - 1;
      a.acc = acc_dev;
      const int tbits = k == 0 ? len[k] : 4 + len[k];
      const size_t smem = elem << tbits;
      const unsigned blocks = (unsigned)(1ull << (n - tbits));
      if (dtype == 0) {
        cudaFuncSetAttribute(sv_pass_kernel<double2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        sv_pass_kernel<double2><<<blocks, kSvThreads, smem, stream>>>(a);
      } else {
        cudaFuncSetAttribute(sv_pass_kernel<float2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        sv_pass_kernel<float2><<<blocks, kSvThreads, smem, stream>>>(a);
      }
      ++*launches;
      err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  if (per_edge) {
    SvArgs a{};
    a.psi = psi;
    a.n = n;
    a.m = m;
    a.edges = edges_dev;
    a.acc = acc_dev;
    for (int e0 = 0; e0 < m; e0 += 16) {
      if (dtype == 0)
        sv_edge_kernel<double2><<<1024, kSvThreads, 0, stream>>>(a, e0);
      else
        sv_edge_kernel<float2><<<1024, kSvThreads, 0, stream>>>(a, e0);
      ++*launches;
      err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  }
  return cudaSuccess;
}

}  // namespace qtc
