// Full-Hilbert-space reference on the GPU (the comparison method of Section 5:
// simulate the whole 2^n state).  QAOA Max-Cut of Section 4.1: |+>^n, then per
// layer the diagonal phase exp(-i gamma/2 sum_e z_a z_b) and exp(-i beta X) on
// every qubit; finally <C> = sum_x |psi_x|^2 cut(x) (Eqs. 9-10) and, on request,
// <Z_a Z_b> per edge.
//
// Layout: qubit q is bit q of the element index.  A pass moves tiles of 2^tb
// elements through shared memory (64 KB: 2^13 complex64 or 2^12 complex128,
// two or three CTAs per SM).  Pass 0 of a layer holds qubits 0..tb-1
// (contiguous tiles) and applies the layer's phase on load; every further pass
// mixes its own group of qubits and carries as many low qubits along
// (unmixed) as fill the tile, so tiles stay full and rows contiguous.  The
// qubits above pass 0 are split evenly over the fewest passes.  The mixer's
// 2x2 rotation is applied to the pass's own qubits three at a time on eight
// elements held in registers.
// The last pass of the last layer accumulates |psi|^2 cut(x).
//
// cut(x) without a loop over vertices: with the tile's vertices T and the
// block's fixed bits f on the other vertices F,
//   cut(x) = c0(f) + sum_{a in T} t_a coef_a(f) + W[t],
// c0 = cut edges inside F plus edges from T to F whose F end is 1,
// coef_a = deg_F(a) - 2 |N_F(a) and f|, W = cut edges inside T (a host-built
// table per pass layout).  The linear term comes from two per-block tables.
// The phase and rotation values are computed once per launch (FP64 angles).
#include <cuda_runtime.h>

#include <vector>

#include "exec_common.cuh"
#include "sv_launch.h"

namespace qtc {

constexpr int kSvThreads = 512;
constexpr int kSvMaxEdges = 512;

template <typename T> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

int sv_tile_bits(int dtype) { return dtype == 0 ? 12 : 13; }

int sv_passes(int n, int tmax, int* lo, int* len, int* rl) {
  lo[0] = 0;
  len[0] = n < tmax ? n : tmax;
  rl[0] = 0;
  const int rest = n - len[0];
  if (rest <= 0) return 1;
  const int per = tmax - 4;                    // at least 4 carried qubits per pass
  const int k = (rest + per - 1) / per;
  int q = len[0];
  for (int i = 0; i < k; ++i) {
    const int l = rest / k + (i < rest % k ? 1 : 0);
    lo[1 + i] = q;
    len[1 + i] = l;
    rl[1 + i] = tmax - l;
    q += l;
  }
  return 1 + k;
}

// Tile vertex of tile bit j for a pass (lo = 0: bits 0..len-1; else the
// carried bits 0..rl-1 then lo..lo+len-1).
static inline int tile_vertex(int lo, int rl, int j) {
  return lo == 0 || j < rl ? j : lo + j - rl;
}

std::vector<uint16_t> sv_cut_table(const std::vector<uint32_t>& adj, int n, int lo, int len,
                                   int rl) {
  const int tb = lo == 0 ? len : rl + len;
  std::vector<int> va(tb);
  for (int j = 0; j < tb; ++j) va[j] = tile_vertex(lo, rl, j);
  std::vector<std::pair<int, int>> inner;  // tile-internal edges as tile bit pairs
  for (int j = 0; j < tb; ++j)
    for (int k = j + 1; k < tb; ++k)
      if ((adj[va[j]] >> va[k]) & 1u) inner.emplace_back(j, k);
  std::vector<uint16_t> w((size_t)1 << tb);
  for (uint32_t t = 0; t < (1u << tb); ++t) {
    int c = 0;
    for (auto& e : inner) c += ((t >> e.first) ^ (t >> e.second)) & 1u;
    w[t] = (uint16_t)c;
  }
  (void)n;
  return w;
}

struct SvArgs {
  void* psi;
  int n, m;
  const uint32_t* adj;       // per qubit: bit mask of its neighbours (n <= 32)
  const void* phase;         // per layer m + 1 values exp(-i gamma (m - 2c) / 2)
  const void* rot;           // per layer (cos beta, sin beta)
  const uint16_t* wcut;      // cut edges inside the tile (passes that need cut(x)), else null
  int layer;
  int lo, len, rl;           // pass: tile bits 0..len-1 (lo = 0) or 0..rl-1 and lo..lo+len-1
  int first;                 // 1: the state is |+>, do not read it
  int last;                  // 1: accumulate <C> after this pass
  double* acc;               // [<C>, <ZZ> per edge]
};

// Sets up the per-launch tables: phase[layer][c] and rot[layer].
template <typename T>
__global__ void sv_setup_kernel(const double* params, int p, int m, T* phase, T* rot) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * (m + 1) + p;
       i += gridDim.x * blockDim.x) {
    double sn, cs;
    if (i < p * (m + 1)) {
      const int layer = i / (m + 1), c = i % (m + 1);
      sincos(-0.5 * params[layer] * (double)(m - 2 * c), &sn, &cs);
      phase[i] = from_d2<T>(make_double2(cs, sn));
    } else {
      const int layer = i - p * (m + 1);
      sincos(params[p + layer], &sn, &cs);
      rot[layer] = from_d2<T>(make_double2(cs, sn));
    }
  }
}

// exp(-i beta X) on the pair (x0, x1) = amplitudes with the qubit at 0 and 1:
// [[c, -i s], [-i s, c]].
template <typename T, typename R>
__device__ __forceinline__ void rx_pair(T& x0, T& x1, R c, R s) {
  const T a = x0, b = x1;
  x0.x = c * a.x + s * b.y;
  x0.y = c * a.y - s * b.x;
  x1.x = c * b.x + s * a.y;
  x1.y = c * b.y - s * a.x;
}

// The rotation on k = 1..3 consecutive qubit bits of 2^k amplitudes in registers.
template <int K, typename T, typename R>
__device__ __forceinline__ void rx_bits(T (&v)[8], R c, R s) {
#pragma unroll
  for (int q = 0; q < K; ++q)
#pragma unroll
    for (int i = 0; i < (1 << K); ++i)
      if (!((i >> q) & 1)) rx_pair(v[i], v[i | (1 << q)], c, s);
}

// One mixer round on tile bits b..b+K-1: groups of 2^K amplitudes.
template <int K, typename T, typename R>
__device__ __forceinline__ void rx_round(T* tile, uint32_t tsize, int b, R c, R s) {
  const uint32_t ngroups = tsize >> K;
  const uint32_t lowm = (1u << b) - 1u;
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const uint32_t base = (g & lowm) | ((g & ~lowm) << K);
    T v[8];
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) v[i] = tile[base | ((uint32_t)i << b)];
    rx_bits<K>(v, c, s);
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) tile[base | ((uint32_t)i << b)] = v[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(kSvThreads) sv_pass_kernel(const SvArgs a) {
  using R = typename RealOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ T s_phase[kSvMaxEdges + 1];
  __shared__ int s_lo[128], s_hi[64], s_coef[16];
  __shared__ int s_c0;
  __shared__ double s_red[kSvThreads / 32];
  const int n = a.n;
  const bool pass0 = a.lo == 0;
  const int rl = a.rl;
  const int tb = pass0 ? a.len : rl + a.len;
  const uint32_t tsize = 1u << tb;
  const uint64_t blk = blockIdx.x;
  auto gidx = [&](uint32_t t) -> uint64_t {
    if (pass0) return (blk << a.len) | t;
    const uint64_t low = t & ((1u << rl) - 1u), mid = t >> rl;
    const uint64_t below = blk & ((1ull << (a.lo - rl)) - 1);  // bits rl..lo-1
    const uint64_t above = blk >> (a.lo - rl);                   // bits lo+len..
    return low | (below << rl) | (mid << a.lo) | (above << (a.lo + a.len));
  };
  const bool need_cut = a.wcut != nullptr;
  if (need_cut) {
    const uint32_t full = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const uint32_t tmask =
        pass0 ? (uint32_t)(tsize - 1u) : (((1u << rl) - 1u) | (((1u << a.len) - 1u) << a.lo));
    const uint32_t fm = full & ~tmask;
    const uint32_t f = (uint32_t)gidx(0);  // this block's fixed bits (tile bits zero)
    if (threadIdx.x < 32) {
      int part = 0;
      const int v = threadIdx.x;
      if (v < n) {
        const uint32_t adj_f = a.adj[v] & fm;
        if ((tmask >> v) & 1u)
          part = __popc(adj_f & f);          // tile vertex at 0: edges to fixed ones at 1
        else if ((f >> v) & 1u)
          part = __popc(adj_f & ~f);         // fixed-fixed cut edges, counted from the 1 end
      }
      for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if (v == 0) s_c0 = part;
    }
    if (threadIdx.x < (unsigned)tb) {
      const int j = threadIdx.x;
      const int v = pass0 || j < rl ? j : a.lo + j - rl;
      const uint32_t adj_f = a.adj[v] & fm;
      s_coef[j] = __popc(adj_f) - 2 * __popc(adj_f & f);
    }
    __syncthreads();
    if (threadIdx.x < 128) {
      const int u = threadIdx.x;
      int sl = 0, sh = 0;
      for (int j = 0; j < 7 && j < tb; ++j) sl += ((u >> j) & 1) * s_coef[j];
      for (int j = 7; j < tb && u < 64; ++j) sh += ((u >> (j - 7)) & 1) * s_coef[j];
      s_lo[u] = sl;
      if (u < 64) s_hi[u] = sh;
    }
  }
  if (pass0) {
    const T* ph = reinterpret_cast<const T*>(a.phase) + (size_t)a.layer * (a.m + 1);
    for (int c = threadIdx.x; c <= a.m; c += blockDim.x) s_phase[c] = ph[c];
  }
  const T rot = reinterpret_cast<const T*>(a.rot)[a.layer];
  const R cb = rot.x, sb = rot.y;
  __syncthreads();
  auto cut = [&](uint32_t t) -> int {
    return s_c0 + s_lo[t & 127u] + s_hi[t >> 7] + (int)__ldg(a.wcut + t);
  };
  T* psi = reinterpret_cast<T*>(a.psi);
  const R amp0 = (R)exp2(-0.5 * n);

  // Load.  With at least one element per thread, lanes hold consecutive tile
  // elements (coalesced loads, conflict-free stores) and pass 0 mixes tile
  // qubits 0..4 with shuffles (the partner of lane l for qubit q is l ^ 2^q:
  // x' = c x - i s partner, the same on both sides of the pair).
  const bool full_warps = tsize >= (uint32_t)blockDim.x;
  const int shuffled = pass0 && full_warps ? (tb < 5 ? tb : 5) : 0;
  constexpr int kBatch = 8;
  for (uint32_t t0 = 0; t0 < tsize; t0 += kBatch * blockDim.x) {
    T v[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const uint32_t t = t0 + k * blockDim.x + threadIdx.x;
      if (t < tsize) {
        if (pass0 && a.first) {
          v[k].x = amp0;
          v[k].y = 0;
        } else {
          v[k] = psi[gidx(t)];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const uint32_t t = t0 + k * blockDim.x + threadIdx.x;
      if (pass0 && t < tsize) {
        const T ph = s_phase[cut(t)];
        const T x = v[k];
        v[k].x = x.x * ph.x - x.y * ph.y;
        v[k].y = x.x * ph.y + x.y * ph.x;
      }
      if (t0 + k * blockDim.x < tsize)  // uniform: whole warps
        for (int q = 0; q < shuffled; ++q) {
          const R px = __shfl_xor_sync(0xffffffffu, v[k].x, 1u << q);
          const R py = __shfl_xor_sync(0xffffffffu, v[k].y, 1u << q);
          const R x = v[k].x, y = v[k].y;
          v[k].x = cb * x + sb * py;
          v[k].y = cb * y - sb * px;
        }
      if (t < tsize) tile[t] = v[k];
    }
  }
  // the remaining qubits of the pass, three at a time
  for (int b = pass0 ? shuffled : rl; b < tb; b += 3) {
    __syncthreads();
    const int k = tb - b < 3 ? tb - b : 3;
    if (k == 3) rx_round<3>(tile, tsize, b, cb, sb);
    else if (k == 2) rx_round<2>(tile, tsize, b, cb, sb);
    else rx_round<1>(tile, tsize, b, cb, sb);
  }
  __syncthreads();
  R part = 0;
  for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) {
    const T v = tile[t];
    psi[gidx(t)] = v;
    if (a.last) part += (v.x * v.x + v.y * v.y) * (R)cut(t);
  }
  if (!a.last) return;
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[w];
    atomicAdd(&a.acc[0], sum);
  }
}

// <Z_a Z_b> for edges [e0, e0 + 16): one pass over the state.
template <typename T>
__global__ void __launch_bounds__(256) sv_edge_kernel(void* psi_v, int n, int m,
                                                      const int2* edges, double* acc, int e0) {
  __shared__ double s_red[16][256 / 32];
  const T* psi = reinterpret_cast<const T*>(psi_v);
  const int ne = min(16, m - e0);
  double sums[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) sums[k] = 0.0;
  int2 ed[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) ed[k] = k < ne ? edges[e0 + k] : make_int2(0, 0);
  const uint64_t total = 1ull << n;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const double2 d = to_d2(psi[x]);
    const double pr = d.x * d.x + d.y * d.y;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t diff = ((x >> ed[k].x) ^ (x >> ed[k].y)) & 1u;
      sums[k] += diff ? -pr : pr;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    double v = sums[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < ne) {
    double v = 0.0;
    for (int w = 0; w < 256 / 32; ++w) v += s_red[threadIdx.x][w];
    atomicAdd(&acc[1 + e0 + threadIdx.x], v);
  }
}

template <typename T>
static cudaError_t sv_launch_t(void* psi, int n, int m, const uint32_t* adj_dev,
                               const int2* edges_dev, const double* params_dev, int p,
                               const SvTables& tabs, double* acc_dev, int per_edge,
                               cudaStream_t stream, int* launches) {
  int lo[16], len[16], rl[16];
  const int passes = sv_passes(n, sv_tile_bits(sizeof(T) == 16 ? 0 : 1), lo, len, rl);
  *launches = 0;
  cudaError_t err = cudaMemsetAsync(acc_dev, 0, sizeof(double) * (1 + m), stream);
  if (err != cudaSuccess) return err;
  T* phase = reinterpret_cast<T*>(tabs.scratch);
  T* rot = phase + (size_t)p * (m + 1);
  sv_setup_kernel<T><<<4, 256, 0, stream>>>(params_dev, p, m, phase, rot);
  ++*launches;
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  for (int layer = 0; layer < p; ++layer)
    for (int k = 0; k < passes; ++k) {
      SvArgs a{};
      a.psi = psi;
      a.n = n;
      a.m = m;
      a.adj = adj_dev;
      a.phase = phase;
      a.rot = rot;
      a.layer = layer;
      a.lo = lo[k];
      a.len = len[k];
      a.rl = rl[k];
      a.first = layer == 0 && k == 0;
      a.last = layer == p - 1 && k == passes - 1;
      a.wcut = k == 0 ? tabs.wcut_first : (a.last ? tabs.wcut_last : nullptr);
      a.acc = acc_dev;
      const int tb = k == 0 ? len[k] : rl[k] + len[k];
      const size_t smem = sizeof(T) << tb;
      const unsigned blocks = (unsigned)(1ull << (n - tb));
      cudaFuncSetAttribute(sv_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      sv_pass_kernel<T><<<blocks, kSvThreads, smem, stream>>>(a);
      ++*launches;
      err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  if (per_edge)
    for (int e0 = 0; e0 < m; e0 += 16) {
      sv_edge_kernel<T><<<1024, 256, 0, stream>>>(psi, n, m, edges_dev, acc_dev, e0);
      ++*launches;
      err = cudaGetLastError();
      if (err != cudaSuccess) return err;
    }
  return cudaSuccess;
}

cudaError_t sv_qaoa_launch(int dtype, void* psi, int n, int m, const uint32_t* adj_dev,
                           const int2* edges_dev, const double* params_dev, int p,
                           const SvTables& tabs, double* acc_dev, int per_edge,
                           cudaStream_t stream, int* launches) {
  if (dtype == 0)
    return sv_launch_t<double2>(psi, n, m, adj_dev, edges_dev, params_dev, p, tabs, acc_dev,
                                per_edge, stream, launches);
  return sv_launch_t<float2>(psi, n, m, adj_dev, edges_dev, params_dev, p, tabs, acc_dev,
                             per_edge, stream, launches);
}

}  // namespace qtc
