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
// 2x2 rotation is applied to the pass's own qubits on elements held in
// registers (and lane bits by shuffles).
// The last pass of the last layer accumulates |psi|^2 cut(x).
//
// The rotation [[c, -i s], [-i s, c]] (c = cos beta, s = sin beta) is applied
// without its larger factor f (c when |c| >= |s|, else s): x0' = x0 - i t x1
// with t = s / c, or x0' = u x0 - i x1 with u = c / s, two fused multiply-adds
// per element and qubit instead of four.  A layer therefore leaves the state
// divided by F = f^n; the next layer's phase table carries F (applied with the
// phase), and the last layer's F scales the stored state and F^2 the sum for
// <C>.  |f| >= 1/sqrt(2), so the stored amplitudes stay within
// 2^(-n/2) .. 1 of the unit-norm state's scale.
//
// cut(x) without a loop over vertices: with the tile's vertices T and the
// block's fixed bits f on the other vertices F,
//   cut(x) = c0(f) + sum_{a in T} t_a coef_a(f) + W[t],
// c0 = cut edges inside F plus edges from T to F whose F end is 1,
// coef_a = deg_F(a) - 2 |N_F(a) and f|, W = cut edges inside T (a host-built
// table per pass layout).  The linear term comes from two per-block tables.
// The phase and rotation values are computed once per launch (FP64 angles).
#include <cuda_runtime.h>

#include <algorithm>
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
  int store;                 // 0: the pass's result is not needed in memory (last pass, no
                             // per-edge values): it is only reduced into <C>
  const double2* scale;      // (F, F^2) of the last layer (see the rotation above)
  double* acc;               // [<C>, <ZZ> per edge]
};

// Per-block tables for cut(x) = c0(f) + sum_{a in T} t_a coef_a(f) + W[t]
// (tile vertices T, the block's fixed bits f) and the layer's phase values.
struct SvBlock {
  int lo[128], hi[64], coef[16];
  int c0;
};

template <typename T>
__device__ __forceinline__ uint64_t sv_gidx(const SvArgs& a, uint64_t blk, uint32_t t) {
  if (a.lo == 0) return (blk << a.len) | t;
  const int rl = a.rl;
  const uint64_t low = t & ((1u << rl) - 1u), mid = t >> rl;
  const uint64_t below = blk & ((1ull << (a.lo - rl)) - 1);  // bits rl..lo-1
  const uint64_t above = blk >> (a.lo - rl);                   // bits lo+len..
  return low | (below << rl) | (mid << a.lo) | (above << (a.lo + a.len));
}

template <typename T>
__device__ void sv_block_setup(const SvArgs& a, uint64_t blk, int tb, SvBlock& sb, T* s_phase) {
  const int n = a.n;
  const bool pass0 = a.lo == 0;
  const int rl = a.rl;
  if (a.wcut != nullptr) {
    const uint32_t tsize = 1u << tb;
    const uint32_t full = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const uint32_t tmask =
        pass0 ? (uint32_t)(tsize - 1u) : (((1u << rl) - 1u) | (((1u << a.len) - 1u) << a.lo));
    const uint32_t fm = full & ~tmask;
    const uint32_t f = (uint32_t)sv_gidx<T>(a, blk, 0);  // fixed bits (tile bits zero)
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
      if (v == 0) sb.c0 = part;
    }
    if (threadIdx.x < (unsigned)tb) {
      const int j = threadIdx.x;
      const int v = pass0 || j < rl ? j : a.lo + j - rl;
      const uint32_t adj_f = a.adj[v] & fm;
      sb.coef[j] = __popc(adj_f) - 2 * __popc(adj_f & f);
    }
    __syncthreads();
    if (threadIdx.x < 128) {
      const int u = threadIdx.x;
      int sl = 0, sh = 0;
      for (int j = 0; j < 7 && j < tb; ++j) sl += ((u >> j) & 1) * sb.coef[j];
      for (int j = 7; j < tb && u < 64; ++j) sh += ((u >> (j - 7)) & 1) * sb.coef[j];
      sb.lo[u] = sl;
      if (u < 64) sb.hi[u] = sh;
    }
  }
  if (pass0) {
    const T* ph = reinterpret_cast<const T*>(a.phase) + (size_t)a.layer * (a.m + 1);
    for (int c = threadIdx.x; c <= a.m; c += blockDim.x) s_phase[c] = ph[c];
  }
  __syncthreads();
}

// Sets up the per-launch tables: phase[layer][c] (times the previous layer's
// F), rot[layer] = (t or u, 1 when the cos form) and scale = (F, F^2) of the
// last layer.
template <typename T>
__global__ void sv_setup_kernel(const double* params, int n, int p, int m, T* phase, T* rot,
                                double2* scale) {
  auto form = [&](int layer, double* r, double* f) {
    double sn, cs;
    sincos(params[p + layer], &sn, &cs);
    const bool kc = fabs(cs) >= fabs(sn);
    *r = kc ? sn / cs : cs / sn;
    *f = kc ? cs : sn;
    return kc;
  };
  auto layer_scale = [&](int layer) {
    double r, f, F = 1.0;
    form(layer, &r, &f);
    for (int i = 0; i < n; ++i) F *= f;
    return F;
  };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * (m + 1) + p + 1;
       i += gridDim.x * blockDim.x) {
    double sn, cs;
    if (i < p * (m + 1)) {
      const int layer = i / (m + 1), c = i % (m + 1);
      sincos(-0.5 * params[layer] * (double)(m - 2 * c), &sn, &cs);
      const double F = layer > 0 ? layer_scale(layer - 1) : 1.0;
      phase[i] = from_d2<T>(make_double2(F * cs, F * sn));
    } else if (i < p * (m + 1) + p) {
      const int layer = i - p * (m + 1);
      double r, f;
      const bool kc = form(layer, &r, &f);
      rot[layer] = from_d2<T>(make_double2(r, kc ? 1.0 : 0.0));
    } else {
      const double F = layer_scale(p - 1);
      *scale = make_double2(F, F * F);
    }
  }
}

// exp(-i beta X) on the pair (x0, x1) = amplitudes with the qubit at 0 and 1,
// without the factor f: KC: x0' = x0 - i t x1; else x0' = u x0 - i x1 (r = t
// or u; the same on both sides of the pair).
template <bool KC, typename T, typename R>
__device__ __forceinline__ void rxs_pair(T& x0, T& x1, R r) {
  const T a = x0, b = x1;
  if (KC) {
    x0.x = a.x + r * b.y;
    x0.y = a.y - r * b.x;
    x1.x = b.x + r * a.y;
    x1.y = b.y - r * a.x;
  } else {
    x0.x = r * a.x + b.y;
    x0.y = r * a.y - b.x;
    x1.x = r * b.x + a.y;
    x1.y = r * b.y - a.x;
  }
}

// The same with the partner amplitude in another lane (bit q of the lane).
template <bool KC, typename T, typename R>
__device__ __forceinline__ void rxs_shfl(T& v, R r, int q) {
  const R px = __shfl_xor_sync(0xffffffffu, v.x, 1u << q);
  const R py = __shfl_xor_sync(0xffffffffu, v.y, 1u << q);
  if (KC) {
    v.x = v.x + r * py;
    v.y = v.y - r * px;
  } else {
    v.x = r * v.x + py;
    v.y = r * v.y - px;
  }
}

// The rotation on k = 1..3 consecutive qubit bits of 2^k amplitudes in registers.
template <int K, bool KC, typename T, typename R>
__device__ __forceinline__ void rx_bits(T (&v)[8], R r) {
#pragma unroll
  for (int q = 0; q < K; ++q)
#pragma unroll
    for (int i = 0; i < (1 << K); ++i)
      if (!((i >> q) & 1)) rxs_pair<KC>(v[i], v[i | (1 << q)], r);
}

// One mixer round on tile bits b..b+K-1: groups of 2^K amplitudes.
template <int K, bool KC, typename T, typename R>
__device__ __forceinline__ void rx_round(T* tile, uint32_t tsize, int b, R r) {
  const uint32_t ngroups = tsize >> K;
  const uint32_t lowm = (1u << b) - 1u;
  for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const uint32_t base = (g & lowm) | ((g & ~lowm) << K);
    T v[8];
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) v[i] = tile[base | ((uint32_t)i << b)];
    rx_bits<K, KC>(v, r);
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
  __shared__ SvBlock s_sb;
  __shared__ double s_red[kSvThreads / 32];
  const int n = a.n;
  const bool pass0 = a.lo == 0;
  const int rl = a.rl;
  const int tb = pass0 ? a.len : rl + a.len;
  const uint32_t tsize = 1u << tb;
  const uint64_t blk = blockIdx.x;
  auto gidx = [&](uint32_t t) -> uint64_t { return sv_gidx<T>(a, blk, t); };
  sv_block_setup<T>(a, blk, tb, s_sb, s_phase);
  const T rot = reinterpret_cast<const T*>(a.rot)[a.layer];
  const R rr = rot.x;
  const bool kc = rot.y != (R)0;
  auto cut = [&](uint32_t t) -> int {
    return s_sb.c0 + s_sb.lo[t & 127u] + s_sb.hi[t >> 7] + (int)__ldg(a.wcut + t);
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
          if (kc) rxs_shfl<true>(v[k], rr, q);
          else rxs_shfl<false>(v[k], rr, q);
        }
      if (t < tsize) tile[t] = v[k];
    }
  }
  // the remaining qubits of the pass, three at a time
  for (int b = pass0 ? shuffled : rl; b < tb; b += 3) {
    __syncthreads();
    const int k = tb - b < 3 ? tb - b : 3;
    if (kc) {
      if (k == 3) rx_round<3, true>(tile, tsize, b, rr);
      else if (k == 2) rx_round<2, true>(tile, tsize, b, rr);
      else rx_round<1, true>(tile, tsize, b, rr);
    } else {
      if (k == 3) rx_round<3, false>(tile, tsize, b, rr);
      else if (k == 2) rx_round<2, false>(tile, tsize, b, rr);
      else rx_round<1, false>(tile, tsize, b, rr);
    }
  }
  __syncthreads();
  R part = 0;
  const R fin = a.last ? (R)a.scale->x : (R)1;
  for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) {
    T v = tile[t];
    if (a.last) {
      part += (v.x * v.x + v.y * v.y) * (R)cut(t);
      v.x *= fin;
      v.y *= fin;
    }
    if (a.store) psi[gidx(t)] = v;
  }
  if (!a.last) return;
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[w];
    atomicAdd(&a.acc[0], sum * a.scale->y);
  }
}

// A full tile (2^tb elements, tb = sv_tile_bits) with 2^K elements per
// thread held in registers.  In every layout lanes are tile bits 0..4
// (consecutive elements: coalesced global access, conflict-free shared
// memory) and the registers are K consecutive tile bits r0..r0+K-1; the warp
// index fills the other bits.  The load layout has the registers on the top
// K bits, which are mixed right after the load (pass 0: after the phase);
// mixed lane bits use shuffles; the bits in between are mixed in rounds
// through shared memory, K at a time (one store and one load per element);
// the pass stores from its last layout.  Bits below the pass's carried range
// (rl, passes after the first) are not mixed.  Per layout a thread computes
// its base tile index, global offset and linear cut term once; register r
// adds r << r0 to the tile index, its deposit to the global offset and its
// bits' cut coefficients.
template <int K, bool KC, typename T, typename R>
__device__ __forceinline__ void rx_reg_bits(T (&v)[1 << K], int r0, int lo, int hi, R r) {
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (r0 + q >= lo && r0 + q < hi)
#pragma unroll
      for (int i = 0; i < (1 << K); ++i)
        if (!((i >> q) & 1)) rxs_pair<KC>(v[i], v[i | (1 << q)], r);
}

template <typename T, int K>
__global__ void __launch_bounds__(kSvThreads, 2) sv_tile_kernel(const SvArgs a) {
  using R = typename RealOf<T>::type;
  constexpr int NR = 1 << K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ T s_phase[kSvMaxEdges + 1];
  __shared__ uint32_t s_adj[32];
  __shared__ int s_coef[16];
  __shared__ int s_c0;
  __shared__ double s_red[kSvThreads / 32];
  const int n = a.n;
  const bool pass0 = a.lo == 0;
  const int tb = pass0 ? a.len : a.rl + a.len;   // K + 9 (512 threads)
  const int mix_lo = pass0 ? 0 : a.rl;           // lowest mixed tile bit
  const uint64_t n_tiles = 1ull << (n - tb);
  const bool need_cut = a.wcut != nullptr;       // pass 0 and the last pass
  // once per CTA: adjacency masks, the layer's phase table, the rotation
  if (threadIdx.x < 32) s_adj[threadIdx.x] = (int)threadIdx.x < n ? a.adj[threadIdx.x] : 0u;
  if (pass0) {
    const T* ph = reinterpret_cast<const T*>(a.phase) + (size_t)a.layer * (a.m + 1);
    for (int c = threadIdx.x; c <= a.m; c += blockDim.x) s_phase[c] = ph[c];
  }
  const T rot = reinterpret_cast<const T*>(a.rot)[a.layer];
  const R rr = rot.x;
  const bool kc = rot.y != (R)0;   // the form of the layer's rotation (uniform)
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t full = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint32_t tmask = pass0 ? (uint32_t)((1u << tb) - 1u)
                               : (((1u << a.rl) - 1u) | (((1u << a.len) - 1u) << a.lo));
  const uint32_t low_mask = pass0 ? 0xFFFFFFFFu : ((1u << a.rl) - 1u);
  auto gbits = [&](uint32_t tbits) -> uint64_t {   // tile bits -> global bits
    return pass0 ? (uint64_t)tbits
                 : ((uint64_t)(tbits & low_mask) | ((uint64_t)(tbits >> a.rl) << a.lo));
  };
  T* psi = reinterpret_cast<T*>(a.psi);
  R part = 0;
  __syncthreads();
  for (uint64_t blk = blockIdx.x; blk < n_tiles; blk += gridDim.x) {
    if (need_cut) {
      // this tile's cut terms from its fixed bits f (see the file comment)
      const uint32_t fm = full & ~tmask;
      const uint32_t f = (uint32_t)sv_gidx<T>(a, blk, 0);
      __syncthreads();   // the previous tile's readers of s_c0 / s_coef are done
      if (threadIdx.x < 32) {
        int c = 0;
        const int v = threadIdx.x;
        if (v < n) {
          const uint32_t adj_f = s_adj[v] & fm;
          if ((tmask >> v) & 1u) c = __popc(adj_f & f);
          else if ((f >> v) & 1u) c = __popc(adj_f & ~f);
        }
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (v == 0) s_c0 = c;
      }
      if (threadIdx.x < (unsigned)tb) {
        const int j = threadIdx.x;
        const int v = pass0 || j < a.rl ? j : a.lo + j - a.rl;
        const uint32_t adj_f = s_adj[v] & fm;
        s_coef[j] = __popc(adj_f) - 2 * __popc(adj_f & f);
      }
      __syncthreads();
    }
    // register bits r0..r0+K-1 of a layout: tile index, global offset, linear
    // cut term and the registers' cut coefficients
    uint32_t tbase = 0;
    uint64_t gbase = 0;
    int lin = 0, cr[K];
    auto set_layout = [&](int r0) {
      const uint32_t wl = w & ((1u << (r0 - 5)) - 1u), wh = w >> (r0 - 5);
      tbase = lane | (wl << 5) | (wh << (r0 + K));
      gbase = sv_gidx<T>(a, blk, tbase);
      if (need_cut) {
        lin = s_c0;
        for (int j = 0; j < tb; ++j)
          if ((tbase >> j) & 1u) lin += s_coef[j];
#pragma unroll
        for (int k = 0; k < K; ++k) cr[k] = s_coef[r0 + k];
      }
    };
    auto cut_of = [&](int r0, int r) -> int {
      int c = lin;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if ((r >> k) & 1) c += cr[k];
      return c + (int)__ldg(a.wcut + (tbase | ((uint32_t)r << r0)));
    };
    T v[NR];
    int r0 = tb - K;
    set_layout(r0);
    if (pass0 && a.first) {
      const R amp0 = (R)exp2(-0.5 * n);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        v[r].x = amp0;
        v[r].y = 0;
      }
    } else {
#pragma unroll
      for (int r = 0; r < NR; ++r) v[r] = psi[gbase | gbits((uint32_t)r << r0)];
    }
    if (pass0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T ph = s_phase[cut_of(r0, r)];
        const T x = v[r];
        v[r].x = x.x * ph.x - x.y * ph.y;
        v[r].y = x.x * ph.y + x.y * ph.x;
      }
    }
    if (kc) rx_reg_bits<K, true>(v, r0, mix_lo, tb, rr);
    else rx_reg_bits<K, false>(v, r0, mix_lo, tb, rr);
    // lane bits (tile bits 0..4) that the pass mixes: shuffles
    for (int q = mix_lo; q < 5; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (kc) rxs_shfl<true>(v[r], rr, q);
        else rxs_shfl<false>(v[r], rr, q);
      }
    // bits 5..tb-K-1 in rounds of K through shared memory
    for (int b = 5; b < tb - K; b += K) {
      const int hi = min(b + K, tb - K);
      if (hi <= mix_lo) continue;   // carried bits only
      __syncthreads();   // earlier readers of the tile are done
#pragma unroll
      for (int r = 0; r < NR; ++r) tile[tbase | ((uint32_t)r << r0)] = v[r];
      __syncthreads();
      r0 = min(b, tb - 2 * K);
      set_layout(r0);
#pragma unroll
      for (int r = 0; r < NR; ++r) v[r] = tile[tbase | ((uint32_t)r << r0)];
      if (kc) rx_reg_bits<K, true>(v, r0, max(b, mix_lo), hi, rr);
      else rx_reg_bits<K, false>(v, r0, max(b, mix_lo), hi, rr);
    }
    if (!a.last) {
#pragma unroll
      for (int r = 0; r < NR; ++r) psi[gbase | gbits((uint32_t)r << r0)] = v[r];
      continue;
    }
    const R fin = (R)a.scale->x;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      part += (v[r].x * v[r].x + v[r].y * v[r].y) * (R)cut_of(r0, r);
      if (a.store) {
        T o = v[r];
        o.x *= fin;
        o.y *= fin;
        psi[gbase | gbits((uint32_t)r << r0)] = o;
      }
    }
  }
  if (!a.last) return;
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0) s_red[w] = (double)part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += s_red[i];
    atomicAdd(&a.acc[0], sum * a.scale->y);
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
  const int tmax = sv_tile_bits(sizeof(T) == 16 ? 0 : 1);
  int dev = 0, sms = 0;
  cudaError_t aerr = cudaGetDevice(&dev);
  if (aerr == cudaSuccess) aerr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (aerr != cudaSuccess) return aerr;
  if (sms < 1) sms = 1;
  const int passes = sv_passes(n, tmax, lo, len, rl);
  *launches = 0;
  cudaError_t err = cudaMemsetAsync(acc_dev, 0, sizeof(double) * (1 + m), stream);
  if (err != cudaSuccess) return err;
  T* phase = reinterpret_cast<T*>(tabs.scratch);
  T* rot = phase + (size_t)p * (m + 1);
  double2* scale = reinterpret_cast<double2*>(
      (reinterpret_cast<uintptr_t>(rot + p) + 15) & ~static_cast<uintptr_t>(15));
  sv_setup_kernel<T><<<4, 256, 0, stream>>>(params_dev, n, p, m, phase, rot, scale);
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
      a.store = !(a.last && !per_edge);
      a.scale = scale;
      a.acc = acc_dev;
      const int tb = k == 0 ? len[k] : rl[k] + len[k];
      const size_t smem = sizeof(T) << tb;
      const unsigned blocks = (unsigned)(1ull << (n - tb));
      if (tb == tmax) {
        // full tiles: registers hold 2^K elements per thread (K + 9 = tb)
        // one CTA per resident slot (two per SM), each walking tiles
        constexpr int K = sizeof(T) == 16 ? 3 : 4;
        cudaFuncSetAttribute(sv_tile_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        const unsigned grid = std::min<unsigned>(blocks, 2u * (unsigned)sms);
        sv_tile_kernel<T, K><<<grid, kSvThreads, smem, stream>>>(a);
      } else {
        cudaFuncSetAttribute(sv_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        sv_pass_kernel<T><<<blocks, kSvThreads, smem, stream>>>(a);
      }
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
