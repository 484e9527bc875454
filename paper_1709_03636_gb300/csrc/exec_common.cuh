// Device helpers shared by the executors: complex arithmetic, gate tensors,
// execution teams and the bit-map contraction of one op (Eq. 1 with batch
// indices).
#pragma once

#include <cuda_runtime.h>

#include "device_program.h"

namespace qtc {

constexpr int kMaxParams = 64;

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <typename T> __device__ __forceinline__ T from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

// Values (and derivatives with respect to params[slot]) of one gate table
// entry, element index bit k = label k (see LeafKind).
__device__ inline void gate_tensor(const GateSpec& s, const double* params, double2* val,
                            double2* der) {
  const double theta = s.constant + (s.slot >= 0 ? s.coeff * params[s.slot] : 0.0);
  const double dth = s.slot >= 0 ? s.coeff : 0.0;  // d theta / d param
  const int rank = leaf_rank_of(s.kind);
  const int n = 1 << rank;
  for (int i = 0; i < n; ++i) {
    val[i] = make_double2(0.0, 0.0);
    der[i] = make_double2(0.0, 0.0);
  }
  const double r = 0.70710678118654752440;
  double sh, ch;
  sincos(0.5 * theta, &sh, &ch);
  switch (s.kind) {
    case LK_ZERO: case LK_PROJ0: val[0].x = 1.0; break;
    case LK_PROJ1: val[1].x = 1.0; break;
    case LK_PLUS: val[0].x = r; val[1].x = r; break;
    case LK_ZDIAG: val[0].x = 1.0; val[1].x = -1.0; break;
    case LK_H:
      for (int i = 0; i < 4; ++i) val[i].x = (i == 3) ? -r : r;
      break;
    case LK_X: case LK_OBS_X: val[2].x = 1.0; val[1].x = 1.0; break;
    case LK_Y: case LK_OBS_Y:
      val[2].y = -1.0;  // [0][1] = -i  (index out=0 | in=1 << 1)
      val[1].y = 1.0;   // [1][0] = +i
      break;
    case LK_Z: case LK_OBS_Z: val[0].x = 1.0; val[3].x = -1.0; break;
    case LK_RX:  // cos(t/2) I - i sin(t/2) X, [out, in]
      val[0].x = ch; val[3].x = ch; val[1].y = -sh; val[2].y = -sh;
      der[0].x = -0.5 * sh * dth; der[3].x = -0.5 * sh * dth;
      der[1].y = -0.5 * ch * dth; der[2].y = -0.5 * ch * dth;
      break;
    case LK_RZ: case LK_RZDIAG: {
      // diag(exp(-i t/2), exp(+i t/2)); dense form at [0][0] and [1][1]
      const int i1 = s.kind == LK_RZ ? 3 : 1;
      val[0] = make_double2(ch, -sh);
      val[i1] = make_double2(ch, sh);
      der[0] = make_double2(-0.5 * sh * dth, -0.5 * ch * dth);
      der[i1] = make_double2(-0.5 * sh * dth, 0.5 * ch * dth);
      break;
    }
    case LK_ZZDIAG: case LK_ZZ:
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double zz = (a == b) ? 1.0 : -1.0;  // z_a z_b
          const int idx = s.kind == LK_ZZDIAG ? (a | b << 1) : (a | b << 1 | a << 2 | b << 3);
          val[idx] = make_double2(ch, -zz * sh);  // exp(-i zz t/2)
          // d/dt = -i zz/2 * value
          der[idx] = make_double2(-0.5 * sh * dth, -0.5 * zz * ch * dth);
        }
      break;
    case LK_CNOT:
      for (int c = 0; c < 2; ++c)
        for (int t = 0; t < 2; ++t) val[c | (t ^ c) << 1 | c << 2 | t << 3].x = 1.0;
      break;
    default: break;
  }
  if (s.conj)
    for (int i = 0; i < n; ++i) {
      val[i].y = -val[i].y;
      der[i].y = -der[i].y;
    }
}

// A team is one warp (small networks, kWarp) or the whole CTA.
template <bool kWarp>
struct Team {
  int tid, size, id;
  __device__ Team() {
    if (kWarp) {
      tid = threadIdx.x & 31;
      size = 32;
      id = threadIdx.x >> 5;
    } else {
      tid = threadIdx.x;
      size = blockDim.x;
      id = 0;
    }
  }
  __device__ __forceinline__ void sync() const {
    if (kWarp)
      __syncwarp();
    else
      __syncthreads();
  }
};

// Element pointer of an op offset: gate table below table_elems, else the
// team's own arena.
template <typename T>
__device__ __forceinline__ T* resolve(uint32_t off, T* table, T* arena, uint32_t table_elems) {
  return off < table_elems ? table + off : arena + (off - table_elems);
}

// out = sum over the summed bits of a * b for every output element; the
// team's threads (team.tid of team.size) share the outputs.
template <typename T, typename TeamT>
__device__ __forceinline__ void contract_op(const SOp& op, T* out, const T* a, const T* b,
                                            const TeamT& team) {
  const uint32_t nout = 1u << op.rc;
  const uint32_t ny = 1u << op.ry;
  for (uint32_t c = team.tid; c < nout; c += team.size) {
    uint32_t oa = 0, ob = 0;
    for (int i = 0; i < op.rc; ++i) {
      const uint32_t bit = (c >> i) & 1u;
      if (op.p1[i] != kAbsent) oa |= bit << op.p1[i];
      if (op.p2[i] != kAbsent) ob |= bit << op.p2[i];
    }
    T acc = czero<T>();
    for (uint32_t y = 0; y < ny; ++y) {
      uint32_t ya = 0, yb = 0;
      for (int j = 0; j < op.ry; ++j) {
        const uint32_t bit = (y >> j) & 1u;
        if (op.y1[j] != kAbsent) ya |= bit << op.y1[j];
        if (op.y2[j] != kAbsent) yb |= bit << op.y2[j];
      }
      acc = cfma(a[oa | ya], b[ob | yb], acc);
    }
    out[c] = acc;
  }
}

}  // namespace qtc
