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

__device__ __forceinline__ void sincos_r(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

// Values (and derivatives with respect to params[slot]) of one gate table
// entry, element index bit k = label k (see LeafKind), written straight into
// val and der (der may be null: no derivative wanted).  The angle is formed in
// FP64; sine and cosine are taken in the element precision (FP32 for
// complex64: GB300's FP64 pipe is slow, and the tensor is stored in FP32).
template <typename T>
__device__ inline void gate_tensor(const GateSpec& s, const double* params, T* val, T* der_out) {
  T scratch[16];
  T* der = der_out ? der_out : scratch;
  using R = decltype(T::x);
  const double theta = s.constant + (s.slot >= 0 ? s.coeff * params[s.slot] : 0.0);
  const R dth = s.slot >= 0 ? (R)s.coeff : R(0);  // d theta / d param
  const int rank = leaf_rank_of(s.kind);
  const int n = 1 << rank;
  for (int i = 0; i < n; ++i) {
    val[i] = T{R(0), R(0)};
    der[i] = T{R(0), R(0)};
  }
  const R r = R(0.70710678118654752440);
  const R half = R(0.5);
  R sh, ch;
  sincos_r((R)(0.5 * theta), &sh, &ch);
  switch (s.kind) {
    case LK_ZERO: case LK_PROJ0: val[0].x = R(1); break;
    case LK_PROJ1: val[1].x = R(1); break;
    case LK_PLUS: val[0].x = r; val[1].x = r; break;
    case LK_ZDIAG: val[0].x = R(1); val[1].x = R(-1); break;
    case LK_H:
      for (int i = 0; i < 4; ++i) val[i].x = (i == 3) ? -r : r;
      break;
    case LK_X: case LK_OBS_X: val[2].x = R(1); val[1].x = R(1); break;
    case LK_Y: case LK_OBS_Y:
      val[2].y = R(-1);  // [0][1] = -i  (index out=0 | in=1 << 1)
      val[1].y = R(1);   // [1][0] = +i
      break;
    case LK_Z: case LK_OBS_Z: val[0].x = R(1); val[3].x = R(-1); break;
    case LK_RX:  // cos(t/2) I - i sin(t/2) X, [out, in]
      val[0].x = ch; val[3].x = ch; val[1].y = -sh; val[2].y = -sh;
      der[0].x = -half * sh * dth; der[3].x = -half * sh * dth;
      der[1].y = -half * ch * dth; der[2].y = -half * ch * dth;
      break;
    case LK_RZ: case LK_RZDIAG: {
      // diag(exp(-i t/2), exp(+i t/2)); dense form at [0][0] and [1][1]
      const int i1 = s.kind == LK_RZ ? 3 : 1;
      val[0] = T{ch, -sh};
      val[i1] = T{ch, sh};
      der[0] = T{-half * sh * dth, -half * ch * dth};
      der[i1] = T{-half * sh * dth, half * ch * dth};
      break;
    }
    case LK_ZZDIAG: case LK_ZZ:
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const R zz = (a == b) ? R(1) : R(-1);  // z_a z_b
          const int idx = s.kind == LK_ZZDIAG ? (a | b << 1) : (a | b << 1 | a << 2 | b << 3);
          val[idx] = T{ch, -zz * sh};  // exp(-i zz t/2)
          // d/dt = -i zz/2 * value
          der[idx] = T{-half * sh * dth, -half * zz * ch * dth};
        }
      break;
    case LK_CNOT:
      for (int c = 0; c < 2; ++c)
        for (int t = 0; t < 2; ++t) val[c | (t ^ c) << 1 | c << 2 | t << 3].x = R(1);
      break;
    case LK_OBS_I: val[0].x = R(1); val[3].x = R(1); break;
    case LK_ONES: val[0].x = R(1); val[1].x = R(1); break;
    case LK_OBS_P0: val[0].x = R(1); break;
    case LK_OBS_P1: val[3].x = R(1); break;
    case LK_CNOTX:  // [t_out, c, t_in]: 1 where t_out = t_in xor c
      for (int i = 0; i < 8; ++i) val[i].x = ((i & 1) == (((i >> 1) ^ (i >> 2)) & 1)) ? R(1) : R(0);
      break;
    case LK_DEPOL: case LK_DEPHASE: case LK_AMPDAMP: {
      // sum_k K[ko][ki] conj(K[bo][bi]) at index ko | bo<<1 | ki<<2 | bi<<3, in
      // closed form (all real): depolarizing (1-s) I(x)I + s/3 (XX* + YY* + ZZ*),
      // dephasing (1-s) I(x)I + s ZZ*, amplitude damping K0 K0* + K1 K1*
      const R st = (R)s.constant;
      for (int i = 0; i < 16; ++i) {
        const int ko = i & 1, bo = (i >> 1) & 1, ki = (i >> 2) & 1, bi = (i >> 3) & 1;
        const bool keep = ko == ki && bo == bi;
        const R zz = (ko ^ bo) ? R(-1) : R(1);   // Z[ko][ko] Z[bo][bo]
        R v = R(0);
        if (s.kind == LK_DEPOL) {
          if (keep) v = (R(1) - st) + st / R(3) * zz;
          else if (ko != ki && bo != bi && ko == bo) v = R(2) * st / R(3);  // XX* + YY*
        } else if (s.kind == LK_DEPHASE) {
          if (keep) v = (R(1) - st) + st * zz;
        } else {
          if (keep) v = (ko ? sqrt(R(1) - st) : R(1)) * (bo ? sqrt(R(1) - st) : R(1));
          else if (ko == 0 && bo == 0 && ki == 1 && bi == 1) v = st;
        }
        val[i].x = v;
      }
      break;
    }
    default:
      break;
  }
  if (s.conj)
    for (int i = 0; i < n; ++i) {
      val[i].y = -val[i].y;
      der[i].y = -der[i].y;
    }
}

// Writes every gate table entry (values, and derivatives for parameterised
// entries) into the table at the start of shared memory; all threads of the
// CTA take part.
template <typename T>
__device__ __forceinline__ void build_gate_table(const GateEntryDev* gates, int n_gates,
                                                 const double* params, T* table,
                                                 const GateEntryDev* inline_gates = nullptr,
                                                 int n_inline = 0) {
  for (int e = threadIdx.x; e < n_gates; e += blockDim.x) {
    const GateEntryDev g = e < n_inline ? inline_gates[e] : gates[e];
    gate_tensor<T>(g.spec, params, table + g.val_off,
                   g.spec.slot >= 0 ? table + g.der_off : nullptr);
  }
}

// Sum of v over aligned groups of `width` lanes (a power of two <= 32); every
// lane of the group receives it.
template <typename T>
__device__ __forceinline__ T warp_csum(T v, uint32_t width) {
  for (uint32_t off = 1; off < width; off <<= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// One warp: grad[2 slot], grad[2 slot + 1] += sum_j g[j] * d[j] over cnt
// terms (at most 16 for a leaf), in the element precision.  grad holds one
// network's partial derivatives; the sums over networks are taken in FP64.
template <typename T, typename G>
__device__ __forceinline__ void warp_leaf_dot(const T* g, const T* d, uint32_t cnt,
                                              uint32_t lane, G* grad, uint32_t slot) {
  T acc = czero<T>();
  for (uint32_t j = lane; j < cnt; j += 32) acc = cfma(g[j], d[j], acc);
  acc = warp_csum(acc, cnt < 32 ? cnt : 32u);
  if (lane == 0) {
    grad[2 * slot] += (G)acc.x;
    grad[2 * slot + 1] += (G)acc.y;
  }
}

// Explicit shared-memory accesses on 32-bit shared addresses (the warp
// program loop addresses its operands this way, never through generic
// pointers).  Ordered with respect to barriers and each other.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
template <typename T> __device__ __forceinline__ T lds_c(uint32_t a);
template <> __device__ __forceinline__ float2 lds_c<float2>(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
template <> __device__ __forceinline__ double2 lds_c<double2>(uint32_t a) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts_c(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts_c(uint32_t a, double2 v) {
  asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only) and the wait for all
// of this thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Adds one to a counter with acquire-release semantics at GPU scope and
// returns the old value.  Called by one thread after a CTA barrier, it
// publishes the writes of the whole CTA (the barrier orders them before it)
// and, for the CTA that sees the last count, makes every other CTA's
// published writes visible.
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

constexpr int kReduceThreads = 128;   // threads of the final reduction

// Final reduction of the last CTA (threads < kReduceThreads take part; all
// threads of the CTA must call it): <C> = sum_e w_e (1 - Re s_e)/2 and
// d<C>/dparam_q = -1/2 sum_e w_e Re ds_e/dparam_q (Section 4.1), in FP64, one
// pass over the per-network rows (stride 2 + 2P: s_e, then ds_e/dparam as
// complex pairs).  out = [<C>, gradient (P), Re s_e per network (N)].
// s_part holds (1 + P) * kReduceThreads / 32 doubles.
__device__ inline void reduce_network_rows(const volatile double* res, const double* weights,
                                           int N, int P, bool qaoa_reduce, double* out,
                                           double* s_part) {
  constexpr int kW = kReduceThreads / 32;
  const int stride = 2 + 2 * P;
  const int nq = 1 + P;
  const int tid = threadIdx.x;
  if (tid < kReduceThreads) {
    for (int q0 = 0; q0 < nq; q0 += 8) {
      double part[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) part[i] = 0.0;
      for (int e = tid; e < N; e += kReduceThreads) {
        const double w = weights[e];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int q = q0 + i;
          if (q == 0)
            part[i] += w * 0.5 * (1.0 - res[(size_t)e * stride]);
          else if (q < nq)
            part[i] += -0.5 * w * res[(size_t)e * stride + 2 + 2 * (q - 1)];
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (q0 + i >= nq) break;
        double v = part[i];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0) s_part[(q0 + i) * kW + tid / 32] = v;
      }
    }
    for (int e = tid; e < N; e += kReduceThreads) out[1 + P + e] = res[(size_t)e * stride];
  }
  __syncthreads();
  for (int q = tid; q < nq; q += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kW; ++w) t += s_part[q * kW + w];
    out[q] = qaoa_reduce ? t : 0.0;
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
