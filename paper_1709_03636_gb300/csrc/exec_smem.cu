// Shared-memory network executor.
//
// One CTA contracts one whole network at a time, every tensor held in shared
// memory: the gate tensors are materialised from the parameters (FP64 math,
// stored in the contraction type), then the plan's pairwise contractions
// (Eq. 1, with batch indices for hyperedges) run one after another, then the
// adjoint sweep (when asked) accumulates d(scalar)/d(params).  CTAs take
// networks from a global queue; the last CTA to finish reduces the per-network
// scalars to the Max-Cut objective <C> = sum_e (1 - <Z_u Z_v>_e)/2 of
// Section 4.1 and its gradient, in FP64, and re-arms the counters.
#include <cuda_runtime.h>

#include "device_program.h"
#include "exec_launch.h"

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
__device__ void gate_tensor(const GateSpec& s, const double* params, double2* val,
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

template <typename T, bool kWarp>
__device__ __forceinline__ void contract_op(const SOp& op, T* out, const T* a, const T* b,
                                            const Team<kWarp>& team) {
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

constexpr int kMaxTeams = 8;

template <typename T, bool kWarp>
__global__ void __launch_bounds__(256) smem_exec_kernel(const ProgramDev prog) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_grad[kMaxTeams][2 * kMaxParams];
  __shared__ unsigned int s_task[kMaxTeams];
  __shared__ int s_last;
  __shared__ double s_red[256];
  T* table = reinterpret_cast<T*>(smem_raw);

  // gate table (leaf values) in FP64, stored in the contraction type
  for (int e = threadIdx.x; e < prog.n_gates; e += blockDim.x) {
    const GateEntryDev g = prog.gates[e];
    double2 val[16], der[16];
    gate_tensor(g.spec, prog.params, val, der);
    const int n = 1 << g.rank;
    for (int i = 0; i < n; ++i) {
      table[g.val_off + i] = from_d2<T>(val[i]);
      if (g.spec.slot >= 0) table[g.der_off + i] = from_d2<T>(der[i]);
    }
  }
  __syncthreads();

  const Team<kWarp> team;
  unsigned char* team_base = smem_raw + prog.table_bytes + (size_t)team.id * prog.team_bytes;
  SOp* stage = reinterpret_cast<SOp*>(team_base);
  T* arena = reinterpret_cast<T*>(team_base + (size_t)prog.stage_ops * sizeof(SOp));
  double* grad = s_grad[team.id];
  const int P = prog.n_params;
  const int stride = 2 + 2 * P;
  constexpr int kWords = sizeof(SOp) / sizeof(uint4);
  for (;;) {
    if (team.tid == 0) s_task[team.id] = atomicAdd(&prog.counters[0], 1u);
    for (int i = team.tid; i < 2 * P; i += team.size) grad[i] = 0.0;
    team.sync();
    const unsigned int t = s_task[team.id];
    if (t >= (unsigned)prog.n_tasks) break;
    const TaskDev task = prog.tasks[t];
    for (uint32_t base = 0; base < task.op_count; base += prog.stage_ops) {
      // stage a chunk of the op list with one cooperative copy
      const uint32_t n = min(prog.stage_ops, task.op_count - base);
      const uint4* src = reinterpret_cast<const uint4*>(prog.ops + task.op_begin + base);
      uint4* dst = reinterpret_cast<uint4*>(stage);
      for (uint32_t w = team.tid; w < n * kWords; w += team.size) dst[w] = src[w];
      team.sync();
      for (uint32_t k = 0; k < n; ++k) {
        const SOp& op = stage[k];
        switch (op.code) {
          case SOP_CONTRACT:
            contract_op<T, kWarp>(op, resolve(op.out, table, arena, prog.table_elems),
                                  resolve(op.in1, table, arena, prog.table_elems),
                                  resolve(op.in2, table, arena, prog.table_elems), team);
            break;
          case SOP_LEAFGRAD:
            if (threadIdx.x % team.size < 32) {
              const T* g = resolve(op.in1, table, arena, prog.table_elems);
              const T* d = resolve(op.in2, table, arena, prog.table_elems);
              const uint32_t cnt = 1u << op.rc;
              double2 acc = make_double2(0.0, 0.0);
              for (uint32_t j = threadIdx.x & 31; j < cnt; j += 32) {
                const double2 gj = to_d2(g[j]);
                const double2 dj = to_d2(d[j]);
                acc.x += gj.x * dj.x - gj.y * dj.y;
                acc.y += gj.x * dj.y + gj.y * dj.x;
              }
              for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
              }
              if ((threadIdx.x & 31) == 0) {
                grad[2 * op.out] += acc.x;
                grad[2 * op.out + 1] += acc.y;
              }
            }
            break;
          case SOP_RESULT:
            if (team.tid == 0) {
              const double2 v = to_d2(*resolve(op.in1, table, arena, prog.table_elems));
              prog.results[(size_t)task.net * stride] = v.x;
              prog.results[(size_t)task.net * stride + 1] = v.y;
            }
            break;
          case SOP_SEED:
            if (team.tid == 0)
              *resolve(op.out, table, arena, prog.table_elems) =
                  from_d2<T>(make_double2(1.0, 0.0));
            break;
          default:
            break;
        }
        team.sync();
      }
    }
    for (int i = team.tid; i < 2 * P; i += team.size)
      prog.results[(size_t)task.net * stride + 2 + i] = prog.want_grad ? grad[i] : 0.0;
    team.sync();
  }

  // the last CTA reduces in FP64 and re-arms the counters
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(&prog.counters[1], 1u);
    s_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int N = prog.n_nets;
  const volatile double* res = prog.results;
  // quantities: q = 0 -> <C>, q = 1 + k -> d<C>/dparam_k
  for (int q = 0; q < 1 + P; ++q) {
    double part = 0.0;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
      const double w = prog.weights[e];
      if (q == 0)
        part += w * 0.5 * (1.0 - res[(size_t)e * stride]);
      else
        part += -0.5 * w * res[(size_t)e * stride + 2 + 2 * (q - 1)];
    }
    s_red[threadIdx.x] = part;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off) s_red[threadIdx.x] += s_red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) prog.out[q] = prog.qaoa_reduce ? s_red[0] : 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < N; e += blockDim.x) prog.out[1 + P + e] = res[(size_t)e * stride];
  if (threadIdx.x == 0) {
    prog.counters[0] = 0;
    prog.counters[1] = 0;
  }
}

template <typename T, bool kWarp>
static const void* kernel_ptr() {
  return (const void*)smem_exec_kernel<T, kWarp>;
}

static const void* select_kernel(int dtype, bool warp) {
  if (dtype == 0) return warp ? kernel_ptr<double2, true>() : kernel_ptr<double2, false>();
  return warp ? kernel_ptr<float2, true>() : kernel_ptr<float2, false>();
}

cudaError_t smem_exec_configure(int dtype, bool warp_teams, size_t smem_bytes, size_t max_dynamic,
                                int block, int* blocks_per_sm) {
  const void* fn = select_kernel(dtype, warp_teams);
  // the attribute is per kernel, shared by every prepared program: always
  // raise it to the device limit so a smaller program never lowers it below
  // what a larger one needs
  if (smem_bytes > max_dynamic) return cudaErrorInvalidValue;
  cudaError_t err =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dynamic);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem_bytes);
}

cudaError_t smem_exec_launch(const ProgramDev& prog, int dtype, bool warp_teams, int grid,
                             int block, size_t smem_bytes, cudaStream_t stream) {
  if (dtype == 0) {
    if (warp_teams)
      smem_exec_kernel<double2, true><<<grid, block, smem_bytes, stream>>>(prog);
    else
      smem_exec_kernel<double2, false><<<grid, block, smem_bytes, stream>>>(prog);
  } else {
    if (warp_teams)
      smem_exec_kernel<float2, true><<<grid, block, smem_bytes, stream>>>(prog);
    else
      smem_exec_kernel<float2, false><<<grid, block, smem_bytes, stream>>>(prog);
  }
  return cudaGetLastError();
}

}  // namespace qtc
