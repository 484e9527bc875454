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

#include <type_traits>

#include "device_program.h"
#include "exec_common.cuh"
#include "exec_launch.h"

namespace qtc {

constexpr int kMaxTeams = 8;

// One CONTRACT op of a warp team from its pre-expanded offset tables: lane
// handles outputs c = 32 j + lane.
template <typename T>
__device__ __forceinline__ void warp_contract(const WOp& op, T* out, const T* a, const T* b,
                                              uint32_t lane) {
  const uint32_t nout = 1u << op.rc, ny = 1u << op.ry;
  const uint32_t alo = op.a_lo[lane], blo = op.b_lo[lane];
  for (uint32_t j = 0; 32 * j < nout; ++j) {
    const uint32_t c = 32 * j + lane;
    if (c >= nout) break;
    const uint32_t oa = alo | op.a_hi[j], ob = blo | op.b_hi[j];
    T acc = czero<T>();
    for (uint32_t y = 0; y < ny; ++y) acc = cfma(a[oa | op.ya[y]], b[ob | op.yb[y]], acc);
    out[c] = acc;
  }
}

__device__ __forceinline__ uint32_t op_slot(const WOp& op) { return op.slot; }
__device__ __forceinline__ uint32_t op_slot(const SOp& op) { return op.out; }

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

  using OpT = typename std::conditional<kWarp, WOp, SOp>::type;
  const Team<kWarp> team;
  unsigned char* team_base = smem_raw + prog.table_bytes + (size_t)team.id * prog.team_bytes;
  OpT* stage = reinterpret_cast<OpT*>(team_base);
  T* arena = reinterpret_cast<T*>(team_base + (size_t)prog.stage_ops * sizeof(OpT));
  const OpT* ops = kWarp ? reinterpret_cast<const OpT*>(prog.wops)
                         : reinterpret_cast<const OpT*>(prog.ops);
  double* grad = s_grad[team.id];
  const int P = prog.n_params;
  const int stride = 2 + 2 * P;
  constexpr int kWords = sizeof(OpT) / sizeof(uint4);
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
      const uint4* src = reinterpret_cast<const uint4*>(ops + task.op_begin + base);
      uint4* dst = reinterpret_cast<uint4*>(stage);
      for (uint32_t w = team.tid; w < n * kWords; w += team.size) dst[w] = src[w];
      team.sync();
      for (uint32_t k = 0; k < n; ++k) {
        const OpT& op = stage[k];
        switch (op.code) {
          case SOP_CONTRACT:
            if constexpr (kWarp) {
              warp_contract<T>(op, resolve<T>(op.out, table, arena, prog.table_elems),
                               resolve<T>(op.in1, table, arena, prog.table_elems),
                               resolve<T>(op.in2, table, arena, prog.table_elems), team.tid);
            } else {
              contract_op<T>(op, resolve(op.out, table, arena, prog.table_elems),
                             resolve(op.in1, table, arena, prog.table_elems),
                             resolve(op.in2, table, arena, prog.table_elems), team);
            }
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
                const uint32_t slot = kWarp ? op_slot(op) : op.out;
                grad[2 * slot] += acc.x;
                grad[2 * slot + 1] += acc.y;
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
  if (threadIdx.x == 0) prog.out[1 + P + N] = 0.0;  // status: this executor never waits
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
