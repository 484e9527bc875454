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
// handles outputs c = 32 j + lane (j < 2^(rc - 5), up to 64 for rank 11).
// Ops with zero or one summed bit (most of them) take straight-line paths
// whose operand loads issue together.  With WOPF_LEAFGRAD the op also adds
// sum_c out[c] * der[c] to the parameter gradient (the leaf-gradient dot of
// the adjoint, fused).
template <typename T>
__device__ __forceinline__ void warp_contract(const WOp& op, const uint4 head, T* out,
                                              const T* a, const T* b, const T* table,
                                              decltype(T::x)* grad, uint32_t lane) {
  const uint32_t rc = (head.x >> 8) & 0xffu, ry = (head.x >> 16) & 0xffu;
  const bool leafgrad = ((head.x >> 24) & WOPF_LEAFGRAD) != 0;
  const uint32_t nout = 1u << rc, ny = 1u << ry;
  const uint32_t alo = op.a_lo[lane], blo = op.b_lo[lane];
  const uint32_t ay1 = op.ya[1], by1 = op.yb[1];
  const uint32_t nj = (nout + 31) >> 5;
  T dot = czero<T>();
  if (ry <= 1) {
    // four output chunks at a time: their operand loads issue together
    for (uint32_t j0 = 0; j0 < nj; j0 += 4) {
      T a0[4], b0[4], a1[4], b1[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t j = j0 + u < nj ? j0 + u : j0;
        const uint32_t oa = alo | op.a_hi[j], ob = blo | op.b_hi[j];
        a0[u] = a[oa];
        b0[u] = b[ob];
        a1[u] = a[oa | ay1];
        b1[u] = b[ob | by1];
      }
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t c = 32 * (j0 + u) + lane;
        T acc = cfma(a0[u], b0[u], czero<T>());
        if (ry == 1) acc = cfma(a1[u], b1[u], acc);
        if (j0 + u < nj && c < nout) {
          out[c] = acc;
          if (leafgrad) dot = cfma(acc, table[(head.w & 0xffffu) + c], dot);
        }
      }
    }
  } else {
    // 4..256 summed terms (ny a power of two >= 4): four accumulators, the
    // loads of four terms issued together
    for (uint32_t j = 0; j < nj; ++j) {
      const uint32_t c = 32 * j + lane;
      const uint32_t oa = alo | op.a_hi[j];
      const uint32_t ob = blo | op.b_hi[j];
      T acc4[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
      for (uint32_t y = 0; y < ny; y += 4) {
        T av[4], bv[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
          const uint32_t yy = y + u;
          av[u] = a[oa | op.ya[yy & 15] | op.ya_hi[yy >> 4]];
          bv[u] = b[ob | op.yb[yy & 15] | op.yb_hi[yy >> 4]];
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) acc4[u] = cfma(av[u], bv[u], acc4[u]);
      }
      T acc = acc4[0];
#pragma unroll
      for (uint32_t u = 1; u < 4; ++u) {
        acc.x += acc4[u].x;
        acc.y += acc4[u].y;
      }
      if (c < nout) {
        out[c] = acc;
        if (leafgrad) dot = cfma(acc, table[(head.w & 0xffffu) + c], dot);
      }
    }
  }
  if (leafgrad) {
    dot = warp_csum(dot, nout < 32 ? nout : 32u);
    if (lane == 0) {
      const uint32_t slot = head.z >> 16;
      grad[2 * slot] += dot.x;
      grad[2 * slot + 1] += dot.y;
    }
  }
}

// One bundle step of a warp program: every lane computes its own output
// element (one or two summed terms, Eq. 1) of the op its lane group belongs
// to.  Leaf-gradient lanes form out * d(leaf)/dparam (or the plain product);
// with few parameters each lane adds its term to its own accumulator of the
// slot (lacc_s: this lane's column, one row of 32 per slot), otherwise the
// lane group sums with shuffles and its first lane adds the sum to the slot.
// Every offset counts elements from base_s, the warp's gate-table copy, which
// its arena follows.  All shared-memory loads of the step issue before any
// arithmetic (one round trip per step): lanes without a second term read
// their first operands again (ya1 = yb1 = 0), lanes without a leaf
// derivative read table element 0, and lanes that add no leaf-gradient term
// read the accumulator of slot 0.
// Ops summing four to sixteen terms spread them over lane pairs (two terms
// a lane) and add the pairs with `prounds` shuffle rounds (the step's most).
template <typename T>
__device__ __forceinline__ void warp_bundle(const uint4 L, uint32_t rounds, uint32_t prounds,
                                            uint32_t base_s, decltype(T::x)* grad,
                                            uint32_t lacc_s, bool lane_grad, uint32_t n_params,
                                            uint32_t res_s, uint32_t lane) {
  constexpr uint32_t kE = sizeof(T);
  const uint32_t kind = L.x & 0xffu, flags = (L.x >> 8) & 0xffu;
  const uint32_t gwp = (L.x >> 16) & 0xffu, slot = L.x >> 24;
  const uint32_t gw = gwp & 7u;
  const uint32_t pa = base_s + (L.y >> 16) * kE, pb = base_s + (L.z & 0xffffu) * kE;
  const uint32_t pl = lacc_s + (slot < n_params ? slot : 0u) * (32u * kE);
  const T a0 = lds_c<T>(pa), b0 = lds_c<T>(pb);
  const T a1 = lds_c<T>(pa + (L.w & 0xffffu) * kE), b1 = lds_c<T>(pb + (L.w >> 16) * kE);
  const T d = lds_c<T>(base_s + (L.z >> 16) * kE);
  T s = czero<T>();
  if (lane_grad) s = lds_c<T>(pl);
  T acc = cfma(a0, b0, czero<T>());
  if (flags & WLF_Y1) acc = cfma(a1, b1, acc);
  if (prounds) {
    const uint32_t pd = (gwp >> 3) & 7u, pr = gwp >> 6;
    for (uint32_t r = 0; r < prounds; ++r) {
      const decltype(T::x) ox = __shfl_xor_sync(0xffffffffu, acc.x, 1u << (pd + r));
      const decltype(T::x) oy = __shfl_xor_sync(0xffffffffu, acc.y, 1u << (pd + r));
      if (r < pr) {
        acc.x += ox;
        acc.y += oy;
      }
    }
  }
  if (kind == WL_SEED) acc = from_d2<T>(make_double2(1.0, 0.0));
  if (flags & WLF_STORE) sts_c(base_s + (L.y & 0xffffu) * kE, acc);
  if (kind == WL_RESULT) sts_c(res_s, to_d2(a0));
  if (rounds & kWHasLeafGrad) {
    T v = czero<T>();
    if (flags & WLF_LG_MUL) v = cfma(acc, d, v);
    else if (flags & WLF_LG_ADD) v = acc;
    if (lane_grad) {
      if (flags & (WLF_LG_MUL | WLF_LG_ADD)) {
        s.x += v.x;
        s.y += v.y;
        sts_c(pl, s);
      }
      return;
    }
    for (uint32_t r = 0; r < (rounds & 0x7fu); ++r) {
      const decltype(T::x) ox = __shfl_xor_sync(0xffffffffu, v.x, 1u << r);
      const decltype(T::x) oy = __shfl_xor_sync(0xffffffffu, v.y, 1u << r);
      if (r < gw) {
        v.x += ox;
        v.y += oy;
      }
    }
    if ((flags & (WLF_LG_MUL | WLF_LG_ADD)) && (lane & ((1u << gw) - 1u)) == 0) {
      atomicAdd(&grad[2 * slot], v.x);
      atomicAdd(&grad[2 * slot + 1], v.y);
    }
  }
}

// A warp team's own copy of the gate table.  With at most 32 gates, lane g
// takes the sine and cosine of gate g's half angle; every element is then one
// complex multiply-add of its coefficient record with its gate's pair,
// shuffled from that lane (the same code for every kind; the records of 128
// elements are loaded before any is used).  Otherwise the lanes stride over
// the gates in closed form.
template <typename T>
__device__ __forceinline__ void build_warp_gate_table(const ProgramDev& prog, T* table,
                                                      uint32_t table_s, uint32_t lane) {
  using R = decltype(T::x);
  using Rec = typename std::conditional<sizeof(R) == 4, TabCoef32, TabCoef64>::type;
  if (prog.n_gates > 32 || prog.coef == nullptr) {
    for (int e = (int)lane; e < prog.n_gates; e += 32) {
      const GateEntryDev g = e < kInlineGates ? prog.gates_inline[e] : prog.gates[e];
      gate_tensor<T>(g.spec, prog.params, table + g.val_off,
                     g.spec.slot >= 0 ? table + g.der_off : nullptr);
    }
    return;
  }
  const Rec* rec = static_cast<const Rec*>(prog.coef);
  const uint32_t ne = prog.table_elems;
  // One memory round trip before the sines: the first 128 records, the
  // lane's gate entry and the parameters (lane k holds params[k] and
  // params[k + 32], shuffled to the gates that use them) load together.
  Rec r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t j = 32 * k + lane;
    r[k] = j < ne ? rec[j] : Rec{};
  }
  const int P = prog.n_params;
  double p_lo = 0.0, p_hi = 0.0;
  if (prog.n_inline_params > 0) {
    // passed by value (host-pointer calls): lane k selects entry k
#pragma unroll
    for (int k = 0; k < kInlineParams; ++k)
      if ((int)lane == k && k < prog.n_inline_params) p_lo = prog.params_inline[k];
  } else {
    p_lo = (int)lane < P ? prog.params[lane] : 0.0;
    p_hi = (int)lane + 32 < P ? prog.params[lane + 32] : 0.0;
  }
  GateSpec spec{};
  spec.slot = -1;
  if ((int)lane < prog.n_gates)
    spec = ((int)lane < kInlineGates ? prog.gates_inline[lane] : prog.gates[lane]).spec;
  const int slot = spec.slot < 0 ? 0 : spec.slot;
  const double v_lo = __shfl_sync(0xffffffffu, p_lo, slot & 31);
  const double v_hi = __shfl_sync(0xffffffffu, p_hi, slot & 31);
  R c = R(1), s = R(0);
  if ((int)lane < prog.n_gates) {
    const double theta =
        spec.constant + (spec.slot >= 0 ? spec.coeff * (slot < 32 ? v_lo : v_hi) : 0.0);
    sincos_r((R)(0.5 * theta), &s, &c);
  }
  for (uint32_t j0 = 0; j0 < ne; j0 += 128) {
    if (j0 > 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t j = j0 + 32 * k + lane;
        r[k] = j < ne ? rec[j] : Rec{};
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t j = j0 + 32 * k + lane;
      const R cj = __shfl_sync(0xffffffffu, c, r[k].gate & 31u);
      const R sj = __shfl_sync(0xffffffffu, s, r[k].gate & 31u);
      T v;
      v.x = fma((R)r[k].a[0], cj, fma((R)r[k].a[2], sj, (R)r[k].a[4]));
      v.y = fma((R)r[k].a[1], cj, fma((R)r[k].a[3], sj, (R)r[k].a[5]));
      if (j < ne) sts_c(table_s + j * (uint32_t)sizeof(T), v);
    }
  }
}

// Read-only loads of streamed warp steps (global memory, not written while
// the kernel runs).
__device__ __forceinline__ uint4 ldg_u4(const void* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ uint32_t ldg_u32(const void* p) {
  return __ldg(reinterpret_cast<const unsigned int*>(p));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Streamed steps: the queue holds steps k .. k + 3 in registers; step
// k + kStreamAhead is prefetched into L2 so that the queue's loads hit it.
constexpr uint32_t kStreamAhead = 16;

// kStream (warp teams whose step lists do not fit shared memory beside their
// arenas): steps are read from global memory through a four-deep register
// queue per lane (header word and the lane's descriptor) instead of being
// staged; a solo step's op is read where it lies.
template <typename T, bool kWarp, bool kStream = false>
__global__ void __maxnreg__(kExecMaxRegs) smem_exec_kernel(const ProgramDev prog) {
  using R = decltype(T::x);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one network's partial derivatives per team, in the element precision
  __shared__ R s_grad[kMaxTeams][2 * kMaxParams];
  __shared__ unsigned int s_task[kMaxTeams];
  __shared__ double2 s_res[kMaxTeams];   // the network's scalar, per team
  __shared__ int s_last[kMaxTeams];

  // A CTA team reads the gate table at the start of shared memory; a warp
  // team keeps its own copy between its staged steps and its arena, so its
  // table and arena offsets run on from one another.
  using OpT = typename std::conditional<kWarp, WStep, SOp>::type;
  const Team<kWarp> team;
  const int P = prog.n_params;
  const int teams_per_cta = blockDim.x / team.size;
  unsigned char* team_base = smem_raw + prog.table_bytes + (size_t)team.id * prog.team_bytes;
  OpT* stage = reinterpret_cast<OpT*>(team_base);
  T* after_stage = reinterpret_cast<T*>(team_base + (size_t)prog.stage_ops * sizeof(OpT));
  const bool lane_grad = kWarp && prog.want_grad && P <= kWarpLaneGradSlots;
  T* table = kWarp ? after_stage + (lane_grad ? 32 * P : 0) : reinterpret_cast<T*>(smem_raw);
  T* arena = kWarp ? table + prog.table_elems : after_stage;
  const OpT* ops = kWarp ? reinterpret_cast<const OpT*>(prog.wsteps)
                         : reinterpret_cast<const OpT*>(prog.ops);
  R* grad = s_grad[team.id];
  const int stride = 2 + 2 * P;
  constexpr int kWords = sizeof(OpT) / sizeof(uint4);
  const uint32_t stage_s = smem_u32(stage), table_s = smem_u32(table);
  const uint32_t lacc_s = smem_u32(after_stage) + team.tid * (uint32_t)sizeof(T);
  const uint32_t res_s = smem_u32(&s_res[team.id]);

  // Each team's first network is fixed by its position (no queue round
  // trip); its first op chunk is copied asynchronously while the gate table
  // (leaf values and derivatives) is built.  Later networks come from the
  // queue, numbered after the statically assigned ones.
  unsigned int t = blockIdx.x * teams_per_cta + team.id;
  TaskDev task{};
  // streamed steps: the register queue (steps k .. k + 3 of the current task)
  uint32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;
  uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0, q2 = q0, q3 = q0;
  bool primed = false;
  if (kStream && t < (unsigned)prog.n_tasks) {
    // with a fixed stride the first steps are read before the task record
    // arrives (only within the task's own stride)
    if (prog.task_stride) {
      const WStep* gs = prog.wsteps + (size_t)t * prog.task_stride;
      const uint32_t m = min(prog.task_stride, 4u);
      if (m > 0) { h0 = ldg_u32(&gs[0]); q0 = ldg_u4(&gs[0].lane[team.tid]); }
      if (m > 1) { h1 = ldg_u32(&gs[1]); q1 = ldg_u4(&gs[1].lane[team.tid]); }
      if (m > 2) { h2 = ldg_u32(&gs[2]); q2 = ldg_u4(&gs[2].lane[team.tid]); }
      if (m > 3) { h3 = ldg_u32(&gs[3]); q3 = ldg_u4(&gs[3].lane[team.tid]); }
      primed = true;
    }
    task = prog.tasks[t];
  } else if (t < (unsigned)prog.n_tasks) {
    uint4* dst = reinterpret_cast<uint4*>(stage);
    if (kWarp && prog.task_stride) {
      // fixed stride: the copy starts before the task record arrives
      const uint4* src = reinterpret_cast<const uint4*>(ops + (size_t)t * prog.task_stride);
      for (uint32_t w = team.tid; w < prog.stage_ops * kWords; w += team.size)
        cp_async16(dst + w, src + w);
      task = prog.tasks[t];
    } else {
      task = prog.tasks[t];
      const uint32_t n = min(prog.stage_ops, task.op_count);
      const uint4* src = reinterpret_cast<const uint4*>(ops + task.op_begin);
      for (uint32_t w = team.tid; w < n * kWords; w += team.size) cp_async16(dst + w, src + w);
    }
  }
  if (kWarp)
    build_warp_gate_table<T>(prog, table, table_s, team.tid);
  else
    build_gate_table<T>(prog.gates, prog.n_gates, prog.params, table, prog.gates_inline,
                        kInlineGates);
  cp_async_wait_all();
  team.sync();  // a warp team's table and steps are its own
  bool staged = true;
  while (t < (unsigned)prog.n_tasks) {
    const double w_net = prog.weights[task.net];  // used once the network is done
    for (int i = team.tid; i < 2 * P; i += team.size) grad[i] = R(0);
    if (lane_grad)
      for (int q = 0; q < P; ++q) sts_c(lacc_s + q * 32u * (uint32_t)sizeof(T), czero<T>());
    if constexpr (kStream) {
      const WStep* gs = prog.wsteps + task.op_begin;
      const uint32_t n = task.op_count;
      if (!primed) {
        if (n > 0) { h0 = ldg_u32(&gs[0]); q0 = ldg_u4(&gs[0].lane[team.tid]); }
        if (n > 1) { h1 = ldg_u32(&gs[1]); q1 = ldg_u4(&gs[1].lane[team.tid]); }
        if (n > 2) { h2 = ldg_u32(&gs[2]); q2 = ldg_u4(&gs[2].lane[team.tid]); }
        if (n > 3) { h3 = ldg_u32(&gs[3]); q3 = ldg_u4(&gs[3].lane[team.tid]); }
      }
      primed = false;
      for (uint32_t k = 4; k < min(n, kStreamAhead); ++k) prefetch_l2(&gs[k].lane[team.tid]);
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t h = h0;  // solo | rounds << 8
        const uint4 L = q0;
        h0 = h1; q0 = q1;
        h1 = h2; q1 = q2;
        h2 = h3; q2 = q3;
        if (k + 4 < n) {
          h3 = ldg_u32(&gs[k + 4]);
          q3 = ldg_u4(&gs[k + 4].lane[team.tid]);
        }
        if (k + kStreamAhead < n) prefetch_l2(&gs[k + kStreamAhead].lane[team.tid]);
        if (!(h & 0xffu)) {
          warp_bundle<T>(L, (h >> 8) & 0xffu, (h >> 16) & 0xffu, table_s, grad, lacc_s,
                         lane_grad, (uint32_t)P, res_s, team.tid);
        } else {
          // solo step, its op read in place
          const WOp& w = gs[k].op;
          const uint4 head = ldg_u4(&w);
          const uint32_t code = head.x & 0xffu;
          T* out = resolve<T>(head.y & 0xffffu, table, arena, prog.table_elems);
          T* in1 = resolve<T>(head.y >> 16, table, arena, prog.table_elems);
          T* in2 = resolve<T>(head.z & 0xffffu, table, arena, prog.table_elems);
          if (code == SOP_CONTRACT) {
            warp_contract<T>(w, head, out, in1, in2, table, grad, team.tid);
          } else if (code == SOP_LEAFGRAD) {
            warp_leaf_dot<T>(in1, in2, 1u << ((head.x >> 8) & 0xffu), team.tid, grad,
                             head.z >> 16);
          } else if (code == SOP_RESULT) {
            if (team.tid == 0) s_res[team.id] = to_d2(*in1);
          } else if (code == SOP_SEED) {
            if (team.tid == 0) *out = from_d2<T>(make_double2(1.0, 0.0));
          }
        }
        team.sync();
      }
    }
    for (uint32_t base = 0; !kStream && base < task.op_count; base += prog.stage_ops) {
      const uint32_t n = min(prog.stage_ops, task.op_count - base);
      if (!staged) {
        // stage a chunk of the op list with one cooperative copy
        team.sync();
        const uint4* src = reinterpret_cast<const uint4*>(ops + task.op_begin + base);
        uint4* dst = reinterpret_cast<uint4*>(stage);
        for (uint32_t w = team.tid; w < n * kWords; w += team.size) dst[w] = src[w];
      }
      staged = false;
      team.sync();
      // warp programs: the next step's header and this lane's descriptor are
      // loaded while the current step runs
      uint32_t h_next = 0;
      uint4 l_next = make_uint4(0, 0, 0, 0);
      if (kWarp) {
        h_next = lds_u32(stage_s);
        l_next = lds_u4(stage_s + 16 + 16 * team.tid);
      }
      for (uint32_t k = 0; k < n; ++k) {
        const OpT& op = stage[k];
        if constexpr (kWarp) {
          const uint32_t h = h_next;  // solo | rounds << 8
          const uint4 L = l_next;
          if (k + 1 < n) {
            const uint32_t nxt = stage_s + (k + 1) * (uint32_t)sizeof(WStep);
            h_next = lds_u32(nxt);
            l_next = lds_u4(nxt + 16 + 16 * team.tid);
          }
          if (!(h & 0xffu)) {
            warp_bundle<T>(L, (h >> 8) & 0xffu, (h >> 16) & 0xffu, table_s, grad, lacc_s,
                           lane_grad, (uint32_t)P, res_s, team.tid);
          } else {
            // solo step; header word: code, rc, ry, flags | out, in1 | in2, slot | der
            const WOp& w = op.op;
            const uint4 head = *reinterpret_cast<const uint4*>(&w);
            const uint32_t code = head.x & 0xffu;
            T* out = resolve<T>(head.y & 0xffffu, table, arena, prog.table_elems);
            T* in1 = resolve<T>(head.y >> 16, table, arena, prog.table_elems);
            T* in2 = resolve<T>(head.z & 0xffffu, table, arena, prog.table_elems);
            if (code == SOP_CONTRACT) {
              warp_contract<T>(w, head, out, in1, in2, table, grad, team.tid);
            } else if (code == SOP_LEAFGRAD) {
              warp_leaf_dot<T>(in1, in2, 1u << ((head.x >> 8) & 0xffu), team.tid, grad,
                               head.z >> 16);
            } else if (code == SOP_RESULT) {
              if (team.tid == 0) s_res[team.id] = to_d2(*in1);
            } else if (code == SOP_SEED) {
              if (team.tid == 0) *out = from_d2<T>(make_double2(1.0, 0.0));
            }
          }
        } else {
          switch (op.code) {
            case SOP_CONTRACT:
              contract_op<T>(op, resolve(op.out, table, arena, prog.table_elems),
                             resolve(op.in1, table, arena, prog.table_elems),
                             resolve(op.in2, table, arena, prog.table_elems), team);
              break;
            case SOP_LEAFGRAD:
              if (team.tid < 32)
                warp_leaf_dot<T>(resolve(op.in1, table, arena, prog.table_elems),
                                 resolve(op.in2, table, arena, prog.table_elems), 1u << op.rc,
                                 team.tid, grad, op.out);
              break;
            case SOP_RESULT:
              if (team.tid == 0) s_res[team.id] = to_d2(*resolve(op.in1, table, arena,
                                                                prog.table_elems));
              break;
            case SOP_SEED:
              if (team.tid == 0)
                *resolve(op.out, table, arena, prog.table_elems) =
                    from_d2<T>(make_double2(1.0, 0.0));
              break;
            default:
              break;
          }
        }
        team.sync();
      }
    }
    if (lane_grad) {
      // sum the lanes' accumulators into the network's slots
      for (int q = 0; q < P; ++q) {
        T v = warp_csum(lds_c<T>(lacc_s + q * 32u * (uint32_t)sizeof(T)), 32u);
        if (team.tid == 0) {
          grad[2 * q] += v.x;
          grad[2 * q + 1] += v.y;
        }
      }
      team.sync();
    }
    // the network's row (scalar and derivatives), its entry of the output,
    // and its weighted terms of <C> and of the gradient (Section 4.1) added
    // into the FP64 sums (atomics carried out in L2: the order of the terms
    // over networks is not fixed, so sums can differ in the last bits
    // between runs)
    double* row = prog.results + (size_t)task.net * stride;
    if (team.tid == 0) {
      const double2 sv = s_res[team.id];
      row[0] = sv.x;
      row[1] = sv.y;
      prog.out[1 + P + task.net] = sv.x;
      atomicAdd(&prog.acc[0], 0.5 * w_net * (1.0 - sv.x));
    }
    for (int i = team.tid; i < 2 * P; i += team.size)
      row[2 + i] = prog.want_grad ? (double)grad[i] : 0.0;
    if (prog.want_grad)
      for (int q = team.tid; q < P; q += team.size)
        atomicAdd(&prog.acc[1 + q], -0.5 * w_net * (double)grad[2 * q]);
    // networks beyond the statically assigned ones come from the queue
    const unsigned int n_static = gridDim.x * teams_per_cta;
    if (n_static >= (unsigned)prog.n_tasks) break;
    if (team.tid == 0) s_task[team.id] = n_static + atomicAdd(&prog.counters[0], 1u);
    team.sync();
    t = s_task[team.id];
    if (t < (unsigned)prog.n_tasks) task = prog.tasks[t];
  }

  // A team counts itself out after its last queue fetch (its first thread's
  // release, after the team barrier, covers the team's writes and sums); the
  // last team out copies the sums to the output, clears them and re-arms the
  // counters (no team touches them afterwards).
  team.sync();
  if (team.tid == 0)
    s_last[team.id] = atomic_add_acq_rel(&prog.counters[1], 1u) == gridDim.x * teams_per_cta - 1;
  team.sync();
  if (!s_last[team.id]) return;
  for (int q = team.tid; q <= P; q += team.size) {
    const double v = reinterpret_cast<volatile double*>(prog.acc)[q];
    prog.out[q] = prog.qaoa_reduce ? v : 0.0;
    prog.acc[q] = 0.0;
  }
  if (team.tid == 0) {
    prog.out[1 + P + prog.n_nets] = 0.0;  // status: this executor never waits
    prog.counters[0] = 0;
    prog.counters[1] = 0;
  }
  // Host-polled completion: every lane's writes are fenced at system scope
  // (the other teams' per-network entries are covered by cumulativity: the
  // counter's acquire observed them), then one release store of the sequence
  // number tells the host the output is complete.
  if (prog.done) {
    __threadfence_system();
    team.sync();
    if (team.tid == 0)
      asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(prog.done), "l"(prog.seq)
                   : "memory");
  }
}

template <typename T, bool kWarp, bool kStream>
static const void* kernel_ptr() {
  return (const void*)smem_exec_kernel<T, kWarp, kStream>;
}

// mode: 0 CTA teams, 1 warp teams with staged steps, 2 warp teams with
// streamed steps
template <typename T>
static const void* select_mode(int mode) {
  if (mode == 2) return kernel_ptr<T, true, true>();
  return mode == 1 ? kernel_ptr<T, true, false>() : kernel_ptr<T, false, false>();
}

static const void* select_kernel(int dtype, int mode) {
  return dtype == 0 ? select_mode<double2>(mode) : select_mode<float2>(mode);
}

cudaError_t smem_exec_configure(int dtype, int mode, size_t smem_bytes, size_t max_dynamic,
                                int block, int* blocks_per_sm) {
  const void* fn = select_kernel(dtype, mode);
  // the attribute is per kernel, shared by every prepared program: always
  // raise it to the device limit so a smaller program never lowers it below
  // what a larger one needs
  if (smem_bytes > max_dynamic) return cudaErrorInvalidValue;
  cudaError_t err =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dynamic);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem_bytes);
}

cudaError_t smem_exec_launch(const ProgramDev& prog, int dtype, int mode, int grid, int block,
                             size_t smem_bytes, cudaStream_t stream) {
  if (dtype == 0) {
    if (mode == 2)
      smem_exec_kernel<double2, true, true><<<grid, block, smem_bytes, stream>>>(prog);
    else if (mode == 1)
      smem_exec_kernel<double2, true><<<grid, block, smem_bytes, stream>>>(prog);
    else
      smem_exec_kernel<double2, false><<<grid, block, smem_bytes, stream>>>(prog);
  } else {
    if (mode == 2)
      smem_exec_kernel<float2, true, true><<<grid, block, smem_bytes, stream>>>(prog);
    else if (mode == 1)
      smem_exec_kernel<float2, true><<<grid, block, smem_bytes, stream>>>(prog);
    else
      smem_exec_kernel<float2, false><<<grid, block, smem_bytes, stream>>>(prog);
  }
  return cudaGetLastError();
}

}  // namespace qtc
