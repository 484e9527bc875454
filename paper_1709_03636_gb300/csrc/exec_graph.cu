// Graph executor: networks whose tensors do not fit one CTA's shared memory.
//
// One persistent launch per wave of networks.  The task list holds two kinds
// of tasks, ordered so that every task's producers come earlier:
//  * shared-memory subtree programs (the ops of the shared-memory executor,
//    whose operands may also live in the global work buffer), and
//  * chunks of a global contraction C = sum_y A * B (Eq. 1, batch indices
//    kept) with bit-map addressing: rows of 256 outputs, one per thread, and
//    the summed index tabulated in shared memory; for small outputs with long
//    sums the chunks split the summed index and the last chunk to arrive adds
//    the partial sums in chunk order (deterministic).
// CTAs take tasks in list order and wait for the counters of the task's
// producers.  Every wait is bounded in time: on expiry the CTA sets the error
// flag, and every CTA stops taking tasks once the flag is set.  The last CTA
// of the final wave reduces the per-network rows to the Max-Cut objective
// <C> = sum_e (1 - <Z_u Z_v>_e)/2 (Section 4.1) and its gradient in FP64,
// records the status, and re-arms the counters.
#include <cuda_bf16.h>

#include "exec_common.cuh"
#include "exec_launch.h"
#include "qtc.h"

namespace qtc {

constexpr int kGraphBlock = 256;   // threads per team

// A team of 256 threads runs one task at a time.  The instantiation without
// tensor-core tasks has one team per CTA (4 CTAs per SM); the one with them
// has four teams in a 1024-thread CTA (the runtime keeps one such CTA per
// SM), synchronised with named barriers 1..4.
template <int kTeams>
struct GTeam {
  int tid, size, id;
  __device__ GTeam() : tid(threadIdx.x % kGraphBlock), size(kGraphBlock),
                       id(threadIdx.x / kGraphBlock) {}
  __device__ __forceinline__ void sync() const {
    if (kTeams == 1)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(kGraphBlock) : "memory");
  }
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t runs_offset(const GRuns& r, uint32_t idx) {
  uint32_t off = 0;
  for (int k = 0; k < r.n; ++k) off |= ((idx >> r.src[k]) & ((1u << r.len[k]) - 1u)) << r.dst[k];
  return off;
}

template <typename T> __device__ __forceinline__ T load_l2(const T* p);
template <> __device__ __forceinline__ float2 load_l2<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 load_l2<double2>(const double2* p) {
  return __ldcg(p);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

// Called by the team's first warp: waits until every producer counter of
// `task` reaches its target; false when the error flag is (or becomes) set or
// the bound expires.  Lane i polls producer counter i (32 at a time), so the
// checks cost one memory round trip instead of one per producer; all 32 lanes
// get the same answer.
__device__ bool wait_for_producers_warp(const GraphProgDev& prog, const GTask& task,
                                        uint32_t lane) {
  volatile unsigned* err = prog.counters + CTR_ERROR;
  if (__any_sync(0xffffffffu, *err != 0u)) return false;
  const unsigned long long t0 = now_ns();
  for (uint32_t base = 0; base < task.wait_count; base += 32) {
    const uint32_t i = base + lane;
    const bool mine = i < task.wait_count;
    WaitDev w{};
    if (mine) w = prog.waits[task.wait_begin + i];
    const unsigned* c = prog.counters + ctr_index(mine ? w.counter : 0u);
    unsigned sleep_ns = 64;   // exponential backoff, capped at 1 us
    for (;;) {
      const bool done = !mine || ld_acquire(c) >= w.target;
      if (__all_sync(0xffffffffu, done)) break;
      if (__any_sync(0xffffffffu, *err != 0u)) return false;
      const bool late = (long long)(now_ns() - t0) > prog.wait_limit_ns;
      if (__any_sync(0xffffffffu, late)) {
        if (lane == 0) atomicCAS(prog.counters + CTR_ERROR, 0u, (unsigned)QTC_ERR_TIMEOUT);
        return false;
      }
      __nanosleep(sleep_ns);
      if (sleep_ns < 1024) sleep_ns <<= 1;
    }
  }
  return true;
}

// Publishes the team's writes, then adds to a completion counter.
template <int kTeams>
__device__ __forceinline__ void signal_done(const GraphProgDev& prog, uint32_t ctr,
                                            const GTeam<kTeams>& team) {
  __threadfence();
  team.sync();
  if (team.tid == 0 && ctr != 0xFFFFFFFFu) atomicAdd(prog.counters + ctr_index(ctr), 1u);
}

template <typename T>
__device__ __forceinline__ T* locate(uint32_t off, bool global, T* gbase, T* table, T* arena,
                                     uint32_t table_elems) {
  return global ? gbase + off : resolve(off, table, arena, table_elems);
}

template <typename T, int kTeams>
__device__ void run_smem_task(const GraphProgDev& prog, const GTask& task, T* table,
                              unsigned char* work, double* s_grad, const GTeam<kTeams>& team) {
  const int P = prog.n_params;
  const int stride = 2 + 2 * P;
  for (int i = team.tid; i < 2 * P; i += team.size) s_grad[i] = 0.0;
  SOp* stage = reinterpret_cast<SOp*>(work);
  T* arena = reinterpret_cast<T*>(work + (size_t)prog.stage_ops * sizeof(SOp));
  T* gbase = reinterpret_cast<T*>(prog.gbase);
  constexpr int kWords = sizeof(SOp) / sizeof(uint4);
  for (uint32_t base = 0; base < task.b; base += prog.stage_ops) {
    const uint32_t n = min(prog.stage_ops, task.b - base);
    team.sync();
    const uint4* src = reinterpret_cast<const uint4*>(prog.ops + task.a + base);
    uint4* dst = reinterpret_cast<uint4*>(stage);
    for (uint32_t w = team.tid; w < n * kWords; w += team.size) dst[w] = src[w];
    team.sync();
    for (uint32_t k = 0; k < n; ++k) {
      const SOp& op = stage[k];
      T* out = locate(op.out, (op.flags & SOPF_OUT_GLOBAL) != 0, gbase, table, arena,
                      prog.table_elems);
      T* in1 = locate(op.in1, (op.flags & SOPF_IN1_GLOBAL) != 0, gbase, table, arena,
                      prog.table_elems);
      T* in2 = locate(op.in2, (op.flags & SOPF_IN2_GLOBAL) != 0, gbase, table, arena,
                      prog.table_elems);
      switch (op.code) {
        case SOP_CONTRACT:
          contract_op<T>(op, out, in1, in2, team);
          break;
        case SOP_LEAFGRAD:
          if (team.tid < 32)
            warp_leaf_dot<T>(in1, in2, 1u << op.rc, team.tid, s_grad, op.out);
          break;
        case SOP_RESULT:
          if (team.tid == 0) {
            const double2 v = to_d2(*in1);
            prog.results[(size_t)task.net * stride] = v.x;
            prog.results[(size_t)task.net * stride + 1] = v.y;
          }
          break;
        case SOP_SEED:
          if (team.tid == 0) *out = from_d2<T>(make_double2(1.0, 0.0));
          break;
        default:
          break;
      }
      team.sync();
    }
  }
  for (int i = team.tid; i < 2 * P; i += team.size)
    if (s_grad[i] != 0.0) atomicAdd(&prog.results[(size_t)task.net * stride + 2 + i], s_grad[i]);
  signal_done(prog, task.signal, team);
}

// sum over y = y0, y0 + step, ... < y1 of A[oa | ya[y]] * B[ob | yb[y]] with
// eight independent accumulators, so that eight load pairs are in flight
// (long summed indices are otherwise latency bound); fixed summation order.
template <typename T>
__device__ __forceinline__ T ysum(const T* A, const T* B, uint32_t oa, uint32_t ob,
                                  const uint32_t* ya, const uint32_t* yb, uint32_t y0,
                                  uint32_t y1, uint32_t step) {
  T acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = czero<T>();
  uint32_t y = y0;
  for (; y + 7 * step < y1; y += 8 * step) {
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      const uint32_t yy = y + u * step;
      acc[u] = cfma(A[oa | ya[yy]], B[ob | yb[yy]], acc[u]);
    }
  }
  for (; y < y1; y += step) acc[0] = cfma(A[oa | ya[y]], B[ob | yb[y]], acc[0]);
  return cadd(cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3])),
              cadd(cadd(acc[4], acc[5]), cadd(acc[6], acc[7])));
}

// Rows r0..r1 of a chunk whose summed index has NY values: R rows at a
// time with every term's operands loaded before any product, so R * NY load
// pairs are in flight per thread.  Rows past r1 load row r1 - 1 again and
// store nothing.
template <typename T, uint32_t R, uint32_t NY>
__device__ __forceinline__ void rows_unrolled(const T* A, const T* B, T* C, const uint32_t* rowa,
                                              const uint32_t* rowb, uint32_t a_lo, uint32_t b_lo,
                                              const uint32_t* ya, const uint32_t* yb, uint32_t r0,
                                              uint32_t r1, uint32_t rowlen, uint32_t tid) {
  uint32_t yav[NY], ybv[NY];
#pragma unroll
  for (uint32_t y = 0; y < NY; ++y) {
    yav[y] = ya[y];
    ybv[y] = yb[y];
  }
  for (uint32_t row = r0; row < r1; row += R) {
    T av[R][NY], bv[R][NY];
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t rr = min(row + r, r1 - 1) - r0;
      const uint32_t oa = rowa[rr] | a_lo, ob = rowb[rr] | b_lo;
#pragma unroll
      for (uint32_t y = 0; y < NY; ++y) {
        av[r][y] = A[oa | yav[y]];
        bv[r][y] = B[ob | ybv[y]];
      }
    }
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      T acc = czero<T>();
#pragma unroll
      for (uint32_t y = 0; y < NY; ++y) acc = cfma(av[r][y], bv[r][y], acc);
      if (row + r < r1) C[(row + r) * rowlen + tid] = acc;
    }
  }
}

// Rows of a GSF_ROWS step, four at a time: row k of a group reads A element
// ia(k) and B element ib(k) of the group's distinct ones (GRS_ZX: A varies
// with row bit 1, B with bit 0; GRS_ZZ: one A, four B; GRS_XX: four A, one
// B), two summed values per pass, so a pass issues 8 (ZX) or 10 loads for 8
// terms instead of 16.  nr is a multiple of four; rowc holds each row's
// output offset.
template <typename T, int kShare>
__device__ __forceinline__ void rows_shared(const T* A, const T* B, T* C, const uint32_t* rowa,
                                            const uint32_t* rowb, const uint32_t* rowc,
                                            uint32_t a_lo, uint32_t b_lo, const uint32_t* ya,
                                            const uint32_t* yb, uint32_t nr, uint32_t n_y,
                                            uint32_t tid) {
  constexpr int NA = kShare == GRS_ZZ ? 1 : (kShare == GRS_ZX ? 2 : 4);
  constexpr int NB = kShare == GRS_XX ? 1 : (kShare == GRS_ZX ? 2 : 4);
  auto ia = [](int k) { return kShare == GRS_ZZ ? 0 : (kShare == GRS_ZX ? k >> 1 : k); };
  auto ib = [](int k) { return kShare == GRS_XX ? 0 : (kShare == GRS_ZX ? k & 1 : k); };
  for (uint32_t r = 0; r < nr; r += 4) {
    uint32_t oa[NA], ob[NB];
#pragma unroll
    for (int i = 0; i < NA; ++i) oa[i] = rowa[r + (kShare == GRS_ZX ? 2 * i : i)] | a_lo;
#pragma unroll
    for (int i = 0; i < NB; ++i) ob[i] = rowb[r + i] | b_lo;
    T acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = czero<T>();
    for (uint32_t y = 0; y < n_y; y += 2) {
      const uint32_t ay0 = ya[y], by0 = yb[y], ay1 = ya[y + 1], by1 = yb[y + 1];
      T av[NA][2], bv[NB][2];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        av[i][0] = A[oa[i] | ay0];
        av[i][1] = A[oa[i] | ay1];
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        bv[i][0] = B[ob[i] | by0];
        bv[i][1] = B[ob[i] | by1];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        acc[k] = cfma(av[ia(k)][1], bv[ib(k)][1], cfma(av[ia(k)][0], bv[ib(k)][0], acc[k]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) C[rowc[r + k] + tid] = acc[k];
  }
}

// Rows of a GRS_FIXA / GRS_FIXB step (1, 2 or 4 summed values): groups of 2^G
// rows read the fixed operand S once per summed value and the other operand
// O per row, 2^G x NY loads of O in flight per thread.  Kept out of line so
// its registers do not weigh on the rest of the chunk code.
template <typename T, uint32_t NY, uint32_t G>
__device__ __noinline__ void rows_fixed(const T* S, const T* O, T* C, const uint32_t* rows_s,
                                        const uint32_t* rows_o, const uint32_t* rowc,
                                        uint32_t s_lo, uint32_t o_lo, const uint32_t* ys,
                                        const uint32_t* yo, uint32_t nr, uint32_t tid) {
  constexpr uint32_t NG = 1u << G;
  uint32_t ysv[NY], yov[NY];
#pragma unroll
  for (uint32_t y = 0; y < NY; ++y) {
    ysv[y] = ys[y];
    yov[y] = yo[y];
  }
  for (uint32_t r = 0; r < nr; r += NG) {
    const uint32_t os = rows_s[r] | s_lo;
    T sv[NY], ov[NG][NY];
#pragma unroll
    for (uint32_t y = 0; y < NY; ++y) sv[y] = S[os | ysv[y]];
#pragma unroll
    for (uint32_t k = 0; k < NG; ++k) {
      const uint32_t oo = rows_o[r + k] | o_lo;
#pragma unroll
      for (uint32_t y = 0; y < NY; ++y) ov[k][y] = O[oo | yov[y]];
    }
#pragma unroll
    for (uint32_t k = 0; k < NG; ++k) {
      T acc = czero<T>();
#pragma unroll
      for (uint32_t y = 0; y < NY; ++y) acc = cfma(ov[k][y], sv[y], acc);
      C[rowc[r + k] + tid] = acc;
    }
  }
}

template <typename T>
__device__ __forceinline__ void rows_fixed_dispatch(const T* A, const T* B, T* C,
                                                    const uint32_t* rowa, const uint32_t* rowb,
                                                    const uint32_t* rowc, uint32_t a_lo,
                                                    uint32_t b_lo, const uint32_t* ya,
                                                    const uint32_t* yb, uint32_t nr, uint32_t n_y,
                                                    bool fix_b, uint32_t tid) {
  const T* S = fix_b ? B : A;
  const T* O = fix_b ? A : B;
  const uint32_t* rs = fix_b ? rowb : rowa;
  const uint32_t* ro = fix_b ? rowa : rowb;
  const uint32_t sl = fix_b ? b_lo : a_lo, ol = fix_b ? a_lo : b_lo;
  const uint32_t* ys = fix_b ? yb : ya;
  const uint32_t* yo = fix_b ? ya : yb;
  if (n_y == 1) rows_fixed<T, 1, grs_fix_bits(1)>(S, O, C, rs, ro, rowc, sl, ol, ys, yo, nr, tid);
  else if (n_y == 2) rows_fixed<T, 2, grs_fix_bits(2)>(S, O, C, rs, ro, rowc, sl, ol, ys, yo, nr, tid);
  else rows_fixed<T, 4, grs_fix_bits(4)>(S, O, C, rs, ro, rowc, sl, ol, ys, yo, nr, tid);
}

// ---- tile tasks: footprints staged through shared memory -------------------

// Copies the footprint (2^nf elements) of an operand at element offset
// `base`: footprint index j -> operand element base | ff(j).  Index bit 0 is
// the operand's bit 0, so element pairs (complex64) are contiguous.
template <typename T>
__device__ __forceinline__ void stage_footprint(T* dst, const T* src, uint32_t base,
                                                const GRuns& ff, uint32_t nf, uint32_t tid,
                                                uint32_t nthreads) {
  constexpr uint32_t per = 16 / sizeof(T);   // elements per 16-byte copy
  const uint32_t n = 1u << nf;
  if (per == 2 && nf == 0) {
    if (tid == 0) dst[0] = src[base];
    return;
  }
  for (uint32_t j = tid * per; j < n; j += nthreads * per)
    cp_async16(dst + j, src + (base | runs_offset(ff, j)));
}

template <typename T>
__device__ __forceinline__ T shfl_xor_c(T v, int m);
template <>
__device__ __forceinline__ float2 shfl_xor_c<float2>(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <>
__device__ __forceinline__ double2 shfl_xor_c<double2>(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// The contraction of one outer output value o over outer summed values
// [q0, q1): 2^kOut register accumulators per thread, summed over the tile's
// register-summed bits, then over summed lane and warp bits; the owners
// write the C tile into shared memory (Cs, footprint order).
template <typename T, int kTeams, int kOut>
__device__ void tile_contract(const GStep& st, const T* Ag, const T* Bg, T* As, T* Bs, T* Cs,
                              T* red, const uint2* soff, uint32_t o, uint32_t q0, uint32_t q1,
                              const GTeam<kTeams>& team) {
  const GTileMap& tm = st.tile;
  const bool sa = (tm.staged & 1) != 0, sb = (tm.staged & 2) != 0;
  const uint32_t tid = team.tid, lane = tid & 31u, warp = tid >> 5;
  const uint32_t a_lw = runs_offset(tm.tfa, tid), b_lw = runs_offset(tm.tfb, tid);
  uint32_t ak[1 << kOut], bk[1 << kOut];
#pragma unroll
  for (int k = 0; k < (1 << kOut); ++k) {
    ak[k] = a_lw | runs_offset(tm.tfa, (uint32_t)k << 8);
    bk[k] = b_lw | runs_offset(tm.tfb, (uint32_t)k << 8);
  }
  T acc[1 << kOut];
#pragma unroll
  for (int k = 0; k < (1 << kOut); ++k) acc[k] = czero<T>();
  const uint32_t abase = runs_offset(tm.oa, o), bbase = runs_offset(tm.ob, o);
  const uint32_t ns = 1u << tm.ns;
  for (uint32_t q = q0; q < q1; ++q) {
    const uint32_t aq = abase | runs_offset(tm.qa, q), bq = bbase | runs_offset(tm.qb, q);
    if (sa) stage_footprint(As, Ag, aq, tm.ffa, tm.nfa, tid, team.size);
    if (sb) stage_footprint(Bs, Bg, bq, tm.ffb, tm.nfb, tid, team.size);
    if (sa || sb) {
      cp_async_wait_all();
      team.sync();
    }
    const T* Ab = sa ? As : Ag + aq;
    const T* Bb = sb ? Bs : Bg + bq;
    uint32_t s = 0;
    for (; s + 1 < ns; s += 2) {
      const uint2 o0 = soff[s], o1 = soff[s + 1];
#pragma unroll
      for (int k = 0; k < (1 << kOut); ++k) {
        const T a0 = Ab[ak[k] | o0.x], b0 = Bb[bk[k] | o0.y];
        const T a1 = Ab[ak[k] | o1.x], b1 = Bb[bk[k] | o1.y];
        acc[k] = cfma(a1, b1, cfma(a0, b0, acc[k]));
      }
    }
    for (; s < ns; ++s) {
      const uint2 o0 = soff[s];
#pragma unroll
      for (int k = 0; k < (1 << kOut); ++k) acc[k] = cfma(Ab[ak[k] | o0.x], Bb[bk[k] | o0.y], acc[k]);
    }
    if (sa || sb) team.sync();   // the footprints are refilled (or reused) next
  }
  // summed lane bits: butterfly over those bits, every lane gets the sum
#pragma unroll
  for (int m = 0; m < 5; ++m)
    if ((tm.sum_lane_mask >> m) & 1u) {
#pragma unroll
      for (int k = 0; k < (1 << kOut); ++k) acc[k] = cadd(acc[k], shfl_xor_c(acc[k], 1 << m));
    }
  const bool lane_owner = (lane & tm.sum_lane_mask) == 0;
  if (tm.sum_warp_mask) {
#pragma unroll
    for (int k = 0; k < (1 << kOut); ++k) red[((uint32_t)k << 8) | tid] = acc[k];
    team.sync();
    if ((warp & tm.sum_warp_mask) == 0 && lane_owner) {
#pragma unroll
      for (int k = 0; k < (1 << kOut); ++k) {
        T sum = czero<T>();
        for (uint32_t w2 = 0; w2 < 8; ++w2)
          if ((w2 & ~(uint32_t)tm.sum_warp_mask) == warp) sum = cadd(sum, red[((uint32_t)k << 8) | (w2 << 5) | lane]);
        acc[k] = sum;
      }
    }
  }
  if ((warp & tm.sum_warp_mask) == 0 && lane_owner) {
    const uint32_t c_lw = runs_offset(tm.tfc, tid);
#pragma unroll
    for (int k = 0; k < (1 << kOut); ++k) Cs[c_lw | runs_offset(tm.tfc, (uint32_t)k << 8)] = acc[k];
  }
  team.sync();
}

// A tile whose operands are read where they are (nothing staged): per
// thread the tile offsets are formed once, every outer output value o is
// contracted in registers (global or table loads, lanes over the lead
// operand's lowest bits), reduced over summed lane bits by shuffles and over
// summed warp bits through shared memory, and the owners store their outputs
// to C (or, split, to the chunk's partial slot in C-footprint order)
// directly.  Returns the split arrival like run_tile's staged form.
template <typename T, int kTeams, int kOut>
__device__ void tile_direct(const GStep& st, const GTask& task, const T* Ag, const T* Bg, T* C,
                            T* partial, T* red, const uint2* soff, const GTeam<kTeams>& team) {
  const GTileMap& tm = st.tile;
  const bool split = (st.flags & GSF_SPLIT) != 0;
  const uint32_t tid = team.tid, lane = tid & 31u, warp = tid >> 5;
  const uint32_t a_lw = runs_offset(tm.tfa, tid), b_lw = runs_offset(tm.tfb, tid);
  uint32_t ak[1 << kOut], bk[1 << kOut], ck[1 << kOut];
#pragma unroll
  for (int k = 0; k < (1 << kOut); ++k) {
    const uint32_t t = tid | ((uint32_t)k << 8);
    ak[k] = a_lw | runs_offset(tm.tfa, (uint32_t)k << 8);
    bk[k] = b_lw | runs_offset(tm.tfb, (uint32_t)k << 8);
    const uint32_t fc = runs_offset(tm.tfc, t);   // C-footprint index
    ck[k] = split ? fc : runs_offset(tm.ffc, fc);
  }
  const bool owner = (lane & tm.sum_lane_mask) == 0 && (warp & tm.sum_warp_mask) == 0;
  const uint32_t nq = 1u << tm.nq, no = 1u << tm.no, ns = 1u << tm.ns;
  uint32_t o0, o1, q0, q1;
  if (split) {
    o0 = 0;
    o1 = 1;
    q0 = task.b * tm.q_per_chunk;
    q1 = min(q0 + tm.q_per_chunk, nq);
  } else {
    o0 = task.b * tm.o_per_chunk;
    o1 = min(o0 + tm.o_per_chunk, no);
    q0 = 0;
    q1 = nq;
  }
  for (uint32_t o = o0; o < o1; ++o) {
    T acc[1 << kOut];
#pragma unroll
    for (int k = 0; k < (1 << kOut); ++k) acc[k] = czero<T>();
    const uint32_t abase = runs_offset(tm.oa, o), bbase = runs_offset(tm.ob, o);
    for (uint32_t q = q0; q < q1; ++q) {
      const T* Ab = Ag + (abase | runs_offset(tm.qa, q));
      const T* Bb = Bg + (bbase | runs_offset(tm.qb, q));
      uint32_t sidx = 0;
      for (; sidx + 3 < ns; sidx += 4) {
        const uint2 o0_ = soff[sidx], o1_ = soff[sidx + 1], o2_ = soff[sidx + 2], o3_ = soff[sidx + 3];
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) {
          const T a0 = Ab[ak[k] | o0_.x], b0 = Bb[bk[k] | o0_.y];
          const T a1 = Ab[ak[k] | o1_.x], b1 = Bb[bk[k] | o1_.y];
          const T a2 = Ab[ak[k] | o2_.x], b2 = Bb[bk[k] | o2_.y];
          const T a3 = Ab[ak[k] | o3_.x], b3 = Bb[bk[k] | o3_.y];
          acc[k] = cfma(a3, b3, cfma(a2, b2, cfma(a1, b1, cfma(a0, b0, acc[k]))));
        }
      }
      for (; sidx < ns; ++sidx) {
        const uint2 oo = soff[sidx];
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) acc[k] = cfma(Ab[ak[k] | oo.x], Bb[bk[k] | oo.y], acc[k]);
      }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m)
      if ((tm.sum_lane_mask >> m) & 1u) {
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) acc[k] = cadd(acc[k], shfl_xor_c(acc[k], 1 << m));
      }
    if (tm.sum_warp_mask) {
#pragma unroll
      for (int k = 0; k < (1 << kOut); ++k) red[((uint32_t)k << 8) | tid] = acc[k];
      team.sync();
      if (owner) {
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) {
          T sum = czero<T>();
          for (uint32_t w2 = 0; w2 < 8; ++w2)
            if ((w2 & ~(uint32_t)tm.sum_warp_mask) == warp)
              sum = cadd(sum, red[((uint32_t)k << 8) | (w2 << 5) | lane]);
          acc[k] = sum;
        }
      }
      team.sync();
    }
    if (owner) {
      if (split) {
        T* dst = partial + ((size_t)task.b << tm.nfc);
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) dst[ck[k]] = acc[k];
      } else {
        const uint32_t cbase = runs_offset(tm.oc, o);
#pragma unroll
        for (int k = 0; k < (1 << kOut); ++k) C[cbase | ck[k]] = acc[k];
      }
    }
  }
}

// A tile task: for each outer output value of the chunk (or, split, the
// chunk's outer summed values) contract the tile, then copy the C tile out
// (or into the chunk's partial slot; the last chunk of a split step adds the
// partials in chunk order).
template <typename T, int kTeams>
__device__ void run_tile(const GraphProgDev& prog, const GTask& task, T* table,
                         unsigned char* work, const GStep& st, int& s_last,
                         const GTeam<kTeams>& team) {
  const GTileMap& tm = st.tile;
  const bool sa = (tm.staged & 1) != 0, sb = (tm.staged & 2) != 0;
  const bool split = (st.flags & GSF_SPLIT) != 0;
  T* gb = reinterpret_cast<T*>(prog.gbase);
  const T* Ag = (st.flags & GSF_A_TABLE) ? table + st.a_off : gb + st.a_off;
  const T* Bg = (st.flags & GSF_B_TABLE) ? table + st.b_off : gb + st.b_off;
  constexpr uint32_t min_fp = sizeof(T) == 8 ? 2 : 1;
  const uint32_t fa = sa ? max(min_fp, 1u << tm.nfa) : 0, fb = sb ? max(min_fp, 1u << tm.nfb) : 0;
  uint32_t ab = fa + fb;
  if (tm.sum_warp_mask) ab = max(ab, 256u << tm.kout);
  const uint32_t fc = max(min_fp, 1u << tm.nfc);
  T* As = reinterpret_cast<T*>(work);
  T* Bs = As + fa;
  T* Cs = As + ab;
  uint2* soff = reinterpret_cast<uint2*>(work + (((size_t)(ab + fc) * sizeof(T) + 15) & ~size_t(15)));
  const uint32_t tid = team.tid;
  const uint32_t shift = 8u + tm.kout;
  for (uint32_t s = tid; s < (1u << tm.ns); s += team.size)
    soff[s] = make_uint2(runs_offset(tm.tfa, s << shift), runs_offset(tm.tfb, s << shift));
  team.sync();
  const uint32_t nq = 1u << tm.nq, no = 1u << tm.no;
  uint32_t o0, o1, q0, q1;
  if (split) {
    o0 = 0;
    o1 = 1;
    q0 = task.b * tm.q_per_chunk;
    q1 = min(q0 + tm.q_per_chunk, nq);
  } else {
    o0 = task.b * tm.o_per_chunk;
    o1 = min(o0 + tm.o_per_chunk, no);
    q0 = 0;
    q1 = nq;
  }
  constexpr uint32_t per = 16 / sizeof(T);
  T* C = gb + st.c_off;
  T* partial = gb + st.partial_off;
  if (tm.staged == 0) {
    // read in place: no footprints, outputs stored by their owners
    switch (tm.kout) {
      case 0: tile_direct<T, kTeams, 0>(st, task, Ag, Bg, C, partial, As, soff, team); break;
      case 1: tile_direct<T, kTeams, 1>(st, task, Ag, Bg, C, partial, As, soff, team); break;
      default: tile_direct<T, kTeams, 2>(st, task, Ag, Bg, C, partial, As, soff, team); break;
    }
    o1 = o0;   // done
  }
  for (uint32_t o = o0; o < o1; ++o) {
    switch (tm.kout) {
      case 0: tile_contract<T, kTeams, 0>(st, Ag, Bg, As, Bs, Cs, As, soff, o, q0, q1, team); break;
      case 1: tile_contract<T, kTeams, 1>(st, Ag, Bg, As, Bs, Cs, As, soff, o, q0, q1, team); break;
      default: tile_contract<T, kTeams, 2>(st, Ag, Bg, As, Bs, Cs, As, soff, o, q0, q1, team); break;
    }
    // C tile out: 16-byte stores (footprint bit 0 is C's bit 0)
    const uint32_t n = 1u << tm.nfc;
    if (split) {
      T* dst = partial + (size_t)task.b * n;
      for (uint32_t j = tid; j < n; j += team.size) dst[j] = Cs[j];
    } else if (per == 2 && tm.nfc >= 1) {
      const uint32_t cbase = runs_offset(tm.oc, o);
      for (uint32_t j = tid * 2; j < n; j += team.size * 2)
        *reinterpret_cast<float4*>(C + (cbase | runs_offset(tm.ffc, j))) =
            *reinterpret_cast<const float4*>(Cs + j);
    } else {
      const uint32_t cbase = runs_offset(tm.oc, o);
      for (uint32_t j = tid; j < n; j += team.size) C[cbase | runs_offset(tm.ffc, j)] = Cs[j];
    }
    team.sync();
  }
  if (!split) {
    signal_done(prog, st.done_ctr, team);
    return;
  }
  __threadfence();
  team.sync();
  if (tid == 0)
    s_last = atomicAdd(prog.counters + ctr_index(st.arrive_ctr), 1u) == st.n_chunks - 1;
  team.sync();
  if (!s_last) return;
  __threadfence();
  const uint32_t n = 1u << tm.nfc;
  if (st.flags & GSF_LEAFGRAD) {
    // dS/dparam += sum_c dS/dleaf[c] * dleaf[c]/dparam  (leaf has <= 16 entries)
    if (tid < 32) {
      double2 prod = make_double2(0.0, 0.0);
      if (tid < n) {
        T total = czero<T>();
        for (uint32_t k = 0; k < st.n_chunks; ++k)
          total = cadd(total, load_l2(partial + (size_t)k * n + tid));
        const double2 t = to_d2(total);
        const double2 d = to_d2(table[st.der_off + runs_offset(tm.ffc, tid)]);
        prod.x = t.x * d.x - t.y * d.y;
        prod.y = t.x * d.y + t.y * d.x;
      }
      for (int off = 16; off > 0; off >>= 1) {
        prod.x += __shfl_down_sync(0xffffffffu, prod.x, off);
        prod.y += __shfl_down_sync(0xffffffffu, prod.y, off);
      }
      if (tid == 0) {
        const size_t row = (size_t)st.net * (2 + 2 * prog.n_params);
        atomicAdd(&prog.results[row + 2 + 2 * st.slot], prod.x);
        atomicAdd(&prog.results[row + 3 + 2 * st.slot], prod.y);
      }
    }
  } else {
    for (uint32_t j = tid; j < n; j += team.size) {
      T total = czero<T>();
      for (uint32_t k = 0; k < st.n_chunks; ++k)
        total = cadd(total, load_l2(partial + (size_t)k * n + j));
      C[runs_offset(tm.ffc, j)] = total;
    }
  }
  signal_done(prog, st.done_ctr, team);
}

// ---- paired loads: summed bit 0 is bit 0 of both operands ------------------

__device__ __forceinline__ float4 ld_pair(const float2* p) {
  return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ float2 cfma2(float4 a, float4 b, float2 acc) {
  return cfma(make_float2(a.z, a.w), make_float2(b.z, b.w),
              cfma(make_float2(a.x, a.y), make_float2(b.x, b.y), acc));
}

// sum over y of A[oa | ya[y]] B[ob | yb[y]] for n_y >= 8 summed values, two
// at a time (y, y + 1 adjacent in both operands): eight 16-byte loads in
// flight per thread, four accumulators.
__device__ __forceinline__ float2 ysum_pair(const float2* A, const float2* B, uint32_t oa,
                                            uint32_t ob, const uint32_t* ya, const uint32_t* yb,
                                            uint32_t n_y) {
  float2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
  for (uint32_t y = 0; y < n_y; y += 8) {
    float4 a[4], b[4];
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
      a[u] = ld_pair(A + (oa | ya[y + 2 * u]));
      b[u] = ld_pair(B + (ob | yb[y + 2 * u]));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = cfma2(a[u], b[u], acc[u]);
  }
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}

// R rows at a time, n_y = 2 * NP summed values as NP pairs per row.
template <uint32_t R, uint32_t NP>
__device__ __forceinline__ void rows_pair(const float2* A, const float2* B, float2* C,
                                          const uint32_t* rowa, const uint32_t* rowb,
                                          uint32_t a_lo, uint32_t b_lo, const uint32_t* ya,
                                          const uint32_t* yb, uint32_t r0, uint32_t r1,
                                          uint32_t rowlen, uint32_t tid) {
  uint32_t yav[NP], ybv[NP];
#pragma unroll
  for (uint32_t k = 0; k < NP; ++k) {
    yav[k] = ya[2 * k];
    ybv[k] = yb[2 * k];
  }
  for (uint32_t row = r0; row < r1; row += R) {
    float4 av[R][NP], bv[R][NP];
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t rr = min(row + r, r1 - 1) - r0;
      const uint32_t oa = rowa[rr] | a_lo, ob = rowb[rr] | b_lo;
#pragma unroll
      for (uint32_t k = 0; k < NP; ++k) {
        av[r][k] = ld_pair(A + (oa | yav[k]));
        bv[r][k] = ld_pair(B + (ob | ybv[k]));
      }
    }
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (uint32_t k = 0; k < NP; ++k) acc = cfma2(av[r][k], bv[r][k], acc);
      if (row + r < r1) C[(row + r) * rowlen + tid] = acc;
    }
  }
}

// rows_shared for complex64 steps with paired loads (summed bit 0 is bit 0
// of both operands): two 16-byte pairs per distinct element and pass, so a
// ZX group of four rows issues 8 loads for 16 terms.  Out of line, like
// rows_fixed.
template <int kShare>
__device__ __noinline__ void rows_shared_pair(const float2* A, const float2* B, float2* C,
                                              const uint32_t* rowa, const uint32_t* rowb,
                                              const uint32_t* rowc, uint32_t a_lo, uint32_t b_lo,
                                              const uint32_t* ya, const uint32_t* yb,
                                              uint32_t nr, uint32_t n_y, uint32_t tid) {
  constexpr int NA = kShare == GRS_ZZ ? 1 : (kShare == GRS_ZX ? 2 : 4);
  constexpr int NB = kShare == GRS_XX ? 1 : (kShare == GRS_ZX ? 2 : 4);
  auto ia = [](int k) { return kShare == GRS_ZZ ? 0 : (kShare == GRS_ZX ? k >> 1 : k); };
  auto ib = [](int k) { return kShare == GRS_XX ? 0 : (kShare == GRS_ZX ? k & 1 : k); };
  for (uint32_t r = 0; r < nr; r += 4) {
    uint32_t oa[NA], ob[NB];
#pragma unroll
    for (int i = 0; i < NA; ++i) oa[i] = rowa[r + (kShare == GRS_ZX ? 2 * i : i)] | a_lo;
#pragma unroll
    for (int i = 0; i < NB; ++i) ob[i] = rowb[r + i] | b_lo;
    float2 acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = make_float2(0.f, 0.f);
    for (uint32_t y = 0; y < n_y; y += 4) {
      const uint32_t ay0 = ya[y], by0 = yb[y], ay1 = ya[y + 2], by1 = yb[y + 2];
      float4 av[NA][2], bv[NB][2];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        av[i][0] = ld_pair(A + (oa[i] | ay0));
        av[i][1] = ld_pair(A + (oa[i] | ay1));
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        bv[i][0] = ld_pair(B + (ob[i] | by0));
        bv[i][1] = ld_pair(B + (ob[i] | by1));
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        acc[k] = cfma2(av[ia(k)][1], bv[ib(k)][1], cfma2(av[ia(k)][0], bv[ib(k)][0], acc[k]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) C[rowc[r + k] + tid] = acc[k];
  }
}

// Rows of a complex64 step with paired loads; false for other element types.
template <typename T>
__device__ __forceinline__ bool rows_paired(const T* A, const T* B, T* C, const uint32_t* rowa,
                                            const uint32_t* rowb, uint32_t a_lo, uint32_t b_lo,
                                            const uint32_t* ya, const uint32_t* yb, uint32_t r0,
                                            uint32_t r1, uint32_t rowlen, uint32_t tid,
                                            uint32_t n_y) {
  if constexpr (sizeof(T) != 8) {
    return false;
  } else {
    const float2* a = reinterpret_cast<const float2*>(A);
    const float2* b = reinterpret_cast<const float2*>(B);
    float2* c = reinterpret_cast<float2*>(C);
    if (n_y == 2)
      rows_pair<8, 1>(a, b, c, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
    else if (n_y == 4)
      rows_pair<4, 2>(a, b, c, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
    else if (n_y == 8)
      rows_pair<2, 4>(a, b, c, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
    else
      for (uint32_t row = r0; row < r1; ++row)
        c[row * rowlen + tid] =
            ysum_pair(a, b, rowa[row - r0] | a_lo, rowb[row - r0] | b_lo, ya, yb, n_y);
    return true;
  }
}

// Split chunk with lanes over the summed index (its low bits are the
// operands' lowest): warp w sums outputs c = w, w + 8, ... over the chunk's
// cnt values, lanes 32 apart, four accumulators, then a shuffle reduction.
template <typename T>
__device__ __forceinline__ T warp_ysum(const T* A, const T* B, uint32_t oa, uint32_t ob,
                                       const uint32_t* ya, const uint32_t* yb, uint32_t cnt,
                                       uint32_t lane) {
  T acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = czero<T>();
  uint32_t y = lane;
  for (; y + 96 < cnt; y += 128) {
    T av[4], bv[4];
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) {
      av[u] = A[oa | ya[y + 32 * u]];
      bv[u] = B[ob | yb[y + 32 * u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = cfma(av[u], bv[u], acc[u]);
  }
  for (; y < cnt; y += 32) acc[0] = cfma(A[oa | ya[y]], B[ob | yb[y]], acc[0]);
  T sum = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
  for (int off = 16; off > 0; off >>= 1) sum = cadd(sum, shfl_xor_c(sum, off));
  return sum;
}

template <typename T, int kTeams, bool kTile>
__device__ void run_chunk(const GraphProgDev& prog, const GTask& task, T* table,
                          unsigned char* work, GStep& s_step, int& s_last,
                          const GTeam<kTeams>& team) {
  {
    const uint4* src = reinterpret_cast<const uint4*>(prog.steps + task.a);
    for (uint32_t w = team.tid; w < sizeof(GStep) / sizeof(uint4); w += team.size)
      reinterpret_cast<uint4*>(&s_step)[w] = src[w];
  }
  team.sync();
  const GStep& st = s_step;
  if constexpr (kTile) {
    if (st.flags & GSF_TILE) {
      run_tile<T, kTeams>(prog, task, table, work, st, s_last, team);
      return;
    }
  }
  T* gb = reinterpret_cast<T*>(prog.gbase);
  const T* A = (st.flags & GSF_A_TABLE) ? table + st.a_off : gb + st.a_off;
  const T* B = (st.flags & GSF_B_TABLE) ? table + st.b_off : gb + st.b_off;
  uint32_t* ya = reinterpret_cast<uint32_t*>(work);
  uint32_t* yb = ya + kYTab;
  T* red = reinterpret_cast<T*>(yb + kYTab);
  const uint32_t tid = team.tid;
  const uint32_t nout = 1u << st.rc;
  const uint64_t ny = 1ull << st.ry;

  if (!(st.flags & GSF_SPLIT)) {
    T* C = gb + st.c_off;
    const uint32_t rowlen = nout < kGRow ? nout : kGRow;
    const uint32_t nrows = nout / rowlen;
    const uint32_t r0 = task.b * st.chunk;
    const uint32_t r1 = min(r0 + st.chunk, nrows);
    const bool active = tid < rowlen;
    const uint32_t a_lo = runs_offset(st.ca, tid), b_lo = runs_offset(st.cb, tid);
    if (ny <= kYTab) {
      // offsets of the summed index and of this chunk's rows, tabulated once
      uint32_t* rowa = reinterpret_cast<uint32_t*>(red + kGraphBlock);
      uint32_t* rowb = rowa + kMaxChunkRows;
      uint32_t* rowc = rowb + kMaxChunkRows;
      const bool shared_rows = (st.flags & GSF_ROWS) != 0;
      for (uint32_t y = tid; y < ny; y += team.size) {
        ya[y] = runs_offset(st.ya, y);
        yb[y] = runs_offset(st.yb, y);
      }
      for (uint32_t r = tid; r < r1 - r0; r += team.size) {
        const uint32_t o = shared_rows ? runs_offset(st.rows, r0 + r) : r0 + r;
        rowa[r] = runs_offset(st.ca, o * rowlen);
        rowb[r] = runs_offset(st.cb, o * rowlen);
        rowc[r] = o * rowlen;
      }
      team.sync();
      constexpr uint32_t R = 4;
      const uint32_t n_y = (uint32_t)ny;
      if (active && shared_rows && st.share >= GRS_FIXA) {
        rows_fixed_dispatch(A, B, C, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y,
                            st.share == GRS_FIXB, tid);
      } else if (active && shared_rows && (st.flags & GSF_YPAIR) && sizeof(T) == 8) {
        const float2* a2 = reinterpret_cast<const float2*>(A);
        const float2* b2 = reinterpret_cast<const float2*>(B);
        float2* c2 = reinterpret_cast<float2*>(C);
        if (st.share == GRS_ZX)
          rows_shared_pair<GRS_ZX>(a2, b2, c2, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
        else if (st.share == GRS_ZZ)
          rows_shared_pair<GRS_ZZ>(a2, b2, c2, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
        else
          rows_shared_pair<GRS_XX>(a2, b2, c2, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
      } else if (active && shared_rows) {
        if (st.share == GRS_ZX)
          rows_shared<T, GRS_ZX>(A, B, C, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
        else if (st.share == GRS_ZZ)
          rows_shared<T, GRS_ZZ>(A, B, C, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
        else
          rows_shared<T, GRS_XX>(A, B, C, rowa, rowb, rowc, a_lo, b_lo, ya, yb, r1 - r0, n_y, tid);
      } else if (active && (st.flags & GSF_YPAIR) &&
          rows_paired(A, B, C, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid, n_y)) {
        // complex64 element pairs along summed bit 0
      } else if (active && r1 - r0 < R) {
        // few rows with long sums: the summed index unrolled instead
        for (uint32_t row = r0; row < r1; ++row)
          C[row * rowlen + tid] = ysum(A, B, rowa[row - r0] | a_lo, rowb[row - r0] | b_lo, ya,
                                       yb, 0u, n_y, 1u);
      } else if (active && n_y == 1) {
        rows_unrolled<T, 8, 1>(A, B, C, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
      } else if (active && n_y == 2) {
        rows_unrolled<T, 4, 2>(A, B, C, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
      } else if (active && n_y == 4) {
        rows_unrolled<T, 2, 4>(A, B, C, rowa, rowb, a_lo, b_lo, ya, yb, r0, r1, rowlen, tid);
      } else if (active) {
        // four rows at a time: eight independent loads in flight per thread
        for (uint32_t row = r0; row < r1; row += R) {
          uint32_t oa[R], ob[R];
          T acc[R];
#pragma unroll
          for (uint32_t r = 0; r < R; ++r) {
            const uint32_t rr = min(row + r, r1 - 1) - r0;
            oa[r] = rowa[rr] | a_lo;
            ob[r] = rowb[rr] | b_lo;
            acc[r] = czero<T>();
          }
          // two summed values per pass (n_y >= 8 here): sixteen loads in flight
          for (uint32_t y = 0; y < n_y; y += 2) {
            const uint32_t ay0 = ya[y], by0 = yb[y], ay1 = ya[y + 1], by1 = yb[y + 1];
            T av[R][2], bv[R][2];
#pragma unroll
            for (uint32_t r = 0; r < R; ++r) {
              av[r][0] = A[oa[r] | ay0];
              bv[r][0] = B[ob[r] | by0];
              av[r][1] = A[oa[r] | ay1];
              bv[r][1] = B[ob[r] | by1];
            }
#pragma unroll
            for (uint32_t r = 0; r < R; ++r)
              acc[r] = cfma(av[r][1], bv[r][1], cfma(av[r][0], bv[r][0], acc[r]));
          }
#pragma unroll
          for (uint32_t r = 0; r < R; ++r)
            if (row + r < r1) C[(row + r) * rowlen + tid] = acc[r];
        }
      }
    } else {
      // one row per chunk; the summed index in passes of kYTab values
      const uint32_t hi = r0 * rowlen;
      const uint32_t oa = runs_offset(st.ca, hi) | a_lo;
      const uint32_t ob = runs_offset(st.cb, hi) | b_lo;
      T acc = czero<T>();
      for (uint64_t y0 = 0; y0 < ny; y0 += kYTab) {
        team.sync();
        for (uint32_t y = tid; y < kYTab; y += team.size) {
          ya[y] = runs_offset(st.ya, (uint32_t)(y0 + y));
          yb[y] = runs_offset(st.yb, (uint32_t)(y0 + y));
        }
        team.sync();
        if (active) acc = cadd(acc, ysum(A, B, oa, ob, ya, yb, 0u, kYTab, 1u));
      }
      if (active) C[hi + tid] = acc;
    }
    signal_done(prog, st.done_ctr, team);
    return;
  }

  // split: outputs <= 256, chunk task.b sums y in [y0, y0 + cnt)
  const uint32_t groups = team.size / nout;
  const uint32_t c = tid % nout, g = tid / nout;
  const uint64_t y0 = (uint64_t)task.b * st.chunk;
  const uint32_t cnt = (uint32_t)min((uint64_t)st.chunk, ny - y0);
  for (uint32_t y = tid; y < cnt; y += team.size) {
    ya[y] = runs_offset(st.ya, (uint32_t)(y0 + y));
    yb[y] = runs_offset(st.yb, (uint32_t)(y0 + y));
  }
  team.sync();
  T* partial = gb + st.partial_off;
  if (st.flags & GSF_LANES_Y) {
    const uint32_t lane = tid & 31u, warp = tid >> 5, n_warps = team.size >> 5;
    for (uint32_t cc = warp; cc < nout; cc += n_warps) {
      const T sum = warp_ysum(A, B, runs_offset(st.ca, cc), runs_offset(st.cb, cc), ya, yb, cnt,
                              lane);
      if (lane == 0) partial[(size_t)task.b * nout + cc] = sum;
    }
  } else {
    const uint32_t oa = runs_offset(st.ca, c), ob = runs_offset(st.cb, c);
    T acc = czero<T>();
    if (g < groups) acc = ysum(A, B, oa, ob, ya, yb, g, cnt, groups);
    red[tid] = acc;
    team.sync();
    if (tid < nout) {
      T sum = czero<T>();
      for (uint32_t k = 0; k < groups; ++k) sum = cadd(sum, red[k * nout + tid]);
      partial[(size_t)task.b * nout + tid] = sum;
    }
  }
  __threadfence();
  team.sync();
  if (tid == 0)
    s_last = atomicAdd(prog.counters + ctr_index(st.arrive_ctr), 1u) == st.n_chunks - 1;
  team.sync();
  if (!s_last) return;
  __threadfence();
  T total = czero<T>();
  if (tid < nout)
    for (uint32_t k = 0; k < st.n_chunks; ++k)
      total = cadd(total, load_l2(partial + (size_t)k * nout + tid));
  if (st.flags & GSF_LEAFGRAD) {
    // dS/dparam += sum_c dS/dleaf[c] * dleaf[c]/dparam  (leaf has <= 16 entries)
    if (tid < 32) {
      double2 prod = make_double2(0.0, 0.0);
      if (tid < nout) {
        const double2 t = to_d2(total);
        const double2 d = to_d2(table[st.der_off + tid]);
        prod.x = t.x * d.x - t.y * d.y;
        prod.y = t.x * d.y + t.y * d.x;
      }
      for (int off = 16; off > 0; off >>= 1) {
        prod.x += __shfl_down_sync(0xffffffffu, prod.x, off);
        prod.y += __shfl_down_sync(0xffffffffu, prod.y, off);
      }
      if (tid == 0) {
        const size_t row = (size_t)st.net * (2 + 2 * prog.n_params);
        atomicAdd(&prog.results[row + 2 + 2 * st.slot], prod.x);
        atomicAdd(&prog.results[row + 3 + 2 * st.slot], prod.y);
      }
    }
  } else if (tid < nout) {
    gb[st.c_off + tid] = total;
  }
  signal_done(prog, st.done_ctr, team);
}

// ---- tensor-core GEMM tasks (split BF16, tcgen05, accumulator in TMEM) ----

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle.  lbo = byte stride
// between core matrices (8 rows x 16 bytes) along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the tensor cores' arrival on `mbar` with `parity`.
__device__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long limit_ns) {
  const unsigned long long t0 = now_ns();
  while (!mbar_try_wait(mbar, parity))
    if ((long long)(now_ns() - t0) > limit_ns) return false;
  return true;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Byte offset of element (row r, real k index kk) in a K-major tile of 32 BF16
// per row made of 8x8 core matrices (rows 16 bytes apart, core matrices 128
// bytes apart along K, 512 bytes apart along the rows).
__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t kk) {
  return ((((r >> 3) << 2) + (kk >> 3)) << 7) + ((r & 7u) << 4) + ((kk & 7u) << 1);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// One tile (128 rows m x 64 complex columns n, one batch index) of a complex
// GEMM.  The complex product becomes a real GEMM with K' = 2K and N' = 2N:
// A' row m = (Re A[m][k], Im A[m][k]) interleaved over k, and B'^T row 2n =
// (Re B[k][n], -Im B[k][n]), row 2n + 1 = (Im B[k][n], Re B[k][n]), so that the
// accumulator columns 2n and 2n + 1 are Re C[m][n] and Im C[m][n].
template <typename T, int kTeams>
__device__ bool run_tc(const GraphProgDev& prog, const GTask& task, unsigned char* work,
                       TStep& s_ts, uint32_t tmem, uint32_t mbar, uint32_t& phase,
                       const GTeam<kTeams>& team) {
  {
    const uint4* src = reinterpret_cast<const uint4*>(prog.tsteps + task.a);
    for (uint32_t w = team.tid; w < sizeof(TStep) / sizeof(uint4); w += team.size)
      reinterpret_cast<uint4*>(&s_ts)[w] = src[w];
  }
  team.sync();
  const TStep& ts = s_ts;
  T* gb = reinterpret_cast<T*>(prog.gbase);
  const T* A = gb + ts.a_off;
  const T* B = gb + ts.b_off;
  T* C = gb + ts.c_off;
  const uint32_t per_b = ts.m_tiles * ts.n_tiles;
  const uint32_t bi = task.b / per_b, rem = task.b % per_b;
  const uint32_t mt = rem / ts.n_tiles, nt = rem % ts.n_tiles;
  const uint32_t M = 1u << ts.mb, K = 1u << ts.kb;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(work) + 127) & ~uintptr_t(127));
  unsigned char* a_hi = base;
  unsigned char* a_lo = base + 8192;
  unsigned char* b_hi = base + 16384;
  unsigned char* b_lo = base + 24576;
  const uint32_t tid = team.tid;
  // loaders: A by (row, 8 consecutive k), B by (column, 4 consecutive k)
  const uint32_t a_r = tid & 127u, a_k0 = (tid >> 7) * 8;
  const uint32_t m_g = mt * kTcRows + a_r;
  const bool m_ok = m_g < M;
  const uint32_t a_row = m_ok ? (runs_offset(ts.am, m_g) | runs_offset(ts.ab, bi)) : 0;
  const uint32_t b_c = tid & 63u, b_k0 = (tid >> 6) * 4;
  const uint32_t n_g = nt * kTcCols + b_c;
  const uint32_t b_col = runs_offset(ts.bn, n_g) | runs_offset(ts.bbt, bi);
  const uint32_t nk = (K + kTcK - 1) / kTcK;
  // the operands of K slice kc + 1 are loaded into registers while the MMAs
  // of slice kc run (the shared-memory stage is single, so they are stored
  // after the MMAs complete)
  T av[8], bv[4];
  // the K maps are bit permutations: offset(kc * 16 + kl) = offset(kc * 16) |
  // offset(kl), so each thread keeps the offsets of its own k within a slice
  uint32_t akl[8], bkl[4];
#pragma unroll
  for (uint32_t j = 0; j < 8; ++j) akl[j] = runs_offset(ts.ak, a_k0 + j);
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j) bkl[j] = runs_offset(ts.bk, b_k0 + j);
  auto load_slice = [&](uint32_t kc) {
    const uint32_t ka = a_row | runs_offset(ts.ak, kc * kTcK);
    const uint32_t kb = b_col | runs_offset(ts.bk, kc * kTcK);
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t k = kc * kTcK + a_k0 + j;
      av[j] = (m_ok && k < K) ? A[ka | akl[j]] : czero<T>();
    }
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t k = kc * kTcK + b_k0 + j;
      bv[j] = k < K ? B[kb | bkl[j]] : czero<T>();
    }
  };
  load_slice(0);
  for (uint32_t kc = 0; kc < nk; ++kc) {
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t kl = a_k0 + j;
      const double2 v = to_d2(av[j]);
      __nv_bfloat16 rh, rl, ih, il;
      split_bf16((float)v.x, rh, rl);
      split_bf16((float)v.y, ih, il);
      const uint32_t off = core_offset(a_r, 2 * kl);
      *reinterpret_cast<uint32_t*>(a_hi + off) = pack_bf16(rh, ih);
      *reinterpret_cast<uint32_t*>(a_lo + off) = pack_bf16(rl, il);
    }
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t kl = b_k0 + j;
      const double2 v = to_d2(bv[j]);
      __nv_bfloat16 rh, rl, ih, il;
      split_bf16((float)v.x, rh, rl);
      split_bf16((float)v.y, ih, il);
      const uint32_t o0 = core_offset(2 * b_c, 2 * kl), o1 = core_offset(2 * b_c + 1, 2 * kl);
      *reinterpret_cast<uint32_t*>(b_hi + o0) = pack_bf16(rh, __hneg(ih));
      *reinterpret_cast<uint32_t*>(b_lo + o0) = pack_bf16(rl, __hneg(il));
      *reinterpret_cast<uint32_t*>(b_hi + o1) = pack_bf16(ih, rh);
      *reinterpret_cast<uint32_t*>(b_lo + o1) = pack_bf16(il, rl);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    team.sync();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_addr(a_hi), al = smem_addr(a_lo);
      const uint32_t bh = smem_addr(b_hi), bl = smem_addr(b_lo);
      for (uint32_t ks = 0; ks < 2; ++ks) {
        const uint32_t off = ks * 256;  // 16 reals = two core matrices along K
        const uint32_t acc = (kc | ks) != 0;
        tc_mma(tmem, smem_desc(ah + off, 128, 512), smem_desc(bh + off, 128, 512), acc);
        tc_mma(tmem, smem_desc(ah + off, 128, 512), smem_desc(bl + off, 128, 512), 1);
        tc_mma(tmem, smem_desc(al + off, 128, 512), smem_desc(bh + off, 128, 512), 1);
      }
      tc_commit(mbar);
    }
    if (kc + 1 < nk) load_slice(kc + 1);
    const bool ok = mbar_wait_bounded(mbar, phase, prog.wait_limit_ns);
    phase ^= 1u;
    if (!ok) {
      atomicCAS(prog.counters + CTR_ERROR, 0u, (unsigned)QTC_ERR_TIMEOUT);
      return false;
    }
  }
  tc_fence_after();
  const uint32_t warp = tid >> 5, lane = tid & 31u;
  const uint32_t sub = warp & 3u, half = warp >> 2;
  const uint32_t row = sub * 32 + lane;
  const uint32_t m = mt * kTcRows + row;
  const uint32_t c_row = (m < M) ? (runs_offset(ts.cm, m) | runs_offset(ts.cb, bi)) : 0;
  for (uint32_t c16 = 0; c16 < 4; ++c16) {
    const uint32_t col = half * 64 + c16 * 16;
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((sub * 32u) << 16) + col));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (m < M)
      for (uint32_t q = 0; q < 8; ++q) {
        const uint32_t n = nt * kTcCols + (col >> 1) + q;
        C[c_row | runs_offset(ts.cn, n)] =
            from_d2<T>(make_double2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1])));
      }
  }
  tc_fence_before();
  signal_done(prog, ts.done_ctr, team);
  return true;
}

// kTc: the program has tensor-core GEMM tasks.  Programs without them use the
// instantiation that contains no tensor-core code (one 256-thread team per
// CTA, four CTAs per SM), so its registers and schedule are those of the
// memory-bound task kinds alone.  The tensor-core instantiation runs four
// teams in one 1024-thread CTA per SM and gives each team 128 columns of
// tensor memory.
// kHiOcc (complex64, no tensor cores): registers capped for five 256-thread
// CTAs per SM instead of four (some spilling); helps programs dominated by
// large memory-bound steps, hurts others (chosen per batch by tuning).
// kTile: the program has steps in tile form (a separate instantiation keeps
// the tile code's registers out of the row and split paths).
template <typename T, bool kTc, bool kHiOcc = false, bool kTile = false>
__global__ void __launch_bounds__(kGraphBlock*(kTc ? 4 : 1),
                                  kTc ? 1 : kHiOcc ? 5 : sizeof(T) == 8 ? 4 : 2)
    graph_exec_kernel(const GraphProgDev prog) {
  constexpr int kTeams = kTc ? 4 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ GStep s_step[kTeams];
  __shared__ TStep s_tstep[kTc ? kTeams : 1];
  __shared__ double s_grad[kTeams][2 * kMaxParams];
  __shared__ double s_red[(1 + kMaxParams) * kReduceThreads / 32];
  __shared__ unsigned int s_task[kTeams];
  __shared__ int s_flag[kTeams];
  __shared__ int s_last[kTeams];
  __shared__ int s_final;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_mbar[kTeams];
  const GTeam<kTeams> team;
  T* table = reinterpret_cast<T*>(smem_raw);
  unsigned char* work = smem_raw + prog.table_bytes + (size_t)team.id * prog.arena_bytes;
  // tensor memory: the CTA allocates kTeams x 128 columns once (at most one
  // such CTA is resident per SM, 512 columns per SM)
  uint32_t tmem = 0, phase = 0;
  bool tc_pending = false;
  if (kTc && prog.tmem_cols > 0) {
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_addr(&s_tmem)),
                   "r"(prog.tmem_cols * kTeams)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x < kTeams) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_mbar[threadIdx.x])),
                   "r"(1)
                   : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
  }
  build_gate_table<T>(prog.gates, prog.n_gates, prog.params, table);
  __syncthreads();
  if (kTc && prog.tmem_cols > 0) {
    tc_fence_after();
    tmem = s_tmem + (uint32_t)(team.id * prog.tmem_cols);
  }

  for (;;) {
    if (team.tid < 32) {
      unsigned int t = 0;
      if (team.tid == 0) t = atomicAdd(&prog.counters[CTR_QUEUE], 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      bool ok = t < (unsigned)prog.n_tasks;
      if (ok) ok = wait_for_producers_warp(prog, prog.tasks[t], team.tid);
      if (team.tid == 0) {
        s_task[team.id] = t;
        s_flag[team.id] = ok;
      }
    }
    team.sync();
    if (!s_flag[team.id]) break;
    const GTask task = prog.tasks[s_task[team.id]];
    if (task.kind == GT_SMEM) {
      run_smem_task<T, kTeams>(prog, task, table, work, s_grad[team.id], team);
    } else if (task.kind == GT_CHUNK) {
      run_chunk<T, kTeams, kTile>(prog, task, table, work, s_step[team.id], s_last[team.id], team);
    } else if (kTc && prog.tmem_cols > 0) {
      if (!run_tc<T, kTeams>(prog, task, work, s_tstep[kTc ? team.id : 0], tmem,
                             smem_addr(&s_mbar[team.id]), phase, team)) {
        tc_pending = true;
        team.sync();
        break;
      }
    }
    team.sync();
  }
  if (kTc && prog.tmem_cols > 0) {
    // a GEMM whose completion wait expired may still be running: wait for it
    // once more (bounded) before the tensor memory is given back
    if (tc_pending)
      mbar_wait_bounded(smem_addr(&s_mbar[team.id]), phase ^ 1u, prog.wait_limit_ns);
    tc_fence_before();
  }
  __syncthreads();
  if (kTc && prog.tmem_cols > 0 && threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "r"(prog.tmem_cols * kTeams)
                 : "memory");
  }

  // the last CTA reduces (final wave), records the status and re-arms
  if (threadIdx.x == 0) {
    __threadfence();
    s_final = atomicAdd(&prog.counters[CTR_BLOCKS], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_final) return;
  __threadfence();
  volatile unsigned* vc = prog.counters;
  const unsigned err = vc[CTR_ERROR] | vc[CTR_RESERVED];
  __syncthreads();
  if (threadIdx.x == 0) prog.counters[CTR_RESERVED] = err;  // sticky across waves
  if (prog.final_wave) {
    const int P = prog.n_params;
    const int N = prog.n_nets;
    const int stride = 2 + 2 * P;
    const volatile double* res = prog.results;
    reduce_network_rows(res, prog.weights, N, P, prog.qaoa_reduce != 0, prog.out, s_red);
    if (threadIdx.x == 0) prog.out[1 + P + N] = (double)err;
    if (prog.raw_out)
      for (int i = threadIdx.x; i < N * stride; i += blockDim.x) prog.raw_out[i] = res[i];
    __syncthreads();
    for (int i = threadIdx.x; i < N * stride; i += blockDim.x) prog.results[i] = 0.0;
    if (threadIdx.x == 0) prog.counters[CTR_RESERVED] = 0;
  }
  for (int i = threadIdx.x; i < prog.n_counters; i += blockDim.x)
    prog.counters[ctr_index(i)] = 0;
  if (threadIdx.x == 0) {
    prog.counters[CTR_QUEUE] = 0;
    prog.counters[CTR_BLOCKS] = 0;
    prog.counters[CTR_ERROR] = 0;
  }
}

static const void* graph_kernel(int dtype, bool tc, bool hi_occ, bool tiles) {
  if (dtype == 0) {
    if (tc) return (const void*)graph_exec_kernel<double2, true>;
    return tiles ? (const void*)graph_exec_kernel<double2, false, false, true>
                 : (const void*)graph_exec_kernel<double2, false>;
  }
  if (tc) return (const void*)graph_exec_kernel<float2, true>;
  if (tiles) return (const void*)graph_exec_kernel<float2, false, false, true>;
  return hi_occ ? (const void*)graph_exec_kernel<float2, false, true>
                : (const void*)graph_exec_kernel<float2, false>;
}

cudaError_t graph_exec_configure(int dtype, bool tc, bool hi_occ, bool tiles, size_t smem_bytes,
                                 size_t max_dynamic, int* blocks_per_sm) {
  const void* fn = graph_kernel(dtype, tc, hi_occ, tiles);
  if (smem_bytes > max_dynamic) return cudaErrorInvalidValue;
  cudaError_t err =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dynamic);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn,
                                                       kGraphBlock * (tc ? 4 : 1), smem_bytes);
}

cudaError_t graph_exec_launch(const GraphProgDev& prog, int dtype, bool hi_occ, bool tiles,
                              int grid, size_t smem_bytes, cudaStream_t stream) {
  const bool tc = prog.tmem_cols > 0;
  if (dtype == 0) {
    if (tc)
      graph_exec_kernel<double2, true><<<grid, 4 * kGraphBlock, smem_bytes, stream>>>(prog);
    else if (tiles)
      graph_exec_kernel<double2, false, false, true>
          <<<grid, kGraphBlock, smem_bytes, stream>>>(prog);
    else
      graph_exec_kernel<double2, false><<<grid, kGraphBlock, smem_bytes, stream>>>(prog);
  } else {
    if (tc)
      graph_exec_kernel<float2, true><<<grid, 4 * kGraphBlock, smem_bytes, stream>>>(prog);
    else if (tiles)
      graph_exec_kernel<float2, false, false, true>
          <<<grid, kGraphBlock, smem_bytes, stream>>>(prog);
    else if (hi_occ)
      graph_exec_kernel<float2, false, true><<<grid, kGraphBlock, smem_bytes, stream>>>(prog);
    else
      graph_exec_kernel<float2, false><<<grid, kGraphBlock, smem_bytes, stream>>>(prog);
  }
  return cudaGetLastError();
}

}  // namespace qtc
