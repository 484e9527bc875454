// Plain structures shared by the host lowering and the CUDA kernels.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define QTC_HD __host__ __device__
#else
#define QTC_HD
#endif

namespace qtc {

// Leaf tensor kinds.  Storage convention: label k of a leaf is bit k of the
// element index.
//   rank 1: (a)
//   rank 2 gate [out, in]:   index = out | in << 1, value U[out][in]
//   rank 2 observable [bra, ket]: index = bra | ket << 1, value O[bra][ket]
//   ZZDIAG (a, b):           index = a | b << 1, value exp(-i t z_a z_b / 2)
//   rank 4 [a_out, b_out, a_in, b_in]: value U[(a_out b_out), (a_in b_in)]
enum LeafKind : uint8_t {
  LK_ZERO = 0, LK_PLUS = 1, LK_PROJ0 = 2, LK_PROJ1 = 3,
  LK_H = 4, LK_X = 5, LK_Y = 6, LK_Z = 7, LK_RX = 8, LK_RZ = 9,
  LK_ZDIAG = 10, LK_RZDIAG = 11, LK_ZZDIAG = 12,
  LK_ZZ = 13, LK_CNOT = 14,
  LK_OBS_X = 15, LK_OBS_Y = 16, LK_OBS_Z = 17,
  LK_COUNT = 18
};

QTC_HD inline int leaf_rank_of(int kind) {
  switch (kind) {
    case LK_ZERO: case LK_PLUS: case LK_PROJ0: case LK_PROJ1:
    case LK_ZDIAG: case LK_RZDIAG:
      return 1;
    case LK_ZZ: case LK_CNOT:
      return 4;
    default:
      return 2;
  }
}

// A gate table entry: the tensor of `kind` at angle coeff*params[slot] +
// constant, complex conjugated when conj != 0 (bra side).
struct GateSpec {
  uint8_t kind;
  uint8_t conj;
  int16_t slot;        // -1: no parameter
  uint32_t pad;
  double coeff;
  double constant;
};

struct GateEntryDev {
  GateSpec spec;
  uint32_t val_off;    // element offset of the values in the table region
  uint32_t der_off;    // element offset of d(values)/d(params[slot])
  uint32_t rank;
  uint32_t pad;
};

enum SOpCode : uint8_t {
  SOP_CONTRACT = 0,    // out[c] = sum_y in1[.] * in2[.]  (Eq. 1, bit maps)
  SOP_LEAFGRAD = 1,    // grad[out] += sum_j in1[j] * in2[j], 2^rc terms
  SOP_RESULT = 2,      // network scalar = in1[0]
  SOP_SEED = 3         // out[0] = 1 (adjoint of the root)
};

constexpr int kMaxSmemRank = 16;
constexpr uint8_t kAbsent = 0xFF;

// One shared-memory op.  Offsets are element offsets from the start of the
// task's shared memory (gate table region first, then the arena).  For
// CONTRACT, output bit i reads in1 bit p1[i] and in2 bit p2[i] (kAbsent: the
// operand does not carry that label); summed bit j reads in1 bit y1[j] and
// in2 bit y2[j].
struct alignas(16) SOp {
  uint8_t code, rc, ry, pad0;
  uint32_t out, in1, in2;
  uint8_t p1[kMaxSmemRank], p2[kMaxSmemRank];
  uint8_t y1[kMaxSmemRank], y2[kMaxSmemRank];
};

struct TaskDev {
  uint32_t op_begin, op_count;
  uint32_t net;
  uint32_t arena_elems;
};

// Kernel argument of the shared-memory executor.
struct ProgramDev {
  const GateEntryDev* gates;
  int n_gates;
  uint32_t table_elems;        // gate values + derivatives, in elements
  uint32_t table_bytes;        // table region, rounded to 16 bytes
  uint32_t team_bytes;         // per team: staged ops, then its arena
  uint32_t stage_ops;          // ops staged per team at a time
  const TaskDev* tasks;
  int n_tasks;
  const SOp* ops;
  int n_params;
  int n_nets;
  const double* weights;       // per network, for <C>
  const double* params;        // device, n_params
  double* results;             // per network: Re s, Im s, (Re, Im) ds/dparam_k
  double* out;                 // [<C>, d<C>/dparam (n_params), Re s per network]
  unsigned int* counters;      // [0] task queue, [1] finished blocks, [2] error
  int want_grad;
  int qaoa_reduce;             // 1: reduce to the Max-Cut objective
};

}  // namespace qtc
