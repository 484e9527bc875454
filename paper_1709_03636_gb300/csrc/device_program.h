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
//   CNOTX [t_out, c, t_in]: 1 where t_out = t_in xor c (sparse CNOT: the
//     control wire is shared, as for diagonal gates)
//   channel [ket_out, bra_out, ket_in, bra_in] (DEPOL, DEPHASE, AMPDAMP; the
//     strength is the spec's constant): sum_k K_k[ket_out][ket_in]
//     conj(K_k[bra_out][bra_in])
enum LeafKind : uint8_t {
  LK_ZERO = 0, LK_PLUS = 1, LK_PROJ0 = 2, LK_PROJ1 = 3,
  LK_H = 4, LK_X = 5, LK_Y = 6, LK_Z = 7, LK_RX = 8, LK_RZ = 9,
  LK_ZDIAG = 10, LK_RZDIAG = 11, LK_ZZDIAG = 12,
  LK_ZZ = 13, LK_CNOT = 14,
  LK_OBS_X = 15, LK_OBS_Y = 16, LK_OBS_Z = 17,
  LK_DEPOL = 18, LK_DEPHASE = 19, LK_AMPDAMP = 20,
  LK_OBS_I = 21,          // [bra, ket] identity: closes a wire explicitly
  LK_CNOTX = 22,          // CNOT as XOR [t_out, c, t_in]; the control is a hyperedge
  LK_ONES = 23,           // [a] = (1, 1): closes a shared ket/bra wire (trace)
  LK_OBS_P0 = 24, LK_OBS_P1 = 25,   // [bra, ket] projectors |0><0|, |1><1|
  LK_COUNT = 26
};

QTC_HD inline int leaf_rank_of(int kind) {
  switch (kind) {
    case LK_ZERO: case LK_PLUS: case LK_PROJ0: case LK_PROJ1:
    case LK_ZDIAG: case LK_RZDIAG: case LK_ONES:
      return 1;
    case LK_ZZ: case LK_CNOT: case LK_DEPOL: case LK_DEPHASE: case LK_AMPDAMP:
      return 4;
    case LK_CNOTX:
      return 3;
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

// One element of the gate table as coefficients (see gate_coef.cpp):
// value = (a0 + i a1) cos(t/2) + (a2 + i a3) sin(t/2) + (a4 + i a5), with
// t the angle of gate `gate`; derivative elements carry their own
// coefficients.  One record per table element (padding: zeros).
struct alignas(16) TabCoef32 {
  float a[6];
  uint32_t gate;
  uint32_t pad;
};
struct alignas(16) TabCoef64 {
  double a[6];
  uint32_t gate;
  uint32_t pad[3];
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

// Operand locations: by default an op offset is an element offset into the
// task's shared memory (gate table first, then the arena); a flagged operand
// is an element offset into the global work buffer (graph executor only).
enum SOpFlag : uint8_t {
  SOPF_OUT_GLOBAL = 1,
  SOPF_IN1_GLOBAL = 2,
  SOPF_IN2_GLOBAL = 4
};

constexpr int kMaxSmemRank = 16;
constexpr uint8_t kAbsent = 0xFF;

// One shared-memory op.  Offsets are element offsets from the start of the
// task's shared memory (gate table region first, then the arena).  For
// CONTRACT, output bit i reads in1 bit p1[i] and in2 bit p2[i] (kAbsent: the
// operand does not carry that label); summed bit j reads in1 bit y1[j] and
// in2 bit y2[j].
struct alignas(16) SOp {
  uint8_t code, rc, ry, flags;
  uint32_t out, in1, in2;
  uint8_t p1[kMaxSmemRank], p2[kMaxSmemRank];
  uint8_t y1[kMaxSmemRank], y2[kMaxSmemRank];
};

// The same ops for networks run one per warp (every tensor of rank <= 11,
// at most 8 summed bits per op): the bit maps are pre-expanded into offset
// tables.  Output element c = 32 j + lane of a CONTRACT reads
// in1[a_lo[lane] | a_hi[j] | ya[y & 15] | ya_hi[y >> 4]] and in2 likewise.
// A CONTRACT flagged WOPF_LEAFGRAD produces dS/dleaf and also adds
// sum_c out[c] * table[der + c] to the parameter gradient slot `slot` (the
// leaf-gradient dot fused into the op that produces it).
constexpr int kWarpMaxRank = 11;
constexpr int kWarpMaxSummed = 8;
// With at most this many parameters a warp team keeps one complex gradient
// accumulator per (parameter, lane) in shared memory, right after its staged
// steps; each lane adds its own leaf-gradient terms there without shuffles.
constexpr int kWarpLaneGradSlots = 8;

enum WOpFlag : uint8_t { WOPF_LEAFGRAD = 1 };

struct alignas(16) WOp {
  uint8_t code, rc, ry, flags;
  uint16_t out, in1, in2, slot;   // element offsets (team relative), gradient slot
  uint16_t der, pad0;             // WOPF_LEAFGRAD: table offset of d(leaf)/dparam
  uint16_t a_lo[32], b_lo[32];    // output bits 0..4
  uint16_t ya[16], yb[16];        // summed bits 0..3
  uint16_t a_hi[64], b_hi[64];    // output bits 5..10
  uint16_t ya_hi[16], yb_hi[16];  // summed bits 4..7
};
static_assert(sizeof(WOp) == 528, "WOp is staged as 33 16-byte words");

// Warp programs are sequences of steps.  A bundle step packs mutually
// independent small ops into aligned lane groups of one warp (the host
// schedules the op graph of the network; hazards are tracked per element):
// each lane computes at most one output element with at most two summed
// terms, or two of the 4-16 terms of one output whose lanes are then added
// by shuffles.  A solo step runs one WOp on the whole warp (the other ops:
// outputs above 32 elements, or more lanes than the warp has).
enum WLaneKind : uint8_t { WL_IDLE = 0, WL_CONTRACT = 1, WL_RESULT = 2, WL_SEED = 3 };
enum WLaneFlag : uint8_t {
  WLF_STORE = 1,    // write the lane's output element
  WLF_Y1 = 2,       // add the second summed term
  WLF_LG_MUL = 4,   // leaf gradient: group-sum of out * d(leaf)/dparam into slot
  WLF_LG_ADD = 8    // leaf gradient: group-sum of the product itself into slot
};
// Lane offsets count elements from the start of the warp's gate-table copy
// (the table, then the warp's arena).
// WStep::rounds bit 7: some lane adds a leaf gradient (low bits: rounds).
// WLane::gw packs three fields: bits 0-2 log2 of the op's lane-group width;
// for an op summing 2^ry terms (ry = 2..4) spread over 2^(ry-1) lanes per
// output (each lane two terms), bits 3-5 the log2 distance between those
// lanes (the op's rc) and bits 6-7 the shuffle rounds that add them (ry - 1);
// only the lane of the first pair stores and adds leaf-gradient terms.
// WStep::pad[0]: the most such rounds of any lane of the step.
constexpr uint8_t kWHasLeafGrad = 0x80;

// Unused fields are zero: every lane's loads stay at valid offsets.
struct alignas(16) WLane {
  uint8_t kind, flags, gw, slot;   // gw: log2 of the op's lane-group width;
                                   // slot: parameter of a leaf-gradient lane
  uint16_t c_off, a_off, b_off;    // output, first-term operands
  uint16_t der_off;                // WLF_LG_MUL: table offset of d(leaf)/dparam
  uint16_t ya1, yb1;               // WLF_Y1: element deltas of the second term
};

struct alignas(16) WStep {
  uint8_t solo;     // 1: `op` runs on the whole warp
  uint8_t rounds;   // kWHasLeafGrad | shuffle rounds of the leaf-gradient group sums
  uint8_t pad[14];
  union {
    WLane lane[32];
    WOp op;
  };
};
static_assert(sizeof(WStep) == 544, "WStep is staged as 34 16-byte words");

struct TaskDev {
  uint32_t op_begin, op_count;
  uint32_t net;
  uint32_t arena_elems;
};

// Kernel argument of the shared-memory executor.
// Gate table entries passed in the kernel parameters (the rest, if any, are
// read from `gates`): building the gate table then waits only for the
// parameter values themselves.
constexpr int kInlineGates = 16;
// Parameter values a host-pointer call passes in the kernel parameters (the
// warp gate table then reads no parameter from host memory).
constexpr int kInlineParams = 8;

struct ProgramDev {
  const GateEntryDev* gates;
  int n_gates;
  GateEntryDev gates_inline[kInlineGates];   // the first min(n_gates, 16) entries
  const void* coef;            // warp teams: TabCoef32 (complex64) or TabCoef64 per
                               // table element
  uint32_t table_elems;        // gate values + derivatives, in elements
  uint32_t table_bytes;        // table region, rounded to 16 bytes
  uint32_t team_bytes;         // per team: staged ops, then its arena
  uint32_t stage_ops;          // ops staged per team at a time
  uint32_t task_stride;        // warp teams: task t's steps start at t * task_stride
                               // (0: at tasks[t].op_begin)
  const TaskDev* tasks;
  int n_tasks;
  const SOp* ops;              // CTA teams
  const WStep* wsteps;         // warp teams
  int n_params;
  int n_nets;
  const double* weights;       // per network, for <C>
  const double* params;        // device, n_params
  double* results;             // per network: Re s, Im s, (Re, Im) ds/dparam_k
  double* acc;                 // [1 + n_params]: sums over networks of w (1 - Re s)/2 and
                               // -w/2 Re ds/dparam_k; zero between launches
  double* out;                 // [<C>, d<C>/dparam (n_params), Re s per network]
  unsigned int* counters;      // [0] task queue, [1] finished blocks, [2] error
  int want_grad;
  int qaoa_reduce;             // 1: reduce to the Max-Cut objective
  unsigned long long* done;    // optional (host-mapped): set to seq once out is
  unsigned long long seq;      // visible to the host (system-scope release)
  int n_inline_params;         // > 0: params[0 .. n) also in params_inline
  double params_inline[kInlineParams];
};

// ---- graph executor: shared-memory subtrees and global-memory steps ---------

constexpr int kMaxRuns = 12;
constexpr uint32_t kGRow = 256;      // output elements per row of a global step
constexpr uint32_t kYTab = 4096;     // summed-index offsets tabulated per pass
constexpr uint32_t kMaxChunkRows = 64;  // rows of one normal chunk

// Maps bits of one index (output c or summed y) to bits of an operand index:
// offset = OR_r ((idx >> src[r]) & (2^len[r] - 1)) << dst[r].  Labels kept
// in the same relative order in both tensors form few runs.
struct GRuns {
  uint8_t n;
  uint8_t src[kMaxRuns];
  uint8_t len[kMaxRuns];
  uint8_t dst[kMaxRuns];
};

enum GStepFlag : uint16_t {
  GSF_A_TABLE = 1,     // operand A is a gate table entry (shared memory)
  GSF_B_TABLE = 2,
  GSF_SPLIT = 4,       // chunks split the summed index; the last chunk reduces
  GSF_LEAFGRAD = 8,    // output is dS/dleaf: reduce it against d(leaf)/dparam
  GSF_TILE = 16,       // staged through shared memory in tiles (the tile fields)
  GSF_YPAIR = 32,      // summed bit 0 is bit 0 of A and of B (both in global memory):
                       //   complex64 terms are read as 16-byte element pairs
  GSF_LANES_Y = 64,    // split: the summed index's low bits are A's (or B's) lowest
                       //   bits, so a warp's lanes run over it (one warp per output)
  GSF_ROWS = 128       // rows taken four at a time in the order of `rows`, so that the
                       //   four share operand elements (`share`): fewer loads per term
};

// How the four rows of a GSF_ROWS group share operands: row-counter bit 0 and
// bit 1 map to output labels missing from A (A's element is the same for both
// values) or from B.
enum GRowShare : uint8_t {
  GRS_ZX = 1,   // bit 0 not in A, bit 1 not in B: two A and two B elements per term
  GRS_ZZ = 2,   // neither bit in A: one A and four B elements per term
  GRS_XX = 3,   // neither bit in B: four A and one B element per term
  // short sums (1, 2 or 4 summed values): groups of 2^grs_fix_bits(ny) rows whose
  // counter bits all miss one operand, read once per group for all its rows
  GRS_FIXA = 4, // A's elements are the same for the whole group
  GRS_FIXB = 5  // B's elements are the same for the whole group
};

// Row-counter bits of a GRS_FIXA / GRS_FIXB group for ny summed values: 16
// rows for one value, 8 for two, 4 for four (16 loads of the other operand
// in flight per thread).
constexpr int grs_fix_bits(uint32_t ny) { return ny == 1 ? 4 : (ny == 2 ? 3 : 2); }

// Tile form of a global step.  The step's labels split into tile labels
// (varying inside one task) and outer labels: outer output labels (one task
// per value o) and outer summed labels (values q, looped over inside a task,
// or cut into chunks whose partial sums the last chunk adds when the whole
// output lies in the tile).  For every q a task copies the A and B elements
// of its tile (an operand's footprint: the tile labels it holds, in its own
// bit order, so that its lowest bits come first and the copies are
// contiguous 16-byte transfers) into shared memory, contracts there, and
// finally copies its C tile (footprint likewise) out.  Tile index bits:
// [0, 5) lanes, [5, 8) warps, [8, 8 + kout) output labels held in registers,
// the rest summed labels looped over in registers.  Lane and warp bits that
// are summed labels are reduced by shuffles and through shared memory.
constexpr int kTileMaxOut = 2;        // output bits held in registers
constexpr int kTileMaxRegSum = 8;     // summed bits looped over in registers
constexpr uint32_t kTileBudgetBytes = 40960;   // footprints per team

struct GTileMap {
  uint8_t nv, nfa, nfb, nfc;  // tile bits; footprint bits of A, B, C
  uint8_t no, nq;             // outer output bits, outer summed bits
  uint8_t kout, ns;           // register output bits, register summed bits
  uint32_t q_per_chunk;       // outer summed values per chunk (split)
  uint32_t o_per_chunk;       // outer output values per chunk (not split)
  uint8_t sum_lane_mask;      // lane bits that are summed labels
  uint8_t sum_warp_mask;      // warp bits that are summed labels
  uint8_t staged;             // bit 0: A's footprint is copied to shared memory, bit 1: B's
                              //   (otherwise the tile reads the operand where it is)
  uint8_t pad[5];
  GRuns tfa, tfb, tfc;        // tile index -> footprint index (table operand:
                              //   -> its element index)
  GRuns ffa, ffb, ffc;        // footprint index -> operand element index
  GRuns oa, ob, oc;           // outer output index -> operand element index
  GRuns qa, qb;               // outer summed index -> operand element index
};

// One contraction C = sum_y A * B in global memory (Eq. 1), cut into chunks.
// Normal: chunk k computes output rows [k*chunk, (k+1)*chunk) of 256
// elements (one element per thread and row).  Split (outputs <= 256): chunk k
// sums y in [k*chunk, (k+1)*chunk) into partial slot k; the last chunk to
// arrive adds the partials in slot order and writes C (or, for LEAFGRAD,
// accumulates sum_c C[c] * dleaf[c] into the parameter gradient).
struct alignas(16) GStep {
  uint32_t c_off, a_off, b_off;
  uint32_t partial_off;     // split: element offset of n_chunks * 2^rc partials
  uint32_t n_chunks, chunk; // normal: rows per chunk; split: y values per chunk
  uint32_t arrive_ctr;      // split: arrivals (dependency-counter index)
  uint32_t done_ctr;        // completion counter (target n_chunks; split: 1)
  uint32_t der_off;         // leafgrad: table offset of d(leaf)/dparam
  uint32_t net;
  uint16_t flags;
  int16_t slot;             // leafgrad: parameter slot
  uint8_t rc, ry, share, pad1;  // share: GRowShare of a GSF_ROWS step
  GRuns ca, cb;             // output bits -> A bits, B bits
  GRuns ya, yb;             // summed bits -> A bits, B bits
  GRuns rows;               // GSF_ROWS: row counter bits -> output row bits
  GTileMap tile;            // GSF_TILE
};

// One complex GEMM C[b][m][n] = sum_k A[b][m][k] B[b][k][n] (Eq. 1 with the
// batch labels b, free labels m of A and n of B, summed labels k) on the
// tensor cores.  Each FP32 operand component is split into BF16 hi + lo and
// the products hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory.
// Every tensor offset is a bit gather from the logical (b, m, k, n) indices.
// A task computes one tile of 128 rows m by 64 complex columns n.
constexpr uint32_t kTcRows = 128;      // m per tile (the MMA's M)
constexpr uint32_t kTcCols = 64;       // complex n per tile (MMA N = 128 reals)
constexpr uint32_t kTcK = 16;          // complex k per shared-memory stage

struct alignas(16) TStep {
  uint32_t c_off, a_off, b_off;
  uint32_t done_ctr;
  uint32_t net;
  uint32_t m_tiles, n_tiles;
  uint8_t mb, kb, nb, bb;   // log2 of M, K, N and of the batch
  GRuns am, ak, ab;         // A offset from m, k, b
  GRuns bk, bn, bbt;        // B offset from k, n, b
  GRuns cm, cn, cb;         // C offset from m, n, b
};

enum GTaskKind : uint8_t { GT_SMEM = 0, GT_CHUNK = 1, GT_TC = 2 };

struct GTask {
  uint8_t kind;
  uint8_t pad[3];
  uint32_t a;              // SMEM: first op; CHUNK, TC: step index
  uint32_t b;              // SMEM: op count; CHUNK: chunk index; TC: tile index
  uint32_t net;
  uint32_t wait_begin;     // into the wait list
  uint32_t wait_count;
  uint32_t signal;         // SMEM: counter incremented when done (~0u: none)
  uint32_t pad2;
};

struct WaitDev {
  uint32_t counter;
  uint32_t target;
};

// Counter layout: fixed slots in the first 128-byte line, then the
// dependency counters of the wave, one per 128-byte line (teams poll them
// while producers increment others: no two share a line).
enum CounterSlot : uint32_t {
  CTR_QUEUE = 0, CTR_BLOCKS = 1, CTR_ERROR = 2, CTR_RESERVED = 3
};
constexpr uint32_t kCtrHead = 32;     // words before the first dependency counter
constexpr uint32_t kCtrStride = 32;   // words per dependency counter
QTC_HD inline uint64_t ctr_index(uint32_t dep) { return kCtrHead + (uint64_t)dep * kCtrStride; }
QTC_HD inline uint64_t ctr_words(uint32_t n_dep) { return kCtrHead + (uint64_t)n_dep * kCtrStride; }

// Kernel argument of the graph executor (one launch per wave).
struct GraphProgDev {
  const GateEntryDev* gates;
  int n_gates;
  uint32_t table_elems;
  uint32_t table_bytes;        // gate table region, 16-byte rounded
  uint32_t arena_bytes;        // shared-memory arena of SMEM tasks
  uint32_t stage_ops;          // ops staged at a time
  const GTask* tasks;
  int n_tasks;
  const SOp* ops;
  const GStep* steps;
  const TStep* tsteps;         // tensor-core GEMMs
  const WaitDev* waits;
  void* gbase;                 // global work buffer of the wave
  int tmem_cols;               // tensor memory columns per CTA (0: no GEMM tasks)
  int n_params;
  int n_nets;
  int n_counters;              // dependency counters of this wave
  int final_wave;              // 1: reduce, then clear the result rows
  const double* weights;
  const double* params;
  double* results;             // per network: Re s, Im s, (Re, Im) ds/dparam_k
  double* raw_out;             // optional copy of the result rows (final wave)
  double* out;                 // [<C>, d<C>/dparam, Re s per network, status]
  unsigned int* counters;
  int want_grad;
  int qaoa_reduce;
  long long wait_limit_ns;     // bound of every dependency wait
};

}  // namespace qtc
