// Internal host-side structures of the contraction engine.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "qtc.h"
#include "device_program.h"

namespace qtc {

// Threads per CTA of the shared-memory executor (CTA teams), and networks per
// CTA when one warp runs one network.
constexpr int kExecBlock = 128;
constexpr int kWarpTeamsPerCta = 4;

// ---- errors ---------------------------------------------------------------
// Internal code throws Error; every C-ABI entry point catches it, stores the
// message in the thread-local buffer and returns the status.
struct Error {
  qtc_status status;
  std::string msg;
};
[[noreturn]] void fail(qtc_status s, const char* fmt, ...);
void set_last_error(const std::string& msg);

inline void cuda_check(cudaError_t err, const char* what) {
  if (err != cudaSuccess)
    fail(QTC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(err), cudaGetErrorString(err));
}

// Runs f, turning an Error (or a host exception) into a status code and the
// thread-local message.
template <typename F>
qtc_status guarded(F&& f) {
  try {
    f();
    return QTC_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host out of memory");
    return QTC_ERR_INVALID;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return QTC_ERR_INVALID;
  }
}

// Restores the caller's current device on scope exit.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    cuda_check(cudaGetDevice(&prev), "cudaGetDevice");
    if (prev != dev) cuda_check(cudaSetDevice(dev), "cudaSetDevice");
  }
  ~DeviceScope() {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != prev && prev >= 0) cudaSetDevice(prev);
  }
};

// ---- SplitMix64 (Steele, Lea and Flood 2014) -------------------------------
struct SplitMix64 {
  uint64_t state;
  explicit SplitMix64(uint64_t seed) : state(seed) {}
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // integer in [0, k) by the multiply-high map
  uint64_t below(uint64_t k) {
    return (uint64_t)(((unsigned __int128)next() * k) >> 64);
  }
};

// ---- circuits (Section 2, Section 4.1) -----------------------------------
struct Gate {
  int kind;        // qtc_gate
  int q[2];
  int nq;
  int slot;        // parameter slot or -1
  double coeff, constant;
};

struct Circuit {
  int n = 0;
  int n_params = 0;
  int p = 0;                                  // QAOA depth (0: generic)
  std::vector<Gate> gates;
  std::vector<std::pair<int, int>> edges;     // QAOA graph edges
};

bool gate_is_diagonal(int kind);
bool gate_is_channel(int kind);

// ---- networks ---------------------------------------------------------------
// One leaf tensor: the gate table entry that gives its values and its labels
// in storage order (label k <-> bit k of the element index).
struct Leaf {
  GateSpec spec;
  std::vector<int> labels;
};

struct Network {
  int n_labels = 0;
  int n_params = 0;
  std::vector<Leaf> leaves;
};

Network build_network(const Circuit& c, const qtc_observable& obs, bool lightcone,
                      bool diag);

// ---- plans (Algorithms 1 and 2) -------------------------------------------
struct Step {
  int a, b;        // operand tensor ids
};

struct Plan {
  Network net;
  std::vector<Step> steps;
  // labels of every tensor id (leaves 0..L-1, step results L..L+S-1) in
  // storage order: bit k of an element index is labels[k]
  std::vector<std::vector<int>> labels;
  int max_rank = 0;
  double cmacs = 0, bytes_c64 = 0, lg_width = 0;
};

Plan make_plan(const Network& net, const qtc_plan_opts& opts);

// ---- leaf tensors as coefficients (gate_coef.cpp) ---------------------------
// A, B, C (2^rank each) with element = A cos(t/2) + B sin(t/2) + C.
void gate_coefficients(const GateSpec& s, std::complex<double>* A, std::complex<double>* B,
                       std::complex<double>* C);
// The warp executor's coefficient records, one per table element.
std::vector<uint8_t> coefficient_table(const std::vector<GateEntryDev>& gates,
                                       uint32_t table_elems, int dtype);
// Host evaluation: val and der (nullable) as interleaved complex doubles.
void leaf_values(const GateSpec& s, const double* params, double* val, double* der);

// ---- lowering --------------------------------------------------------------
// Deduplicated gate table shared by every network of a batch.
struct GateTable {
  std::vector<GateSpec> specs;
  int add(const GateSpec& s);    // index of s, adding it if new
};

struct LoweredNet {
  std::vector<SOp> ops;
  uint32_t arena_elems = 0;      // per-task shared-memory arena, in elements
  bool fits = false;
};

// One network's shared-memory ops as warp steps (lane-packed bundles of
// independent small ops, solo steps for the rest), appended to `out`.
void build_warp_steps(const std::vector<SOp>& ops, uint32_t table_elems, uint32_t arena_elems,
                      std::vector<WStep>& out);
// Host check of a warp program's every access against its team region.
void validate_warp_steps(const WStep* steps, size_t n, uint32_t team_elems, int n_params);

// Lowers one plan to a shared-memory op program.  table_elems: size of the
// gate value + derivative region that precedes the arena.  Intermediates and
// adjoints of at most private_below elements keep arena buffers of their own
// (no write-after-read ordering between ops that would reuse that memory);
// UINT32_MAX: every buffer.
LoweredNet lower_smem(const Plan& plan, const std::vector<int>& leaf_gate,
                      const std::vector<uint32_t>& gate_val_off,
                      const std::vector<uint32_t>& gate_der_off,
                      uint32_t table_elems, bool want_grad, uint32_t max_elems,
                      uint32_t private_below = 0);

// ---- graph lowering (networks larger than one CTA's shared memory) ---------


struct GraphLimits {
  int small_rank = 10;               // tensors of higher rank live in global memory
  int task_terms_log2 = 16;          // multiply-adds per chunk task of a global step
  uint64_t subtree_elems = 4096;     // elements of all values of one subtree
  uint32_t arena_elems = 8192;       // shared-memory arena of one subtree task
  bool tensor_cores = false;         // split-BF16 GEMM tasks for GEMM-shaped steps
  bool reuse_global = true;          // place global tensors by live range (memory reuse)
  bool reuse_with_deps = false;      // also where it takes new write-after-read dependencies
  int checkpoint_segments = 1;       // > 1: adjoint recomputes dropped values per segment
  int tile_mode = 0;                 // global steps in tile form: 0 never; staged through
                                     // shared memory: 1 steps with two operands in global
                                     // memory, 2 every step that tiles; read in place:
                                     // 3 steps summing >= 3 labels, 4 every step that tiles
  size_t elem = 8;                   // bytes per element
};

// Tile form of a global step (tile_plan.cpp): fills g.tile, g.n_chunks and
// the GSF_TILE / GSF_SPLIT flags when the step tiles (g's rc, ry and bit maps
// already set); false leaves g as it was.
bool encode_tile(GStep& g, const std::vector<int>& lc, const std::vector<int>& la,
                 const std::vector<int>& lb, bool a_table, bool b_table, size_t elem,
                 int task_terms_log2, bool direct);
// Shared memory of a team's work region a tile task needs.
size_t tile_region_bytes(const GStep& g, size_t elem);
// Host emulation of one tile step on seeded random operands against the
// plain contraction over its bit maps: the largest absolute difference.
double emulate_tile_step(const GStep& g, uint64_t seed);
double emulate_rows_step(const GStep& g, uint64_t seed);

// A unit is one shared-memory subtree task or one global step (its chunks);
// its counter reaches `target` when it is complete.
struct GUnit {
  int kind = GT_SMEM;
  std::vector<SOp> ops;              // GT_SMEM
  GStep step{};                      // GT_CHUNK
  TStep tstep{};                     // GT_TC
  uint32_t arena_elems = 0;
  std::vector<int> deps;             // units that must be complete first
  int depth = 0;
  uint32_t target = 1;
};

// A global tensor's placement: element offset and size in the network's
// work-buffer region, its live range over the units (creation order), the
// units that write it and every unit that touches it.
struct GBuffer {
  uint64_t at, size;
  int first, last;
  std::vector<int> writers, users;
};

struct NetGraph {
  std::vector<GUnit> units;
  uint64_t global_elems = 0;         // global buffers of this network (elements)
  uint64_t unshared_elems = 0;       // the same with a region per tensor (no reuse)
  std::vector<GBuffer> buffers;      // placement by live range (empty without reuse)
  int checkpoint_segments = 1;       // segments the adjoint sweep recomputes by
  int recomputed_segments = 0;       // of which recomputed (all but the last)
  bool fits = true;
  std::string why;
};

// Overlaps the network's global tensors whose uses are ordered: where every
// unit touching one already precedes (through the dependencies) every unit
// writing the other, or, with add_deps, wherever their live ranges in unit
// order are disjoint, adding the write-after-read dependencies that takes.
// Rewrites every work-buffer offset; global_elems becomes the peak.
void place_global_buffers(NetGraph& ng, const std::vector<uint64_t>& vbase,
                          const std::vector<uint64_t>& vsize, bool add_deps);
// Host check of that placement (ordering of every reuse; no live overlap).
void check_global_placement(const NetGraph& ng);

// Lowers one plan to units: maximal subtrees of small steps run in shared
// memory (and are recomputed for the adjoint sweep), the other steps are
// chunked global contractions.  Global offsets are network-local.
NetGraph lower_graph(const Plan& plan, const std::vector<int>& leaf_gate,
                     const std::vector<uint32_t>& gate_val_off,
                     const std::vector<uint32_t>& gate_der_off, uint32_t table_elems,
                     bool want_grad, const GraphLimits& lim);

// How programs are formed: force_graph runs even small networks through the
// graph executor; small_rank <= 0 keeps the default threshold (10).
struct ProgramOptions {
  size_t wave_cap_bytes = (size_t)8 << 30;
  bool force_graph = false;
  int small_rank = 0;
  int tile_mode = 0;               // see GraphLimits::tile_mode
  int task_terms_log2 = 16;        // multiply-adds per chunk task of a global step
  int subtree_bytes = 32768;       // values of one shared-memory subtree task
  int warp_teams = 1;              // 0: one network per CTA; 1: per warp where it fits;
                                   // 2: per warp, steps always streamed
  int sm_count = 152;              // SMs of the device the program is laid out for
  bool graph_hi_occupancy = false; // graph executor: the five-CTAs-per-SM instantiation
  bool operator==(const ProgramOptions& o) const {
    return wave_cap_bytes == o.wave_cap_bytes && force_graph == o.force_graph &&
           small_rank == o.small_rank && task_terms_log2 == o.task_terms_log2 &&
           tile_mode == o.tile_mode &&
           subtree_bytes == o.subtree_bytes && warp_teams == o.warp_teams &&
           sm_count == o.sm_count && graph_hi_occupancy == o.graph_hi_occupancy;
  }
};

// One wave of the graph executor: its tasks, op lists, global steps, waits,
// work-buffer size and dependency counters.
struct WaveHost {
  std::vector<GTask> tasks;
  std::vector<SOp> ops;
  std::vector<GStep> steps;
  std::vector<TStep> tsteps;
  std::vector<WaitDev> waits;
  uint64_t global_elems = 0;
  uint32_t n_counters = 0;
};

// Host copy of a batch's device program for one element type and gradient
// flag.  Shared-memory form: the gate table, one task per network (largest
// first) and the op lists.  Graph form (some network does not fit one CTA's
// shared memory): waves of graph-executor tasks.
struct HostProgram {
  int dtype = 0, want_grad = 0;
  size_t max_dynamic = 0;          // shared-memory budget it was lowered for
  std::vector<GateEntryDev> gates;
  std::vector<TaskDev> tasks;
  std::vector<SOp> ops;            // CTA teams (empty for warp teams)
  std::vector<WStep> wsteps;       // warp teams
  std::vector<uint8_t> coef;       // warp teams: gate table coefficient records
  std::vector<double> weights;
  uint32_t table_elems = 0, max_arena = 0;
  uint32_t table_bytes = 0;        // gate table region, 16-byte rounded
  uint32_t team_bytes = 0;         // per team: staged ops + arena
  uint32_t stage_ops = 0;          // ops staged per team at a time
  uint32_t task_stride = 0;        // warp steps of task t start at t * task_stride (0: packed)
  bool warp_teams = false;         // one network per warp (small networks)
  bool stream_steps = false;       // warp teams read their steps from global memory
  int n_teams = 1;                 // teams per CTA
  int block = kExecBlock;          // threads per CTA
  size_t smem = 0;                 // dynamic shared memory per CTA, bytes
  int n_nets = 0, n_params = 0;
  int qaoa_reduce = 1;
  uint64_t serial = 0;             // process-unique id of this program
  ProgramOptions options;          // options it was built with
  bool graph = false;
  std::vector<WaveHost> waves;
  uint32_t work_bytes = 0;         // graph form: shared memory after the table
  uint64_t max_global_elems = 0;
  uint64_t sum_global_elems = 0;   // over networks: each network's placed peak
  uint64_t sum_unshared_elems = 0; // over networks: a region per global tensor
  int max_checkpoint_segments = 1; // most checkpoint segments of any network
  uint32_t max_counters = 0;
  bool tensor_cores = false;       // some wave has tensor-core GEMM tasks
  bool tiles = false;              // some wave has steps in tile form
};

// Built once per (batch, dtype, want_grad, budget, options) and cached in the
// batch.
const HostProgram& host_program(qtc_batch* b, int dtype, int want_grad, size_t max_dynamic,
                                const ProgramOptions& opts = ProgramOptions());

// Fills hp's graph form (hp.dtype, want_grad and table_elems already set).
void build_graph_program(HostProgram& hp, const std::vector<Plan>& plans,
                         const std::vector<std::vector<int>>& leaf_gate,
                         const std::vector<uint32_t>& val_off,
                         const std::vector<uint32_t>& der_off, size_t max_dynamic,
                         const ProgramOptions& opts);

inline size_t elem_bytes(int dtype) { return dtype == QTC_C128 ? 16 : 8; }

// Dynamic shared memory a CTA of the executor may use: the opt-in limit
// minus 16 KB for the kernel's static shared memory (about 10 KB).
inline size_t max_dynamic_smem(size_t optin) { return optin > 16384 ? optin - 16384 : 0; }


}  // namespace qtc
