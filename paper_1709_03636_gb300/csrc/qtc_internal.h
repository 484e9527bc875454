// Internal host-side structures of the contraction engine.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "qtc.h"
#include "device_program.h"

namespace qtc {

// ---- errors ---------------------------------------------------------------
// Internal code throws Error; every C-ABI entry point catches it, stores the
// message in the thread-local buffer and returns the status.
struct Error {
  qtc_status status;
  std::string msg;
};
[[noreturn]] void fail(qtc_status s, const char* fmt, ...);
void set_last_error(const std::string& msg);

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

// Lowers one plan to a shared-memory op program.  table_elems: size of the
// gate value + derivative region that precedes the arena.
LoweredNet lower_smem(const Plan& plan, const std::vector<int>& leaf_gate,
                      const std::vector<uint32_t>& gate_val_off,
                      const std::vector<uint32_t>& gate_der_off,
                      uint32_t table_elems, bool want_grad, uint32_t max_elems);

}  // namespace qtc
