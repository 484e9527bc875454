// C ABI of the engine (declared in include/qtc.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <memory>
#include <thread>

#include <cuda_runtime.h>

#include "exec_launch.h"
#include "qtc_internal.h"
#include "sv_launch.h"

namespace qtc {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(qtc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  throw Error{s, buf};
}


// A batch's program resident in one engine's arena.
struct Prepared {
  const void* engine = nullptr;
  uint64_t generation = 0;
  int dtype = 0;
  int want_grad = 0;
  ProgramDev prog{};
  int grid = 0, block = 0;
  size_t smem = 0;
  bool warp_teams = false;
  bool stream = false;               // warp teams: steps streamed from global memory
  bool graph = false;
  bool hi_occ = false;               // graph form: the five-CTAs-per-SM instantiation
  bool tiles = false;                // graph form: the instantiation with tile steps
  int per_sm = 0;                    // resident CTAs per SM reported by the runtime
  std::vector<GraphProgDev> waves;   // graph form: one launch each
  double* raw = nullptr;             // graph form: copy of the result rows
};

}  // namespace qtc

using namespace qtc;

struct qtc_engine {
  int device = 0;
  char* arena = nullptr;
  size_t bytes = 0;
  size_t used = 0;
  uint64_t generation = 1;
  int sm_count = 0;
  size_t smem_optin = 0;
  int last_launches = 0;
  ProgramOptions options;                    // wave limit, graph forcing
  double wait_limit_ms = 10000.0;            // bound of every device-side wait

  // Program tables grow from the front of the arena; the graph executor's
  // work buffer sits at the back and is shared by every graph program of the
  // engine (their launches are ordered on the caller's stream).
  size_t work = 0;

  char* alloc(size_t n) {
    size_t at = (used + 255) & ~size_t(255);
    if (at + n > bytes - work)
      fail(QTC_ERR_ARENA, "arena of %zu bytes is too small: need %zu more at offset %zu (%zu "
           "reserved for the work buffer)", bytes, n, at, work);
    used = at + n;
    return arena + at;
  }

  void reserve_work(size_t n) {
    n = (n + 255) & ~size_t(255);
    if (n <= work) return;
    if (used + n > bytes)
      fail(QTC_ERR_ARENA, "arena of %zu bytes is too small: the work buffer needs %zu bytes and "
           "program tables use %zu", bytes, n, used);
    work = n;
  }

  char* work_base() const { return arena + bytes - work; }

  // Host-pointer calls pass parameters and results through a small pinned,
  // device-mapped host buffer: the kernel reads and writes it in place, so a
  // call is one launch with no copies.  The shared-memory executor also
  // publishes a sequence number there once its results are visible, and the
  // call returns on that (its launch may still be retiring): a reallocation
  // or the engine's end waits for the device first.
  double* staging_host = nullptr;
  double* staging_dev = nullptr;
  size_t staging_elems = 0;
  uint64_t seq = 0;

  double* staging(size_t n) {
    if (n > staging_elems) {
      if (staging_host) {
        cuda_check(cudaDeviceSynchronize(), "synchronise before freeing the staging buffer");
        cuda_check(cudaFreeHost(staging_host), "free staging buffer");
      }
      staging_host = nullptr;
      staging_elems = 0;
      void* h = nullptr;
      cuda_check(cudaHostAlloc(&h, sizeof(double) * n, cudaHostAllocMapped),
                 "allocate staging buffer");
      staging_host = (double*)h;
      staging_elems = n;
      void* d = nullptr;
      cuda_check(cudaHostGetDevicePointer(&d, h, 0), "map staging buffer");
      staging_dev = (double*)d;
    }
    return staging_host;
  }

  ~qtc_engine() {
    if (staging_host) {
      int cur = -1;
      cudaGetDevice(&cur);
      cudaSetDevice(device);
      cudaDeviceSynchronize();
      cudaFreeHost(staging_host);
      if (cur >= 0) cudaSetDevice(cur);
    }
  }
};

// Device tables of the state-vector reference for one circuit and engine.
struct SvPrepared {
  const void* engine = nullptr;
  uint64_t generation = 0;
  uint32_t* adj = nullptr;
  int2* edges = nullptr;
  double* params = nullptr;
  double* acc = nullptr;
  SvTables tabs[2];   // per dtype (0: complex double, 1: complex float)
};

struct qtc_circuit {
  Circuit c;
  std::vector<SvPrepared> sv;
};
struct qtc_network {
  Network net;
};
struct qtc_batch {
  Circuit circuit;
  std::vector<Plan> plans;
  std::vector<std::pair<int, int>> obs_edges;
  std::vector<double> weights;
  int qaoa_reduce = 1;
  std::vector<Prepared> prepared;
  std::vector<std::unique_ptr<HostProgram>> host_programs;
};
struct qtc_plan {
  Plan plan;
  std::unique_ptr<qtc_batch> single;  // one-network batch for qtc_contract
};

template <typename V>
static V* upload(qtc_engine* e, const std::vector<V>& v, cudaStream_t stream, const char* what) {
  V* d = (V*)e->alloc(sizeof(V) * std::max<size_t>(v.size(), 1));
  if (!v.empty())
    cuda_check(cudaMemcpyAsync(d, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice, stream),
               what);
  return d;
}

extern "C" const char* qtc_last_error(void) { return g_last_error.c_str(); }

// ---- engine ------------------------------------------------------------------

extern "C" qtc_status qtc_engine_create(int device, void* arena, size_t arena_bytes,
                                        qtc_engine** out) {
  return guarded([&] {
    if (!out) fail(QTC_ERR_INVALID, "null output handle");
    if (!arena || ((uintptr_t)arena & 255)) fail(QTC_ERR_INVALID, "arena must be 256-byte aligned");
    int count = 0;
    cuda_check(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
    if (device < 0 || device >= count) fail(QTC_ERR_INVALID, "device %d of %d", device, count);
    auto e = std::make_unique<qtc_engine>();
    e->device = device;
    e->arena = (char*)arena;
    // the work buffer sits at the back of the arena: a length that is a
    // multiple of 256 keeps its start (and every element in it) aligned
    e->bytes = arena_bytes & ~size_t(255);
    int v = 0;
    cuda_check(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device), "SM count");
    e->sm_count = v;
    e->options.sm_count = v;
    cuda_check(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device),
               "shared memory limit");
    e->smem_optin = (size_t)v;
    *out = e.release();
  });
}

extern "C" void qtc_engine_destroy(qtc_engine* e) { delete e; }

extern "C" qtc_status qtc_engine_reset(qtc_engine* e) {
  return guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    e->used = 0;
    e->work = 0;
    e->generation += 1;
  });
}

extern "C" int qtc_engine_last_launches(const qtc_engine* e) { return e ? e->last_launches : 0; }

extern "C" qtc_status qtc_engine_set_limits(qtc_engine* e, size_t max_wave_bytes,
                                            double wait_limit_ms) {
  return guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    if (max_wave_bytes < (1u << 20)) fail(QTC_ERR_INVALID, "wave limit below 1 MiB");
    if (!(wait_limit_ms > 0.0)) fail(QTC_ERR_INVALID, "wait limit must be positive");
    e->options.wave_cap_bytes = max_wave_bytes;
    e->wait_limit_ms = wait_limit_ms;
    e->generation += 1;  // programs are re-prepared with the new limits
    e->used = 0;
    e->work = 0;
  });
}

extern "C" qtc_status qtc_engine_set_graph_options(qtc_engine* e, int force_graph,
                                                   int small_rank) {
  return guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    if (small_rank < 0 || small_rank > 16) fail(QTC_ERR_INVALID, "small rank %d", small_rank);
    e->options.force_graph = force_graph != 0;
    e->options.small_rank = small_rank;
    e->generation += 1;
    e->used = 0;
    e->work = 0;
  });
}

extern "C" qtc_status qtc_engine_set_task_options(qtc_engine* e, int task_terms_log2,
                                                  int subtree_bytes, int warp_teams,
                                                  int graph_hi_occupancy) {
  return guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    if (task_terms_log2 < 12 || task_terms_log2 > 20)
      fail(QTC_ERR_INVALID, "task size 2^%d multiply-adds (12..20)", task_terms_log2);
    if (subtree_bytes < 4096 || subtree_bytes > 32768)
      fail(QTC_ERR_INVALID, "subtree of %d bytes (4096..32768)", subtree_bytes);
    e->options.task_terms_log2 = task_terms_log2;
    e->options.subtree_bytes = subtree_bytes;
    if (warp_teams < 0 || warp_teams > 2)
      fail(QTC_ERR_INVALID, "warp_teams %d (0..2)", warp_teams);
    e->options.warp_teams = warp_teams;
    e->options.graph_hi_occupancy = graph_hi_occupancy != 0;
    e->generation += 1;
    e->used = 0;
    e->work = 0;
  });
}

extern "C" qtc_status qtc_engine_set_tile_mode(qtc_engine* e, int mode) {
  return guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    if (mode < 0 || mode > 4) fail(QTC_ERR_INVALID, "tile mode %d (0..4)", mode);
    e->options.tile_mode = mode;
    e->generation += 1;
    e->used = 0;
    e->work = 0;
  });
}

extern "C" qtc_status qtc_selftest_tile_steps(qtc_batch* b, int dtype, int want_grad,
                                              int force_graph, int small_rank, int tile_mode,
                                              int max_bits, double* max_err, int32_t* n_checked) {
  return guarded([&] {
    if (!b || !max_err || !n_checked) fail(QTC_ERR_INVALID, "null argument");
    ProgramOptions opts;
    opts.force_graph = force_graph != 0;
    opts.small_rank = small_rank;
    opts.tile_mode = tile_mode;
    const HostProgram& hp = host_program(b, dtype, want_grad, max_dynamic_smem(232448), opts);
    double err = 0;
    int n = 0;
    uint64_t seed = 1;
    for (const WaveHost& w : hp.waves)
      for (const GStep& st : w.steps)
        if ((st.flags & GSF_TILE) && st.rc + st.ry <= max_bits) {
          err = std::max(err, emulate_tile_step(st, seed++));
          ++n;
        } else if ((st.flags & GSF_ROWS) && st.rc + st.ry <= max_bits) {
          err = std::max(err, emulate_rows_step(st, seed++));
          ++n;
        }
    *max_err = err;
    *n_checked = n;
  });
}

extern "C" qtc_status qtc_selftest_wait_timeout(qtc_engine* e, void* stream) {
  qtc_status result = QTC_OK;
  qtc_status st = guarded([&] {
    if (!e) fail(QTC_ERR_INVALID, "null engine");
    DeviceScope scope(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    // one task waiting for a counter that nothing signals
    std::vector<GTask> tasks(1);
    tasks[0] = GTask{};
    tasks[0].kind = GT_SMEM;
    tasks[0].wait_begin = 0;
    tasks[0].wait_count = 1;
    tasks[0].signal = 0xFFFFFFFFu;
    std::vector<WaitDev> waits{{0u, 1u}};
    const size_t mark = e->used;
    GraphProgDev d{};
    d.tasks = upload(e, tasks, s, "upload tasks");
    d.n_tasks = 1;
    d.waits = upload(e, waits, s, "upload waits");
    d.n_counters = 1;
    d.final_wave = 1;
    auto* cnt = (unsigned int*)e->alloc(sizeof(unsigned int) * ctr_words(1));
    auto* out = (double*)e->alloc(sizeof(double) * 2);
    auto* params = (double*)e->alloc(sizeof(double));
    auto* res = (double*)e->alloc(sizeof(double) * 2);
    d.counters = cnt;
    d.out = out;
    d.params = params;
    d.results = res;
    d.wait_limit_ns = (long long)(e->wait_limit_ms * 1e6);
    d.table_bytes = 0;
    d.arena_bytes = 0;
    d.stage_ops = 1;
    cuda_check(cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * ctr_words(1), s), "clear");
    int per_sm = 0;
    const size_t max_dyn = max_dynamic_smem(e->smem_optin);
    const size_t smem = 2 * (size_t)kYTab * sizeof(uint32_t) + 256 * 16;
    cuda_check(graph_exec_configure(1, false, false, false, smem, max_dyn, &per_sm), "configure");
    cuda_check(graph_exec_launch(d, 1, false, false, 1, smem, s), "launch");
    double host_out[2] = {0, 0};
    cuda_check(cudaMemcpyAsync(host_out, out, sizeof host_out, cudaMemcpyDeviceToHost, s), "read");
    cuda_check(cudaStreamSynchronize(s), "synchronise");
    e->used = mark;
    if (host_out[1] != 0.0) {
      result = (qtc_status)(int)host_out[1];
      set_last_error("the forged dependency wait expired as intended");
    }
  });
  return st != QTC_OK ? st : result;
}

// ---- circuits ------------------------------------------------------------------

extern "C" qtc_status qtc_circuit_create(int n, int n_params, qtc_circuit** out) {
  return guarded([&] {
    if (!out) fail(QTC_ERR_INVALID, "null output handle");
    if (n <= 0 || n > 4096) fail(QTC_ERR_INVALID, "qubit count %d", n);
    if (n_params < 0 || n_params > 64) fail(QTC_ERR_INVALID, "parameter count %d (max 64)", n_params);
    auto c = std::make_unique<qtc_circuit>();
    c->c.n = n;
    c->c.n_params = n_params;
    *out = c.release();
  });
}

static void add_gate(Circuit& c, int kind, const int32_t* qubits, int slot, double coeff,
                     double constant) {
  Gate g{};
  g.kind = kind;
  g.slot = slot;
  g.coeff = coeff;
  g.constant = constant;
  switch (kind) {
    case QTC_GATE_H: case QTC_GATE_X: case QTC_GATE_Y: case QTC_GATE_Z:
    case QTC_GATE_RX: case QTC_GATE_RZ:
      g.nq = 1;
      break;
    case QTC_GATE_ZZ: case QTC_GATE_CNOT:
      g.nq = 2;
      break;
    case QTC_GATE_DEPOLARIZE: case QTC_GATE_DEPHASE: case QTC_GATE_AMPDAMP:
      g.nq = 1;
      if (slot != -1) fail(QTC_ERR_INVALID, "a channel's strength is a constant (slot -1)");
      if (!(constant >= 0.0 && constant <= 1.0))
        fail(QTC_ERR_INVALID, "channel strength %g outside [0, 1]", constant);
      g.coeff = 0.0;
      break;
    default:
      fail(QTC_ERR_INVALID, "unknown gate kind %d", kind);
  }
  if (!qubits) fail(QTC_ERR_INVALID, "null qubit list");
  for (int k = 0; k < g.nq; ++k) {
    if (qubits[k] < 0 || qubits[k] >= c.n) fail(QTC_ERR_INVALID, "qubit %d out of range", qubits[k]);
    g.q[k] = qubits[k];
  }
  if (g.nq == 2 && g.q[0] == g.q[1]) fail(QTC_ERR_INVALID, "two-qubit gate on one qubit");
  const bool parametric = kind == QTC_GATE_RX || kind == QTC_GATE_RZ || kind == QTC_GATE_ZZ;
  if (slot >= 0 && (!parametric || slot >= c.n_params))
    fail(QTC_ERR_INVALID, "parameter slot %d invalid for gate kind %d", slot, kind);
  if (slot < -1) fail(QTC_ERR_INVALID, "parameter slot %d", slot);
  if (!std::isfinite(coeff) || !std::isfinite(constant)) fail(QTC_ERR_INVALID, "non-finite angle");
  c.gates.push_back(g);
}

extern "C" qtc_status qtc_circuit_add_gate(qtc_circuit* c, int gate, const int32_t* qubits,
                                           int slot, double coeff, double constant) {
  return guarded([&] {
    if (!c) fail(QTC_ERR_INVALID, "null circuit");
    add_gate(c->c, gate, qubits, slot, coeff, constant);
  });
}

// QAOA Max-Cut circuit of Section 4.1; channel >= 0 adds that channel on
// every qubit after each layer's mixer.
static qtc_circuit* make_qaoa(int n, const int32_t* edges, int m, int p, int channel,
                              double strength) {
  if (n <= 1 || n > 4096) fail(QTC_ERR_INVALID, "qubit count %d", n);
  if (p <= 0 || 2 * p > 64) fail(QTC_ERR_INVALID, "depth p = %d (1..32)", p);
  if (m <= 0 || !edges) fail(QTC_ERR_INVALID, "empty edge list");
  auto c = std::make_unique<qtc_circuit>();
  Circuit& cc = c->c;
  cc.n = n;
  cc.n_params = 2 * p;
  cc.p = p;
  std::vector<std::pair<int, int>> seen;
  for (int i = 0; i < m; ++i) {
    int a = edges[2 * i], b = edges[2 * i + 1];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b)
      fail(QTC_ERR_INVALID, "edge %d = (%d, %d) invalid", i, a, b);
    std::pair<int, int> key(std::min(a, b), std::max(a, b));
    if (std::find(seen.begin(), seen.end(), key) != seen.end())
      fail(QTC_ERR_INVALID, "edge (%d, %d) repeated", a, b);
    seen.push_back(key);
    cc.edges.push_back({a, b});
  }
  for (int q = 0; q < n; ++q) add_gate(cc, QTC_GATE_H, &q, -1, 0, 0);
  for (int k = 0; k < p; ++k) {
    for (auto& e : cc.edges) {
      int32_t qs[2] = {e.first, e.second};
      add_gate(cc, QTC_GATE_ZZ, qs, k, 1.0, 0.0);        // exp(-i gamma_k ZZ/2)
    }
    for (int q = 0; q < n; ++q) add_gate(cc, QTC_GATE_RX, &q, p + k, 2.0, 0.0);  // RX(2 beta_k)
    if (channel >= 0)
      for (int q = 0; q < n; ++q) add_gate(cc, channel, &q, -1, 0.0, strength);
  }
  return c.release();
}

extern "C" qtc_status qtc_circuit_qaoa(int n, const int32_t* edges, int m, int p,
                                       qtc_circuit** out) {
  return guarded([&] {
    if (!out) fail(QTC_ERR_INVALID, "null output handle");
    *out = make_qaoa(n, edges, m, p, -1, 0.0);
  });
}

extern "C" qtc_status qtc_circuit_qaoa_noisy(int n, const int32_t* edges, int m, int p,
                                             int channel, double strength, qtc_circuit** out) {
  return guarded([&] {
    if (!out) fail(QTC_ERR_INVALID, "null output handle");
    if (channel != QTC_GATE_DEPOLARIZE && channel != QTC_GATE_DEPHASE &&
        channel != QTC_GATE_AMPDAMP)
      fail(QTC_ERR_INVALID, "gate kind %d is not a noise channel", channel);
    *out = make_qaoa(n, edges, m, p, channel, strength);
  });
}

extern "C" void qtc_circuit_destroy(qtc_circuit* c) { delete c; }

// ---- networks and plans ----------------------------------------------------------

extern "C" qtc_status qtc_network_build(const qtc_circuit* c, const qtc_observable* obs,
                                        int lightcone, int diag_mode, qtc_network** out) {
  return guarded([&] {
    if (!c || !obs || !out) fail(QTC_ERR_INVALID, "null argument");
    auto n = std::make_unique<qtc_network>();
    n->net = build_network(c->c, *obs, lightcone != 0, diag_mode != 0);
    *out = n.release();
  });
}

extern "C" qtc_status qtc_network_leaf_values(const qtc_network* n, int leaf,
                                              const double* params, double* val, double* der) {
  return guarded([&] {
    if (!n || !val) fail(QTC_ERR_INVALID, "null argument");
    if (leaf < 0 || leaf >= (int)n->net.leaves.size())
      fail(QTC_ERR_INVALID, "leaf %d of %zu", leaf, n->net.leaves.size());
    const GateSpec& s = n->net.leaves[leaf].spec;
    if (s.slot >= 0 && !params) fail(QTC_ERR_INVALID, "leaf %d needs params", leaf);
    leaf_values(s, params, val, der);
  });
}

extern "C" qtc_status qtc_network_leaves(const qtc_network* n, int32_t* counts, int32_t* kind,
                                         int32_t* conj, int32_t* slot, double* coeff,
                                         double* constant, int32_t* labels) {
  return guarded([&] {
    if (!n) fail(QTC_ERR_INVALID, "null network");
    const Network& net = n->net;
    if (counts) {
      counts[0] = (int32_t)net.leaves.size();
      counts[1] = net.n_labels;
    }
    for (size_t i = 0; i < net.leaves.size(); ++i) {
      const Leaf& l = net.leaves[i];
      if (kind) kind[i] = l.spec.kind;
      if (conj) conj[i] = l.spec.conj;
      if (slot) slot[i] = l.spec.slot;
      if (coeff) coeff[i] = l.spec.coeff;
      if (constant) constant[i] = l.spec.constant;
      if (labels)
        for (int k = 0; k < 4; ++k)
          labels[4 * i + k] = k < (int)l.labels.size() ? l.labels[k] : -1;
    }
  });
}

extern "C" void qtc_network_destroy(qtc_network* n) { delete n; }

static qtc_plan_opts default_opts() {
  qtc_plan_opts o{};
  o.kind = QTC_ORDER_LG;
  o.seed = 0;
  o.max_rejections = 10;
  o.restarts = 8;
  o.budget_ms = 0;
  return o;
}

extern "C" qtc_status qtc_plan_create(const qtc_network* n, const qtc_plan_opts* opts,
                                      qtc_plan** out) {
  return guarded([&] {
    if (!n || !out) fail(QTC_ERR_INVALID, "null argument");
    auto p = std::make_unique<qtc_plan>();
    p->plan = make_plan(n->net, opts ? *opts : default_opts());
    *out = p.release();
  });
}

extern "C" qtc_status qtc_plan_reuse(const qtc_plan* like, const qtc_network* n,
                                     qtc_plan** out) {
  return guarded([&] {
    if (!like || !n || !out) fail(QTC_ERR_INVALID, "null argument");
    const Network& a = like->plan.net;
    const Network& b = n->net;
    if (a.n_labels != b.n_labels || a.leaves.size() != b.leaves.size())
      fail(QTC_ERR_INVALID, "networks differ in structure (%zu vs %zu leaves)", a.leaves.size(),
           b.leaves.size());
    for (size_t i = 0; i < a.leaves.size(); ++i)
      if (a.leaves[i].labels != b.leaves[i].labels)
        fail(QTC_ERR_INVALID, "networks differ in structure at leaf %zu", i);
    auto p = std::make_unique<qtc_plan>();
    p->plan = like->plan;
    p->plan.net = b;   // same labels, the new tensor values
    *out = p.release();
  });
}

extern "C" qtc_status qtc_plan_stats(const qtc_plan* p, qtc_plan_info* info) {
  return guarded([&] {
    if (!p || !info) fail(QTC_ERR_INVALID, "null argument");
    const Plan& pl = p->plan;
    info->n_tensors = (int)pl.net.leaves.size();
    info->n_labels = pl.net.n_labels;
    info->n_steps = (int)pl.steps.size();
    info->max_rank = pl.max_rank;
    info->cmacs = pl.cmacs;
    info->bytes_c64 = pl.bytes_c64;
    info->lg_width = pl.lg_width;
  });
}

extern "C" qtc_status qtc_plan_steps(const qtc_plan* p, int32_t* lhs, int32_t* rhs) {
  return guarded([&] {
    if (!p || !lhs || !rhs) fail(QTC_ERR_INVALID, "null argument");
    for (size_t s = 0; s < p->plan.steps.size(); ++s) {
      lhs[s] = p->plan.steps[s].a;
      rhs[s] = p->plan.steps[s].b;
    }
  });
}

extern "C" qtc_status qtc_plan_step_shapes(const qtc_plan* p, int32_t* shapes) {
  return guarded([&] {
    if (!p || !shapes) fail(QTC_ERR_INVALID, "null argument");
    const Plan& pl = p->plan;
    const int L = (int)pl.net.leaves.size();
    auto has = [](const std::vector<int>& v, int x) {
      return std::find(v.begin(), v.end(), x) != v.end();
    };
    for (size_t s = 0; s < pl.steps.size(); ++s) {
      const auto& la = pl.labels[pl.steps[s].a];
      const auto& lb = pl.labels[pl.steps[s].b];
      const auto& lc = pl.labels[L + s];
      int nb = 0, nx = 0, ny = 0, nz = 0;
      for (int x : la) {
        if (has(lc, x)) (has(lb, x) ? nb : nx) += 1;
        else ny += 1;
      }
      for (int x : lb)
        if (!has(la, x)) (has(lc, x) ? nz : ny) += 1;
      shapes[4 * s] = nb;
      shapes[4 * s + 1] = nx;
      shapes[4 * s + 2] = ny;
      shapes[4 * s + 3] = nz;
    }
  });
}

extern "C" void qtc_plan_destroy(qtc_plan* p) { delete p; }

// ---- batches --------------------------------------------------------------------

extern "C" qtc_status qtc_batch_create(const qtc_circuit* c, const int32_t* obs_edges, int m,
                                       int lightcone, int diag_mode, const qtc_plan_opts* opts,
                                       qtc_batch** out) {
  return guarded([&] {
    if (!c || !out) fail(QTC_ERR_INVALID, "null argument");
    auto b = std::make_unique<qtc_batch>();
    b->circuit = c->c;
    if (obs_edges) {
      if (m <= 0) fail(QTC_ERR_INVALID, "observable edge count %d", m);
      for (int i = 0; i < m; ++i) b->obs_edges.push_back({obs_edges[2 * i], obs_edges[2 * i + 1]});
    } else {
      if (c->c.edges.empty()) fail(QTC_ERR_INVALID, "circuit has no QAOA edges; pass obs_edges");
      b->obs_edges = c->c.edges;
    }
    const qtc_plan_opts o = opts ? *opts : default_opts();
    const int N = (int)b->obs_edges.size();
    b->plans.resize(N);
    b->weights.assign(N, 1.0);
    std::vector<Error> errors(N, Error{QTC_OK, ""});
    auto work = [&](int i) {
      try {
        qtc_observable obs{};
        obs.kind = QTC_OBS_ZZ;
        obs.u = b->obs_edges[i].first;
        obs.v = b->obs_edges[i].second;
        Network net = build_network(b->circuit, obs, lightcone != 0, diag_mode != 0);
        qtc_plan_opts oi = o;
        oi.seed = o.seed + 0x9E3779B97F4A7C15ull * (uint64_t)i;
        b->plans[i] = make_plan(net, oi);
      } catch (const Error& e) {
        errors[i] = e;
      }
    };
    unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < hw; ++t)
      pool.emplace_back([&, t] {
        for (int i = (int)t; i < N; i += (int)hw) work(i);
      });
    for (auto& th : pool) th.join();
    for (auto& e : errors)
      if (e.status != QTC_OK) throw e;
    *out = b.release();
  });
}

extern "C" qtc_status qtc_batch_stats(const qtc_batch* b, qtc_batch_info* info) {
  return guarded([&] {
    if (!b || !info) fail(QTC_ERR_INVALID, "null argument");
    std::memset(info, 0, sizeof *info);
    info->n_networks = (int)b->plans.size();
    info->n_params = b->circuit.n_params;
    for (const Plan& p : b->plans) {
      const int L = (int)p.net.leaves.size(), S = (int)p.steps.size();
      std::vector<char> need(L + S, 0);
      for (int i = 0; i < L; ++i) need[i] = p.net.leaves[i].spec.slot >= 0;
      for (int s = 0; s < S; ++s) need[L + s] = need[p.steps[s].a] || need[p.steps[s].b];
      for (int s = 0; s < S; ++s) {
        const auto& la = p.labels[p.steps[s].a];
        const auto& lb = p.labels[p.steps[s].b];
        std::vector<int> u(la);
        for (int x : lb)
          if (std::find(la.begin(), la.end(), x) == la.end()) u.push_back(x);
        const double ec = std::ldexp(1.0, (int)p.labels[L + s].size());
        for (int side = 0; side < 2; ++side) {
          const int x = side ? p.steps[s].b : p.steps[s].a;
          const int y = side ? p.steps[s].a : p.steps[s].b;
          if (!need[x]) continue;
          info->grad_cmacs += std::ldexp(1.0, (int)u.size());
          info->grad_bytes_c64 += 8.0 * (ec + std::ldexp(1.0, (int)p.labels[x].size()) +
                                         std::ldexp(1.0, (int)p.labels[y].size()));
        }
      }
      info->max_rank = std::max(info->max_rank, p.max_rank);
      info->n_steps_total += (int)p.steps.size();
      info->cmacs += p.cmacs;
      info->bytes_c64 += p.bytes_c64;
      if (p.max_rank <= kMaxSmemRank) info->n_smem_networks += 1;
      else info->n_global_networks += 1;
    }
  });
}

// Algorithmic bytes of one network's evaluation (forward; with want_grad
// also the adjoint sweep's two contractions per step that needs them).
static double network_cost(const Plan& p, bool want_grad) {
  double cost = p.bytes_c64;
  if (!want_grad) return cost;
  const int L = (int)p.net.leaves.size(), S = (int)p.steps.size();
  std::vector<char> need(L + S, 0);
  for (int i = 0; i < L; ++i) need[i] = p.net.leaves[i].spec.slot >= 0;
  for (int s = 0; s < S; ++s) need[L + s] = need[p.steps[s].a] || need[p.steps[s].b];
  for (int s = 0; s < S; ++s) {
    const double ec = std::ldexp(1.0, (int)p.labels[L + s].size());
    for (int side = 0; side < 2; ++side) {
      const int x = side ? p.steps[s].b : p.steps[s].a;
      const int y = side ? p.steps[s].a : p.steps[s].b;
      if (!need[x]) continue;
      cost += 8.0 * (ec + std::ldexp(1.0, (int)p.labels[x].size()) +
                     std::ldexp(1.0, (int)p.labels[y].size()));
    }
  }
  return cost;
}

extern "C" qtc_status qtc_batch_partition(const qtc_batch* b, int n_parts, int want_grad,
                                          int32_t* part_of_net, double* part_cost) {
  return guarded([&] {
    if (!b || !part_of_net) fail(QTC_ERR_INVALID, "null argument");
    if (n_parts < 1) fail(QTC_ERR_INVALID, "%d parts", n_parts);
    const int N = (int)b->plans.size();
    std::vector<double> cost(N);
    for (int i = 0; i < N; ++i) cost[i] = network_cost(b->plans[i], want_grad != 0);
    // longest processing time first: the costliest network goes to the part
    // with the least work so far (ties: the lower network, the lower part)
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<double> load(n_parts, 0.0);
    for (int i : order) {
      int best = 0;
      for (int k = 1; k < n_parts; ++k)
        if (load[k] < load[best]) best = k;
      part_of_net[i] = best;
      load[best] += cost[i];
    }
    if (part_cost)
      for (int k = 0; k < n_parts; ++k) part_cost[k] = load[k];
  });
}

extern "C" qtc_status qtc_batch_subset(const qtc_batch* b, const int32_t* nets, int k,
                                       qtc_batch** out) {
  return guarded([&] {
    if (!b || !out || (k > 0 && !nets)) fail(QTC_ERR_INVALID, "null argument");
    if (k < 1) fail(QTC_ERR_INVALID, "a subset of %d networks", k);
    auto s = std::make_unique<qtc_batch>();
    s->circuit = b->circuit;
    s->qaoa_reduce = b->qaoa_reduce;
    for (int j = 0; j < k; ++j) {
      const int i = nets[j];
      if (i < 0 || i >= (int)b->plans.size()) fail(QTC_ERR_INVALID, "network %d out of range", i);
      s->plans.push_back(b->plans[i]);
      s->obs_edges.push_back(b->obs_edges[i]);
      s->weights.push_back(b->weights[i]);
    }
    *out = s.release();
  });
}

extern "C" void qtc_batch_destroy(qtc_batch* b) { delete b; }

// ---- device programs ---------------------------------------------------------------

const HostProgram& qtc::host_program(qtc_batch* b, int dtype, int want_grad,
                                     size_t max_dynamic, const ProgramOptions& opts) {
  if (dtype != QTC_C128 && dtype != QTC_C64 && dtype != QTC_SPLIT_BF16)
    fail(QTC_ERR_INVALID, "unknown dtype %d", dtype);
  want_grad = want_grad ? 1 : 0;
  for (const auto& hp : b->host_programs)
    if (hp->dtype == dtype && hp->want_grad == want_grad && hp->max_dynamic == max_dynamic &&
        hp->options == opts)
      return *hp;
  const size_t elem = elem_bytes(dtype);
  const int P = b->circuit.n_params;
  const int N = (int)b->plans.size();

  // gate table shared by all networks
  GateTable table;
  std::vector<std::vector<int>> leaf_gate(N);
  for (int i = 0; i < N; ++i)
    for (const Leaf& leaf : b->plans[i].net.leaves) leaf_gate[i].push_back(table.add(leaf.spec));
  const int G = (int)table.specs.size();
  std::vector<uint32_t> val_off(G), der_off(G);
  uint32_t at = 0;
  for (int g = 0; g < G; ++g) {
    val_off[g] = at;
    at += 1u << leaf_rank_of(table.specs[g].kind);
  }
  for (int g = 0; g < G; ++g) {
    der_off[g] = at;
    if (table.specs[g].slot >= 0) at += 1u << leaf_rank_of(table.specs[g].kind);
  }
  const uint32_t table_elems = (at + 1u) & ~1u;
  const uint32_t max_elems = (uint32_t)(max_dynamic / elem);

  static std::atomic<uint64_t> next_serial{1};
  auto hp = std::make_unique<HostProgram>();
  hp->serial = next_serial++;
  hp->dtype = dtype;
  hp->want_grad = want_grad;
  hp->max_dynamic = max_dynamic;
  hp->n_nets = N;
  hp->n_params = P;
  hp->qaoa_reduce = b->qaoa_reduce;
  hp->weights = b->weights;
  hp->table_elems = table_elems;
  hp->options = opts;
  hp->gates.resize(G);
  for (int g = 0; g < G; ++g) {
    hp->gates[g].spec = table.specs[g];
    hp->gates[g].val_off = val_off[g];
    hp->gates[g].der_off = der_off[g];
    hp->gates[g].rank = (uint32_t)leaf_rank_of(table.specs[g].kind);
  }
  std::vector<int> order(N);
  for (int i = 0; i < N; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->plans[x].cmacs > b->plans[y].cmacs; });
  bool all_fit = !opts.force_graph;
  for (int i : order) {
    if (!all_fit) break;
    LoweredNet ln = lower_smem(b->plans[i], leaf_gate[i], val_off, der_off, table_elems,
                               want_grad != 0, max_elems);
    if (!ln.fits) {
      all_fit = false;
      break;
    }
    TaskDev t{};
    t.op_begin = (uint32_t)hp->ops.size();
    t.op_count = (uint32_t)ln.ops.size();
    t.net = (uint32_t)i;
    t.arena_elems = ln.arena_elems;
    hp->tasks.push_back(t);
    hp->ops.insert(hp->ops.end(), ln.ops.begin(), ln.ops.end());
    hp->max_arena = std::max(hp->max_arena, ln.arena_elems);
  }
  if (!all_fit) {
    // some network is too large for one CTA: the graph executor runs them all
    hp->tasks.clear();
    hp->ops.clear();
    hp->max_arena = 0;
    build_graph_program(*hp, b->plans, leaf_gate, val_off, der_off, max_dynamic, opts);
    b->host_programs.push_back(std::move(hp));
    return *b->host_programs.back();
  }
  // Networks of rank <= 11 whose ops sum over <= 8 labels may run one per
  // warp (warp programs); the others use the whole CTA, which stages its op
  // list in chunks.
  uint32_t max_ops = 1;
  int max_rank = 0;
  for (const TaskDev& t : hp->tasks) max_ops = std::max(max_ops, t.op_count);
  for (const Plan& pl : b->plans) max_rank = std::max(max_rank, pl.max_rank);
  auto round16 = [](size_t x) { return (uint32_t)((x + 15) & ~size_t(15)); };
  // warp teams need every op within the pre-expanded tables, and every
  // element of the table copy and arena within a 16-bit lane offset
  bool warp_ok = opts.warp_teams != 0 && max_rank <= kWarpMaxRank &&
                 (size_t)table_elems + hp->max_arena <= 0xffffu;
  for (const SOp& op : hp->ops)
    if (op.code == SOP_CONTRACT && (op.rc > kWarpMaxRank || op.ry > kWarpMaxSummed))
      warp_ok = false;
  // CTA teams share one gate table at the start of shared memory; a warp team
  // keeps its own copy right before its arena ([steps | lane gradient
  // accumulators | table | arena]), so every operand of a warp step is an
  // offset from one base.
  // stage 0 (warp teams): steps streamed from global memory, no stage region
  auto layout = [&](bool warp, uint32_t stage, int teams = kWarpTeamsPerCta) {
    hp->warp_teams = warp;
    hp->stream_steps = warp && stage == 0;
    hp->n_teams = warp ? teams : 1;
    hp->block = warp ? 32 * teams : kExecBlock;
    hp->stage_ops = stage;
    const size_t op_bytes = warp ? sizeof(WStep) : sizeof(SOp);
    hp->table_bytes = warp ? 0 : round16((size_t)table_elems * elem);
    const size_t lane_grad = (warp && want_grad && P <= kWarpLaneGradSlots) ? (size_t)P * 32 : 0;
    hp->team_bytes = round16((size_t)stage * op_bytes +
                             (lane_grad + hp->max_arena + (warp ? table_elems : 0)) * elem);
    hp->smem = hp->table_bytes + (size_t)hp->n_teams * hp->team_bytes;
    return hp->smem <= max_dynamic;
  };
  auto try_layout = [&](bool warp, uint32_t first) {
    for (uint32_t stage = first;; stage /= 2) {
      if (layout(warp, stage)) return true;
      if (stage <= 4) return false;
    }
  };
  bool ok = false;
  // Schedule each network's ops into warp steps (lane-packed bundles), three
  // ways: with an arena buffer per intermediate and adjoint (ops that would
  // reuse memory no longer wait for its last reader, so independent subtrees
  // share steps); with buffers of their own for the small tensors only (<= 32
  // elements: the lane-packed ops); and with the reused arena.  Each can run
  // with its whole step list staged in shared memory or streamed from global
  // memory (no stage region), with 4, 2 or 1 warp teams per CTA.  The layout
  // taken is the one with the fewest (rounds of resident teams) x (steps of
  // the longest network); the reused arena with smaller stages is the last
  // resort.
  struct WarpCand {
    std::vector<TaskDev> tasks;
    std::vector<WStep> wsteps;
    uint32_t max_steps = 1, max_arena = 0;
  };
  std::vector<WarpCand> cands;
  for (int pass = 0; warp_ok && pass < 3; ++pass) {
    const bool reuse = pass == 2;
    const uint32_t private_below = pass == 0 ? UINT32_MAX : 32u;
    WarpCand c;
    c.tasks = hp->tasks;
    bool fit = true;
    for (TaskDev& t : c.tasks) {
      std::vector<SOp> net_ops(hp->ops.begin() + t.op_begin,
                               hp->ops.begin() + t.op_begin + t.op_count);
      const uint32_t begin = (uint32_t)c.wsteps.size();
      if (!reuse) {
        LoweredNet ln = lower_smem(b->plans[t.net], leaf_gate[t.net], val_off, der_off,
                                   table_elems, want_grad != 0, max_elems, private_below);
        if (!ln.fits || (size_t)table_elems + ln.arena_elems > 0xffffu) {
          fit = false;
          break;
        }
        t.arena_elems = ln.arena_elems;
        net_ops = std::move(ln.ops);
      }
      build_warp_steps(net_ops, table_elems, t.arena_elems, c.wsteps);
      c.max_arena = std::max(c.max_arena, t.arena_elems);
      t.op_begin = begin;
      t.op_count = (uint32_t)c.wsteps.size() - begin;
      c.max_steps = std::max(c.max_steps, t.op_count);
    }
    if (fit) cands.push_back(std::move(c));
  }
  // (complex128 programs that need streamed steps or fewer teams per CTA
  // measured slower on warps than on a CTA per network: they stay staged
  // with four teams, or run on CTA teams)
  const bool wide = dtype == QTC_C128;
  const uint32_t shared_arena = hp->max_arena;
  const size_t sm_smem = 233472;  // shared memory of one SM
  int best = -1, best_teams = 0;
  bool best_stream = false;
  double best_cost = 0;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    hp->max_arena = cands[ci].max_arena;
    const uint32_t stage = std::min<uint32_t>(cands[ci].max_steps, 128);
    for (int teams = kWarpTeamsPerCta; teams >= (wide ? kWarpTeamsPerCta : 1); teams /= 2)
      for (int stream = opts.warp_teams == 2 ? 1 : 0; stream < (wide ? 1 : 2); ++stream) {
        if (!layout(true, stream ? 0 : stage, teams)) continue;
        const size_t per_sm = std::max<size_t>(
            1, std::min<size_t>(kExecCtasPerSmByRegs, sm_smem / (hp->smem + 12288)));
        const double slots = (double)opts.sm_count * (double)per_sm * teams;
        const double rounds = std::ceil((double)hp->tasks.size() / slots);
        const double cost = rounds * cands[ci].max_steps * (stream ? 1.05 : 1.0);
        if (best < 0 || cost < best_cost) {
          best = (int)ci;
          best_teams = teams;
          best_stream = stream != 0;
          best_cost = cost;
        }
      }
  }
  if (best >= 0) {
    WarpCand& c = cands[best];
    hp->max_arena = c.max_arena;
    ok = layout(true, best_stream ? 0 : std::min<uint32_t>(c.max_steps, 128), best_teams);
  } else if (!cands.empty()) {
    WarpCand& c = cands.back();  // the reused arena, smaller stages
    hp->max_arena = c.max_arena;
    ok = try_layout(true, std::min<uint32_t>(c.max_steps, 128));
    if (ok) best = (int)cands.size() - 1;
  }
  if (ok) {
    WarpCand& c = cands[best];
    // With a fixed stride per task a team starts reading its first task's
    // steps without first reading the task record; taken when the padding
    // costs little.
    const size_t padded = c.tasks.size() * c.max_steps;
    if (padded <= c.wsteps.size() + c.wsteps.size() / 2 ||
        padded * sizeof(WStep) <= (16u << 20)) {
      std::vector<WStep> fixed(padded);
      for (size_t i = 0; i < c.tasks.size(); ++i) {
        std::copy(c.wsteps.begin() + c.tasks[i].op_begin,
                  c.wsteps.begin() + c.tasks[i].op_begin + c.tasks[i].op_count,
                  fixed.begin() + i * c.max_steps);
        c.tasks[i].op_begin = (uint32_t)(i * c.max_steps);
      }
      c.wsteps = std::move(fixed);
      hp->task_stride = c.max_steps;
    }
    hp->tasks = std::move(c.tasks);
    hp->wsteps = std::move(c.wsteps);
    for (const TaskDev& t : hp->tasks)
      validate_warp_steps(hp->wsteps.data() + t.op_begin, t.op_count,
                          table_elems + t.arena_elems, P);
    hp->coef = coefficient_table(hp->gates, table_elems, dtype);
    hp->ops.clear();
  } else {
    hp->max_arena = shared_arena;
  }
  if (!ok) ok = try_layout(false, std::min<uint32_t>(max_ops, 64));
  if (!ok)
    fail(QTC_ERR_UNSUPPORTED, "program needs %zu bytes of shared memory (limit %zu)", hp->smem,
         max_dynamic);
  b->host_programs.push_back(std::move(hp));
  return *b->host_programs.back();
}

// Uploads a graph-form program: tables per wave, one work buffer shared by
// the waves (they run one after another on the stream), zeroed counters and
// result rows.
static Prepared& prepare_graph(qtc_engine* e, qtc_batch* b, const HostProgram& hp,
                               cudaStream_t stream, size_t max_dyn) {
  DeviceScope scope(e->device);
  const int P = hp.n_params, N = hp.n_nets;
  const size_t stride = 2 + 2 * (size_t)P;
  Prepared pr;
  pr.engine = e;
  pr.generation = e->generation;
  pr.dtype = hp.dtype;
  pr.want_grad = hp.want_grad;
  pr.graph = true;
  auto* dg = upload(e, hp.gates, stream, "upload gates");
  auto* dw = upload(e, hp.weights, stream, "upload weights");
  auto* dparams = (double*)e->alloc(sizeof(double) * std::max(P, 1));
  auto* dres = (double*)e->alloc(sizeof(double) * N * stride);
  auto* draw = (double*)e->alloc(sizeof(double) * N * stride);
  auto* dout = (double*)e->alloc(sizeof(double) * (2 + P + N));
  const size_t n_ctr = ctr_words(hp.max_counters);
  auto* dcnt = (unsigned int*)e->alloc(sizeof(unsigned int) * n_ctr);
  std::vector<GraphProgDev> waves;
  for (const WaveHost& w : hp.waves) {
    GraphProgDev d{};
    d.tasks = upload(e, w.tasks, stream, "upload tasks");
    d.n_tasks = (int)w.tasks.size();
    d.ops = upload(e, w.ops, stream, "upload ops");
    d.steps = upload(e, w.steps, stream, "upload steps");
    d.tsteps = upload(e, w.tsteps, stream, "upload GEMM steps");
    d.waits = upload(e, w.waits, stream, "upload waits");
    d.n_counters = (int)w.n_counters;
    waves.push_back(d);
  }
  e->reserve_work(std::max<size_t>(256, hp.max_global_elems * elem_bytes(hp.dtype)));
  cuda_check(cudaMemsetAsync(dcnt, 0, sizeof(unsigned int) * n_ctr, stream), "clear counters");
  cuda_check(cudaMemsetAsync(dres, 0, sizeof(double) * N * stride, stream), "clear results");
  cuda_check(cudaStreamSynchronize(stream), "prepare sync");
  int per_sm = 0;
  pr.tiles = hp.tiles && !hp.tensor_cores;
  pr.hi_occ = hp.options.graph_hi_occupancy && hp.dtype == QTC_C64 && !hp.tensor_cores &&
              !pr.tiles;
  cuda_check(graph_exec_configure(hp.dtype == QTC_C128 ? 0 : 1, hp.tensor_cores, pr.hi_occ,
                                  pr.tiles, hp.smem, max_dyn, &per_sm),
             "configure graph executor");
  if (per_sm < 1) fail(QTC_ERR_UNSUPPORTED, "graph executor does not fit on an SM");
  // tensor memory: 512 columns per SM shared by the resident CTAs; a GEMM
  // tile needs 128 fp32 columns (N = 128 reals)
  int tmem_cols = 0;
  if (hp.tensor_cores) {
    // one 1024-thread CTA per SM, four teams of 128 columns each
    if (per_sm > 1)
      fail(QTC_ERR_UNSUPPORTED, "%d resident CTAs per SM leave too little tensor memory",
           per_sm);
    tmem_cols = 128;
  }
  size_t max_tasks = 1;
  for (const WaveHost& w : hp.waves) max_tasks = std::max(max_tasks, w.tasks.size());
  pr.grid = (int)std::max<size_t>(1, std::min<size_t>(max_tasks, (size_t)e->sm_count * per_sm));
  pr.smem = hp.smem;
  pr.per_sm = per_sm;
  for (size_t i = 0; i < waves.size(); ++i) {
    GraphProgDev& d = waves[i];
    d.gates = dg;
    d.n_gates = (int)hp.gates.size();
    d.table_elems = hp.table_elems;
    d.table_bytes = hp.table_bytes;
    d.arena_bytes = hp.work_bytes;
    d.stage_ops = hp.stage_ops;
    d.gbase = nullptr;  // the engine's work buffer, set at launch
    d.n_params = P;
    d.n_nets = N;
    d.final_wave = i + 1 == waves.size();
    d.weights = dw;
    d.params = dparams;
    d.results = dres;
    d.raw_out = draw;
    d.out = dout;
    d.counters = dcnt;
    d.want_grad = hp.want_grad;
    d.qaoa_reduce = hp.qaoa_reduce;
    d.wait_limit_ns = (long long)(e->wait_limit_ms * 1e6);
    d.tmem_cols = tmem_cols;
  }
  pr.waves = waves;
  pr.raw = draw;
  pr.prog.params = dparams;
  pr.prog.out = dout;
  pr.prog.results = dres;
  b->prepared.push_back(pr);
  return b->prepared.back();
}

static Prepared& prepare(qtc_engine* e, qtc_batch* b, int dtype, int want_grad,
                         cudaStream_t stream) {
  want_grad = want_grad ? 1 : 0;
  for (Prepared& p : b->prepared)
    if (p.engine == e && p.generation == e->generation && p.dtype == dtype &&
        p.want_grad == want_grad)
      return p;
  const size_t max_dyn = max_dynamic_smem(e->smem_optin);
  const HostProgram& hp = host_program(b, dtype, want_grad, max_dyn, e->options);
  const int P = hp.n_params;
  const int N = hp.n_nets;
  const int G = (int)hp.gates.size();
  if (hp.graph) return prepare_graph(e, b, hp, stream, max_dyn);

  DeviceScope scope(e->device);
  Prepared pr;
  pr.engine = e;
  pr.generation = e->generation;
  pr.dtype = dtype;
  pr.want_grad = want_grad;
  ProgramDev& d = pr.prog;
  auto* dg = (GateEntryDev*)e->alloc(sizeof(GateEntryDev) * G);
  auto* dt = (TaskDev*)e->alloc(sizeof(TaskDev) * hp.tasks.size());
  auto* dops = (SOp*)e->alloc(sizeof(SOp) * std::max<size_t>(1, hp.ops.size()));
  auto* dwsteps = (WStep*)e->alloc(sizeof(WStep) * std::max<size_t>(1, hp.wsteps.size()));
  auto* dcoef = e->alloc(std::max<size_t>(16, hp.coef.size()));
  auto* dw = (double*)e->alloc(sizeof(double) * N);
  auto* dparams = (double*)e->alloc(sizeof(double) * std::max(P, 1));
  auto* dres = (double*)e->alloc(sizeof(double) * (size_t)N * (2 + 2 * P));
  auto* dacc = (double*)e->alloc(sizeof(double) * (1 + P));
  auto* dout = (double*)e->alloc(sizeof(double) * (2 + P + N));
  auto* dcnt = (unsigned int*)e->alloc(sizeof(unsigned int) * 4);
  cuda_check(cudaMemcpyAsync(dg, hp.gates.data(), sizeof(GateEntryDev) * G, cudaMemcpyHostToDevice, stream), "upload gates");
  cuda_check(cudaMemcpyAsync(dt, hp.tasks.data(), sizeof(TaskDev) * hp.tasks.size(), cudaMemcpyHostToDevice, stream), "upload tasks");
  if (!hp.ops.empty())
    cuda_check(cudaMemcpyAsync(dops, hp.ops.data(), sizeof(SOp) * hp.ops.size(), cudaMemcpyHostToDevice, stream), "upload ops");
  if (!hp.wsteps.empty())
    cuda_check(cudaMemcpyAsync(dwsteps, hp.wsteps.data(), sizeof(WStep) * hp.wsteps.size(),
                               cudaMemcpyHostToDevice, stream),
               "upload warp steps");
  if (!hp.coef.empty())
    cuda_check(cudaMemcpyAsync(dcoef, hp.coef.data(), hp.coef.size(), cudaMemcpyHostToDevice,
                               stream),
               "upload gate coefficients");
  cuda_check(cudaMemcpyAsync(dw, hp.weights.data(), sizeof(double) * N, cudaMemcpyHostToDevice, stream), "upload weights");
  cuda_check(cudaMemsetAsync(dcnt, 0, sizeof(unsigned int) * 4, stream), "clear counters");
  cuda_check(cudaMemsetAsync(dacc, 0, sizeof(double) * (1 + P), stream), "clear sums");
  cuda_check(cudaStreamSynchronize(stream), "prepare sync");
  d.gates = dg;
  d.n_gates = G;
  for (int g = 0; g < G && g < kInlineGates; ++g) d.gates_inline[g] = hp.gates[g];
  d.table_elems = hp.table_elems;
  d.table_bytes = hp.table_bytes;
  d.team_bytes = hp.team_bytes;
  d.stage_ops = hp.stage_ops;
  d.task_stride = hp.task_stride;
  d.coef = dcoef;
  d.tasks = dt;
  d.n_tasks = (int)hp.tasks.size();
  d.ops = dops;
  d.wsteps = dwsteps;
  d.n_params = P;
  d.n_nets = N;
  d.weights = dw;
  d.params = dparams;
  d.results = dres;
  d.acc = dacc;
  d.out = dout;
  d.counters = dcnt;
  d.want_grad = want_grad;
  d.qaoa_reduce = hp.qaoa_reduce;
  pr.block = hp.block;
  pr.smem = hp.smem;
  int per_sm = 0;
  pr.warp_teams = hp.warp_teams;
  pr.stream = hp.stream_steps;
  cuda_check(smem_exec_configure(dtype == QTC_C128 ? 0 : 1,
                                 pr.warp_teams ? (pr.stream ? 2 : 1) : 0, pr.smem, max_dyn,
                                 pr.block, &per_sm),
             "configure executor");
  if (per_sm < 1) fail(QTC_ERR_UNSUPPORTED, "executor does not fit on an SM (%zu bytes)", pr.smem);
  const int ctas = ((int)hp.tasks.size() + hp.n_teams - 1) / hp.n_teams;
  pr.grid = std::max(1, std::min(ctas, e->sm_count * per_sm));
  pr.per_sm = per_sm;
  b->prepared.push_back(pr);
  return b->prepared.back();
}

static void launch(qtc_engine* e, const Prepared& pr, const double* params_dev, double* out_dev,
                   cudaStream_t stream, unsigned long long* done = nullptr,
                   uint64_t seq = 0, const double* host_params = nullptr) {
  if (pr.graph) {
    for (const GraphProgDev& w : pr.waves) {
      GraphProgDev d = w;
      d.params = params_dev;
      d.out = out_dev;
      d.gbase = e->work_base();
      cuda_check(graph_exec_launch(d, pr.dtype == QTC_C128 ? 0 : 1, pr.hi_occ, pr.tiles,
                                   pr.grid, pr.smem, stream),
                 "launch graph executor");
    }
    e->last_launches = (int)pr.waves.size();
    return;
  }
  ProgramDev d = pr.prog;
  d.params = params_dev;
  d.out = out_dev;
  d.done = done;
  d.seq = seq;
  d.n_inline_params = 0;
  if (host_params && d.n_params > 0 && d.n_params <= kInlineParams) {
    d.n_inline_params = d.n_params;
    for (int k = 0; k < d.n_params; ++k) d.params_inline[k] = host_params[k];
  }
  cuda_check(smem_exec_launch(d, pr.dtype == QTC_C128 ? 0 : 1,
                              pr.warp_teams ? (pr.stream ? 2 : 1) : 0, pr.grid, pr.block,
                              pr.smem, stream),
             "launch executor");
  e->last_launches = 1;
}

extern "C" qtc_status qtc_batch_program_info(qtc_batch* b, int dtype, int want_grad,
                                              int force_graph, int small_rank,
                                              size_t max_wave_bytes, size_t smem_limit,
                                              qtc_program_info* info) {
  return guarded([&] {
    if (!b || !info) fail(QTC_ERR_INVALID, "null argument");
    ProgramOptions opts;
    opts.force_graph = force_graph != 0;
    opts.small_rank = small_rank;
    if (max_wave_bytes) opts.wave_cap_bytes = max_wave_bytes;
    const size_t max_dyn = max_dynamic_smem(smem_limit ? smem_limit : (size_t)232448);
    const HostProgram& hp = host_program(b, dtype, want_grad, max_dyn, opts);
    std::memset(info, 0, sizeof *info);
    info->graph = hp.graph ? 1 : 0;
    info->smem_bytes = (int)hp.smem;
    info->stage_ops = (int)hp.stage_ops;
    double tables = sizeof(GateEntryDev) * hp.gates.size();
    if (hp.graph) {
      info->n_waves = (int)hp.waves.size();
      for (const WaveHost& w : hp.waves) {
        info->n_tasks += (int)w.tasks.size();
        info->n_global_steps += (int)(w.steps.size() + w.tsteps.size());
        info->n_gemm_steps += (int)w.tsteps.size();
        for (const GTask& t : w.tasks) info->n_smem_tasks += t.kind == GT_SMEM;
        tables += sizeof(GTask) * w.tasks.size() + sizeof(SOp) * w.ops.size() +
                  sizeof(GStep) * w.steps.size() + sizeof(TStep) * w.tsteps.size() +
                  sizeof(WaitDev) * w.waits.size();
      }
      info->work_bytes = (double)hp.max_global_elems * elem_bytes(dtype);
      info->net_global_bytes = (double)hp.sum_global_elems * elem_bytes(dtype);
      info->net_global_bytes_unshared = (double)hp.sum_unshared_elems * elem_bytes(dtype);
      info->checkpoint_segments = hp.max_checkpoint_segments;
    } else {
      info->n_waves = 1;
      info->n_tasks = info->n_smem_tasks = (int)hp.tasks.size();
      tables += sizeof(TaskDev) * hp.tasks.size() + sizeof(SOp) * hp.ops.size() +
                sizeof(WStep) * hp.wsteps.size();
      info->warp_teams = hp.warp_teams ? 1 : 0;
      info->n_ops = (int)hp.ops.size();
      for (const TaskDev& t : hp.tasks)
        if (hp.warp_teams) {
          info->n_warp_steps += (int)t.op_count;
          info->max_warp_steps = std::max(info->max_warp_steps, (int)t.op_count);
          for (uint32_t k = 0; k < t.op_count; ++k)
            info->n_solo_steps += hp.wsteps[t.op_begin + k].solo ? 1 : 0;
        }
    }
    info->table_bytes = tables;
  });
}

extern "C" qtc_status qtc_batch_launch_info(qtc_engine* e, qtc_batch* b, int dtype,
                                             int want_grad, int32_t* out) {
  return guarded([&] {
    if (!e || !b || !out) fail(QTC_ERR_INVALID, "null argument");
    DeviceScope scope(e->device);
    const Prepared& pr = prepare(e, b, dtype, want_grad, nullptr);
    out[0] = pr.grid;
    out[1] = pr.graph ? (pr.waves.empty() || pr.waves[0].tmem_cols == 0 ? 256 : 1024) : pr.block;
    out[2] = (int32_t)pr.smem;
    out[3] = pr.per_sm;
    out[4] = pr.graph ? (int32_t)pr.waves.size() : 1;
    out[5] = pr.graph && !pr.waves.empty() ? pr.waves[0].tmem_cols : 0;
  });
}

extern "C" qtc_status qtc_batch_prepare(qtc_engine* e, qtc_batch* b, int dtype, int want_grad,
                                        void* stream) {
  return guarded([&] {
    if (!e || !b) fail(QTC_ERR_INVALID, "null argument");
    prepare(e, b, dtype, want_grad, (cudaStream_t)stream);
  });
}

extern "C" qtc_status qtc_qaoa_expectation_device(qtc_engine* e, qtc_batch* b,
                                                  const double* params_dev, int dtype,
                                                  int want_grad, void* stream, double* out_dev) {
  return guarded([&] {
    if (!e || !b || !params_dev || !out_dev) fail(QTC_ERR_INVALID, "null argument");
    DeviceScope scope(e->device);
    const Prepared& pr = prepare(e, b, dtype, want_grad, (cudaStream_t)stream);
    launch(e, pr, params_dev, out_dev, (cudaStream_t)stream);
  });
}

// Returns once the kernel has published `seq` at `flag` (an acquire load
// pairs with its system-scope release), or once the stream is idle (results
// visible all the same); a launch or kernel error ends the wait with that error.
static void wait_published(const uint64_t* flag, uint64_t seq, cudaStream_t s) {
  for (uint32_t i = 1;; ++i) {
    if (__atomic_load_n(flag, __ATOMIC_ACQUIRE) == seq) return;
    if ((i & 1023) == 0) {
      const cudaError_t q = cudaStreamQuery(s);
      if (q == cudaSuccess) return;
      if (q != cudaErrorNotReady) cuda_check(q, "executor");
    }
  }
}

extern "C" qtc_status qtc_qaoa_expectation(qtc_engine* e, qtc_batch* b, const double* gammas,
                                           const double* betas, int dtype, int want_grad,
                                           void* stream, double* C_out, double* per_edge_out,
                                           double* grad_out) {
  return guarded([&] {
    if (!e || !b || !gammas || !betas || !C_out) fail(QTC_ERR_INVALID, "null argument");
    if (grad_out && !want_grad) fail(QTC_ERR_INVALID, "grad_out needs want_grad");
    const int p = b->circuit.n_params / 2;
    if (b->circuit.p <= 0) fail(QTC_ERR_INVALID, "the batch's circuit is not a QAOA circuit");
    DeviceScope scope(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    const Prepared& pr = prepare(e, b, dtype, want_grad, s);
    const int P = 2 * p;
    const int N = (int)b->plans.size();
    // parameters, results and the completion word in the engine's mapped
    // staging buffer
    double* params = e->staging((size_t)P + 3 + P + N);
    double* host_out = params + P;
    for (int k = 0; k < p; ++k) {
      params[k] = gammas[k];
      params[p + k] = betas[k];
    }
    if (pr.graph) {
      launch(e, pr, e->staging_dev, e->staging_dev + P, s);
      cuda_check(cudaStreamSynchronize(s), "synchronise stream");
    } else {
      const size_t at = (size_t)P + 2 + P + N;
      auto* flag = reinterpret_cast<uint64_t*>(params + at);
      const uint64_t seq = ++e->seq;
      __atomic_store_n(flag, (uint64_t)0, __ATOMIC_RELAXED);
      launch(e, pr, e->staging_dev, e->staging_dev + P, s,
             reinterpret_cast<unsigned long long*>(e->staging_dev + at), seq, params);
      wait_published(flag, seq, s);
    }
    if (host_out[1 + P + N] != 0.0)
      fail(QTC_ERR_TIMEOUT, "a device-side dependency wait expired (status %g)",
           host_out[1 + P + N]);
    *C_out = host_out[0];
    if (grad_out)
      for (int k = 0; k < P; ++k) grad_out[k] = host_out[1 + k];
    if (per_edge_out)
      for (int i = 0; i < N; ++i) per_edge_out[i] = host_out[1 + P + i];
  });
}

// ---- single network -----------------------------------------------------------------

extern "C" qtc_status qtc_contract(qtc_engine* e, const qtc_plan* p, const double* params,
                                   int dtype, void* stream, double* out_re_im,
                                   double* grad_re_im) {
  return guarded([&] {
    if (!e || !p || !out_re_im) fail(QTC_ERR_INVALID, "null argument");
    const int P = p->plan.net.n_params;
    if (P > 0 && !params) fail(QTC_ERR_INVALID, "null parameters");
    auto* mp = const_cast<qtc_plan*>(p);
    if (!mp->single) {
      mp->single = std::make_unique<qtc_batch>();
      mp->single->circuit.n_params = P;
      mp->single->plans.push_back(p->plan);
      mp->single->weights.assign(1, 1.0);
      mp->single->obs_edges.push_back({0, 0});
      mp->single->qaoa_reduce = 0;
    }
    DeviceScope scope(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int want_grad = grad_re_im ? 1 : 0;
    const Prepared& pr = prepare(e, mp->single.get(), dtype, want_grad, s);
    if (P > 0)
      cuda_check(cudaMemcpyAsync((void*)pr.prog.params, params, sizeof(double) * P,
                                 cudaMemcpyHostToDevice, s), "upload parameters");
    launch(e, pr, pr.prog.params, pr.prog.out, s);
    std::vector<double> res(2 + 2 * P), status(1, 0.0);
    cuda_check(cudaMemcpyAsync(res.data(), pr.graph ? pr.raw : pr.prog.results,
                               sizeof(double) * res.size(), cudaMemcpyDeviceToHost, s),
               "download result");
    cuda_check(cudaMemcpyAsync(status.data(), pr.prog.out + 1 + P + 1, sizeof(double),
                               cudaMemcpyDeviceToHost, s), "download status");
    cuda_check(cudaStreamSynchronize(s), "synchronise stream");
    if (status[0] != 0.0) fail(QTC_ERR_TIMEOUT, "a device-side dependency wait expired");
    out_re_im[0] = res[0];
    out_re_im[1] = res[1];
    if (grad_re_im)
      for (int k = 0; k < 2 * P; ++k) grad_re_im[k] = res[2 + k];
  });
}

// ---- answer strings (Section 3.3) ---------------------------------------------------

extern "C" qtc_status qtc_answer_string(qtc_engine* e, const qtc_circuit* c,
                                        const double* params, int dtype,
                                        const qtc_plan_opts* opts, uint64_t tie_seed,
                                        void* stream, uint8_t* bits_out, double* probs_out) {
  return guarded([&] {
    if (!e || !c || !bits_out || !probs_out) fail(QTC_ERR_INVALID, "null argument");
    const int n = c->c.n;
    if (n <= 0) fail(QTC_ERR_INVALID, "circuit without qubits");
    if (c->c.n_params > 0 && !params) fail(QTC_ERR_INVALID, "null parameters");
    SplitMix64 rng(tie_seed);
    std::vector<uint8_t> bits(n, 2);
    qtc_observable obs{};
    obs.kind = QTC_OBS_PROJECTOR;
    std::unique_ptr<qtc_plan> first;
    double prev = 1.0;
    for (int q = 0; q < n; ++q) {
      // P(prefix, x_q = 0): qubits 0..q-1 projected on their chosen values,
      // qubit q on |0>, the rest traced out; every network has one closing
      // tensor per qubit, so all share the first one's contraction tree
      bits[q] = 0;
      obs.bits = bits.data();
      auto plan = std::make_unique<qtc_plan>();
      Network net = build_network(c->c, obs, false, true);
      if (first) {
        const Network& like = first->plan.net;
        bool same = like.leaves.size() == net.leaves.size();
        for (size_t i = 0; same && i < net.leaves.size(); ++i)
          same = like.leaves[i].labels == net.leaves[i].labels;
        if (!same) fail(QTC_ERR_INVALID, "internal: projector networks differ in structure");
        plan->plan = first->plan;
        plan->plan.net = std::move(net);
      } else {
        plan->plan = make_plan(net, opts ? *opts : default_opts());
      }
      double v[2] = {0.0, 0.0};
      const qtc_status st = qtc_contract(e, plan.get(), params, dtype, stream, v, nullptr);
      if (st != QTC_OK) fail(st, "%s", qtc_last_error());
      const double p0 = v[0], p1 = prev - p0;
      // the likelier value; a tie is broken by the seeded generator
      const bool zero = p0 > p1 || (p0 == p1 && rng.below(2) == 0);
      bits[q] = zero ? 0 : 1;
      prev = zero ? p0 : p1;
      bits_out[q] = bits[q];
      probs_out[q] = prev;
      if (!first) first = std::move(plan);
    }
  });
}

// ---- state-vector reference (full Hilbert space) ----------------------------------

static SvPrepared& sv_prepare(qtc_engine* e, qtc_circuit* c, cudaStream_t s) {
  for (SvPrepared& p : c->sv)
    if (p.engine == e && p.generation == e->generation) return p;
  const Circuit& cc = c->c;
  if (cc.p <= 0) fail(QTC_ERR_INVALID, "the state-vector reference needs a QAOA circuit");
  if (cc.n > 32) fail(QTC_ERR_UNSUPPORTED, "state vector of %d qubits (at most 32)", cc.n);
  if (cc.edges.size() > 512) fail(QTC_ERR_UNSUPPORTED, "more than 512 edges");
  std::vector<uint32_t> adj(cc.n, 0);
  std::vector<int2> edges;
  for (auto& ed : cc.edges) {
    adj[ed.first] |= 1u << ed.second;
    adj[ed.second] |= 1u << ed.first;
    edges.push_back(make_int2(ed.first, ed.second));
  }
  SvPrepared p;
  p.engine = e;
  p.generation = e->generation;
  p.adj = upload(e, adj, s, "upload adjacency");
  p.edges = upload(e, edges, s, "upload edges");
  p.params = (double*)e->alloc(sizeof(double) * 2 * cc.p);
  p.acc = (double*)e->alloc(sizeof(double) * (1 + cc.edges.size()));
  void* scratch = e->alloc((size_t)16 * (cc.p * (cc.edges.size() + 1) + cc.p + 2));
  for (int d = 0; d < 2; ++d) {
    int lo[16], len[16], rl[16];
    const int passes = sv_passes(cc.n, sv_tile_bits(d), lo, len, rl);
    const int l = passes - 1;
    p.tabs[d].scratch = scratch;
    p.tabs[d].wcut_first =
        upload(e, sv_cut_table(adj, cc.n, lo[0], len[0], rl[0]), s, "upload cut table");
    p.tabs[d].wcut_last =
        passes > 1 ? upload(e, sv_cut_table(adj, cc.n, lo[l], len[l], rl[l]), s, "upload cut table")
                   : p.tabs[d].wcut_first;
  }
  cuda_check(cudaStreamSynchronize(s), "prepare sync");
  c->sv.push_back(p);
  return c->sv.back();
}

static void sv_run(qtc_engine* e, qtc_circuit* c, const SvPrepared& p, const double* params_dev,
                   int dtype, int per_edge, cudaStream_t s, double* acc) {
  if (dtype != QTC_C128 && dtype != QTC_C64)
    fail(QTC_ERR_INVALID, "the state vector runs in complex128 or complex64");
  const Circuit& cc = c->c;
  const size_t elem = elem_bytes(dtype);
  e->reserve_work(elem << cc.n);
  int launches = 0;
  const int d = dtype == QTC_C128 ? 0 : 1;
  cuda_check(sv_qaoa_launch(d, e->work_base(), cc.n, (int)cc.edges.size(), p.adj, p.edges,
                            params_dev, cc.p, p.tabs[d], acc, per_edge, s, &launches),
             "launch state vector");
  e->last_launches = launches;
}

extern "C" qtc_status qtc_statevector_qaoa(qtc_engine* e, const qtc_circuit* c,
                                           const double* gammas, const double* betas, int dtype,
                                           int per_edge, void* stream, double* C_out,
                                           double* per_edge_out) {
  return guarded([&] {
    if (!e || !c || !gammas || !betas || !C_out) fail(QTC_ERR_INVALID, "null argument");
    if (per_edge_out && !per_edge) fail(QTC_ERR_INVALID, "per_edge_out needs per_edge");
    DeviceScope scope(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    auto* mc = const_cast<qtc_circuit*>(c);
    const SvPrepared& p = sv_prepare(e, mc, s);
    const int P = mc->c.p, m = (int)mc->c.edges.size();
    std::vector<double> params(2 * P), out(1 + m);
    for (int k = 0; k < P; ++k) {
      params[k] = gammas[k];
      params[P + k] = betas[k];
    }
    cuda_check(cudaMemcpyAsync(p.params, params.data(), sizeof(double) * 2 * P,
                               cudaMemcpyHostToDevice, s), "upload parameters");
    sv_run(e, mc, p, p.params, dtype, per_edge, s, p.acc);
    cuda_check(cudaMemcpyAsync(out.data(), p.acc, sizeof(double) * out.size(),
                               cudaMemcpyDeviceToHost, s), "download results");
    cuda_check(cudaStreamSynchronize(s), "synchronise stream");
    *C_out = out[0];
    if (per_edge_out)
      for (int i = 0; i < m; ++i) per_edge_out[i] = out[1 + i];
  });
}

extern "C" qtc_status qtc_statevector_qaoa_device(qtc_engine* e, const qtc_circuit* c,
                                                  const double* params_dev, int dtype,
                                                  int per_edge, void* stream, double* out_dev) {
  return guarded([&] {
    if (!e || !c || !params_dev || !out_dev) fail(QTC_ERR_INVALID, "null argument");
    DeviceScope scope(e->device);
    cudaStream_t s = (cudaStream_t)stream;
    auto* mc = const_cast<qtc_circuit*>(c);
    const SvPrepared& p = sv_prepare(e, mc, s);
    sv_run(e, mc, p, params_dev, dtype, per_edge, s, out_dev);
  });
}
