// qtc_qaoa_expectation_static: the Max-Cut evaluation without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs inside another framework's memory pool, or a plugin whose host forbids
// device allocations).  The executor's scratch — program tables, per-network
// result rows and counters — lives in a fixed file-scope device array
// instead of an engine arena.
#include <mutex>

#include "exec_launch.h"
#include "qtc_internal.h"

namespace {

constexpr size_t kScratchBytes = QTC_STATIC_SCRATCH_BYTES;

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  void* scratch = nullptr;   // device address of g_static_scratch on this device
  size_t smem_optin = 0;
  int sm_count = 0;
  uint64_t resident = 0;     // serial of the program whose tables are in the array
};

std::mutex g_mutex;
DeviceSetup g_setup[kMaxDevices];

// With the device current: the host-side name of the array is only a
// stand-in, so its device address is resolved here.  The lookup allocates
// nothing and is repeated on every call, so that a module reloaded after a
// device reset (the array may then sit elsewhere, with its contents lost)
// is noticed: a new address forgets which program's tables were resident.
// The device attributes are read once per device.
DeviceSetup& setup_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) qtc::fail(QTC_ERR_INVALID, "device %d out of range", dev);
  DeviceSetup& s = g_setup[dev];
  void* p = nullptr;
  qtc::cuda_check(cudaGetSymbolAddress(&p, g_static_scratch),
                  "cudaGetSymbolAddress(static scratch)");
  if (s.sm_count == 0) {
    int v = 0;
    qtc::cuda_check(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                    "shared memory limit");
    s.smem_optin = (size_t)v;
    qtc::cuda_check(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev), "SM count");
    s.sm_count = v;
  }
  if (p != s.scratch) {
    s.scratch = p;
    s.resident = 0;
  }
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" qtc_status qtc_qaoa_expectation_static(qtc_batch* b, const double* params_dev,
                                                  int dtype, int want_grad, void* stream,
                                                  double* out_dev) {
  using namespace qtc;
  return guarded([&] {
    if (!b || !params_dev || !out_dev) fail(QTC_ERR_INVALID, "null argument");
    int dev = -1;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSetup& setup = setup_device(dev);
    const size_t max_dyn = max_dynamic_smem(setup.smem_optin);
    const HostProgram& hp = host_program(b, dtype, want_grad, max_dyn);
    if (hp.graph)
      fail(QTC_ERR_UNSUPPORTED,
           "this batch has networks larger than one CTA's shared memory; use "
           "qtc_qaoa_expectation_device with an arena");
    const int P = hp.n_params, N = hp.n_nets, G = (int)hp.gates.size();

    // layout of one call inside the array
    const size_t o_gates = 0;
    const size_t o_tasks = align256(o_gates + sizeof(GateEntryDev) * G);
    const size_t o_ops = align256(o_tasks + sizeof(TaskDev) * hp.tasks.size());
    const size_t o_wsteps = align256(o_ops + sizeof(SOp) * hp.ops.size());
    const size_t o_coef = align256(o_wsteps + sizeof(WStep) * hp.wsteps.size());
    const size_t o_weights = align256(o_coef + hp.coef.size());
    const size_t o_results = align256(o_weights + sizeof(double) * N);
    // the FP64 sums and the counters sit together: one clear per call
    const size_t o_acc = align256(o_results + sizeof(double) * (size_t)N * (2 + 2 * P));
    const size_t o_counters = o_acc + ((sizeof(double) * (1 + P) + 15) & ~size_t(15));
    const size_t total = o_counters + sizeof(unsigned int) * 4;
    if (total > kScratchBytes)
      fail(QTC_ERR_ARENA,
           "this batch needs %zu bytes of device scratch; the static scratch array holds %zu "
           "bytes (use qtc_qaoa_expectation_device with an arena instead)",
           total, kScratchBytes);

    char* base = (char*)setup.scratch;
    cudaStream_t s = (cudaStream_t)stream;
    if (setup.resident != hp.serial) {
      cuda_check(cudaMemcpyAsync(base + o_gates, hp.gates.data(), sizeof(GateEntryDev) * G,
                                 cudaMemcpyHostToDevice, s), "upload gates");
      cuda_check(cudaMemcpyAsync(base + o_tasks, hp.tasks.data(),
                                 sizeof(TaskDev) * hp.tasks.size(), cudaMemcpyHostToDevice, s),
                 "upload tasks");
      if (!hp.ops.empty())
        cuda_check(cudaMemcpyAsync(base + o_ops, hp.ops.data(), sizeof(SOp) * hp.ops.size(),
                                   cudaMemcpyHostToDevice, s), "upload ops");
      if (!hp.wsteps.empty())
        cuda_check(cudaMemcpyAsync(base + o_wsteps, hp.wsteps.data(),
                                   sizeof(WStep) * hp.wsteps.size(),
                                   cudaMemcpyHostToDevice, s), "upload warp ops");
      if (!hp.coef.empty())
        cuda_check(cudaMemcpyAsync(base + o_coef, hp.coef.data(), hp.coef.size(),
                                   cudaMemcpyHostToDevice, s), "upload gate coefficients");
      cuda_check(cudaMemcpyAsync(base + o_weights, hp.weights.data(), sizeof(double) * N,
                                 cudaMemcpyHostToDevice, s), "upload weights");
      setup.resident = hp.serial;
    }
    // the sums, the queue and the team counter must start at zero; the array
    // keeps whatever the previous call left there
    cuda_check(cudaMemsetAsync(base + o_acc, 0, o_counters - o_acc + sizeof(unsigned int) * 4, s),
               "clear counters");

    int per_sm = 0;
    const int mode = hp.warp_teams ? (hp.stream_steps ? 2 : 1) : 0;
    cuda_check(smem_exec_configure(dtype == QTC_C128 ? 0 : 1, mode, hp.smem, max_dyn,
                                   hp.block, &per_sm), "configure executor");
    if (per_sm < 1) fail(QTC_ERR_UNSUPPORTED, "executor does not fit on an SM");
    ProgramDev d{};
    d.gates = (const GateEntryDev*)(base + o_gates);
    d.n_gates = G;
    for (int g = 0; g < G && g < kInlineGates; ++g) d.gates_inline[g] = hp.gates[g];
    d.table_elems = hp.table_elems;
    d.table_bytes = hp.table_bytes;
    d.team_bytes = hp.team_bytes;
    d.stage_ops = hp.stage_ops;
    d.task_stride = hp.task_stride;
    d.coef = base + o_coef;
    d.tasks = (const TaskDev*)(base + o_tasks);
    d.n_tasks = (int)hp.tasks.size();
    d.ops = (const SOp*)(base + o_ops);
    d.wsteps = (const WStep*)(base + o_wsteps);
    d.n_params = P;
    d.n_nets = N;
    d.weights = (const double*)(base + o_weights);
    d.params = params_dev;
    d.results = (double*)(base + o_results);
    d.acc = (double*)(base + o_acc);
    d.out = out_dev;
    d.counters = (unsigned int*)(base + o_counters);
    d.want_grad = hp.want_grad;
    d.qaoa_reduce = hp.qaoa_reduce;
    const int ctas = ((int)hp.tasks.size() + hp.n_teams - 1) / hp.n_teams;
    const int grid = std::max(1, std::min(ctas, setup.sm_count * per_sm));
    cuda_check(smem_exec_launch(d, dtype == QTC_C128 ? 0 : 1, mode, grid, hp.block,
                                hp.smem, s),
               "launch executor");
  });
}
