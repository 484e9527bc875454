#!/usr/bin/env python
"""Throughput of QAOA Max-Cut edge-network contraction on GB300.

One step = one evaluation of <C>(gamma, beta) and its gradient for one
graph: every per-edge <Z_u Z_v> light-cone network is contracted (forward
pass) and swept backwards (adjoint), and the per-edge scalars are reduced to
<C> and d<C>/d(gamma, beta) in FP64 - all in one launch of the executor.
The planner (host) runs once before timing, as the paper excludes ordering
time.  `value` is edge networks per second with inputs resident in device
memory; `e2e` is the same through the host-pointer C call (every step, the
parameters go in and the results come out through the engine's pinned,
device-mapped host buffer).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference   # the FP64 CPU oracle on the same metric

With N > 1 (torchrun) every rank contracts its own seeded graph of the
same family (independent problems, weak scaling) and no collective touches
the data path.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS  # noqa: E402

DEFAULT_WORKLOAD = "qaoa_p1_n50_d3"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, per launch) of
# the dominant kernel from one ncu capture of the same workload, reported only
# while the kernel's sources hash to the value recorded with the capture
# (otherwise null: the figure would describe another kernel).
KERNEL_SOURCES = {
    "smem_exec_kernel": ["exec_smem.cu", "exec_common.cuh", "device_program.h",
                         "warp_program.cpp", "api.cpp", "gate_coef.cpp", "lower.cpp"],
    "graph_exec_kernel": ["exec_graph.cu", "exec_common.cuh", "device_program.h", "lower.cpp",
                          "graph_host.cpp"],
}
NCU_TRAFFIC = {
    # (workload, kernel, dtype, want_grad): (bytes per launch, source hash, profile summary)
    ("qaoa_p1_n50_d3", "smem_exec_kernel", "c64", True):
        (640640, "9c63c5f0b746d4c1", "profiles/smem_exec_kernel_qaoa_p1_n50_d3.md"),
}


def kernel_source_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1709_03636_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str, dtype: str, want_grad: bool):
    rec = NCU_TRAFFIC.get((workload, kernel, dtype, want_grad))
    if rec is None or rec[1] != kernel_source_hash(kernel):
        return None, None
    return rec[0], rec[2]

METRIC = "edge-<ZZ> networks/s (value + gradient)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default=None, help="override the workload's element type")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--edges", type=int, default=0,
                    help="contract only the first K edge networks (small profiling cases)")
    ap.add_argument("--dense", action="store_true",
                    help="rank-4 ZZ tensors instead of diagonal (hyperedge) ZZ")
    ap.add_argument("--per-network", action="store_true",
                    help="also time the plain form: one launch per edge network")
    ap.add_argument("--statevector", action="store_true",
                    help="also time the full 2^n state vector on the GPU for the same graph")
    ap.add_argument("--crossover", action="store_true",
                    help="tensor network vs state vector over regularities 3..7 (table)")
    ap.add_argument("--width-sweep", action="store_true",
                    help="time per <C> against the ordering's width, 18-qubit circuits (table)")
    ap.add_argument("--autotune", default=None, metavar="CACHE.json",
                    help="tune the graph executor's task shapes on this workload first "
                         "(cache file, created if missing; no effect on shared-memory batches)")
    ap.add_argument("--noise", default=None, metavar="CHANNEL:STRENGTH",
                    help="noisy QAOA: depolarize|dephase|ampdamp channel of that strength on "
                         "every qubit after each mixer (density-matrix networks)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_workload(base, rank):
    """Rank r contracts the same family's graph with seed (seed + r):
    independent problems, no data exchanged between ranks (weak scaling)."""
    from dataclasses import replace
    return replace(base, graph_seed=base.graph_seed + rank)


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the job is as
    slow as its slowest rank); the identity with one rank."""
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) <= 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, networks_per_rank, seconds_per_step):
    """Whole-job throughput: the networks every rank contracted per step over
    the slowest rank's step time."""
    return world * networks_per_rank / seconds_per_step


def workload_config(w, networks, want_grad, dtype, noise=None):
    cfg = {
        "workload": w.name,
        "graph": f"{w.d}-regular, n={w.n}, configuration model seed {w.graph_seed}",
        "p": w.p,
        "networks_per_step": networks,
        "ordering": w.ordering,
        "form": ("diagonal ZZ (hyperedges)" if w.diag else "rank-4 ZZ") +
                (", light cone" if w.lightcone else ", full network"),
        "want_grad": want_grad,
        "dtype": dtype,
        "l2": "flushed between timed steps (256 MiB write outside the events)",
    }
    if noise:
        cfg["noise"] = f"{noise[0]} channel, strength {noise[1]}, every qubit after each mixer"
    return cfg


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []          # (host time, csv line)
        self.window = (0.0, 0.0)

    def start(self):
        """Start sampling and wait for the first sample, so that nvidia-smi's
        own start-up never overlaps the timed region."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return self
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 10.0:
            time.sleep(0.02)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t_begin, t_end):
        self.window = (t_begin, t_end)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window
        inside = [ln for t, ln in self.lines if t0 <= t <= t1]
        for line in inside:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def oracle_networks_per_s(w, edges, g, b, want_grad, seconds):
    """The FP64 oracle (O-TN, forward-mode gradient) on a bounded sample."""
    from oracle import tensornet as tn
    done = 0
    t0 = time.perf_counter()
    while True:
        for e in edges:
            if want_grad:
                tn.edge_value_grad(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)
            else:
                tn.edge_value(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)
            done += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                return done / el, done, el


def _oracle_share(job):
    """One worker of the all-cores oracle timing: edges k, k + n, ... of the
    workload, repeated for `seconds`."""
    name, k, n, seconds, want_grad = job
    w = WORKLOADS[name]
    edges = w.graph()
    g, b = w.angles()
    from oracle import tensornet as tn
    mine = edges[k::n] or edges[:1]
    done = 0
    t0 = time.perf_counter()
    while True:
        for e in mine:
            if want_grad:
                tn.edge_value_grad(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)
            else:
                tn.edge_value(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)
            done += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                return done, el


def oracle_all_cores(w, want_grad, seconds):
    """The same oracle on every host core: one process per core (spawned, so
    that no child inherits the parent's CUDA context), edges dealt round
    robin; the rate is the sum of the workers' rates."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    jobs = [(w.name, k, n, seconds, want_grad) for k in range(n)]
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_share, jobs)
    return sum(d / el for d, el in res), n, sum(d for d, _ in res)


def run_reference(args):
    """The oracle as the reference arm: same metric, rank 0 only."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    edges = w.graph()
    g, b = w.angles()
    want_grad = True
    sample = edges[:min(len(edges), 25)]
    for _ in range(args.warmup):
        oracle_networks_per_s(w, edges, g, b, want_grad, 0.0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        from oracle import tensornet as tn
        for e in sample:
            tn.edge_value_grad(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)
        times.append(time.perf_counter() - t0)
    per_step = sum(times) / len(times)
    value = len(sample) / per_step
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "networks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": workload_config(w, len(sample), want_grad, "c128"),
        "cpu_baseline": {"value": value, "unit": "networks/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(sample)} of {len(edges)} edge networks per step, "
                                   "FP64 tensor-network oracle with forward-mode gradient"},
        "e2e": {"value": value, "unit": "networks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_1709_03636_gb300 as q
    from paper_1709_03636_gb300 import _lib

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    base = WORKLOADS[args.workload]
    dtype = args.dtype or base.dtype
    want_grad = True
    # rank r contracts graph seed (seed + r): independent problems
    from dataclasses import replace
    w = rank_workload(base, rank)
    if args.dense:
        w = replace(w, diag=False)
    edges = w.graph()
    g, b = w.angles()
    noise = None
    if args.noise:
        kind, strength = args.noise.split(":")
        noise = (kind, float(strength))
    circ = q.Circuit.qaoa(w.n, edges, w.p, noise=noise)
    obs = edges[:args.edges] if args.edges else None
    batch = q.Batch(circ, obs, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
    stats = batch.stats()
    n_nets = stats["n_networks"]
    need = 0
    for grad in (True, False):
        info = batch.program_info(dtype, grad)
        need += info["work_bytes"] + 2 * info["table_bytes"]
    engine = q.Engine(local, arena_bytes=int(need) + (256 << 20))
    tuned = None
    if args.autotune:
        tuned = q.autotune(engine, batch, dtype, want_grad, cache_path=args.autotune)
        tuned = {k: tuned[k] for k in ("small_rank", "task_terms_log2", "subtree_bytes",
                                       "cached")}
    batch.prepare(engine, dtype, want_grad=want_grad)
    batch.prepare(engine, dtype, want_grad=False)
    P = 2 * w.p
    params = torch.tensor(g + b, dtype=torch.float64, device=dev)
    out = torch.zeros(2 + P + n_nets, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def device_step(grad):
        q.qaoa_expectation_device(engine, batch, params, out, dtype, want_grad=grad,
                                  stream=stream)

    def timed(fn, steps):
        # a short device-side sleep first, so that the following steps are all
        # queued before the GPU reaches them: the events then time the GPU
        # alone, not the host's enqueue latency
        torch.cuda._sleep(int(4e6))
        evs = []
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            fn()
            e.record(stream)
            evs.append((s, e))
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in evs]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        device_step(True)
        device_step(False)
    clocks = ClockSampler(local).start()
    barrier()
    wall0 = time.perf_counter()
    step_ms = timed(lambda: device_step(True), args.steps)
    wall = time.perf_counter() - wall0
    clocks.mark(wall0, wall0 + wall)
    launches = args.steps * engine.last_launches
    prog = batch.program_info(dtype, True)
    barrier()
    fwd_ms = timed(lambda: device_step(False), args.steps)
    barrier()

    # end to end through the host-pointer call: pinned params in, results out
    h_gam = torch.tensor(g, dtype=torch.float64).pin_memory()
    h_bet = torch.tensor(b, dtype=torch.float64).pin_memory()
    h_C = torch.zeros(1, dtype=torch.float64).pin_memory()
    h_edge = torch.zeros(n_nets, dtype=torch.float64).pin_memory()
    h_grad = torch.zeros(P, dtype=torch.float64).pin_memory()
    vp = lambda t: q.ctypes.c_void_p(t.data_ptr())  # noqa: E731

    dptr = lambda t: q.ctypes.cast(vp(t), q.ctypes.POINTER(q.ctypes.c_double))  # noqa: E731
    e2e_args = (engine.ptr, batch.ptr, dptr(h_gam), dptr(h_bet), q.DTYPES[dtype], 1,
                q.ctypes.c_void_p(stream.cuda_stream), dptr(h_C), dptr(h_edge), dptr(h_grad))
    e2e_call = _lib.lib.qtc_qaoa_expectation

    def e2e_step():
        _lib.check(e2e_call(*e2e_args))

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    barrier()

    ms = sum(step_ms) / len(step_ms)
    e2e_s = sum(e2e_times) / len(e2e_times)
    fwd = sum(fwd_ms) / len(fwd_ms)
    ms, e2e_s, fwd = max_over_ranks([ms, e2e_s, fwd], dev)
    value = job_rate(world, n_nets, ms * 1e-3)
    elem = 16 if dtype == "c128" else 8
    alg_bytes = (stats["bytes_c64"] + stats["grad_bytes_c64"]) * elem / 8
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    kernel = "graph_exec_kernel" if prog["graph"] else "smem_exec_kernel"
    traffic, traffic_src = ncu_traffic(w.name, kernel, dtype, want_grad) if not noise \
        else (None, None)
    line = {
        "metric": METRIC, "value": value, "unit": "networks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": workload_config(w, n_nets, want_grad, dtype, noise),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "kernel": kernel,
                     "launches_per_step": engine.last_launches,
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_step": alg_bytes},
        "e2e": {"value": job_rate(world, n_nets, e2e_s), "unit": "networks/s",
                "h2d_bytes_per_step": 8 * P,
                # <C>, gradient, per-edge values, status; the shared-memory
                # executor also writes its 8-byte completion word
                "d2h_bytes_per_step": 8 * (2 + P + n_nets + (0 if prog["graph"] else 1))},
        "complex_gflops": {"value": 8.0 * (stats["cmacs"] + (stats["grad_cmacs"] if want_grad
                                                                else 0.0)) / (ms * 1e-3) / 1e9,
                           "unit": "GFLOP/s", "count": "algorithmic, 8 real flops per complex "
                           "multiply-add (forward and adjoint contractions)"},
        "gpu_launches": launches,
        "autotuned": tuned,
        "clocks": clocks.summary(),
        "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)],
        "forward_only": {"value": job_rate(world, n_nets, fwd * 1e-3), "unit": "networks/s",
                         "ms_per_step": fwd},
        "grad_fwd_ratio": ms / fwd,
        "timed_wall_s": wall,
    }
    clocks.stop()
    if args.per_network:
        # the plain form: every edge network is its own batch and launch, c64
        singles = [q.Batch(circ, [e], lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
                   for e in (obs or edges)]
        outs = [torch.zeros(2 + P + 1, dtype=torch.float64, device=dev) for _ in singles]
        for sb in singles:
            sb.prepare(engine, "c64", want_grad=False)

        def per_network_step():
            for sb, o in zip(singles, outs):
                q.qaoa_expectation_device(engine, sb, params, o, "c64", want_grad=False,
                                          stream=stream)

        for _ in range(args.warmup):
            per_network_step()
        pn_ms = timed(per_network_step, args.steps)
        pn = sum(pn_ms) / len(pn_ms)
        line["per_network_c64_forward"] = {
            "value": n_nets / (pn * 1e-3), "unit": "networks/s", "ms_per_step": pn,
            "launches_per_step": len(singles),
            "batched_forward_speedup": pn / fwd}
    if args.statevector:
        out_sv = torch.zeros(1 + len(edges), dtype=torch.float64, device=dev)
        sv_dtype = "c128" if dtype == "c128" else "c64"

        def sv_step():
            q.statevector_expectation_device(engine, circ, params, out_sv, sv_dtype,
                                             stream=stream)

        for _ in range(args.warmup):
            sv_step()
        sv_ms = timed(sv_step, args.steps)
        svt = sum(sv_ms) / len(sv_ms)
        line["statevector_forward"] = {
            "ms_per_eval": svt, "launches": engine.last_launches,
            "tensor_network_forward_ms": fwd, "tn_over_sv_time": fwd / svt,
            "C_statevector": out_sv[0].item(), "C_tensor_network": out[0].item()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not noise:
        rate, done, el = oracle_networks_per_s(w, edges, g, b, want_grad, 10.0)
        line["cpu_baseline"] = {
            "value": rate, "unit": "networks/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} edge networks of {w.name} with gradient in {el:.1f} s "
                      "(FP64 tensor-network oracle, numpy einsum, one thread)"}
        rate_all, cores, done_all = oracle_all_cores(w, want_grad, 10.0)
        line["cpu_baseline_all_cores"] = {
            "value": rate_all, "unit": "networks/s", "cores": cores, "kind": "oracle",
            "sample": f"{done_all} edge networks of {w.name} with gradient, 10 s on each of "
                      f"{cores} processes (one per core, edges dealt round robin)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_width_sweep(args):
    """Time per <C> evaluation (forward, full un-reduced networks, p = 1) of
    18-qubit QAOA circuits on 3- to 7-regular graphs against the width of
    the contraction ordering (largest intermediate rank minus one: the upper
    bound on the treewidth that the ordering certifies), for both orderings
    (Section 5, simulation time against approximate treewidth)."""
    import torch
    import paper_1709_03636_gb300 as q
    from synth import qaoa_angles, random_regular_graph
    dev = torch.device("cuda", 0)
    rows = []
    n = 18
    for d in (3, 4, 5, 6, 7):
        for seed in range(4):
            edges = random_regular_graph(n, d, seed)
            g, b = qaoa_angles(1, seed)
            circ = q.Circuit.qaoa(n, edges, 1)
            params = torch.tensor(g + b, dtype=torch.float64, device=dev)
            for ordering in ("lg", "stoch"):
                bt = q.Batch(circ, lightcone=False, ordering=ordering, seed=seed)
                need = bt.program_info("c64", False)["work_bytes"]
                engine = q.Engine(0, arena_bytes=int(need) + (1 << 30))
                out = torch.zeros(3 + len(edges), dtype=torch.float64, device=dev)
                f = lambda: q.qaoa_expectation_device(engine, bt, params, out, "c64")  # noqa
                for _ in range(2):
                    f()
                torch.cuda.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                for _ in range(args.steps):
                    f()
                s1.record()
                torch.cuda.synchronize()
                st = bt.stats()
                row = {"d": d, "seed": seed, "ordering": ordering, "width": st["max_rank"] - 1,
                       "ms": s0.elapsed_time(s1) / args.steps, "C": out[0].item()}
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
                del engine
                torch.cuda.empty_cache()
    print(json.dumps({"width_sweep": rows}), flush=True)


def run_crossover(args):
    """Time per <C> evaluation (forward) of the light-cone tensor networks, the
    full un-reduced networks and the 2^n state vector, for d = 3..7 at each n."""
    import torch
    import paper_1709_03636_gb300 as q
    from synth import qaoa_angles, random_regular_graph
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    rows = []
    for n in (20, 24, 26):
        for d in (3, 4, 5, 6, 7):
            if (n * d) % 2:
                continue
            edges = random_regular_graph(n, d, 0)
            g, b = qaoa_angles(1, 0)
            circ = q.Circuit.qaoa(n, edges, 1)
            params = torch.tensor(g + b, dtype=torch.float64, device=dev)
            row = {"n": n, "d": d, "edges": len(edges)}
            batches = {"lightcone": q.Batch(circ, lightcone=True),
                       "full": q.Batch(circ, lightcone=False)}
            need = max(bt.program_info("c64", False)["work_bytes"] for bt in batches.values())
            engine = q.Engine(0, arena_bytes=int(need + (8 << 8) * (1 << n) / 256) + (1 << 30))
            for name, bt in batches.items():
                out = torch.zeros(3 + len(edges), dtype=torch.float64, device=dev)
                bt.prepare(engine, "c64", False)
                f = lambda: q.qaoa_expectation_device(engine, bt, params, out, "c64",  # noqa
                                                      stream=stream)
                for _ in range(2):
                    f()
                torch.cuda.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                for _ in range(args.steps):
                    f()
                s1.record(stream)
                torch.cuda.synchronize()
                row[f"tn_{name}_ms"] = s0.elapsed_time(s1) / args.steps
                row[f"tn_{name}_max_rank"] = bt.stats()["max_rank"]
            out_sv = torch.zeros(1 + len(edges), dtype=torch.float64, device=dev)
            f = lambda: q.statevector_expectation_device(engine, circ, params, out_sv, "c64",  # noqa
                                                         stream=stream)
            for _ in range(2):
                f()
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.steps):
                f()
            s1.record(stream)
            torch.cuda.synchronize()
            row["sv_ms"] = s0.elapsed_time(s1) / args.steps
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            del engine
            torch.cuda.empty_cache()
    print(json.dumps({"crossover": rows}), flush=True)


def main():
    args = parse()
    if args.crossover:
        run_crossover(args)
        return
    if args.width_sweep:
        run_width_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
