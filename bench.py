#!/usr/bin/env python
"""Throughput of QAOA Max-Cut edge-network contraction on GB300.

One step = one evaluation of <C>(gamma, beta) and its gradient for one
graph: every per-edge <Z_u Z_v> light-cone network is contracted (forward
pass) and swept backwards (adjoint), and the per-edge scalars are reduced to
<C> and d<C>/d(gamma, beta) in FP64.  The headline workload is the largest
single-GPU one: p = 3 on a 4-regular 60-vertex graph, value and gradient
(120 networks, intermediates of rank up to 24).  The planner (host) runs once
before timing, as the paper excludes ordering time.  `value` is edge
networks per second with inputs resident in device memory; `e2e` is the same
through the host-pointer C call (every step, the parameters go in and the
results come out through the engine's pinned, device-mapped host buffer).
The other workloads are reported on the same line under "configs".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference   # the FP64 CPU oracle on the same metric

With N > 1 (torchrun) the graph's edge networks are sharded over the ranks
(longest processing time first on their algorithmic bytes, the same
partition on every rank) and each step ends with one FP64 all-reduce of the
1 + 2p partial sums: the total work is fixed (strong scaling).
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

DEFAULT_WORKLOAD = "qaoa_p3_n60_d4"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, per launch) of
# the dominant kernel from one ncu capture of the same workload, reported only
# while the kernel's sources hash to the value recorded with the capture
# (otherwise null: the figure would describe another kernel).
KERNEL_SOURCES = {
    "smem_exec_kernel": ["exec_smem.cu", "exec_common.cuh", "device_program.h",
                         "warp_program.cpp", "api.cpp", "gate_coef.cpp", "lower.cpp"],
    "graph_exec_kernel": ["exec_graph.cu", "exec_common.cuh", "device_program.h", "lower.cpp",
                          "graph_host.cpp", "tile_plan.cpp"],
}
NCU_TRAFFIC = {
    # (workload, kernel, dtype, want_grad): (bytes per launch, source hash, profile summary)
    ("qaoa_p1_n50_d3", "smem_exec_kernel", "c64", True):
        (643840, "48e4649410569c71", "profiles/smem_exec_kernel_qaoa_p1_n50_d3.md"),
    ("qaoa_p3_n60_d4", "graph_exec_kernel", "c64", True):
        (23111387648, "8838fa3bffc44c32", "profiles/graph_exec_kernel_qaoa_p3_n60_d4.md"),
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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default=None, help="override the workload's element type")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-mode", type=int, default=None, choices=[0, 1, 2],
                    help="graph executor's tile form of global steps (default: the library's)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads reported under \"configs\"")
    ap.add_argument("--edges", type=int, default=0,
                    help="contract only the first K edge networks (small profiling cases)")
    ap.add_argument("--dense", action="store_true",
                    help="rank-4 ZZ tensors instead of diagonal (hyperedge) ZZ")
    ap.add_argument("--per-network", action="store_true",
                    help="also time the plain form: one launch per edge network")
    ap.add_argument("--crossover", action="store_true",
                    help="tensor network vs state vector over regularities 3..7 (table)")
    ap.add_argument("--width-sweep", action="store_true",
                    help="time per <C> against the ordering's width, 18-qubit circuits (table)")
    ap.add_argument("--autotune", default=None, metavar="CACHE.json",
                    help="tune the graph executor's task shapes on this workload first "
                         "(cache file, created if missing; no effect on shared-memory batches)")
    ap.add_argument("--tune", default="quick", choices=["quick", "off"],
                    help="without --autotune: time six task shapes of the graph executor on "
                         "the headline workload before the timed steps and keep the fastest "
                         "(quick, the default), or run the library defaults (off)")
    ap.add_argument("--noise", default=None, metavar="CHANNEL:STRENGTH",
                    help="noisy QAOA: depolarize|dephase|ampdamp channel of that strength on "
                         "every qubit after each mixer (density-matrix networks)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the job is as
    slow as its slowest rank); the identity with one rank."""
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) <= 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_rate(networks_total, seconds_per_step):
    """Whole-job throughput: every network of the graph (over all ranks)
    per step, over the slowest rank's step time."""
    return networks_total / seconds_per_step


def workload_config(w, networks, want_grad, dtype, noise=None, world=1):
    cfg = {
        "workload": w.name,
        "graph": f"{w.d}-regular, n={w.n}, configuration model seed {w.graph_seed}",
        "p": w.p,
        "networks_per_step": networks,
        "ordering": w.ordering + (f" ({w.restarts} randomised min-fill runs)"
                                  if w.ordering == "lg" else ""),
        "form": ("diagonal ZZ (hyperedges)" if w.diag else "rank-4 ZZ") +
                (", light cone" if w.lightcone else ", full network"),
        "want_grad": want_grad,
        "dtype": dtype,
        "l2": "flushed between timed steps (256 MiB write outside the events); the "
              "largest intermediates (2^20-2^24 complex64) exceed L2 as well",
    }
    if world > 1:
        cfg["parallelism"] = (f"edge networks sharded over {world} ranks (longest processing "
                              "time first on algorithmic bytes), one FP64 all-reduce of the "
                              "1 + 2p sums per step")
    if noise:
        cfg["noise"] = f"{noise[0]} channel, strength {noise[1]}, every qubit after each mixer"
    return cfg


class ClockSampler:
    """nvidia-smi samples (every 20 ms) over the headline workload's
    warm-up and timed phases; the summary covers that whole window and says
    how many samples fell inside the timed steps themselves."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []          # (host time, csv line)
        self.window = (0.0, 0.0)
        self.timed = (0.0, 0.0)

    def start(self):
        """Start sampling and wait for the first sample, so that nvidia-smi's
        own start-up never overlaps the measured phases."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
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

    def mark(self, t_begin, t_end, timed=None):
        self.window = (t_begin, t_end)
        if timed:
            self.timed = timed

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(lines):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
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
        return sm, mx, reasons

    def summary(self):
        t0, t1 = self.window
        sm, mx, reasons = self._parse([ln for t, ln in self.lines if t0 <= t <= t1])
        tt0, tt1 = self.timed
        sm_t, _, _ = self._parse([ln for t, ln in self.lines if tt0 <= t <= tt1])
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "samples_in_timed_steps": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "samples_in_timed_steps": len(sm_t),
                "sm_mhz_timed_steps": statistics.median(sm_t) if sm_t else None,
                "window": "warm-up, value+gradient, forward and end-to-end phases of the "
                          "headline workload"}


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


def cpu_baseline_line(w, want_grad, seconds):
    edges = w.graph()
    g, b = w.angles()
    rate, done, el = oracle_networks_per_s(w, edges, g, b, want_grad, seconds)
    return {"value": rate, "unit": "networks/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} edge networks of {w.name}" + (" with gradient" if want_grad else "")
                      + f" in {el:.1f} s (FP64 tensor-network oracle, numpy einsum, one thread)"}


def run_reference(args):
    """The oracle as the reference arm: same workload and metric, rank 0
    only; each step is a bounded sample (one edge network, value and
    gradient, rotating over the graph's edges)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    edges = w.graph()
    g, b = w.angles()
    want_grad = True
    from oracle import tensornet as tn
    per_step = 1 if w.p >= 3 else min(len(edges), 25)

    def step(k):
        for j in range(per_step):
            e = edges[(k * per_step + j) % len(edges)]
            tn.edge_value_grad(w.n, edges, g, b, e, lightcone=w.lightcone, dense=not w.diag)

    for k in range(args.warmup):
        step(k)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + k)
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = per_step / sec
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "networks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": workload_config(w, per_step, want_grad, "c128"),
        "cpu_baseline": {"value": value, "unit": "networks/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} of {len(edges)} edge networks per step (rotating "
                                   "over the edges), FP64 tensor-network oracle with "
                                   "forward-mode gradient, one thread"},
        "e2e": {"value": value, "unit": "networks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Bench:
    """Device state shared by every workload measured in one run."""

    def __init__(self, q, dev, stream, world, rank):
        import torch
        self.q, self.dev, self.stream, self.world, self.rank = q, dev, stream, world, rank
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.tile_mode = None

    def timed(self, fn, steps):
        """Per-step device times (ms) of `steps` calls of fn, CUDA events on
        the launching stream, L2 flushed between steps outside the events.
        A short device-side sleep first, so that the steps are all queued
        before the GPU reaches them: the events then time the GPU alone."""
        import torch
        torch.cuda._sleep(int(4e6))
        evs = []
        for _ in range(steps):
            self.flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(self.stream)
            fn()
            e.record(self.stream)
            evs.append((s, e))
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in evs]

    def barrier(self):
        import torch
        torch.cuda.synchronize()
        if self.world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def setup(self, w, dtype, grads, noise=None, obs_edges=None, autotune=None, tune=False):
        """Circuit, whole batch, this rank's shard, an engine sized for its
        programs, prepared for every gradient flag in `grads`."""
        import torch
        q = self.q
        edges = w.graph()
        g, b = w.angles()
        circ = q.Circuit.qaoa(w.n, edges, w.p, noise=noise)
        full = q.Batch(circ, obs_edges, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering,
                       restarts=w.restarts)
        batch, mine = q.shard(full, self.rank, self.world, want_grad=max(grads))
        if batch is None:
            raise SystemExit(f"rank {self.rank} has no edge network of {w.name}")
        need = 0
        for grad in grads:
            # room for the tuning candidates too (small_rank 9 keeps more in global memory)
            per = [batch.program_info(dtype, grad, small_rank=sr) for sr in ((0, 9) if tune else (0,))]
            need += max(i["work_bytes"] + 2 * i["table_bytes"] for i in per)
        engine = q.Engine(self.dev.index, arena_bytes=int(need) + (256 << 20))
        if self.tile_mode is not None:
            engine.set_tile_mode(self.tile_mode)
        tuned = None
        if autotune:
            tuned = q.autotune(engine, batch, dtype, max(grads), cache_path=autotune)
            tuned = {k: tuned[k] for k in ("small_rank", "task_terms_log2", "subtree_bytes",
                                           "cached")}
        elif tune and batch.program_info(dtype, max(grads))["graph"]:
            from paper_1709_03636_gb300.tuning import quick_candidates
            t0 = time.time()
            res = q.autotune(engine, batch, dtype, max(grads), candidates=quick_candidates())
            tuned = {k: res[k] for k in ("small_rank", "task_terms_log2", "subtree_bytes")}
            tuned.update(mode="quick: 6 task shapes timed on this batch, untimed setup",
                         trials_ms={f"{t['small_rank']}/{t['task_terms_log2']}": t["ms"]
                                    for t in res["trials"]},
                         tuning_s=round(time.time() - t0, 1))
        for grad in grads:
            batch.prepare(engine, dtype, want_grad=grad)
        P = 2 * w.p
        params = torch.tensor(g + b, dtype=torch.float64, device=self.dev)
        out = torch.zeros(2 + P + len(mine), dtype=torch.float64, device=self.dev)
        return dict(w=w, edges=edges, g=g, b=b, circ=circ, full=full, batch=batch, mine=mine,
                    engine=engine, params=params, out=out, P=P, dtype=dtype, tuned=tuned,
                    n_total=len(full.edges))

    def step_fn(self, st, grad):
        """One evaluation: the rank's launches, then (N > 1) the one FP64
        all-reduce of the 1 + 2p sums."""
        q = self.q
        sums = st["out"][:1 + st["P"]]

        def fn():
            q.qaoa_expectation_device(st["engine"], st["batch"], st["params"], st["out"],
                                      st["dtype"], want_grad=grad, stream=self.stream)
            if self.world > 1:
                q.allreduce_sum(sums)
        return fn

    def roofline(self, st, ms, want_grad, peak, peak_kind, traffic=None, traffic_src=None):
        stats = st["batch"].stats()
        prog = st["batch"].program_info(st["dtype"], want_grad)
        elem = 16 if st["dtype"] == "c128" else 8
        alg = (stats["bytes_c64"] + (stats["grad_bytes_c64"] if want_grad else 0.0)) * elem / 8
        launches = prog["n_waves"] if prog["graph"] else 1
        achieved = alg / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": "graph_exec_kernel" if prog["graph"] else "smem_exec_kernel",
                "launches_per_step": launches, "peak_kind": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_step": alg,
                "algorithmic_bytes_per_launch": alg / launches}

    def e2e(self, st, steps, warmup):
        """The host-pointer C call per step: pinned parameters in, <C>, the
        gradient and the per-edge values out (plus, N > 1, the all-reduce)."""
        import torch
        q = self.q
        from paper_1709_03636_gb300 import _lib
        P, n = st["P"], len(st["mine"])
        h_gam = torch.tensor(st["g"], dtype=torch.float64).pin_memory()
        h_bet = torch.tensor(st["b"], dtype=torch.float64).pin_memory()
        h_C = torch.zeros(1, dtype=torch.float64).pin_memory()
        h_edge = torch.zeros(n, dtype=torch.float64).pin_memory()
        h_grad = torch.zeros(P, dtype=torch.float64).pin_memory()
        dptr = lambda t: q.ctypes.cast(q.ctypes.c_void_p(t.data_ptr()),  # noqa: E731
                                       q.ctypes.POINTER(q.ctypes.c_double))
        args = (st["engine"].ptr, st["batch"].ptr, dptr(h_gam), dptr(h_bet), q.DTYPES[st["dtype"]],
                1, q.ctypes.c_void_p(self.stream.cuda_stream), dptr(h_C), dptr(h_edge),
                dptr(h_grad))
        call = _lib.lib.qtc_qaoa_expectation

        def step():
            _lib.check(call(*args))
            if self.world > 1:
                q.allreduce_sum(torch.cat([h_C, h_grad]).to(self.dev))

        for _ in range(warmup):
            step()
        self.barrier()
        times = []
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step()
            times.append(time.perf_counter() - t0)
        self.barrier()
        prog = st["batch"].program_info(st["dtype"], True)
        d2h = 8 * (2 + P + n + (0 if prog["graph"] else 1))
        return sum(times) / len(times), 8 * P, d2h


def measure_extra(bench, name, dtype, want_grad, steps, warmup, peak, peak_kind, dense=False,
                  cpu_seconds=5.0, statevector=False):
    """One more workload on the same line: device-timed rate, roofline
    fraction and a one-thread oracle sample (rank 0, N = 1)."""
    from dataclasses import replace
    import torch
    w = WORKLOADS[name]
    if dense:
        w = replace(w, diag=False)
    st = bench.setup(w, dtype, [want_grad])
    fn = bench.step_fn(st, want_grad)
    for _ in range(warmup):
        fn()
    bench.barrier()
    ms_list = bench.timed(fn, steps)
    ms = max_over_ranks([sum(ms_list) / len(ms_list)], bench.dev)[0]
    rec = {"dtype": dtype, "want_grad": want_grad,
           "form": ("diagonal ZZ" if w.diag else "rank-4 ZZ") +
                   (", light cone" if w.lightcone else ", full network"),
           "networks_per_step": st["n_total"], "ms_per_step": ms,
           "value": job_rate(st["n_total"], ms * 1e-3), "unit": "networks/s",
           "launches_per_step": st["engine"].last_launches,
           "roofline": bench.roofline(st, ms, want_grad, peak, peak_kind),
           "C": st["out"][0].item()}
    prog = st["batch"].program_info(dtype, want_grad)
    rec["gemm_steps"] = prog["n_gemm_steps"]
    if statevector:
        out_sv = torch.zeros(1 + len(st["edges"]), dtype=torch.float64, device=bench.dev)
        sv_dtype = "c128" if dtype == "c128" else "c64"

        def sv_step():
            bench.q.statevector_expectation_device(st["engine"], st["circ"], st["params"],
                                                   out_sv, sv_dtype, stream=bench.stream)

        for _ in range(warmup):
            sv_step()
        sv = bench.timed(sv_step, steps)
        svt = sum(sv) / len(sv)
        rec["statevector"] = {"ms_per_eval": svt, "tn_over_sv_time": ms / svt,
                              "C": out_sv[0].item(), "bytes_per_eval_hint":
                              "about 3 passes over 2^n complex64"}
    if bench.rank == 0 and bench.world == 1 and cpu_seconds > 0:
        rec["cpu_baseline"] = cpu_baseline_line(w, want_grad, cpu_seconds)
    del st
    torch.cuda.empty_cache()
    return rec


def run_ours(args):
    import torch
    import paper_1709_03636_gb300 as q

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    bench = Bench(q, dev, stream, world, rank)
    bench.tile_mode = args.tile_mode
    peak, peak_kind = measured_peaks()

    from dataclasses import replace
    w = WORKLOADS[args.workload]
    if args.dense:
        w = replace(w, diag=False)
    dtype = args.dtype or w.dtype
    want_grad = True
    noise = None
    if args.noise:
        kind, strength = args.noise.split(":")
        noise = (kind, float(strength))
    obs = w.graph()[:args.edges] if args.edges else None
    st = bench.setup(w, dtype, [True, False], noise=noise, obs_edges=obs,
                     autotune=args.autotune, tune=args.tune == "quick")
    n_total = st["n_total"]
    grad_step, fwd_step = bench.step_fn(st, True), bench.step_fn(st, False)

    clocks = ClockSampler(local).start()
    t_begin = time.perf_counter()
    for _ in range(args.warmup):
        grad_step()
        fwd_step()
    bench.barrier()
    t0 = time.perf_counter()
    step_ms = bench.timed(grad_step, args.steps)
    t1 = time.perf_counter()
    launches = args.steps * st["engine"].last_launches
    bench.barrier()
    fwd_ms = bench.timed(fwd_step, args.steps)
    bench.barrier()
    e2e_s, h2d, d2h = bench.e2e(st, args.steps, args.warmup)
    t_end = time.perf_counter()
    clocks.mark(t_begin, t_end, timed=(t0, t1))

    ms = sum(step_ms) / len(step_ms)
    fwd = sum(fwd_ms) / len(fwd_ms)
    ms, e2e_s, fwd = max_over_ranks([ms, e2e_s, fwd], dev)
    stats = st["batch"].stats()
    kernel = "graph_exec_kernel" if st["batch"].program_info(dtype, True)["graph"] \
        else "smem_exec_kernel"
    traffic, traffic_src = ncu_traffic(w.name, kernel, dtype, want_grad) \
        if not noise and not args.edges and world == 1 else (None, None)
    roof = bench.roofline(st, ms, want_grad, peak, peak_kind, traffic, traffic_src)
    clk = clocks.summary()
    clocks.stop()
    line = {
        "metric": METRIC, "value": job_rate(n_total, ms * 1e-3), "unit": "networks/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(w, n_total, want_grad, dtype, noise, world),
        "roofline": roof,
        "e2e": {"value": job_rate(n_total, e2e_s), "unit": "networks/s",
                "h2d_bytes_per_step": h2d,
                # <C>, gradient, per-edge values, status; the shared-memory
                # executor also writes its 8-byte completion word
                "d2h_bytes_per_step": d2h},
        "complex_gflops": {"value": 8.0 * (stats["cmacs"] + stats["grad_cmacs"]) / (ms * 1e-3)
                           / 1e9, "unit": "GFLOP/s",
                           "count": "algorithmic, 8 real flops per complex multiply-add "
                                    "(forward and adjoint contractions), this rank"},
        "gpu_launches": launches,
        "autotuned": st["tuned"],
        "clocks": clk,
        "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)],
        "forward_only": {"value": job_rate(n_total, fwd * 1e-3), "unit": "networks/s",
                         "ms_per_step": fwd,
                         "roofline": bench.roofline(st, fwd, False, peak, peak_kind)},
        "grad_fwd_ratio": ms / fwd,
        "C": st["out"][0].item(),
        "timed_wall_s": t1 - t0,
    }
    if clk.get("sm_mhz"):
        line["clocks"]["ms_x_median_sm_mhz"] = ms * clk["sm_mhz"]
    if args.per_network:
        line["per_network_c64_forward"] = per_network(bench, st, args, fwd)
    del st
    torch.cuda.empty_cache()
    if not args.no_extras and not args.edges and not noise:
        k, wu = min(args.steps, 20), min(args.warmup, 3)
        cpu_s = 0.0 if args.no_cpu_baseline else 5.0
        extras = {}
        extras["qaoa_p1_n50_d3"] = measure_extra(
            bench, "qaoa_p1_n50_d3", "c64", True, k, wu, peak, peak_kind, cpu_seconds=cpu_s)
        extras["qaoa_p2_n100_d5"] = measure_extra(
            bench, "qaoa_p2_n100_d5", "c64", True, k, wu, peak, peak_kind, cpu_seconds=cpu_s)
        extras["qaoa_p2_n100_d5_dense_split_bf16"] = measure_extra(
            bench, "qaoa_p2_n100_d5", "split_bf16", False, k, wu, peak, peak_kind, dense=True,
            cpu_seconds=cpu_s)
        extras["qaoa_p2_n100_d5_dense_c64"] = measure_extra(
            bench, "qaoa_p2_n100_d5", "c64", False, k, wu, peak, peak_kind, dense=True,
            cpu_seconds=0.0)
        extras["qaoa_p1_n26_d7_full"] = measure_extra(
            bench, "qaoa_p1_n26_d7", "c64", False, k, wu, peak, peak_kind, cpu_seconds=cpu_s,
            statevector=True)
        line["configs"] = extras
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not noise:
        line["cpu_baseline"] = cpu_baseline_line(w, want_grad, 10.0)
        rate_all, cores, done_all = oracle_all_cores(w, want_grad, 10.0)
        line["cpu_baseline_all_cores"] = {
            "value": rate_all, "unit": "networks/s", "cores": cores, "kind": "oracle",
            "sample": f"{done_all} edge networks of {w.name} with gradient, 10 s on each of "
                      f"{cores} processes (one per core, edges dealt round robin)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def per_network(bench, st, args, fwd):
    """The plain form: every edge network its own batch and launch, c64."""
    import torch
    q = bench.q
    w = st["w"]
    singles = [q.Batch(st["circ"], [e], lightcone=w.lightcone, diag=w.diag, ordering=w.ordering,
                       restarts=w.restarts)
               for e in st["batch"].edges]
    outs = [torch.zeros(2 + st["P"] + 1, dtype=torch.float64, device=bench.dev)
            for _ in singles]
    for sb in singles:
        sb.prepare(st["engine"], "c64", want_grad=False)

    def step():
        for sb, o in zip(singles, outs):
            q.qaoa_expectation_device(st["engine"], sb, st["params"], o, "c64", want_grad=False,
                                      stream=bench.stream)

    for _ in range(args.warmup):
        step()
    pn = bench.timed(step, args.steps)
    pn = sum(pn) / len(pn)
    return {"value": len(singles) / (pn * 1e-3), "unit": "networks/s", "ms_per_step": pn,
            "launches_per_step": len(singles), "batched_forward_speedup": pn / fwd}


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
