"""Autotuner for the executors' task shapes.

Networks too large for one CTA's shared memory run on the persistent graph
executor (one launch per wave).  How its work is cut into tasks decides how
well the tasks fill the GPU: the rank above which tensors live in global
memory (`small_rank`), the multiply-adds per chunk task of a global step
(`task_terms_log2`) and the size of a shared-memory subtree task
(`subtree_bytes`).  Batches whose networks fit one CTA's shared memory run on
the shared-memory executor, one network per warp or one per CTA
(`warp_teams`).  `autotune` times each candidate on the batch itself (the
device call, L2 flushed between evaluations, CUDA events), applies the
fastest to the engine and can persist the choice in a JSON cache keyed by the
batch's structure, the dtype, the gradient flag and the GPU, so a later run
applies it without timing.
"""

from __future__ import annotations

import hashlib
import json
import os

DEFAULTS = {"small_rank": 10, "task_terms_log2": 16, "subtree_bytes": 32768,
            "warp_teams": 1, "graph_hi_occupancy": False}


def default_candidates(graph: bool = True):
    """Graph programs: small_rank x task size x subtree size around the
    defaults, on the regular and on the five-CTAs-per-SM kernel build.
    Shared-memory programs: one network per warp (layout by cost, or with
    streamed steps) or one per CTA."""
    if not graph:
        return [dict(DEFAULTS), dict(DEFAULTS, warp_teams=2), dict(DEFAULTS, warp_teams=0)]
    out = []
    for occ in (False, True):
        for sr in (9, 10, 11):
            for tt in (15, 16, 17, 18):
                for sb in (16384, 32768):
                    out.append(dict(DEFAULTS, small_rank=sr, task_terms_log2=tt,
                                    subtree_bytes=sb, graph_hi_occupancy=occ))
    return out


def quick_candidates():
    """A short list for graph programs: the rank above which tensors live in
    global memory (9, 10) x multiply-adds per chunk task (2^16, 2^17, 2^18)."""
    return [dict(DEFAULTS, small_rank=sr, task_terms_log2=tt)
            for sr in (9, 10) for tt in (16, 17, 18)]


def signature(batch, dtype: str, want_grad: bool, device_name: str) -> str:
    """Key of a tuning result: the batch's networks and plans (edges, depth,
    sizes and step counts), the dtype, the gradient flag and the GPU."""
    st = batch.stats()
    h = hashlib.sha1()
    h.update(repr(sorted(tuple(e) for e in batch.edges)).encode())
    h.update(repr((batch.p, st["n_networks"], st["max_rank"], st["n_steps_total"],
                   round(st["cmacs"]), round(st["bytes_c64"]))).encode())
    return f"{h.hexdigest()[:16]}|{dtype}|{int(bool(want_grad))}|{device_name}"


def _load(path):
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _store(path, table):
    if not path:
        return
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(engine, choice: dict):
    """Set the engine's graph-executor options to `choice` (invalidates its
    prepared programs)."""
    engine.set_graph_options(False, int(choice["small_rank"]))
    engine.set_task_options(int(choice["task_terms_log2"]), int(choice["subtree_bytes"]),
                            int(choice.get("warp_teams", 1)),
                            bool(choice.get("graph_hi_occupancy", False)))


def _device_timer(engine, batch, dtype, want_grad, steps, warmup):
    import torch

    from . import qaoa_expectation_device
    dev = torch.device(f"cuda:{engine.device}")
    P = 2 * batch.p
    params = torch.full((P,), 0.3, dtype=torch.float64, device=dev)
    out = torch.zeros(2 + P + len(batch.edges), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run():
        for _ in range(warmup):
            qaoa_expectation_device(engine, batch, params, out, dtype, want_grad=want_grad)
        ts = []
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            qaoa_expectation_device(engine, batch, params, out, dtype, want_grad=want_grad)
            e.record()
            ts.append((s, e))
        torch.cuda.synchronize()
        vals = sorted(s.elapsed_time(e) for s, e in ts)
        return vals[len(vals) // 2]
    return run


def autotune(engine, batch, dtype: str = "c64", want_grad: bool = True, *, cache_path=None,
             candidates=None, steps: int = 5, warmup: int = 2, timer=None,
             device_name=None) -> dict:
    """Pick the fastest graph-executor options for `batch` on `engine` and
    apply them.  Returns the choice with its median time in ms ("ms"), whether
    it came from the cache ("cached") and every candidate's time ("trials").
    `timer`, if given, is called after each candidate is applied and prepared
    and returns its time in ms (the default times the device call)."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name(engine.device)
    key = signature(batch, dtype, want_grad, device_name)
    table = _load(cache_path)
    if key in table:
        choice = dict(DEFAULTS, **table[key])
        apply(engine, choice)
        choice.update(cached=True, trials=[])
        return choice
    graph = bool(batch.program_info(dtype, want_grad)["graph"])
    from . import QtcError
    if timer is None:
        timer = _device_timer(engine, batch, dtype, want_grad, steps, warmup)
    trials = []
    for cand in candidates or default_candidates(graph):
        cand = dict(DEFAULTS, **cand)
        try:
            apply(engine, cand)
            batch.prepare(engine, dtype, want_grad=want_grad)
            ms = float(timer())
        except QtcError as err:  # a candidate that does not fit the arena or the limits
            trials.append(dict(cand, ms=None, error=str(err)))
            continue
        trials.append(dict(cand, ms=ms))
    ok = [t for t in trials if t["ms"] is not None]
    if not ok:
        apply(engine, DEFAULTS)
        raise QtcError(-1, "no autotuning candidate ran: " + "; ".join(
            t.get("error", "") for t in trials))
    best = min(ok, key=lambda t: t["ms"])
    choice = {k: best[k] for k in DEFAULTS}
    apply(engine, choice)
    table[key] = dict(choice, ms=best["ms"])
    _store(cache_path, table)
    return dict(choice, ms=best["ms"], cached=False, trials=trials, graph=graph)
