"""The graph-executor autotuner on a GPU: every candidate computes the same
values (only the task shapes differ), the choice is applied and persisted,
and a second call takes it from the cache."""

import numpy as np
import pytest

import paper_1709_03636_gb300 as q
from synth import WORKLOADS


@pytest.mark.gpu
def test_autotune_keeps_values_and_caches(tmp_path):
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    g, b = w.angles()
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), obs_edges=edges[:4], ordering="lg")
    assert batch.program_info("c64", True)["graph"] == 1
    engine = q.Engine(0, arena_bytes=512 << 20)
    C0, e0, g0 = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    cands = [dict(small_rank=10, task_terms_log2=16, subtree_bytes=32768),
             dict(small_rank=9, task_terms_log2=15, subtree_bytes=16384),
             dict(small_rank=11, task_terms_log2=17, subtree_bytes=32768),
             dict(small_rank=10, task_terms_log2=16, subtree_bytes=32768,
                  graph_hi_occupancy=True)]
    path = tmp_path / "tune.json"
    res = q.autotune(engine, batch, "c64", True, cache_path=str(path), candidates=cands,
                     steps=3, warmup=1)
    assert res["cached"] is False
    assert len([t for t in res["trials"] if t["ms"] is not None]) == len(cands)
    assert engine.task_options == (res["task_terms_log2"], res["subtree_bytes"], 1,
                                   res["graph_hi_occupancy"])
    for cand in cands:
        q.tuning.apply(engine, cand)
        C1, e1, g1 = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
        assert abs(C1 - C0) <= 1e-5 * abs(C0)
        assert np.max(np.abs(np.array(e1) - np.array(e0))) < 1e-5
        assert np.max(np.abs(np.array(g1) - np.array(g0))) <= 1e-4 * np.max(np.abs(g0))
    res2 = q.autotune(engine, batch, "c64", True, cache_path=str(path), candidates=cands)
    assert res2["cached"] is True
    assert (res2["small_rank"], res2["task_terms_log2"]) == (res["small_rank"],
                                                           res["task_terms_log2"])


@pytest.mark.gpu
def test_arena_of_any_length_keeps_the_work_buffer_aligned():
    """The graph executor's global intermediates live at the back of the
    arena; an arena length that is not a multiple of 256 (here +1000 bytes)
    is rounded down so that buffer stays aligned, and the values match those
    from a round arena."""
    import torch
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    g, b = w.angles()
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), obs_edges=edges[:2], ordering="lg")
    ref = q.qaoa_expectation(q.Engine(0, arena_bytes=256 << 20), batch, g, b, "c64",
                             want_grad=True)
    arena = torch.empty((256 << 20) + 1000, dtype=torch.uint8, device="cuda:0")
    got = q.qaoa_expectation(q.Engine(0, arena=arena), batch, g, b, "c64", want_grad=True)
    assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert np.max(np.abs(np.array(got[2]) - np.array(ref[2]))) <= 1e-12 * np.max(np.abs(ref[2]))
