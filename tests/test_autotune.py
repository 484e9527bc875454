"""Host logic of the graph-executor autotuner (no GPU): candidate selection,
skipped candidates, the persisted cache and its key."""

import json

import pytest

import paper_1709_03636_gb300 as q
from paper_1709_03636_gb300 import tuning as at


class FakeEngine:
    device = 0

    def __init__(self):
        self.calls = []
        self.opts = None

    def set_graph_options(self, force_graph=False, small_rank=0):
        self.calls.append(("graph", force_graph, small_rank))
        self.sr = small_rank

    def set_task_options(self, task_terms_log2=16, subtree_bytes=32768, warp_teams=1,
                         graph_hi_occupancy=False):
        self.occ = graph_hi_occupancy
        self.calls.append(("task", task_terms_log2, subtree_bytes, warp_teams))
        self.opts = (self.sr, task_terms_log2, subtree_bytes)
        self.warp = warp_teams


class FakeBatch:
    def __init__(self, graph=True, edges=((0, 1), (1, 2)), p=2):
        self.edges = list(edges)
        self.p = p
        self.graph = graph
        self.prepared = []

    def stats(self):
        return {"n_networks": len(self.edges), "max_rank": 20, "n_steps_total": 300,
                "cmacs": 1e9, "bytes_c64": 2e9}

    def program_info(self, dtype, want_grad):
        return {"graph": int(self.graph)}

    def prepare(self, engine, dtype, want_grad=False):
        if engine.opts == (9, 15, 16384):
            raise q.QtcError(6, "arena too small")
        self.prepared.append(engine.opts)


def test_picks_fastest_skips_failures_and_caches(tmp_path):
    eng, batch = FakeEngine(), FakeBatch()
    times = {(sr, tt, sb): 10.0 + sr - 0.5 * tt + sb / 32768
             for sr in (9, 10, 11) for tt in (15, 16, 17, 18) for sb in (16384, 32768)}
    timer = lambda: times[eng.opts] + (0.1 if eng.occ else 0.0)  # noqa: E731
    path = tmp_path / "tune.json"
    res = at.autotune(eng, batch, "c64", True, cache_path=str(path), timer=timer,
                      device_name="GB300")
    assert (res["small_rank"], res["task_terms_log2"], res["subtree_bytes"]) == (9, 18, 16384)
    assert res["graph_hi_occupancy"] is False
    assert res["cached"] is False
    assert eng.opts == (9, 18, 16384)          # the choice is applied last
    failed = [t for t in res["trials"] if t["ms"] is None]
    assert len(failed) == 2 and "arena" in failed[0]["error"]   # on both kernel builds
    table = json.loads(path.read_text())
    assert len(table) == 1
    # a second call applies the cached choice without timing anything
    eng2 = FakeEngine()
    res2 = at.autotune(eng2, batch, "c64", True, cache_path=str(path),
                       timer=lambda: pytest.fail("timed a cached batch"), device_name="GB300")
    assert res2["cached"] is True and eng2.opts == (9, 18, 16384)


def test_signature_separates_dtype_gradient_device_and_structure():
    b = FakeBatch()
    keys = {at.signature(b, "c64", True, "GB300"), at.signature(b, "c128", True, "GB300"),
            at.signature(b, "c64", False, "GB300"), at.signature(b, "c64", True, "B200"),
            at.signature(FakeBatch(edges=((0, 2), (1, 2))), "c64", True, "GB300")}
    assert len(keys) == 5


def test_shared_memory_batches_choose_warp_or_cta_teams():
    eng = FakeEngine()
    res = at.autotune(eng, FakeBatch(graph=False), "c64", True,
                      timer=lambda: {0: 2.0, 1: 1.5, 2: 1.0}[eng.warp], device_name="GB300")
    assert res["graph"] is False and res["warp_teams"] == 2 and eng.warp == 2
    eng = FakeEngine()
    res = at.autotune(eng, FakeBatch(graph=False), "c128", True,
                      timer=lambda: 3.0 if eng.warp else 2.0, device_name="GB300")
    assert res["warp_teams"] == 0 and eng.warp == 0
    assert eng.opts == (at.DEFAULTS["small_rank"], at.DEFAULTS["task_terms_log2"],
                        at.DEFAULTS["subtree_bytes"])


def test_task_option_ranges_are_checked():
    lib = q.lib
    assert lib.qtc_engine_set_task_options(None, 16, 32768, 1, 0) != 0



def test_quick_candidates_as_the_bench_runs_them():
    """The bench's quick tuning: small_rank 9 and 10 x 2^16, 2^17, 2^18-term
    tasks, nothing else changed; with no cache file the fastest is applied
    and nothing is stored."""
    cands = at.quick_candidates()
    assert [(c["small_rank"], c["task_terms_log2"]) for c in cands] == [
        (9, 16), (9, 17), (9, 18), (10, 16), (10, 17), (10, 18)]
    for c in cands:
        assert {k: v for k, v in c.items() if k not in ("small_rank", "task_terms_log2")} == {
            k: v for k, v in at.DEFAULTS.items() if k not in ("small_rank", "task_terms_log2")}
    eng, batch = FakeEngine(), FakeBatch()
    times = {(sr, tt, 32768): 5.0 + 0.1 * sr - 0.2 * tt for sr in (9, 10) for tt in (16, 17, 18)}
    res = at.autotune(eng, batch, "c64", True, candidates=cands, timer=lambda: times[eng.opts],
                      device_name="GB300")
    assert (res["small_rank"], res["task_terms_log2"]) == (9, 18)
    assert eng.opts == (9, 18, 32768) and len(res["trials"]) == 6 and res["cached"] is False
