"""One graph's edge networks sharded over CPU ranks (gloo, world size 2).

The multi-GPU path splits the edge networks of one graph over the ranks by
the library's longest-processing-time partition (host only, the same on
every rank), evaluates each rank's part and adds the 1 + 2p partial sums
(<C> and its gradient) once in FP64.  Here the ranks are CPU processes: the
partition and the sub-batches come from the library (host side, no GPU),
each rank's partial sums come from the p = 1 closed form of its own edges
(the device evaluation itself needs a GPU; the GPU test of the same split
is in test_gpu_parity.py), and the exchange is the package's allreduce_sum
over gloo.  The sharded totals must equal the single-rank totals to
rounding.
"""

import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _partial_sums(w, edges, mine_edges):
    """<C> and d<C>/d(gamma, beta) summed over this rank's edges (p = 1)."""
    from oracle import closed_form as cf
    g, b = w.angles()
    C = dg = db = 0.0
    for e in mine_edges:
        par = cf.edge_params(w.n, edges, e)
        C += (1.0 - cf.zz_p1(g[0], b[0], *par)) / 2.0
        zg, zb = cf.zz_p1_grad(g[0], b[0], *par)
        dg -= 0.5 * zg
        db -= 0.5 * zb
    return [C, dg, db]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    import paper_1709_03636_gb300 as q
    from synth import WORKLOADS
    rec = {}
    for name in ("qaoa_p1_n12_d3", "qaoa_p1_n50_d3"):
        w = WORKLOADS[name]
        edges = w.graph()
        full = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), lightcone=w.lightcone, diag=w.diag,
                       ordering=w.ordering)
        parts, cost = full.partition(world, want_grad=True)
        sub, mine = q.shard(full, rank, world)
        info = sub.program_info("c64", True)            # host-side program, no GPU
        sums = q.allreduce_sum(_partial_sums(w, edges, [edges[i] for i in mine]))
        rec[name] = {"parts": parts, "cost": cost, "mine": mine,
                     "sub_edges": [list(e) for e in sub.edges],
                     "sub_bytes": sub.stats()["bytes_c64"], "smem": info["smem_bytes"],
                     "sums": sums.tolist()}
    ms = [1.0 + rank, 5.0 - rank, 2.0]               # this rank's step times
    got = bench.max_over_ranks(ms, "cpu")
    rec["max"] = got
    rec["rate"] = bench.job_rate(75, got[0] * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(rec, f)


def test_two_gloo_ranks_shard_one_graph(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import paper_1709_03636_gb300 as q
    from synth import WORKLOADS
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    for name in ("qaoa_p1_n12_d3", "qaoa_p1_n50_d3"):
        w = WORKLOADS[name]
        edges = w.graph()
        a, b = r[0][name], r[1][name]
        # the same partition on both ranks, computed without communication
        assert a["parts"] == b["parts"] and a["cost"] == b["cost"]
        # disjoint parts covering every edge network, each rank's sub-batch
        # holding exactly its edges
        assert sorted(a["mine"] + b["mine"]) == list(range(len(edges)))
        assert not set(a["mine"]) & set(b["mine"])
        for x in (a, b):
            assert [tuple(e) for e in x["sub_edges"]] == [edges[i] for i in x["mine"]]
        # longest processing time first: within 4/3 of the optimum, which is
        # at least the mean part and at least the costliest network
        full = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), lightcone=w.lightcone, diag=w.diag,
                       ordering=w.ordering)
        single = []
        for i in range(len(edges)):
            st = full.subset([i]).stats()
            single.append(st["bytes_c64"] + st["grad_bytes_c64"])
        assert sum(a["cost"]) == pytest.approx(sum(single))
        assert max(a["cost"]) <= 4.0 / 3.0 * max(sum(single) / world, max(single)) * (1 + 1e-12)
        assert a["sub_bytes"] + b["sub_bytes"] == pytest.approx(full.stats()["bytes_c64"])
        # the one exchange: the all-reduced partial sums equal the totals
        want = _partial_sums(w, edges, edges)
        for x in (a, b):
            assert x["sums"] == pytest.approx(want, rel=0, abs=1e-12)
    assert r[0]["max"] == r[1]["max"] == [2.0, 5.0, 2.0]
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(75 / 2e-3)


def test_partition_is_balanced_and_deterministic():
    sys.path.insert(0, ROOT)
    import paper_1709_03636_gb300 as q
    from synth import WORKLOADS
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    full = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), ordering="lg")
    for world in (2, 3, 8):
        parts, cost = full.partition(world, want_grad=True)
        again, _ = full.partition(world, want_grad=True)
        assert parts == again
        assert sorted(set(parts)) == list(range(world))
        # LPT bound: within 4/3 of the optimum, which is at least the mean
        # part and at least the costliest network
        top = max(full.subset([i]).stats()["bytes_c64"] + full.subset([i]).stats()[
            "grad_bytes_c64"] for i in range(len(edges)))
        assert max(cost) <= 4.0 / 3.0 * max(sum(cost) / world, top) * (1 + 1e-12)
    sub, mine = q.shard(full, 0, 1)
    assert sub is full and mine == list(range(len(edges)))


def test_single_rank_is_the_identity(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.max_over_ranks([3.0, 1.0], "cpu") == [3.0, 1.0]
    assert bench.job_rate(75, 12e-6) == pytest.approx(75 / 12e-6)
