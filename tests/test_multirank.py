"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2):
each rank builds its own seeded problem (independent graphs, the same
network count), no data crosses ranks, and the job's rate uses the slowest
rank's time (element-wise maximum over ranks)."""

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
    w = bench.rank_workload(WORKLOADS["qaoa_p1_n12_d3"], rank)
    edges = w.graph()
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), lightcone=True, diag=True, ordering="lg")
    n_nets = batch.stats()["n_networks"]
    info = batch.program_info("c64", True)          # host-side program, no GPU
    ms = [1.0 + rank, 5.0 - rank, 2.0]               # this rank's step times
    got = bench.max_over_ranks(ms, "cpu")
    rate = bench.job_rate(world, n_nets, got[0] * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"seed": w.graph_seed, "edges": sorted(map(list, edges)), "n_nets": n_nets,
                   "smem": info["smem_bytes"], "max": got, "rate": rate}, f)


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert [x["seed"] for x in r] == [r[0]["seed"], r[0]["seed"] + 1]
    assert r[0]["edges"] != r[1]["edges"]              # independent problems
    assert r[0]["n_nets"] == r[1]["n_nets"] == 18      # same work per rank (weak scaling)
    assert r[0]["max"] == r[1]["max"] == [2.0, 5.0, 2.0]
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(2 * 18 / 2e-3)


def test_single_rank_is_the_identity(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.max_over_ranks([3.0, 1.0], "cpu") == [3.0, 1.0]
    assert bench.job_rate(1, 75, 12e-6) == pytest.approx(75 / 12e-6)
