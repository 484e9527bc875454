"""Full-size workloads against the FP64 oracle, element by element.

These are the large cases of the five workloads, run in the launch
configuration the bench times (all edge networks of a graph in one batch):

* dense p=2 n=100 (250 networks) with split-BF16 tensor-core GEMM steps, every
  edge against the oracle's tensor-network contraction (O-TN);
* 7-regular p=1 n=24 and n=26 full un-reduced networks (intermediates of
  2^23-2^24 elements), every edge against the exact p=1 closed form;
* p=3 n=60 (120 networks, value and gradient): every edge's value against
  O-TN; the gradient of the 60+ edges whose oracle contraction stays at rank
  <= 24 (forward mode carries 6 tangents per tensor) against O-TN's, single
  edge networks' gradients against O-TN's and, on two edges, against central
  differences (h = 1e-4) of O-TN.

Tolerances are the workloads' stated bounds: 1e-5 relative on <C> and 1e-4
relative on the gradient; 2e-6 absolute per edge for complex64 (|<ZZ>| <= 1,
FP32 accumulation over a few hundred steps), 1e-4 per edge for split BF16
(three BF16 products, relative error per product about 2^-16).  The oracle
runs in worker processes started with spawn, so that no child inherits
the parent's CUDA context.
"""

import functools
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import closed_form as cf  # noqa: E402
from oracle import tensornet as tn  # noqa: E402
from synth import WORKLOADS  # noqa: E402

C_REL, G_REL, EDGE_C64, EDGE_BF16 = 1e-5, 1e-4, 2e-6, 1e-4


def _oracle_map(fn, items, gb_per_worker=16):
    """fn over items in spawned worker processes, as many as the host's cores
    and memory allow (the oracle's largest p=3 intermediates hold 2^28
    complex128 values)."""
    mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    workers = max(1, min(len(items), os.cpu_count() or 1, 16, int(mem // (gb_per_worker << 30))))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items))


def _oracle_rank(n, edges, g, b, e):
    fs, _ = tn.build_network(n, edges, g, b, e)
    return tn.max_elimination_rank(fs)


@pytest.fixture(scope="module")
def engine():
    return q.Engine(0, arena_bytes=12 << 30)


def test_split_bf16_dense_p2_n100_every_edge_vs_oracle(engine):
    w = WORKLOADS["qaoa_p2_n100_d5"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, lightcone=True, diag=False, ordering="lg")
    assert batch.program_info("split_bf16", False)["n_gemm_steps"] > 0
    ref = np.array([v.real for v in _oracle_map(
        functools.partial(tn.edge_value, w.n, edges, g, b), edges)])
    ref_C = float(np.sum((1.0 - ref) / 2.0))
    for dtype, tol in (("split_bf16", EDGE_BF16), ("c64", EDGE_C64)):
        C, per_edge, _ = q.qaoa_expectation(engine, batch, g, b, dtype)
        err = np.abs(np.array(per_edge) - ref)
        print(f"{dtype}: per-edge max {err.max():.2e} mean {err.mean():.2e}, "
              f"<C> rel {abs(C - ref_C) / abs(ref_C):.2e}")
        assert err.max() < tol
        assert abs(C - ref_C) <= C_REL * abs(ref_C)


@pytest.mark.parametrize("name", ["qaoa_p1_n24_d7", "qaoa_p1_n26_d7"])
def test_d7_full_networks_every_edge_vs_closed_form(engine, name):
    """Un-reduced networks (lightcone = False), the crossover form, whose
    largest intermediates have 2^23-2^24 elements."""
    w = WORKLOADS[name]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, 1)
    batch = q.Batch(circ, lightcone=False, ordering="lg")
    assert batch.stats()["max_rank"] >= 23
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    ref = np.array([cf.zz_p1(g[0], b[0], *cf.edge_params(w.n, edges, e)) for e in edges])
    ref_C = cf.maxcut_p1(w.n, edges, g[0], b[0])
    ref_grad = np.array(cf.maxcut_p1_grad(w.n, edges, g[0], b[0]))
    err = np.abs(np.array(per_edge) - ref)
    print(f"{name}: per-edge max {err.max():.2e}, <C> rel {abs(C - ref_C) / abs(ref_C):.2e}, "
          f"launches {engine.last_launches}")
    assert err.max() < EDGE_C64
    assert abs(C - ref_C) <= C_REL * abs(ref_C)
    assert np.max(np.abs(np.array(grad) - ref_grad)) <= G_REL * np.max(np.abs(ref_grad))


def test_p3_n60_every_edge_value_and_sampled_gradients(engine):
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, ordering="lg", restarts=w.restarts)   # as the bench plans it
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    ref = np.array([v.real for v in _oracle_map(
        functools.partial(tn.edge_value, w.n, edges, g, b), edges)])
    ref_C = float(np.sum((1.0 - ref) / 2.0))
    err = np.abs(np.array(per_edge) - ref)
    print(f"p3 n60: per-edge max {err.max():.2e}, <C> rel {abs(C - ref_C) / abs(ref_C):.2e}")
    assert err.max() < EDGE_C64
    assert abs(C - ref_C) <= C_REL * abs(ref_C)

    # d<C>/dtheta against the sum of O-TN's per-edge gradients (forward mode:
    # every tensor carries 6 tangents, so the edges whose oracle ordering
    # stays at rank <= 24 are taken, most of the graph) for the same networks
    # run as one batch
    light = [i for i, e in enumerate(edges) if _oracle_rank(w.n, edges, g, b, e) <= 24]
    assert len(light) >= 60
    ref_vg = dict(zip(light, _oracle_map(
        functools.partial(tn.edge_value_grad, w.n, edges, g, b), [edges[i] for i in light])))
    sub = batch.subset(light)
    _, _, gs = q.qaoa_expectation(engine, sub, g, b, "c64", want_grad=True)
    want = -0.5 * np.real(sum(ref_vg[i][1] for i in light))
    assert np.max(np.abs(np.array(gs) - want)) <= G_REL * np.max(np.abs(want)), (gs, want)

    # single edge networks: their gradient against O-TN's, and on two edges
    # against central differences of O-TN's value
    sample = light[::max(1, len(light) // 6)][:6]
    fd = _oracle_map(functools.partial(tn.edge_grad_fd, w.n, edges, g, b),
                     [edges[i] for i in sample[:2]])
    for k, i in enumerate(sample):
        _, _, g1 = q.qaoa_expectation(engine, batch.subset([i]), g, b, "c64", want_grad=True)
        want = -0.5 * np.real(ref_vg[i][1])
        scale = max(np.max(np.abs(want)), 1e-3)
        assert np.max(np.abs(np.array(g1) - want)) <= G_REL * scale, (i, g1, want)
        if k < 2:
            want_fd = -0.5 * fd[k]
            assert np.max(np.abs(np.array(g1) - want_fd)) <= G_REL * scale, (i, g1, want_fd)
            # the oracle's two gradients agree to the differences' O(h^2) error
            assert np.max(np.abs(want_fd - want)) <= 1e-7 * scale
