"""Noisy QAOA on the GPU (Section 2's density-matrix form with Kraus
channels) against the density-matrix oracle.

A channel on every qubit after each layer's mixer makes each edge network a
density-matrix network: one rank-4 tensor per channel joins the ket and bra
wires.  The executors run these networks unchanged; the gradient flows
through the channels (constant tensors).  Bounds as for the pure circuits:
complex128 1e-11, complex64 2e-6 per edge and 1e-4 relative on the gradient
(the oracle's gradient is a central difference with h = 1e-4, itself good to
~1e-7 relative).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import density as dm  # noqa: E402
from synth import WORKLOADS, random_regular_graph  # noqa: E402

G2, B2 = [0.45, 1.05], [0.8, 0.35]


@pytest.fixture(scope="module")
def engine():
    return q.Engine(0, arena_bytes=4 << 30)


@pytest.mark.parametrize("channel", dm.CHANNELS)
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-6)])
def test_noisy_p2_value_and_gradient(engine, channel, dtype, tol):
    n, s = 8, 0.07
    edges = random_regular_graph(n, 3, 9)
    circ = q.Circuit.qaoa(n, edges, 2, noise=(channel, s))
    batch = q.Batch(circ, ordering="lg")
    C, per_edge, grad = q.qaoa_expectation(engine, batch, G2, B2, dtype, want_grad=True)
    ref = dm.edge_zz(n, edges, G2, B2, channel, s)
    assert np.max(np.abs(np.array(per_edge) - ref)) < tol
    assert abs(C - dm.maxcut(n, edges, G2, B2, channel, s)) < tol * len(edges)
    ref_g = dm.maxcut_grad(n, edges, G2, B2, channel, s)
    err = np.max(np.abs(np.array(grad) - ref_g)) / np.max(np.abs(ref_g))
    assert err < (1e-6 if dtype == "c128" else 1e-4), err


def test_noisy_full_networks_and_graph_executor(engine):
    """Un-reduced networks, and the light-cone ones forced through the graph
    executor (global-memory steps)."""
    n, s = 8, 0.11
    edges = random_regular_graph(n, 3, 2)
    circ = q.Circuit.qaoa(n, edges, 2, noise=("depolarize", s))
    ref = dm.edge_zz(n, edges, G2, B2, "depolarize", s)
    full = q.Batch(circ, lightcone=False, ordering="lg")
    _, per_edge, _ = q.qaoa_expectation(engine, full, G2, B2, "c128")
    assert np.max(np.abs(np.array(per_edge) - ref)) < 1e-11
    engine.set_graph_options(force_graph=True, small_rank=2)
    try:
        batch = q.Batch(circ, ordering="stoch")
        assert batch.program_info("c128", True, force_graph=True, small_rank=2)["graph"] == 1
        C, per_edge, grad = q.qaoa_expectation(engine, batch, G2, B2, "c128", want_grad=True)
    finally:
        engine.set_graph_options(False, 0)
    assert np.max(np.abs(np.array(per_edge) - ref)) < 1e-11
    ref_g = dm.maxcut_grad(n, edges, G2, B2, "depolarize", s)
    assert np.max(np.abs(np.array(grad) - ref_g)) < 1e-6 * np.max(np.abs(ref_g))


@pytest.mark.parametrize("channel", dm.CHANNELS)
def test_noisy_p1_n50_sampled_edges(engine, channel):
    """The 75-edge p=1 workload with noise: sampled edges against the
    light-cone density matrix (exact for trace-preserving channels)."""
    w = WORKLOADS["qaoa_p1_n50_d3"]
    edges = w.graph()
    g, b = w.angles()
    s = 0.03
    circ = q.Circuit.qaoa(w.n, edges, 1, noise=(channel, s))
    batch = q.Batch(circ, ordering="lg")
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    for i in (0, 11, 40, 74):
        ref = dm.edge_zz_lightcone(w.n, edges, g, b, edges[i], channel, s)
        assert abs(per_edge[i] - ref) < 2e-6
    # the gradient of one edge network alone, through the single-network call
    e = edges[11]
    one = q.Batch(circ, obs_edges=[e], ordering="lg")
    _, _, g1 = q.qaoa_expectation(engine, one, g, b, "c64", want_grad=True)
    ref_g = -0.5 * dm.edge_grad_lightcone(w.n, edges, g, b, e, channel, s)
    assert np.max(np.abs(np.array(g1) - ref_g)) < 1e-4 * max(np.max(np.abs(ref_g)), 1e-3)
