"""The on-GPU full-Hilbert-space reference against the FP64 oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import closed_form as cf  # noqa: E402
from oracle import statevector as sv  # noqa: E402
from synth import WORKLOADS, random_regular_graph  # noqa: E402


@pytest.fixture(scope="module")
def engine():
    return q.Engine(0, arena_bytes=2 << 30)


@pytest.mark.parametrize("n,d,p", [(5, 2, 1), (12, 3, 2), (13, 4, 3), (16, 5, 2)])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-6)])
def test_statevector_matches_oracle(engine, n, d, p, dtype, tol):
    edges = random_regular_graph(n, d, n + p) if d > 2 else [(i, (i + 1) % n) for i in range(n)]
    edges = [tuple(sorted(e)) for e in edges]
    g = [0.3 + 0.5 * k for k in range(p)]
    b = [1.1 - 0.3 * k for k in range(p)]
    circ = q.Circuit.qaoa(n, edges, p)
    C, per_edge = q.statevector_expectation(engine, circ, g, b, dtype, per_edge=True)
    assert abs(C - sv.maxcut_expectation(n, edges, g, b)) < tol * len(edges)
    assert np.max(np.abs(np.array(per_edge) - sv.edge_zz(n, edges, g, b))) < tol


@pytest.mark.parametrize("n,d,p", [(12, 3, 2), (13, 4, 2), (17, 4, 3), (19, 4, 2), (22, 3, 2)])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-6)])
def test_statevector_value_only_matches_oracle(engine, n, d, p, dtype, tol):
    """<C> alone (the last pass reduces the state without storing it), over
    one, two and three passes per layer, against the FP64 oracle."""
    edges = [tuple(sorted(e)) for e in random_regular_graph(n, d, 3 * n + p)]
    g = [0.45 + 0.4 * k for k in range(p)]
    b = [0.9 - 0.25 * k for k in range(p)]
    circ = q.Circuit.qaoa(n, edges, p)
    C, per_edge = q.statevector_expectation(engine, circ, g, b, dtype, per_edge=False)
    assert abs(C - sv.maxcut_expectation(n, edges, g, b)) < tol * len(edges)


@pytest.mark.parametrize("n,d", [(23, 6), (26, 7)])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-5)])
def test_statevector_value_only_p1_closed_form(n, d, dtype, tol):
    """Two and three passes of full tiles (the bench's crossover sizes),
    <C> alone, against the p=1 closed form."""
    edges = random_regular_graph(n, d, 0)
    g, b = [0.61], [0.37]
    eng = q.Engine(0, arena_bytes=(16 << n) + (256 << 20))
    C, _ = q.statevector_expectation(eng, q.Circuit.qaoa(n, edges, 1), g, b, dtype)
    assert abs(C - cf.maxcut_p1(n, edges, g[0], b[0])) < tol * abs(C)


def test_statevector_d7_n20_closed_form(engine):
    w = WORKLOADS["qaoa_p1_n20_d7"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, 1)
    C, per_edge = q.statevector_expectation(engine, circ, g, b, "c64", per_edge=True)
    ref = [cf.zz_p1(g[0], b[0], *cf.edge_params(w.n, edges, e)) for e in edges]
    assert np.max(np.abs(np.array(per_edge) - ref)) < 2e-6
    assert abs(C - cf.maxcut_p1(w.n, edges, g[0], b[0])) < 1e-5 * abs(C)


def test_statevector_device_form_and_tensor_network_agree(engine):
    n = 24
    edges = random_regular_graph(n, 7, 0)
    g, b = [0.6], [0.35]
    circ = q.Circuit.qaoa(n, edges, 1)
    params = torch.tensor(g + b, dtype=torch.float64, device="cuda")
    out = torch.zeros(1 + len(edges), dtype=torch.float64, device="cuda")
    q.statevector_expectation_device(engine, circ, params, out, "c64", per_edge=True)
    torch.cuda.synchronize()
    ref = cf.maxcut_p1(n, edges, g[0], b[0])
    assert abs(out[0].item() - ref) < 1e-5 * ref
    batch = q.Batch(circ, ordering="lg")
    C, per_edge, _ = q.qaoa_expectation(engine, batch, g, b, "c64")
    assert abs(C - out[0].item()) < 1e-5 * ref
    assert np.max(np.abs(np.array(per_edge) - out[1:].cpu().numpy())) < 4e-6
