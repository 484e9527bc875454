"""Parity of the CUDA path with the FP64 oracle (GB300).

Tolerances: complex128 runs agree to 1e-11 absolute; complex64 runs to
1e-5 relative on <C> (and 2e-6 absolute per edge, |<ZZ>| <= 1), gradients to
1e-4 relative (the error bounds the workloads state for FP32 accumulation).
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import closed_form as cf  # noqa: E402
from oracle import statevector as sv  # noqa: E402
from oracle import tensornet as tn  # noqa: E402
from synth import WORKLOADS, random_regular_graph  # noqa: E402

C_REL = 1e-5
G_REL = 1e-4


@pytest.fixture(scope="module")
def engine():
    return q.Engine(0, arena_bytes=1 << 30)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def _grad_close(got, want, rel=G_REL):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(np.max(np.abs(want)), 1e-12)
    assert np.max(np.abs(got - want)) <= rel * scale, (got, want)


def test_qaoa_p1_n12_complex128_matches_statevector(engine):
    w = WORKLOADS["qaoa_p1_n12_d3"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c128", want_grad=True)
    ref_zz = sv.edge_zz(w.n, edges, g, b)
    ref_C, ref_grad = sv.gradient(w.n, edges, g, b)
    assert np.max(np.abs(np.array(per_edge) - ref_zz)) < 1e-11
    assert abs(C - ref_C) < 1e-11
    assert np.max(np.abs(np.array(grad) - ref_grad)) < 1e-10


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_qaoa_p1_n50_matches_closed_form(engine, dtype):
    w = WORKLOADS["qaoa_p1_n50_d3"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, dtype, want_grad=True)
    ref = np.array([cf.zz_p1(g[0], b[0], *cf.edge_params(w.n, edges, e)) for e in edges])
    ref_C = cf.maxcut_p1(w.n, edges, g[0], b[0])
    ref_grad = cf.maxcut_p1_grad(w.n, edges, g[0], b[0])
    tol = 2e-6 if dtype == "c64" else 1e-12
    assert np.max(np.abs(np.array(per_edge) - ref)) < tol
    assert _rel(C, ref_C) < (C_REL if dtype == "c64" else 1e-12)
    _grad_close(grad, ref_grad, G_REL if dtype == "c64" else 1e-10)


def test_qaoa_p2_n100_batched_matches_oracle(engine):
    w = WORKLOADS["qaoa_p2_n100_d5"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, lightcone=True, diag=True, ordering="lg")
    assert batch.stats()["n_networks"] == 250
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    ref_C, ref_grad = tn.maxcut_grad(w.n, edges, g, b)
    ref = np.array([tn.edge_value(w.n, edges, g, b, e).real for e in edges])
    assert np.max(np.abs(np.array(per_edge) - ref)) < 2e-6
    assert _rel(C, ref_C) < C_REL
    _grad_close(grad, ref_grad)
    # the forward-only program (one warp per network, tensors up to rank 11)
    assert batch.program_info("c64", False)["warp_teams"] == 1
    C_f, per_edge_f, _ = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=False)
    assert np.max(np.abs(np.array(per_edge_f) - ref)) < 2e-6
    assert _rel(C_f, ref_C) < C_REL


def test_qaoa_dense_and_diagonal_forms_agree(engine):
    n = 16
    edges = random_regular_graph(n, 3, 21)
    g, b = [0.41, 1.3], [0.72, 0.18]
    circ = q.Circuit.qaoa(n, edges, 2)
    ref = sv.edge_zz(n, edges, g, b)
    for diag in (True, False):
        for ordering in ("lg", "stoch"):
            batch = q.Batch(circ, lightcone=True, diag=diag, ordering=ordering, seed=5)
            _, per_edge, _ = q.qaoa_expectation(engine, batch, g, b, "c128")
            assert np.max(np.abs(np.array(per_edge) - ref)) < 1e-11


def test_qaoa_p1_d7_lightcones(engine):
    w = WORKLOADS["qaoa_p1_n20_d7"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, 1)
    batch = q.Batch(circ, lightcone=True, diag=True, ordering="lg")
    C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    ref = np.array([cf.zz_p1(g[0], b[0], *cf.edge_params(w.n, edges, e)) for e in edges])
    assert np.max(np.abs(np.array(per_edge) - ref)) < 2e-6
    assert _rel(C, cf.maxcut_p1(w.n, edges, g[0], b[0])) < C_REL
    _grad_close(grad, cf.maxcut_p1_grad(w.n, edges, g[0], b[0]))


def test_single_network_contract_and_gradient(engine):
    n = 12
    edges = random_regular_graph(n, 3, 2)
    g, b = [0.9, 0.2], [0.3, 1.2]
    circ = q.Circuit.qaoa(n, edges, 2)
    e = edges[5]
    net = q.Network(circ, "zz", edge=e, lightcone=True, diag=True)
    plan = q.Plan(net, "lg")
    s_ref, ds_ref = tn.edge_value_grad(n, edges, g, b, e, lightcone=True)
    for dtype, tol in (("c128", 1e-11), ("c64", 5e-6)):
        s, ds = q.contract(engine, plan, g + b, dtype, want_grad=True)
        assert abs(s - s_ref) < tol
        assert np.max(np.abs(np.array(ds) - ds_ref)) < 50 * tol


def test_identity_and_amplitude_networks(engine):
    n = 10
    edges = random_regular_graph(n, 3, 8)
    g, b = [0.6, 1.1], [0.25, 0.8]
    circ = q.Circuit.qaoa(n, edges, 2)
    ident = q.Network(circ, "identity", lightcone=False)
    val = q.contract(engine, q.Plan(ident, "lg"), g + b, "c128")
    assert abs(val - 1) < 1e-12
    psi = sv.qaoa_state(n, edges, g, b)
    rng = np.random.default_rng(0)
    for _ in range(4):
        bits = rng.integers(0, 2, n).tolist()
        net = q.Network(circ, "amplitude", bits=bits, lightcone=False)
        amp = q.contract(engine, q.Plan(net, "stoch", seed=1), g + b, "c128")
        assert abs(amp - sv.amplitude(n, edges, g, b, bits)) < 1e-12
    assert abs(np.vdot(psi, psi) - 1) < 1e-12


def test_generic_circuit_pauli_on_gpu(engine):
    from test_host_plans import GENERIC, _full_unitary_reference
    n = 4
    params = [0.37, -1.1, 2.3]
    circ = q.Circuit(n, len(params))
    gates = []
    for i, (gname, qs) in enumerate(GENERIC):
        if gname in ("rx", "rz", "zz"):
            circ.add_gate(gname, qs, i % 3, 1.0, 0.1)
            gates.append((gname, qs, params[i % 3] + 0.1))
        else:
            circ.add_gate(gname, qs)
            gates.append((gname, qs, 0.0))
    for pauli in ("XYZI", "ZIIZ", "IYIX"):
        _, ref = _full_unitary_reference(n, gates, pauli)
        for diag in (True, False):
            net = q.Network(circ, "pauli", pauli=pauli, lightcone=True, diag=diag)
            val = q.contract(engine, q.Plan(net, "lg"), params, "c128")
            assert abs(val - ref) < 1e-12


def test_device_api_graph_capture_and_repeat(engine):
    w = WORKLOADS["qaoa_p1_n50_d3"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, 1)
    batch = q.Batch(circ, ordering="lg")
    C_host, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    params = torch.tensor(g + b, dtype=torch.float64, device="cuda")
    out = torch.zeros(2 + 2 + len(edges), dtype=torch.float64, device="cuda")
    batch.prepare(engine, "c64", want_grad=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        q.qaoa_expectation_device(engine, batch, params, out, "c64", want_grad=True)
    stream.synchronize()
    assert abs(out[0].item() - C_host) < 1e-12
    assert np.allclose(out[1:3].cpu().numpy(), grad, atol=1e-12)
    graph = torch.cuda.CUDAGraph()
    out2 = torch.zeros_like(out)
    with torch.cuda.graph(graph, stream=stream):
        q.qaoa_expectation_device(engine, batch, params, out2, "c64", want_grad=True,
                                  stream=stream)
    for _ in range(3):
        out2.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out2, out)


def test_autograd_function(engine):
    w = WORKLOADS["qaoa_p1_n50_d3"]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, 1)
    batch = q.Batch(circ, ordering="lg")
    theta = torch.tensor(g + b, dtype=torch.float64, requires_grad=True)
    C = q.QAOAExpectation.apply(theta, engine, batch, "c64")
    C.backward()
    ref = cf.maxcut_p1_grad(w.n, edges, g[0], b[0])
    _grad_close(theta.grad.numpy(), ref)
    assert _rel(C.item(), cf.maxcut_p1(w.n, edges, g[0], b[0])) < C_REL


def test_arena_too_small_reports_arena_error():
    small = q.Engine(0, arena_bytes=4096)
    edges = random_regular_graph(20, 3, 0)
    circ = q.Circuit.qaoa(20, edges, 2)
    batch = q.Batch(circ)
    with pytest.raises(q.QtcError, match="ARENA"):
        q.qaoa_expectation(small, batch, [0.1, 0.2], [0.3, 0.4], "c64")


def test_trivial_angles_give_half_the_edges(engine):
    edges = random_regular_graph(30, 3, 4)
    circ = q.Circuit.qaoa(30, edges, 2)
    batch = q.Batch(circ)
    C, per_edge, _ = q.qaoa_expectation(engine, batch, [0.0, 0.0], [0.4, 0.9], "c64")
    assert abs(C - len(edges) / 2) < 1e-6
    assert np.max(np.abs(per_edge)) < 1e-6


@pytest.mark.parametrize("diag", [True, False])
def test_cnot_heavy_circuit_sparse_and_dense(engine, diag):
    """A random 12-qubit circuit of H, RX, RZ and CNOT (sparse XOR CNOT
    tensors in diag mode, dense rank-4 otherwise), full network, against a
    state-vector reference."""
    from test_host_plans import build_generic, random_cnot_circuit, statevector_reference
    n = 12
    gates = random_cnot_circuit(n, 80, 3)
    circ = build_generic(n, gates)
    pauli = "ZIIXIIIIYIIZ"
    ref = statevector_reference(n, gates, pauli)
    net = q.Network(circ, "pauli", pauli=pauli, lightcone=False, diag=diag)
    plan = q.Plan(net, "lg", seed=1)
    assert abs(q.contract(engine, plan, [], "c128") - ref) < 1e-11
    assert abs(q.contract(engine, plan, [], "c64") - ref) < 2e-5


@pytest.mark.parametrize("name", ["qaoa_p1_n50_d3", "qaoa_p2_n100_d5"])
def test_warp_step_modes_agree(name):
    """The same complex64 batch with warp programs whose steps are staged in
    shared memory (default layout), streamed from global memory (forced), and
    on CTA teams: identical math, so results agree to rounding."""
    w = WORKLOADS[name]
    edges = w.graph()
    g, b = w.angles()
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), lightcone=True, diag=True, ordering="lg")
    eng = q.Engine(0, arena_bytes=256 << 20)
    res = {}
    for mode in (1, 2, 0):
        eng.set_task_options(16, 32768, mode)
        res[mode] = q.qaoa_expectation(eng, batch, g, b, "c64", want_grad=True)
    info = batch.program_info("c64", True)
    assert info["warp_teams"] == 1
    for mode in (2, 0):
        C, per_edge, grad = res[mode]
        assert _rel(C, res[1][0]) < 1e-6
        assert np.max(np.abs(np.array(per_edge) - np.array(res[1][1]))) < 2e-6
        _grad_close(grad, res[1][2])


@pytest.mark.parametrize("name", ["qaoa_p1_n50_d3", "qaoa_p2_n100_d5"])
def test_host_call_returns_published_results(engine, name):
    """The host-pointer call returns when the kernel's published sequence
    number arrives, not at stream idle: back-to-back calls with changing
    angles, alternated with the device-pointer call on a second stream, give
    the same per-edge values (bit for bit: same kernel, same inputs) and the
    same FP64 sums up to their summation order."""
    w = WORKLOADS[name]
    edges = w.graph()
    g0, b0 = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, ordering="lg")
    P = 2 * w.p
    params = torch.zeros(P, dtype=torch.float64, device="cuda")
    out = torch.zeros(2 + P + len(edges), dtype=torch.float64, device="cuda")
    batch.prepare(engine, "c64", want_grad=True)
    other = torch.cuda.Stream()
    rng = np.random.default_rng(11)
    for it in range(60):
        g = [x + 0.05 * rng.standard_normal() for x in g0]
        b = [x + 0.05 * rng.standard_normal() for x in b0]
        C_host, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
        params.copy_(torch.tensor(g + b, dtype=torch.float64))
        with torch.cuda.stream(other):
            other.wait_stream(torch.cuda.current_stream())
            q.qaoa_expectation_device(engine, batch, params, out, "c64", want_grad=True,
                                      stream=other)
        other.synchronize()
        ref = out.cpu().numpy()
        assert ref[1 + P + len(edges)] == 0.0
        assert np.array_equal(np.asarray(per_edge), ref[1 + P:1 + P + len(edges)]), it
        assert abs(C_host - ref[0]) <= 1e-12 * abs(ref[0]), it
        assert np.allclose(grad, ref[1:1 + P], rtol=1e-10, atol=1e-13), it
    # one more host call straight after a device call left in flight
    with torch.cuda.stream(other):
        q.qaoa_expectation_device(engine, batch, params, out, "c64", want_grad=True,
                                  stream=other)
    other.synchronize()
    C_last, _, _ = q.qaoa_expectation(engine, batch, g, b, "c64", want_grad=True)
    assert abs(C_last - out[0].item()) <= 1e-12 * abs(out[0].item())


def test_gate_table_parameters_above_slot_32(engine):
    """40 parameters, gates on slots 2 and 33-39 only (fewer than 32 gates):
    the warp gate table takes each gate's angle from the parameter held by
    lane slot - 32.  Value against a full state-vector reference, gradient
    against the complex128 run and against central differences."""
    from test_host_plans import GENERIC, _full_unitary_reference
    n, P = 4, 40
    rng = np.random.default_rng(5)
    params = list(rng.uniform(-2.0, 2.0, P))
    circ = q.Circuit(n, P)
    gates = []
    slots = [33, 2, 39, 35, 36, 37, 34, 38]
    for i, (gname, qs) in enumerate(GENERIC):
        if gname in ("rx", "rz", "zz"):
            k = slots[i % len(slots)]
            circ.add_gate(gname, qs, k, 0.8, 0.1)
            gates.append((gname, qs, 0.8 * params[k] + 0.1))
        else:
            circ.add_gate(gname, qs)
            gates.append((gname, qs, 0.0))
    _, ref = _full_unitary_reference(n, gates, "ZIIZ")
    plan = q.Plan(q.Network(circ, "pauli", pauli="ZIIZ", lightcone=True, diag=True), "lg")
    v64, g64 = q.contract(engine, plan, params, "c64", want_grad=True)
    v128, g128 = q.contract(engine, plan, params, "c128", want_grad=True)
    assert abs(v128 - ref) < 1e-12
    assert abs(v64 - ref) < 2e-6
    _grad_close([z.real for z in g64], [z.real for z in g128], rel=1e-4)
    h = 1e-5
    for k in (2, 33, 39, 0):
        pp, pm = list(params), list(params)
        pp[k] += h
        pm[k] -= h
        fd = (q.contract(engine, plan, pp, "c128") - q.contract(engine, plan, pm, "c128")) / (2 * h)
        assert abs(g128[k] - fd) < 1e-7, (k, g128[k], fd)


@pytest.mark.parametrize("name", ["qaoa_p1_n12_d3", "qaoa_p1_n50_d3"])
def test_sharded_parts_sum_to_the_whole_graph(engine, name):
    """The multi-GPU split run part by part on one GPU: the library's
    partition into 2 and 3 parts, each part's sub-batch evaluated on its own,
    and the parts' <C> and gradient added in FP64 equal the whole batch's
    (complex128, to rounding); the per-edge values are the same networks'."""
    w = WORKLOADS[name]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    full = q.Batch(circ, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
    C, per_edge, grad = q.qaoa_expectation(engine, full, g, b, "c128", want_grad=True)
    for world in (2, 3):
        tot_C, tot_g = 0.0, np.zeros(2 * w.p)
        seen = []
        for rank in range(world):
            sub, mine = q.shard(full, rank, world)
            c, pe, gr = q.qaoa_expectation(engine, sub, g, b, "c128", want_grad=True)
            tot_C += c
            tot_g += np.array(gr)
            assert np.max(np.abs(np.array(pe) - np.array(per_edge)[mine])) < 1e-13
            seen += mine
        assert sorted(seen) == list(range(len(edges)))
        assert abs(tot_C - C) < 1e-12
        assert np.max(np.abs(tot_g - np.array(grad))) < 1e-12
