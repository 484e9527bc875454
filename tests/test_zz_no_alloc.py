"""The evaluation entry point that allocates no device memory.

qtc_qaoa_expectation_static serves callers that cannot call cudaMalloc (and
so cannot give the library an arena): its scratch is a fixed device array
inside the library.  It must give what the arena-based
qtc_qaoa_expectation_device gives, call after call, and refuse batches that
do not fit its array.  This file is collected last on purpose; it passes
both alone in a fresh process and after the other tests.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from paper_1709_03636_gb300 import _lib  # noqa: E402
from synth import WORKLOADS, random_regular_graph  # noqa: E402

# tolerances of the parity tests: per edge 2e-6 absolute, <C> 1e-5 relative,
# gradient 1e-4 relative to its largest component (c64)
EDGE_TOL, C_REL, G_REL = 2e-6, 1e-5, 1e-4


def _static_call(batch, params, out, dtype, want_grad, stream):
    _lib.check(_lib.lib.qtc_qaoa_expectation_static(
        batch.ptr, ctypes.c_void_p(params.data_ptr()), q.DTYPES[dtype], int(want_grad),
        ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out.data_ptr())))


def _close(got, ref, p):
    got, ref = got.cpu().numpy(), ref.cpu().numpy()
    assert abs(got[0] - ref[0]) <= C_REL * abs(ref[0])
    g, rg = got[1:1 + 2 * p], ref[1:1 + 2 * p]
    assert np.max(np.abs(g - rg)) <= G_REL * max(np.max(np.abs(rg)), 1e-12)
    assert np.max(np.abs(got[1 + 2 * p:] - ref[1 + 2 * p:])) <= EDGE_TOL


@pytest.mark.parametrize("name,dtype", [("qaoa_p1_n50_d3", "c64"), ("qaoa_p1_n12_d3", "c128")])
def test_static_entry_point_matches_arena_entry_point(name, dtype):
    w = WORKLOADS[name]
    edges = w.graph()
    g, b = w.angles()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, lightcone=w.lightcone, diag=w.diag, ordering=w.ordering)
    engine = q.Engine(0, arena_bytes=64 << 20)
    stream = torch.cuda.current_stream()
    params = torch.tensor(g + b, dtype=torch.float64, device="cuda")
    ref = torch.zeros(2 + 2 * w.p + len(edges), dtype=torch.float64, device="cuda")
    q.qaoa_expectation_device(engine, batch, params, ref, dtype, want_grad=True)
    for _ in range(2):  # two calls in a row share the array
        out = torch.full_like(ref, float("nan"))
        _static_call(batch, params, out, dtype, True, stream)
        torch.cuda.synchronize()
        _close(out, ref, w.p)


def test_static_entry_point_switches_batches():
    n = 16
    edges = random_regular_graph(n, 3, 3)
    stream = torch.cuda.current_stream()
    engine = q.Engine(0, arena_bytes=64 << 20)
    runs = []
    for p in (1, 2):
        circ = q.Circuit.qaoa(n, edges, p)
        batch = q.Batch(circ, ordering="lg")
        params = torch.tensor([0.3 * (k + 1) for k in range(2 * p)], dtype=torch.float64,
                              device="cuda")
        ref = torch.zeros(2 + 2 * p + len(edges), dtype=torch.float64, device="cuda")
        q.qaoa_expectation_device(engine, batch, params, ref, "c64", want_grad=True)
        runs.append((batch, params, ref, p))
    for batch, params, ref, p in runs + runs:
        out = torch.full_like(ref, float("nan"))
        _static_call(batch, params, out, "c64", True, stream)
        torch.cuda.synchronize()
        _close(out, ref, p)


def test_static_entry_point_rejects_programs_that_do_not_fit():
    w = WORKLOADS["qaoa_p2_n100_d5"]
    edges = w.graph()
    circ = q.Circuit.qaoa(w.n, edges, w.p)
    batch = q.Batch(circ, obs_edges=edges * 3, ordering="lg")  # 750 networks
    params = torch.zeros(2 * w.p, dtype=torch.float64, device="cuda")
    out = torch.zeros(2 + 2 * w.p + 3 * len(edges), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QtcError, match="ARENA.*static scratch"):
        _static_call(batch, params, out, "c64", True, torch.cuda.current_stream())
