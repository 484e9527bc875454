"""Split-BF16 tensor-core GEMM steps (tcgen05) against the oracle.

Dense (rank-4 ZZ) networks have GEMM-shaped steps; with the split-BF16
element type those run on the tensor cores with each FP32 operand split into
BF16 hi + lo and the products hi*hi + hi*lo + lo*hi accumulated in FP32.
Per-product relative error is about 2^-16, so the bound used here is the
workloads' 1e-5 relative on <C> and 1e-4 on the gradient.  The full-size
dense p=2 n=100 workload is checked edge by edge against the oracle in
test_gpu_workloads.py.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import statevector as sv  # noqa: E402
from synth import random_regular_graph  # noqa: E402


@pytest.fixture(scope="module")
def engine():
    return q.Engine(0, arena_bytes=4 << 30)


def test_split_bf16_gemm_steps_match_statevector(engine):
    n = 16
    edges = random_regular_graph(n, 3, 2)
    g, b = [0.45, 1.1], [0.7, 0.3]
    circ = q.Circuit.qaoa(n, edges, 2)
    batch = q.Batch(circ, lightcone=False, diag=False, ordering="lg")
    engine.set_graph_options(force_graph=True, small_rank=6)
    try:
        info = batch.program_info("split_bf16", True, force_graph=True, small_rank=6)
        assert info["n_gemm_steps"] > 0
        C, per_edge, grad = q.qaoa_expectation(engine, batch, g, b, "split_bf16",
                                               want_grad=True)
        C64, per_edge64, grad64 = q.qaoa_expectation(engine, batch, g, b, "c64",
                                                     want_grad=True)
    finally:
        engine.set_graph_options(False, 0)
    ref_C, ref_grad = sv.gradient(n, edges, g, b)
    ref = sv.edge_zz(n, edges, g, b)
    err_edge = np.max(np.abs(np.array(per_edge) - ref))
    err_C = abs(C - ref_C) / abs(ref_C)
    err_g = np.max(np.abs(np.array(grad) - ref_grad)) / np.max(np.abs(ref_grad))
    print(f"split-bf16: edge {err_edge:.2e}, <C> rel {err_C:.2e}, grad rel {err_g:.2e}; "
          f"c64: <C> rel {abs(C64 - ref_C) / abs(ref_C):.2e}")
    assert err_C < 1e-5
    assert err_edge < 1e-4
    assert err_g < 1e-4
