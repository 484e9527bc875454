"""QAOA angle optimisation driven by the adjoint gradient (Section 4.1's
outer loop) against the p=1 closed form.

For p = 1 <C>(gamma, beta) has a closed form (pinned in the oracle tests);
its maximum over (gamma, beta), found on the CPU by scipy from a grid of
starts, is the value the GPU-driven optimiser must reach.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_opt = pytest.importorskip("scipy.optimize")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_1709_03636_gb300 as q  # noqa: E402
from oracle import closed_form as cf  # noqa: E402
from synth import WORKLOADS  # noqa: E402


def closed_form_maximum(n, edges):
    f = lambda x: -cf.maxcut_p1(n, edges, x[0], x[1])  # noqa: E731
    best = None
    for g0 in np.linspace(0.1, 3.0, 7):
        for b0 in np.linspace(0.1, 1.5, 5):
            r = scipy_opt.minimize(f, [g0, b0], method="Nelder-Mead",
                                   options={"xatol": 1e-10, "fatol": 1e-12, "maxiter": 4000})
            if best is None or r.fun < best.fun:
                best = r
    return -best.fun, best.x


def test_adam_on_adjoint_gradient_reaches_the_p1_optimum():
    w = WORKLOADS["qaoa_p1_n50_d3"]
    edges = w.graph()
    engine = q.Engine(0, arena_bytes=256 << 20)
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, 1), ordering="lg")
    c_max, x_max = closed_form_maximum(w.n, edges)
    best, g, b, hist = q.optimize_angles(engine, batch, [0.3], [0.3], steps=400, lr=0.03)
    assert hist[-1] > hist[0]
    # complex64 contractions: <C> good to ~1e-6 relative
    assert abs(best - c_max) < 2e-5 * c_max, (best, c_max, g, b, x_max)
    # the oracle agrees at the optimiser's point, and its gradient vanishes there
    assert abs(cf.maxcut_p1(w.n, edges, g[0], b[0]) - best) < 1e-5 * c_max
    grad = np.array(cf.maxcut_p1_grad(w.n, edges, g[0], b[0]))
    assert np.max(np.abs(grad)) < 2e-2
