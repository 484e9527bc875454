"""Pins of the answer-string oracle (Section 3.3).  CPU only.

* On a product distribution the sequential estimate is exact: it returns the
  most likely string (each qubit's more likely value), with the product of
  the chosen marginals as its probability.
* Its final prefix probability is the probability of the returned string
  itself, p[x], and of |<x|psi>|^2 from the state-vector oracle's amplitude.
* Each chosen prefix probability is at least half of the previous one.
"""

import numpy as np

from oracle import answer
from oracle import statevector as sv
from synth import random_regular_graph


def test_product_distribution_gives_the_most_likely_string():
    rng = np.random.default_rng(4)
    for _ in range(5):
        m = rng.uniform(0.05, 0.95, size=9)
        p = answer.product_distribution(m)
        bits, probs = answer.sequential(p, 9)
        assert bits == [int(x > 0.5) for x in m]
        assert int(np.argmax(p)) == sum(b << q for q, b in enumerate(bits))
        expect = np.cumprod([x if b else 1 - x for x, b in zip(m, bits)])
        assert np.allclose(probs, expect, rtol=1e-12, atol=0)


def test_final_probability_is_the_string_probability():
    n = 10
    edges = random_regular_graph(n, 3, 8)
    g, b = [0.61, 0.23], [0.44, 1.02]
    psi = sv.qaoa_state(n, edges, g, b)
    # qubit q is bit q of the index: reorder the C-order array (qubit 0 last axis)
    p = np.abs(psi.reshape(-1)) ** 2
    bits, probs = answer.sequential(p, n)
    x = sum(bt << q for q, bt in enumerate(bits))
    assert abs(probs[-1] - p[x]) < 1e-14
    assert abs(probs[-1] - abs(sv.amplitude(n, edges, g, b, bits)) ** 2) < 1e-12
    for a, c in zip([1.0] + probs[:-1], probs):
        assert c >= a / 2 - 1e-15
