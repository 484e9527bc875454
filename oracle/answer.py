"""Section 3.3's answer-string estimate from an exact probability vector.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The heuristic fixes the qubits one at a time: with qubits 0..q-1 fixed to
their chosen values, it compares the probabilities of the prefix extended by
x_q = 0 and by x_q = 1 and keeps the larger (a tie is broken at random).
Here those prefix probabilities are plain sums of the exact distribution
p[x] (qubit q = bit q of x), e.g. p = |psi|^2 from ``statevector`` or the
diagonal of a density matrix from ``density``.
"""

from __future__ import annotations

import numpy as np


def sequential(p, n: int, rng=None):
    """(bits, prefix probabilities) of the sequential estimate over p
    (length 2^n, non-negative, summing to one)."""
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    if p.size != 1 << n:
        raise ValueError("p must have 2^n entries")
    rng = rng or np.random.default_rng(0)
    idx = np.arange(p.size)
    mask, pattern = 0, 0
    bits, probs = [], []
    prev = float(p.sum())
    for q in range(n):
        mask |= 1 << q
        p0 = float(p[(idx & mask) == pattern].sum())       # x_q = 0
        p1 = prev - p0
        if p0 > p1 or (p0 == p1 and rng.integers(2) == 0):
            b, prev = 0, p0
        else:
            b, prev = 1, p1
        pattern |= b << q
        bits.append(b)
        probs.append(prev)
    return bits, probs


def product_distribution(marginals):
    """p[x] = prod_q (1 - m_q if x_q = 0 else m_q) for P(x_q = 1) = m_q."""
    n = len(marginals)
    idx = np.arange(1 << n)
    p = np.ones(1 << n)
    for q, m in enumerate(marginals):
        p *= np.where((idx >> q) & 1, m, 1 - m)
    return p
