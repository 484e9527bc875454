"""O-SV: brute-force 2^n state-vector simulation of the QAOA Max-Cut circuit.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Circuit (Section 4.1, with the phase-gate sign of the workloads): start from
|+>^n (H on |0>^n), then for k = 1..p apply the cost layer
``prod_{(a,b) in E} exp(-i gamma_k Z_a Z_b / 2)`` followed by the mixer
``prod_q exp(-i beta_k X_q)`` (= RX(2 beta_k) on every qubit).  The objective
is Eqs. (maxcut objective) and (pairwise clause):
``C = sum_{(a,b)} (1 - Z_a Z_b) / 2``.

Qubit q is bit q of the basis index.  All arithmetic is complex128/float64.
"""

from __future__ import annotations

import numpy as np


def _axis(n: int, q: int) -> int:
    # C-order reshape to (2,)*n puts the most significant bit on axis 0
    return n - 1 - q


def _z(n: int, q: int) -> np.ndarray:
    """Broadcastable +1/-1 eigenvalue array of Z_q."""
    shape = [1] * n
    shape[_axis(n, q)] = 2
    return np.array([1, -1], dtype=np.int8).reshape(shape)


def zz_sum(n: int, edges) -> np.ndarray:
    """sum_{(a,b) in E} z_a(x) z_b(x) for every basis state x, shape (2,)*n."""
    acc = np.zeros((2,) * n, dtype=np.int16)
    for a, b in edges:
        acc = acc + (_z(n, a) * _z(n, b)).astype(np.int16)
    return acc


def _phase_layer(psi: np.ndarray, zz: np.ndarray, m: int, gamma: float) -> np.ndarray:
    # exp(-i gamma/2 * sum_e z_a z_b), looked up per distinct value of the sum
    table = np.exp(-0.5j * gamma * np.arange(-m, m + 1, dtype=np.float64))
    return psi * table[zz.astype(np.int32) + m]


def _mixer_layer(psi: np.ndarray, n: int, beta: float) -> np.ndarray:
    # exp(-i beta X) = cos(beta) I - i sin(beta) X on every qubit
    c, s = np.cos(beta), np.sin(beta)
    for q in range(n):
        psi = c * psi - 1j * s * np.flip(psi, axis=_axis(n, q))
    return psi


def qaoa_state(n: int, edges, gammas, betas) -> np.ndarray:
    """Final state |psi(gamma, beta)> as a (2,)*n complex128 array."""
    if len(gammas) != len(betas):
        raise ValueError("need as many gammas as betas")
    psi = np.full((2,) * n, 2.0 ** (-n / 2), dtype=np.complex128)
    zz = zz_sum(n, edges)
    m = len(edges)
    for g, b in zip(gammas, betas):
        psi = _phase_layer(psi, zz, m, g)
        psi = _mixer_layer(psi, n, b)
    return psi


def zz_expectations(psi: np.ndarray, edges) -> np.ndarray:
    """<Z_a Z_b> for every edge from the 2x2 marginal of |psi|^2."""
    n = psi.ndim
    prob = np.abs(psi) ** 2
    out = np.empty(len(edges))
    for i, (a, b) in enumerate(edges):
        keep = {_axis(n, a), _axis(n, b)}
        others = tuple(ax for ax in range(n) if ax not in keep)
        marg = prob.sum(axis=others)  # 2x2 over (bit of the lower axis, higher)
        out[i] = marg[0, 0] - marg[0, 1] - marg[1, 0] + marg[1, 1]
    return out


def maxcut_expectation(n: int, edges, gammas, betas) -> float:
    """<C> = sum_e (1 - <Z_a Z_b>) / 2."""
    psi = qaoa_state(n, edges, gammas, betas)
    zz = zz_expectations(psi, edges)
    return float(np.sum((1.0 - zz) / 2.0))


def edge_zz(n: int, edges, gammas, betas) -> np.ndarray:
    """Per-edge <Z_a Z_b> in the order of ``edges``."""
    return zz_expectations(qaoa_state(n, edges, gammas, betas), edges)


def identity_expectation(n: int, edges, gammas, betas) -> float:
    """<psi|psi> (unitarity: exactly 1 up to rounding)."""
    psi = qaoa_state(n, edges, gammas, betas)
    return float(np.vdot(psi, psi).real)


def amplitude(n: int, edges, gammas, betas, bits) -> complex:
    """<x|psi> for the basis state with qubit q set to bits[q]."""
    psi = qaoa_state(n, edges, gammas, betas)
    idx = tuple(int(bits[n - 1 - ax]) for ax in range(n))
    return complex(psi[idx])


def gradient(n: int, edges, gammas, betas, observable=None):
    """d<O>/d(gamma_1..p, beta_1..p) by the adjoint method.

    With psi = U_L ... U_1 |+>, each U_j = exp(-i theta_j G_j):
    d<O>/d theta_j = 2 Im <lambda_j| G_j |phi_j>, where phi_j is the state
    after U_j and lambda_j = (U_L ... U_{j+1})^dagger O psi.  Both are
    stepped backwards through U_j^dagger.  G is (1/2) sum_e Z_a Z_b for a cost
    layer and sum_q X_q for a mixer layer.

    ``observable`` is ``None`` for C = sum_e (1 - Z_a Z_b)/2, or an edge
    ``(a, b)`` for Z_a Z_b.  Returns (value, grad) with grad of length 2p
    ordered (gamma_1..gamma_p, beta_1..beta_p).
    """
    p = len(gammas)
    m = len(edges)
    zz = zz_sum(n, edges)
    psi = qaoa_state(n, edges, gammas, betas)
    if observable is None:
        odiag = (m - zz.astype(np.float64)) / 2.0
    else:
        a, b = observable
        odiag = (_z(n, a) * _z(n, b)).astype(np.float64) * np.ones((2,) * n)
    value = float(np.vdot(psi, odiag * psi).real)
    phi = psi
    lam = odiag * psi
    grad = np.zeros(2 * p)
    half_zz = 0.5 * zz.astype(np.float64)
    for k in reversed(range(p)):
        # mixer layer of step k: G = sum_q X_q
        gphi = np.zeros_like(phi)
        for q in range(n):
            gphi += np.flip(phi, axis=_axis(n, q))
        grad[p + k] = 2.0 * np.vdot(lam, gphi).imag
        phi = _mixer_layer(phi, n, -betas[k])
        lam = _mixer_layer(lam, n, -betas[k])
        # cost layer of step k: G = (1/2) sum_e Z_a Z_b
        grad[k] = 2.0 * np.vdot(lam, half_zz * phi).imag
        phi = _phase_layer(phi, zz, m, -gammas[k])
        lam = _phase_layer(lam, zz, m, -gammas[k])
    return value, grad
