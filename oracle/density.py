"""O-DM: density-matrix simulation of the QAOA Max-Cut circuit with noise.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 formulates circuits on density matrices (a gate acts as
rho -> U rho U^dagger on dimension-4 wires), which is what admits operations
that are not unitary.  A channel in Kraus form acts as
rho -> sum_k K_k rho K_k^dagger with sum_k K_k^dagger K_k = I.  The noisy
QAOA model used here is the Section 4.1 circuit (|+>^n, per layer the phase
exp(-i gamma Z_a Z_b / 2) on every edge and exp(-i beta X) on every qubit)
with one channel applied to every qubit after each layer's mixer.

Channels (strength s in [0, 1]):

* ``depolarize``: (1 - s) rho + s/3 (X rho X + Y rho Y + Z rho Z);
* ``dephase``:    (1 - s) rho + s Z rho Z;
* ``ampdamp``:    K0 = [[1, 0], [0, sqrt(1 - s)]], K1 = [[0, sqrt(s)], [0, 0]].

rho is a complex128 array of shape (2,)*2n: axes 0..n-1 are the row bits,
axes n..2n-1 the column bits, qubit q on row axis n-1-q (as in
``statevector``).  Everything is FP64 and plain numpy.
"""

from __future__ import annotations

import numpy as np

from .statevector import zz_sum

_I = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)

CHANNELS = ("depolarize", "dephase", "ampdamp")


def kraus(kind: str, s: float):
    """Kraus operators of a one-qubit channel of strength s."""
    if not 0.0 <= s <= 1.0:
        raise ValueError("channel strength must lie in [0, 1]")
    if kind == "depolarize":
        return [np.sqrt(1 - s) * _I, np.sqrt(s / 3) * _X, np.sqrt(s / 3) * _Y,
                np.sqrt(s / 3) * _Z]
    if kind == "dephase":
        return [np.sqrt(1 - s) * _I, np.sqrt(s) * _Z]
    if kind == "ampdamp":
        k0 = np.array([[1, 0], [0, np.sqrt(1 - s)]], dtype=np.complex128)
        k1 = np.array([[0, np.sqrt(s)], [0, 0]], dtype=np.complex128)
        return [k0, k1]
    raise ValueError(f"unknown channel {kind!r}")


def channel_superop(kind: str, s: float) -> np.ndarray:
    """The channel in the paper's dimension-4 vector order [rho_00, rho_01,
    rho_10, rho_11]: sum_k kron(K_k, conj(K_k)) (as Section 2 does for U)."""
    return sum(np.kron(k, np.conj(k)) for k in kraus(kind, s))


def _row(n: int, q: int) -> int:
    return n - 1 - q


def _col(n: int, q: int) -> int:
    return 2 * n - 1 - q


def apply_1q(rho: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    """rho -> U rho U^dagger on qubit q."""
    r = np.moveaxis(np.tensordot(u, rho, axes=([1], [_row(n, q)])), 0, _row(n, q))
    return np.moveaxis(np.tensordot(np.conj(u), r, axes=([1], [_col(n, q)])), 0, _col(n, q))


def apply_channel(rho: np.ndarray, n: int, q: int, ks) -> np.ndarray:
    """rho -> sum_k K_k rho K_k^dagger on qubit q."""
    return sum(apply_1q(rho, n, q, k) for k in ks)


def initial(n: int) -> np.ndarray:
    """|+><+| on every qubit: every entry 2^-n."""
    return np.full((2,) * (2 * n), 2.0 ** (-n), dtype=np.complex128)


def qaoa_rho(n: int, edges, gammas, betas, channel=None, strength: float = 0.0) -> np.ndarray:
    """Final density matrix of the noisy QAOA circuit (channel after every
    layer's mixer on every qubit; channel None = noiseless)."""
    if len(gammas) != len(betas):
        raise ValueError("need as many gammas as betas")
    rho = initial(n)
    m = len(edges)
    zz = zz_sum(n, edges).astype(np.int64)
    ks = kraus(channel, strength) if channel else None
    for gamma, beta in zip(gammas, betas):
        table = np.exp(-0.5j * gamma * np.arange(-m, m + 1, dtype=np.float64))
        ph = table[zz + m]
        rho = rho * ph.reshape(ph.shape + (1,) * n) * np.conj(ph).reshape((1,) * n + ph.shape)
        c, s = np.cos(beta), np.sin(beta)
        rx = np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
        for q in range(n):
            rho = apply_1q(rho, n, q, rx)
        if ks is not None:
            for q in range(n):
                rho = apply_channel(rho, n, q, ks)
    return rho


def _diag(rho: np.ndarray, n: int) -> np.ndarray:
    return np.real(np.diagonal(rho.reshape(2 ** n, 2 ** n))).reshape((2,) * n)


def edge_zz(n: int, edges, gammas, betas, channel=None, strength: float = 0.0) -> np.ndarray:
    """Tr(rho Z_a Z_b) for every edge."""
    d = _diag(qaoa_rho(n, edges, gammas, betas, channel, strength), n)
    out = []
    for a, b in edges:
        za = np.array([1, -1]).reshape([2 if ax == _row(n, a) else 1 for ax in range(n)])
        zb = np.array([1, -1]).reshape([2 if ax == _row(n, b) else 1 for ax in range(n)])
        out.append(float(np.sum(d * za * zb)))
    return np.array(out)


def maxcut(n: int, edges, gammas, betas, channel=None, strength: float = 0.0) -> float:
    """<C> = sum_e (1 - <Z_a Z_b>)/2 (Eqs. 9-10) under the noisy circuit."""
    return float(np.sum((1.0 - edge_zz(n, edges, gammas, betas, channel, strength)) / 2))


def maxcut_grad(n: int, edges, gammas, betas, channel=None, strength: float = 0.0,
                h: float = 1e-4) -> np.ndarray:
    """d<C>/d(gamma_1..p, beta_1..p) by central differences with step h."""
    x = np.array(list(gammas) + list(betas), dtype=np.float64)
    p = len(gammas)
    g = np.zeros_like(x)
    for i in range(len(x)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fp = maxcut(n, edges, xp[:p], xp[p:], channel, strength)
        fm = maxcut(n, edges, xm[:p], xm[p:], channel, strength)
        g[i] = (fp - fm) / (2 * h)
    return g


def edge_zz_lightcone(n: int, edges, gammas, betas, edge, channel=None, strength: float = 0.0,
                      max_qubits: int = 11) -> float:
    """<Z_u Z_v> for one edge from the density matrix of the radius-p ball
    around it (the induced subgraph, same channel placement).  Exact: a
    trace-preserving channel maps the identity to itself in the Heisenberg
    picture, so channels outside the reverse light cone drop out exactly as
    gates do (see ``lightcone``)."""
    from .lightcone import ball, induced
    u, v = edge
    verts = ball(n, edges, (u, v), len(gammas))
    if len(verts) > max_qubits:
        raise ValueError(f"light cone of {edge} has {len(verts)} qubits")
    sub, index = induced(edges, verts)
    k = sub.index((index[u], index[v])) if (index[u], index[v]) in sub else \
        sub.index((index[v], index[u]))
    return float(edge_zz(len(verts), sub, gammas, betas, channel, strength)[k])


def edge_grad_lightcone(n: int, edges, gammas, betas, edge, channel=None,
                        strength: float = 0.0, h: float = 1e-4) -> np.ndarray:
    """d<Z_u Z_v>/d(gamma_1..p, beta_1..p) by central differences of
    ``edge_zz_lightcone``."""
    x = np.array(list(gammas) + list(betas), dtype=np.float64)
    p = len(gammas)
    g = np.zeros_like(x)
    for i in range(len(x)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (edge_zz_lightcone(n, edges, xp[:p], xp[p:], edge, channel, strength)
                - edge_zz_lightcone(n, edges, xm[:p], xm[p:], edge, channel, strength)) / (2 * h)
    return g
