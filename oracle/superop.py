"""The paper's dimension-4 superoperator network form (Section 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 represents a density matrix rho by the 4-vector
[rho_00, rho_01, rho_10, rho_11], a gate U by the superoperator that maps
rho to U rho U^dagger, initial states and measurements by rank-1 tensors, and
joins them on dimension-4 wires.  With that vector order the superoperator of
a one-qubit gate is U (x) conj(U): entry ((i,j),(k,l)) = U_ik conj(U_jl).
A two-qubit gate is the rank-4 tensor indexed
[control_out, target_out, control_in, target_in], each index a (row, column)
pair of that qubit's density matrix.

The functions below build those tensors and a closed density-matrix network
for a small circuit; it is contracted with the same variable elimination as
O-TN (dimension-agnostic).
"""

from __future__ import annotations

import numpy as np

from .tensornet import Factor, contract

RHO0 = np.array([1.0, 0.0, 0.0, 0.0])


def superop_1q(u):
    """4x4 superoperator of a 2x2 unitary: kron(U, conj(U))."""
    u = np.asarray(u, dtype=np.complex128)
    return np.kron(u, np.conj(u))


def superop_2q(u4):
    """Rank-4 (4,4,4,4) superoperator [c_out, t_out, c_in, t_in] of a 4x4 gate.

    ``u4`` acts on the basis |c t> with index 2*c + t.
    """
    u = np.asarray(u4, dtype=np.complex128).reshape(2, 2, 2, 2)  # [ic, it, kc, kt]
    s = np.einsum("abcd,efgh->aebfcgdh", u, np.conj(u))
    # axes now (ic, jc, it, jt, kc, lc, kt, lt)
    return s.reshape(4, 4, 4, 4)


def measurement(kind):
    """Rank-1 measurement tensors M_Trace, M_X, M_Y, M_Z: entry (i,j) = P_ji."""
    paulis = {
        "I": np.eye(2),
        "X": np.array([[0, 1], [1, 0]]),
        "Y": np.array([[0, -1j], [1j, 0]]),
        "Z": np.array([[1, 0], [0, -1]]),
    }
    p = np.asarray(paulis[kind], dtype=np.complex128)
    return p.T.reshape(4)  # Tr(P rho) = sum_ij P_ji rho_ij


def density_network(n, gates, meas, rho0=RHO0):
    """Closed network of Tr(M rho_out) for a circuit on n qubits.

    gates: list of (tensor, qubits); a one-qubit tensor is [out, in] (4x4), a
    two-qubit tensor is [c_out, t_out, c_in, t_in].  meas: one rank-1
    measurement vector per qubit.
    """
    label = [0]

    def new():
        label[0] += 1
        return label[0] - 1

    cur = {}
    fs = []
    for q in range(n):
        cur[q] = new()
        fs.append(Factor(rho0, (cur[q],)))
    for tensor, qs in gates:
        outs = [new() for _ in qs]
        fs.append(Factor(tensor, tuple(outs) + tuple(cur[q] for q in qs)))
        for q, o in zip(qs, outs):
            cur[q] = o
    for q in range(n):
        fs.append(Factor(meas[q], (cur[q],)))
    return fs


def expectation(n, gates, meas, rho0=RHO0):
    value, _ = contract(density_network(n, gates, meas, rho0))
    return value
