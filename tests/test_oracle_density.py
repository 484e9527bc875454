"""Pins of the density-matrix oracle (noisy QAOA; Section 2's density-matrix
form with Kraus channels).  CPU only.

Each check is against something other than the oracle itself:

* no noise -> the pure-state oracle (itself pinned by matrix exponentials);
* depolarizing after the last mixer scales every <Z_a Z_b> by (1 - 4s/3)^2
  (the channel maps Z to (1 - 4s/3) Z);
* dephasing after the last mixer leaves every <Z_a Z_b> unchanged (it maps Z
  to Z); full amplitude damping there leaves |0..0>, so <Z_a Z_b> = 1;
* trace one, hermiticity and positivity of the noisy state; Kraus
  completeness;
* the paper's own dimension-4 superoperator network (Section 2 tensors,
  contracted by variable elimination) with the channel's superoperator
  sum_k kron(K, conj K), on a two-qubit circuit;
* a planted mistake (K rho K instead of K rho K^dagger) breaks a pin;
* the radius-p light-cone density matrix against the full one.
"""

import numpy as np
import pytest

from oracle import density as dm
from oracle import statevector as sv
from oracle import superop as so
from synth import random_regular_graph

G, B = [0.63, 1.1], [0.41, 0.27]


@pytest.mark.parametrize("kind", dm.CHANNELS)
@pytest.mark.parametrize("s", [0.0, 0.05, 0.5, 1.0])
def test_kraus_completeness(kind, s):
    ks = dm.kraus(kind, s)
    total = sum(k.conj().T @ k for k in ks)
    assert np.allclose(total, np.eye(2), atol=1e-14)


def test_noiseless_matches_pure_state():
    n = 8
    edges = random_regular_graph(n, 3, 5)
    for kind in dm.CHANNELS:
        got = dm.edge_zz(n, edges, G, B, kind, 0.0)
        assert np.max(np.abs(got - sv.edge_zz(n, edges, G, B))) < 1e-12


@pytest.mark.parametrize("s", [0.02, 0.3])
def test_depolarizing_at_the_end_scales_zz(s):
    n = 8
    edges = random_regular_graph(n, 3, 7)
    clean = sv.edge_zz(n, edges, G[:1], B[:1])
    noisy = dm.edge_zz(n, edges, G[:1], B[:1], "depolarize", s)
    assert np.max(np.abs(noisy - (1 - 4 * s / 3) ** 2 * clean)) < 1e-12


def test_dephasing_and_full_damping_at_the_end():
    n = 6
    edges = random_regular_graph(n, 3, 2)
    clean = sv.edge_zz(n, edges, G[:1], B[:1])
    assert np.max(np.abs(dm.edge_zz(n, edges, G[:1], B[:1], "dephase", 0.37) - clean)) < 1e-12
    assert np.max(np.abs(dm.edge_zz(n, edges, G[:1], B[:1], "ampdamp", 1.0) - 1.0)) < 1e-12


@pytest.mark.parametrize("kind", dm.CHANNELS)
def test_noisy_state_is_a_density_matrix(kind):
    n = 6
    edges = random_regular_graph(n, 3, 3)
    rho = dm.qaoa_rho(n, edges, G, B, kind, 0.2).reshape(2 ** n, 2 ** n)
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-13
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12
    # noise lowers the purity below one
    assert np.real(np.trace(rho @ rho)) < 1 - 1e-3


@pytest.mark.parametrize("kind", dm.CHANNELS)
def test_paper_superoperator_network_with_channel(kind):
    """Two qubits, p = 2, channel after each mixer: the Section 2 network of
    kron(U, conj U) gate tensors and sum_k kron(K, conj K) channel tensors,
    closed by M_Z (x) M_Z, against the Kraus-form density matrix."""
    s = 0.23
    h = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    gates = [(so.superop_1q(h), (0,)), (so.superop_1q(h), (1,))]
    for gamma, beta in zip(G, B):
        zz = np.diag(np.exp(-0.5j * gamma * np.array([1, -1, -1, 1])))
        gates.append((so.superop_2q(zz), (0, 1)))
        c, sn = np.cos(beta), np.sin(beta)
        rx = np.array([[c, -1j * sn], [-1j * sn, c]])
        for q in (0, 1):
            gates.append((so.superop_1q(rx), (q,)))
        for q in (0, 1):
            gates.append((dm.channel_superop(kind, s), (q,)))
    value = so.expectation(2, gates, [so.measurement("Z"), so.measurement("Z")])
    ref = dm.edge_zz(2, [(0, 1)], G, B, kind, s)[0]
    assert abs(value.imag) < 1e-13
    assert abs(value.real - ref) < 1e-12


def test_gradient_matches_noiseless_adjoint_at_zero_noise():
    n = 6
    edges = random_regular_graph(n, 3, 4)
    g = dm.maxcut_grad(n, edges, G, B, "depolarize", 0.0)
    _, ref = sv.gradient(n, edges, G, B)
    # central differences with h = 1e-4: truncation error of order h^2
    assert np.max(np.abs(g - ref)) < 1e-6 * np.max(np.abs(ref))


def test_planted_mistake_is_caught():
    """K rho K instead of K rho K^dagger breaks the trace pin for a channel
    with a non-Hermitian Kraus operator (amplitude damping's K1)."""
    n = 4
    edges = random_regular_graph(n, 3, 1)
    rho = dm.qaoa_rho(n, edges, G[:1], B[:1]).copy()
    ks = dm.kraus("ampdamp", 0.4)

    def wrong(r, q):
        out = 0
        for k in ks:
            a = np.moveaxis(np.tensordot(k, r, axes=([1], [n - 1 - q])), 0, n - 1 - q)
            # right-multiplication by K: (a K)[.., j] = sum_l a[.., l] K[l, j]
            out = out + np.moveaxis(np.tensordot(k, a, axes=([0], [2 * n - 1 - q])), 0,
                                    2 * n - 1 - q)
        return out

    bad = wrong(rho, 0).reshape(2 ** n, 2 ** n)
    good = dm.apply_channel(rho, n, 0, ks).reshape(2 ** n, 2 ** n)
    assert abs(np.trace(good) - 1) < 1e-12
    assert abs(np.trace(bad) - 1) > 1e-3


@pytest.mark.parametrize("kind", dm.CHANNELS)
def test_lightcone_density_matches_full(kind):
    """The radius-p ball (p = 1 and 2) against the full density matrix."""
    n = 10
    edges = random_regular_graph(n, 3, 6)
    for p in (1, 2):
        full = dm.edge_zz(n, edges, G[:p], B[:p], kind, 0.15)
        for i in (0, 4, 9):
            got = dm.edge_zz_lightcone(n, edges, G[:p], B[:p], edges[i], kind, 0.15)
            assert abs(got - full[i]) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_lightcone_fd_gradient_matches_adjoint_at_zero_noise(p):
    """The light-cone central-difference gradient (the density oracle's only
    gradient per edge) against the state-vector adjoint on the same ball
    with no noise, and at p = 1 against the closed form's derivatives.  A
    wrong divisor (h instead of 2h), a swapped sign or a parameter slot
    mix-up would each miss these by far more than the O(h^2) truncation."""
    from oracle import closed_form as cf
    from oracle import lightcone as lc
    n = 10
    edges = random_regular_graph(n, 3, 8)
    for i in (0, 5, 13):
        e = edges[i]
        got = dm.edge_grad_lightcone(n, edges, G[:p], B[:p], e, "dephase", 0.0)
        _, ref = lc.edge_gradient(n, edges, G[:p], B[:p], e)
        assert np.max(np.abs(got - np.asarray(ref))) < 1e-7 * max(np.max(np.abs(ref)), 1.0)
        if p == 1:
            dg, db = cf.zz_p1_grad(G[0], B[0], *cf.edge_params(n, edges, e))
            assert abs(got[0] - dg) < 1e-7 and abs(got[1] - db) < 1e-7
