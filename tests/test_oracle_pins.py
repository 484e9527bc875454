"""Pins of the FP64 oracle against things other than itself (CPU only).

* the state vector against scipy's matrix exponential of the full circuit;
* the p=1 closed form and its worked value;
* invariants (unitarity, bounds, symmetries, trivial angles);
* brute force: light cone and tensor network against the full state vector;
* gradients against central finite differences;
* the paper's printed superoperator tables against kron(U, conj(U)).
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import closed_form as cf
from oracle import lightcone as lc
from oracle import statevector as sv
from oracle import superop as so
from oracle import tensornet as tn
from synth import random_regular_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

K4 = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
# 7 vertices, degrees 2..4, several triangles
TRI7 = [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5), (4, 6), (5, 6), (0, 6)]


def _full_matrices(n, edges):
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    z = np.diag([1.0, -1.0]).astype(complex)
    eye = np.eye(2, dtype=complex)

    def op(single, q):
        # qubit q is bit q of the index: kron order puts qubit n-1 first
        mats = [single if k == q else eye for k in reversed(range(n))]
        out = mats[0]
        for m in mats[1:]:
            out = np.kron(out, m)
        return out

    zz = sum(op(z, a) @ op(z, b) for a, b in edges)
    bsum = sum(op(x, q) for q in range(n))
    return zz, bsum, op


@pytest.mark.parametrize("n,edges,gammas,betas", [
    (4, K4, [0.31], [1.2]),
    (5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 2)], [0.7, -0.4], [0.4, 0.9]),
    (6, random_regular_graph(6, 3, 3), [1.1, 0.2, 2.0], [0.3, 0.8, 1.4]),
])
def test_statevector_matches_matrix_exponential(n, edges, gammas, betas):
    zz, bsum, op = _full_matrices(n, edges)
    psi = np.full(2 ** n, 2 ** (-n / 2), dtype=complex)
    for g, b in zip(gammas, betas):
        psi = scipy.linalg.expm(-0.5j * g * zz) @ psi
        psi = scipy.linalg.expm(-1j * b * bsum) @ psi
    ours = sv.qaoa_state(n, edges, gammas, betas).reshape(-1)
    assert np.allclose(ours, psi, atol=1e-12)
    z = np.diag([1.0, -1.0]).astype(complex)
    for i, (a, b) in enumerate(edges):
        ref = np.vdot(psi, op(z, a) @ op(z, b) @ psi).real
        assert abs(sv.zz_expectations(ours.reshape((2,) * n), edges)[i] - ref) < 1e-12


@pytest.mark.parametrize("n,edges", [
    (4, K4), (7, TRI7), (10, random_regular_graph(10, 3, 0)),
    (12, random_regular_graph(12, 4, 1)),
])
@pytest.mark.parametrize("gamma,beta", [(0.7, 0.4), (2.3, 1.1), (-0.9, 0.25)])
def test_closed_form_matches_statevector(n, edges, gamma, beta):
    zz = sv.edge_zz(n, edges, [gamma], [beta])
    for i, e in enumerate(edges):
        assert abs(cf.zz_p1(gamma, beta, *cf.edge_params(n, edges, e)) - zz[i]) < 1e-12


def test_worked_value():
    with open(os.path.join(GOLDEN, "p1_worked_value.json")) as f:
        gold = json.load(f)
    val = cf.zz_p1(gold["gamma"], gold["beta"], gold["degree"], gold["degree"],
                   gold["triangles"])
    assert abs(val - gold["zz"]) < gold["abs_tol"]
    assert abs((1 - val) / 2 - gold["c_edge"]) < gold["abs_tol"]
    # the same number from brute force on a triangle-free 3-regular graph
    edges = random_regular_graph(12, 3, 0)
    zz = sv.edge_zz(12, edges, [gold["gamma"]], [gold["beta"]])
    tri_free = [i for i, e in enumerate(edges) if cf.edge_params(12, edges, e)[2] == 0]
    assert tri_free
    for i in tri_free:
        assert abs(zz[i] - gold["zz"]) < gold["abs_tol"]


def test_closed_form_gradient_matches_adjoint():
    edges = TRI7
    for gamma, beta in [(0.7, 0.4), (2.3, 1.1)]:
        _, grad = sv.gradient(7, edges, [gamma], [beta])
        g, b = cf.maxcut_p1_grad(7, edges, gamma, beta)
        assert abs(grad[0] - g) < 1e-11 and abs(grad[1] - b) < 1e-11


@pytest.mark.parametrize("p", [1, 2, 3])
def test_adjoint_gradient_matches_finite_differences(p):
    n = 8
    edges = random_regular_graph(n, 3, p)
    rng = np.random.default_rng(p)
    gammas = list(rng.uniform(0, math.pi, p))
    betas = list(rng.uniform(0, math.pi / 2, p))
    _, grad = sv.gradient(n, edges, gammas, betas)
    h = 1e-5
    theta = gammas + betas
    for i in range(2 * p):
        tp, tm = list(theta), list(theta)
        tp[i] += h
        tm[i] -= h
        fd = (sv.maxcut_expectation(n, edges, tp[:p], tp[p:])
              - sv.maxcut_expectation(n, edges, tm[:p], tm[p:])) / (2 * h)
        assert abs(fd - grad[i]) < 1e-7


def test_invariants():
    n = 10
    edges = random_regular_graph(n, 3, 7)
    g, b = [0.8, 1.9], [0.3, 1.0]
    base = sv.edge_zz(n, edges, g, b)
    assert np.all(np.abs(base) <= 1 + 1e-12)
    assert abs(sv.identity_expectation(n, edges, g, b) - 1) < 1e-12
    neg = sv.edge_zz(n, edges, [-x for x in g], [-x for x in b])
    shift_b = sv.edge_zz(n, edges, g, [x + math.pi / 2 for x in b])
    shift_g = sv.edge_zz(n, edges, [x + 2 * math.pi for x in g], b)
    assert np.allclose(base, neg, atol=1e-12)
    assert np.allclose(base, shift_b, atol=1e-12)
    assert np.allclose(base, shift_g, atol=1e-12)
    for gg, bb in [([0.0, 0.0], b), (g, [0.0, 0.0])]:
        assert np.allclose(sv.edge_zz(n, edges, gg, bb), 0.0, atol=1e-12)
        assert abs(sv.maxcut_expectation(n, edges, gg, bb) - len(edges) / 2) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("form", [dict(), dict(dense=True), dict(lightcone=False),
                                  dict(dense=True, lightcone=False, hadamard=True)])
def test_tensor_network_matches_statevector(p, form):
    n = 10
    edges = random_regular_graph(n, 3, 11 + p)
    gammas = [0.45 * (k + 1) for k in range(p)]
    betas = [0.35 / (k + 1) for k in range(p)]
    ref = sv.edge_zz(n, edges, gammas, betas)
    for i, e in enumerate(edges):
        s = tn.edge_value(n, edges, gammas, betas, e, **form)
        assert abs(s.real - ref[i]) < 1e-12
        assert abs(s.imag) < 1e-12
    assert abs(tn.identity_value(n, edges, gammas, betas, **form) - 1) < 1e-12


def test_lightcone_matches_full_statevector():
    n = 14
    edges = random_regular_graph(n, 3, 5)
    g, b = [0.6, 1.3], [0.7, 0.2]
    ref = sv.edge_zz(n, edges, g, b)
    got = lc.all_edges_zz(n, edges, g, b)
    assert np.allclose(got, ref, atol=1e-12)


def test_tensor_network_gradient_matches_adjoint():
    n = 9
    edges = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7),
             (7, 8), (8, 0), (1, 5), (3, 7)]
    g, b = [0.5, 1.7, 0.2], [0.9, 0.1, 0.6]
    val, grad = sv.gradient(n, edges, g, b)
    tval, tgrad = tn.maxcut_grad(n, edges, g, b)
    assert abs(val - tval) < 1e-11
    assert np.allclose(grad, tgrad, atol=1e-10)
    for e in edges[:3]:
        v1, g1 = lc.edge_gradient(n, edges, g, b, e)
        s, ds = tn.edge_value_grad(n, edges, g, b, e)
        assert abs(v1 - s.real) < 1e-12
        assert np.allclose(g1, ds.real, atol=1e-11)


def test_amplitudes_match_and_normalise():
    n = 6
    edges = random_regular_graph(n, 3, 2)
    g, b = [0.9, 0.3], [0.2, 1.1]
    total = 0.0
    for x in range(2 ** n):
        bits = [(x >> q) & 1 for q in range(n)]
        a_tn = tn.amplitude(n, edges, g, b, bits)
        a_sv = sv.amplitude(n, edges, g, b, bits)
        assert abs(a_tn - a_sv) < 1e-13
        total += abs(a_tn) ** 2
    assert abs(total - 1.0) < 1e-12


def test_contraction_order_independence():
    n = 12
    edges = random_regular_graph(n, 3, 9)
    g, b = [0.4, 1.2], [0.8, 0.3]
    e = edges[4]
    fs, _ = tn.build_network(n, edges, g, b, e)
    ref, _ = tn.contract(fs)
    rng = np.random.default_rng(0)
    for _ in range(3):
        labels = sorted({l for f in fs for l in f.labels})
        perm = dict(zip(labels, rng.permutation(len(labels)).tolist()))
        shuffled = [tn.Factor(f.value, [perm[l] for l in f.labels]) for f in fs]
        order = rng.permutation(len(shuffled))
        val, _ = tn.contract([shuffled[i] for i in order])
        assert abs(val - ref) < 1e-13


def _golden_superops():
    with open(os.path.join(GOLDEN, "superoperators.json")) as f:
        gold = json.load(f)
    cnot = np.zeros((4, 4, 4, 4))
    for key in gold["CNOT_nonzero_ones"]:
        cnot[tuple(int(c) for c in key)] = 1.0
    m_y = np.array([complex(*re_im) for re_im in gold["M_Y"]])
    return gold, cnot, m_y


def test_paper_superoperator_tables():
    gold, cnot, m_y = _golden_superops()
    x = np.array([[0, 1], [1, 0]])
    y = np.array([[0, -1j], [1j, 0]])
    z = np.diag([1, -1])
    assert np.array_equal(so.superop_1q(x), np.array(gold["X"]))
    assert np.array_equal(so.superop_1q(y), np.array(gold["Y"]))
    # the printed Z tilde is the identity: only the corrected reading matches
    assert not np.array_equal(so.superop_1q(z), np.array(gold["Z_as_printed"]))
    assert np.array_equal(so.superop_1q(z), np.array(gold["Z_corrected"]))
    u_cnot = np.zeros((4, 4))
    for c in range(2):
        for t in range(2):
            u_cnot[2 * c + (t ^ c), 2 * c + t] = 1
    assert np.array_equal(so.superop_2q(u_cnot), cnot)
    assert np.array_equal(so.measurement("I"), np.array(gold["M_Trace"]))
    assert np.array_equal(so.measurement("X"), np.array(gold["M_X"]))
    assert np.array_equal(so.measurement("Y"), m_y)
    assert np.array_equal(so.measurement("Z"), np.array(gold["M_Z"]))
    assert np.array_equal(so.RHO0, np.array(gold["rho0"]))


def test_paper_density_network_matches_statevector():
    """A small circuit in the paper's dim-4 form equals <psi|P|psi>."""
    gold, cnot, m_y = _golden_superops()
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    rx = scipy.linalg.expm(-1j * 0.37 * np.array([[0, 1], [1, 0]]))
    z_tilde = np.array(gold["Z_corrected"])
    gates = [(so.superop_1q(h), (0,)), (cnot, (0, 1)), (np.array(gold["X"]), (2,)),
             (so.superop_1q(rx), (1,)), (np.array(gold["Y"]), (0,)),
             (z_tilde, (1,)), (cnot, (1, 2)), (so.superop_1q(h), (2,))]
    meas = [np.array(gold["M_Z"]), np.array(gold["M_X"]), m_y]
    val = so.expectation(3, gates, meas)
    # plain state-vector reference; qubit q is bit q, kron order qubit 2 first
    eye = np.eye(2)
    paulis = {"X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
              "Z": np.diag([1, -1])}

    def one(u, q):
        mats = [u if k == q else eye for k in (2, 1, 0)]
        return np.kron(np.kron(mats[0], mats[1]), mats[2])

    def cx(c, t):
        m = np.zeros((8, 8))
        for s in range(8):
            m[s ^ (((s >> c) & 1) << t), s] = 1
        return m

    psi = np.zeros(8, dtype=complex)
    psi[0] = 1
    for u in [one(h, 0), cx(0, 1), one(paulis["X"], 2), one(rx, 1), one(paulis["Y"], 0),
              one(paulis["Z"], 1), cx(1, 2), one(h, 2)]:
        psi = u @ psi
    obs = one(paulis["Z"], 0) @ one(paulis["X"], 1) @ one(paulis["Y"], 2)
    ref = np.vdot(psi, obs @ psi)
    assert abs(val - ref) < 1e-13
    assert abs(ref) > 0.1  # a non-trivial expectation


MUTATIONS = {
    "gamma_sign": lambda g: (np.exp(+0.5j * g * np.outer([1, -1], [1, -1])),
                             np.zeros((2, 2))),
    "half_angle_dropped": lambda g: (np.exp(-1j * g * np.outer([1, -1], [1, -1])),
                                     np.zeros((2, 2))),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_oracle_mistakes(name, monkeypatch):
    """A wrong phase gate in O-TN must break its agreement with the closed form."""
    monkeypatch.setattr(tn, "_zz_diag", MUTATIONS[name])
    edges = TRI7
    e = edges[0]
    got = tn.edge_value(7, edges, [0.7], [0.4], e).real
    want = cf.zz_p1(0.7, 0.4, *cf.edge_params(7, edges, e))
    assert abs(got - want) > 1e-3


def test_pins_catch_unconjugated_bra(monkeypatch):
    """Dropping the conjugation of the bra network breaks unitarity <I> = 1."""
    monkeypatch.setattr(np, "conj", lambda a: a)
    edges = TRI7
    val = tn.identity_value(7, edges, [0.7], [0.4], edge=edges[0])
    assert abs(val - 1.0) > 1e-3


@pytest.mark.parametrize("n,p", [(8, 2), (10, 3)])
def test_ring_of_disagrees_optimum(n, p):
    """Ring of disagrees (the 2-regular cycle): once the ring is longer than
    an edge's light cone (n > 2p + 1), the best cut fraction level-p QAOA
    reaches is (2p + 1)/(2p + 2) (Farhi, Goldstone and Gutmann 2014; proved
    through the fermionic mapping by Wang, Hadfield, Jiang and Rieffel 2018).
    Every edge network of the ring is the same up to relabelling, so the
    oracle's value and forward-mode gradient of one edge, maximised over the
    angles from several starts, must reach the bound and never pass it."""
    from scipy.optimize import minimize
    edges = [(i, (i + 1) % n) for i in range(n)]

    def neg(x):
        s, ds = tn.edge_value_grad(n, edges, list(x[:p]), list(x[p:]), edges[0])
        return -(1.0 - s.real) / 2.0, 0.5 * np.asarray(ds).real

    bound = (2 * p + 1) / (2 * p + 2)
    rng = np.random.default_rng(0)
    best = 0.0
    for _ in range(8):
        r = minimize(neg, rng.uniform(-1.5, 1.5, 2 * p), jac=True, method="BFGS",
                     options={"gtol": 1e-10})
        assert -r.fun <= bound + 1e-12
        best = max(best, -r.fun)
    assert abs(best - bound) < 1e-9


def test_tensor_network_finite_differences_match_adjoint():
    """O-TN's central differences (h = 1e-4) against the state-vector adjoint
    gradient of the same edge observable (p = 2), and at p = 1 against the
    closed form's derivatives: a wrong divisor or a swapped parameter slot
    misses by far more than the O(h^2) truncation."""
    from oracle import lightcone as lc
    n = 10
    edges = random_regular_graph(n, 3, 9)
    for p in (1, 2):
        g, b = [0.52, 1.07][:p], [0.33, 0.61][:p]
        for e in (edges[1], edges[7]):
            fd = tn.edge_grad_fd(n, edges, g, b, e)
            _, ref = lc.edge_gradient(n, edges, g, b, e)
            assert np.max(np.abs(fd - np.asarray(ref))) < 1e-7
            if p == 1:
                dg, db = cf.zz_p1_grad(g[0], b[0], *cf.edge_params(n, edges, e))
                assert abs(fd[0] - dg) < 1e-7 and abs(fd[1] - db) < 1e-7
