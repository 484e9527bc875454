"""Host-side logic of libqtc.so on the CPU (no GPU calls).

The library's own networks (read back through qtc_network_leaves) are
contracted in numpy along the library's own plans (qtc_plan_steps); the
result must equal the oracle's state-vector value.  This checks the circuit
-> network builder, the light cone, the diagonal/dense forms and both
orderings without a GPU.  Leaf values are written here from the gate
definitions in include/qtc.h.
"""

import math
import re

import numpy as np
import pytest

from oracle import statevector as sv
from synth import WORKLOADS, random_regular_graph

q = pytest.importorskip("paper_1709_03636_gb300")

R = 1 / math.sqrt(2)


def leaf_tensor(kind, conj, slot, coeff, constant, params):
    t = constant + (coeff * params[slot] if slot >= 0 else 0.0)
    c, s = math.cos(t / 2), math.sin(t / 2)
    e = lambda z: complex(math.cos(z * t / 2), -math.sin(z * t / 2))  # exp(-i z t/2)
    T = {
        0: lambda: np.array([1, 0]),
        1: lambda: np.array([R, R]),
        2: lambda: np.array([1, 0]),
        3: lambda: np.array([0, 1]),
        4: lambda: np.array([[R, R], [R, -R]]),
        5: lambda: np.array([[0, 1], [1, 0]]),
        6: lambda: np.array([[0, -1j], [1j, 0]]),
        7: lambda: np.array([[1, 0], [0, -1]]),
        8: lambda: np.array([[c, -1j * s], [-1j * s, c]]),
        9: lambda: np.diag([e(1), e(-1)]),
        10: lambda: np.array([1, -1]),
        11: lambda: np.array([e(1), e(-1)]),
        12: lambda: np.array([[e(1), e(-1)], [e(-1), e(1)]]),
        15: lambda: np.array([[0, 1], [1, 0]]),
        16: lambda: np.array([[0, -1j], [1j, 0]]),
        17: lambda: np.array([[1, 0], [0, -1]]),
    }
    if kind in (18, 19, 20):
        # channel [ket_out, bra_out, ket_in, bra_in] = sum_k K[ko, ki] conj(K[bo, bi])
        st = constant
        if kind == 18:
            ks = [math.sqrt(1 - st) * np.eye(2)] + [
                math.sqrt(st / 3) * np.array(m) for m in
                ([[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]])]
        elif kind == 19:
            ks = [math.sqrt(1 - st) * np.eye(2), math.sqrt(st) * np.diag([1, -1])]
        else:
            ks = [np.array([[1, 0], [0, math.sqrt(1 - st)]]),
                  np.array([[0, math.sqrt(st)], [0, 0]])]
        v = sum(np.einsum("ac,bd->abcd", np.asarray(k, complex), np.conj(np.asarray(k, complex)))
                for k in ks)
        return v
    if kind == 21:
        return np.eye(2, dtype=complex)
    if kind == 23:  # (1, 1): closes a shared ket/bra wire
        return np.array([1, 1], dtype=complex)
    if kind in (24, 25):  # [bra, ket] projector
        return np.diag([1, 0] if kind == 24 else [0, 1]).astype(complex)
    if kind == 22:  # sparse CNOT [t_out, c, t_in]
        v = np.zeros((2, 2, 2), dtype=complex)
        for cc in range(2):
            for tt in range(2):
                v[tt ^ cc, cc, tt] = 1
        return v
    if kind == 13:
        v = np.zeros((2, 2, 2, 2), dtype=complex)
        for a in range(2):
            for b in range(2):
                v[a, b, a, b] = e(1 if a == b else -1)
    elif kind == 14:
        v = np.zeros((2, 2, 2, 2), dtype=complex)
        for cc in range(2):
            for tt in range(2):
                v[cc, tt ^ cc, cc, tt] = 1
    else:
        v = np.asarray(T[kind](), dtype=complex)
    return np.conj(v) if conj else v


def run_plan(network, plan, params):
    leaves, n_labels = network.leaves()
    tensors = [(leaf_tensor(l["kind"], l["conj"], l["slot"], l["coeff"], l["constant"], params),
                tuple(l["labels"])) for l in leaves]
    count = np.zeros(n_labels, dtype=int)
    for _, ls in tensors:
        for l in ls:
            count[l] += 1
    for a, b in plan.steps():
        (va, la), (vb, lb) = tensors[a], tensors[b]
        both = set(la) | set(lb)
        shared = {l: (l in la) + (l in lb) for l in both}
        out = tuple(sorted(l for l in both if count[l] > shared[l]))
        for l in both:
            count[l] -= shared[l]
        for l in out:
            count[l] += 1
        letters = {l: i for i, l in enumerate(sorted(both))}
        v = np.einsum(va, [letters[l] for l in la], vb, [letters[l] for l in lb],
                      [letters[l] for l in out])
        tensors.append((v, out))
    value, labels = tensors[-1]
    assert labels == ()
    return complex(value)


@pytest.mark.parametrize("ordering", ["lg", "stoch"])
@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("lightcone", [True, False])
@pytest.mark.parametrize("p", [1, 2])
def test_qaoa_networks_and_plans_match_statevector(ordering, diag, lightcone, p):
    n = 8
    edges = random_regular_graph(n, 3, 4 + p)
    gammas = [0.3 + 0.4 * k for k in range(p)]
    betas = [0.9 - 0.3 * k for k in range(p)]
    ref = sv.edge_zz(n, edges, gammas, betas)
    circ = q.Circuit.qaoa(n, edges, p)
    params = gammas + betas
    for i, e in enumerate(edges[:6]):
        net = q.Network(circ, "zz", edge=e, lightcone=lightcone, diag=diag)
        plan = q.Plan(net, ordering, seed=3)
        st = plan.stats()
        assert st["n_steps"] == st["n_tensors"] - 1
        val = run_plan(net, plan, params)
        assert abs(val.real - ref[i]) < 1e-12 and abs(val.imag) < 1e-12


@pytest.mark.parametrize("channel", ["depolarize", "dephase", "ampdamp"])
@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("lightcone", [True, False])
def test_noisy_qaoa_networks_match_density_matrix(channel, diag, lightcone):
    """Channels after every mixer (Section 2's density-matrix form): the
    library's networks and plans against the density-matrix oracle."""
    from oracle import density as dm
    n, p, s = 8, 2, 0.07
    edges = random_regular_graph(n, 3, 9)
    gammas, betas = [0.45, 1.05], [0.8, 0.35]
    ref = dm.edge_zz(n, edges, gammas, betas, channel, s)
    circ = q.Circuit.qaoa(n, edges, p, noise=(channel, s))
    for i, e in enumerate(edges[:4]):
        net = q.Network(circ, "zz", edge=e, lightcone=lightcone, diag=diag)
        for ordering in ("lg", "stoch"):
            val = run_plan(net, q.Plan(net, ordering, seed=5), gammas + betas)
            assert abs(val.real - ref[i]) < 1e-12 and abs(val.imag) < 1e-12


def test_channel_arguments_are_checked():
    edges = random_regular_graph(6, 3, 1)
    with pytest.raises(q.QtcError):
        q.Circuit.qaoa(6, edges, 1, noise=("depolarize", 1.5))
    c = q.Circuit(2, 0)
    with pytest.raises(q.QtcError):
        c.add_gate("dephase", [0], slot=0, constant=0.1)
    c.add_gate("h", [0]).add_gate("ampdamp", [0], constant=0.3)
    with pytest.raises(q.QtcError):
        q.Network(c, "amplitude", bits=[0, 0], lightcone=False)


@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("lightcone", [True, False])
def test_projector_networks_give_prefix_probabilities(diag, lightcone):
    """<psi| prod P |psi> (Section 3.3) for projector patterns, against sums of
    |psi|^2; with lightcone = 0 the networks of all patterns share one
    structure, and one plan serves them all."""
    n = 8
    edges = random_regular_graph(n, 3, 12)
    g, b = [0.52, 1.17], [0.93, 0.31]
    p = np.abs(sv.qaoa_state(n, edges, g, b).reshape(-1)) ** 2
    idx = np.arange(1 << n)
    circ = q.Circuit.qaoa(n, edges, 2)
    first = None
    for bits in ([0, 2, 2, 2, 2, 2, 2, 2], [1, 0, 2, 1, 2, 2, 2, 2], [1, 0, 1, 1, 0, 0, 1, 0],
                 [2, 2, 2, 2, 2, 1, 2, 2]):
        mask = sum(1 << k for k in range(n) if bits[k] != 2)
        pat = sum(bits[k] << k for k in range(n) if bits[k] != 2)
        ref = p[(idx & mask) == pat].sum()
        net = q.Network(circ, "projector", bits=bits, lightcone=lightcone, diag=diag)
        if lightcone:
            plan = q.Plan(net, "lg", seed=2)
        else:
            plan = q.Plan(net, like=first) if first else q.Plan(net, "lg", seed=2)
            first = first or plan
        val = run_plan(net, plan, g + b)
        assert abs(val - ref) < 1e-12


def test_plans_are_binary_trees():
    edges = random_regular_graph(20, 4, 1)
    circ = q.Circuit.qaoa(20, edges, 2)
    for ordering in ["lg", "stoch"]:
        net = q.Network(circ, "zz", edge=edges[3])
        plan = q.Plan(net, ordering, seed=11)
        st = plan.stats()
        L = st["n_tensors"]
        used = set()
        for s, (a, b) in enumerate(plan.steps()):
            assert a != b and a < L + s and b < L + s
            assert a not in used and b not in used
            used.update((a, b))
        assert used == set(range(L + st["n_steps"] - 1))


def test_light_cone_sizes():
    # p=1 on a triangle-free 3-regular graph: 6 qubits, 5 phase gates, 2 RX
    edges = random_regular_graph(50, 3, 0)
    circ = q.Circuit.qaoa(50, edges, 1)
    net = q.Network(circ, "zz", edge=edges[0], diag=True)
    leaves, _ = net.leaves()
    kinds = [l["kind"] for l in leaves]
    n_plus = kinds.count(1)
    assert n_plus in (10, 12) and kinds.count(8) == 4 and kinds.count(10) == 2
    assert kinds.count(12) == 2 * (n_plus // 2 - 1)


def _full_unitary_reference(n, gates, pauli):
    """Plain state-vector reference of a generic circuit (kron-built gates)."""
    eye = np.eye(2)
    mats = {"h": np.array([[1, 1], [1, -1]]) * R, "x": np.array([[0, 1], [1, 0]]),
            "y": np.array([[0, -1j], [1j, 0]]), "z": np.diag([1, -1])}

    def one(u, k):
        out = np.array([[1.0]])
        for j in reversed(range(n)):
            out = np.kron(out, u if j == k else eye)
        return out

    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1
    for g, qs, theta in gates:
        if g in mats:
            u = one(mats[g], qs[0])
        elif g == "rx":
            u = one(np.array([[math.cos(theta / 2), -1j * math.sin(theta / 2)],
                              [-1j * math.sin(theta / 2), math.cos(theta / 2)]]), qs[0])
        elif g == "rz":
            u = one(np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)]), qs[0])
        elif g == "zz":
            zz = one(mats["z"], qs[0]) @ one(mats["z"], qs[1])
            u = np.diag(np.exp(-0.5j * theta * np.diag(zz)))
        elif g == "cnot":
            u = np.zeros((2 ** n, 2 ** n))
            for s in range(2 ** n):
                u[s ^ (((s >> qs[0]) & 1) << qs[1]), s] = 1
        psi = u @ psi
    obs = np.eye(1)
    for j in reversed(range(n)):
        obs = np.kron(obs, mats[pauli[j].lower()] if pauli[j] != "I" else eye)
    return psi, np.vdot(psi, obs @ psi)


GENERIC = [("h", (0,)), ("cnot", (0, 1)), ("rx", (2,)), ("zz", (1, 2)), ("rz", (0,)),
           ("y", (3,)), ("cnot", (3, 0)), ("h", (1,)), ("zz", (0, 3)), ("x", (2,)),
           ("rz", (3,)), ("rx", (1,)), ("z", (0,)), ("cnot", (2, 1))]


@pytest.mark.parametrize("pauli", ["ZIIZ", "XYZI", "IYIX", "ZZZZ"])
@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("lightcone", [True, False])
def test_generic_circuit_pauli_observables(pauli, diag, lightcone):
    n = 4
    params = [0.37, -1.1, 2.3]
    circ = q.Circuit(n, len(params))
    gates = []
    slot = 0
    for g, qs in GENERIC:
        if g in ("rx", "rz", "zz"):
            circ.add_gate(g, qs, slot % 3, 1.5, 0.2)
            gates.append((g, qs, 1.5 * params[slot % 3] + 0.2))
            slot += 1
        else:
            circ.add_gate(g, qs)
            gates.append((g, qs, 0.0))
    _, ref = _full_unitary_reference(n, gates, pauli)
    net = q.Network(circ, "pauli", pauli=pauli, lightcone=lightcone, diag=diag)
    val = run_plan(net, q.Plan(net, "lg"), params)
    assert abs(val - ref) < 1e-12


def random_cnot_circuit(n, n_gates, seed):
    """A CNOT-heavy random circuit: (gate, qubits, angle) with H, RX, RZ, CNOT."""
    rng = np.random.default_rng(seed)
    gates = [("h", (q,), 0.0) for q in range(n)]
    for _ in range(n_gates):
        k = rng.integers(4)
        if k < 2:
            a, b = rng.choice(n, 2, replace=False)
            gates.append(("cnot", (int(a), int(b)), 0.0))
        else:
            gates.append((("rx", "rz")[k - 2], (int(rng.integers(n)),), float(rng.uniform(-3, 3))))
    return gates


def statevector_reference(n, gates, pauli):
    """<psi|P|psi> by applying the gates to a 2^n state one by one."""
    psi = np.zeros((2,) * n, dtype=complex)
    psi[(0,) * n] = 1
    ax = lambda q: n - 1 - q  # noqa: E731
    mats = {"h": np.array([[1, 1], [1, -1]]) * R, "x": np.array([[0, 1], [1, 0]]),
            "y": np.array([[0, -1j], [1j, 0]]), "z": np.diag([1, -1])}
    for g, qs, t in gates:
        if g == "cnot":
            c, tq = qs
            sel = [slice(None)] * n
            sel[ax(c)] = 1
            sub = psi[tuple(sel)].copy()
            t_axis = ax(tq) - (1 if ax(tq) > ax(c) else 0)
            psi[tuple(sel)] = np.flip(sub, axis=t_axis)
            continue
        if g == "rx":
            u = np.array([[math.cos(t / 2), -1j * math.sin(t / 2)],
                          [-1j * math.sin(t / 2), math.cos(t / 2)]])
        elif g == "rz":
            u = np.diag([np.exp(-0.5j * t), np.exp(0.5j * t)])
        else:
            u = mats[g]
        psi = np.moveaxis(np.tensordot(u, psi, axes=([1], [ax(qs[0])])), 0, ax(qs[0]))
    phi = psi
    for q_ in range(n):
        if pauli[q_] != "I":
            phi = np.moveaxis(np.tensordot(mats[pauli[q_].lower()], phi, axes=([1], [ax(q_)])),
                              0, ax(q_))
    return complex(np.vdot(psi, phi))


def build_generic(n, gates):
    circ = q.Circuit(n, 0)
    for g, qs, t in gates:
        circ.add_gate(g, list(qs), -1, 0.0, t)
    return circ


def test_sparse_cnot_matches_and_lowers_cost():
    """CNOT as a rank-3 XOR tensor with a shared control wire (diag mode)
    against the dense rank-4 form: the same value, and a far cheaper
    contraction (multiply-adds of the best of three LG plans, summed over
    random CNOT-heavy circuits; measured ~4x fewer at 8-16 qubits)."""
    n = 8
    cost = {True: 0.0, False: 0.0}
    for seed in range(4):
        gates = random_cnot_circuit(n, 40, seed)
        circ = build_generic(n, gates)
        pauli = "ZIXIYIIZ"
        ref = statevector_reference(n, gates, pauli)
        for diag in (True, False):
            net = q.Network(circ, "pauli", pauli=pauli, lightcone=False, diag=diag)
            plans = [q.Plan(net, "lg", seed=s) for s in range(3)]
            best = min(plans, key=lambda pl: pl.stats()["cmacs"])
            cost[diag] += best.stats()["cmacs"]
            assert abs(run_plan(net, best, []) - ref) < 1e-11
    assert cost[True] < 0.5 * cost[False], cost


def test_generic_amplitudes():
    n = 4
    params = [0.37, -1.1, 2.3]
    circ = q.Circuit(n, len(params))
    gates = []
    for i, (g, qs) in enumerate(GENERIC):
        if g in ("rx", "rz", "zz"):
            circ.add_gate(g, qs, i % 3, 1.0, 0.0)
            gates.append((g, qs, params[i % 3]))
        else:
            circ.add_gate(g, qs)
            gates.append((g, qs, 0.0))
    psi, _ = _full_unitary_reference(n, gates, "IIII")
    for x in range(2 ** n):
        bits = [(x >> k) & 1 for k in range(n)]
        net = q.Network(circ, "amplitude", bits=bits, lightcone=False)
        assert abs(run_plan(net, q.Plan(net, "stoch", seed=x), params) - psi[x]) < 1e-12


def test_invalid_inputs_raise():
    with pytest.raises(q.QtcError, match="INVALID"):
        q.Circuit.qaoa(4, [(0, 0)], 1)
    with pytest.raises(q.QtcError, match="INVALID"):
        q.Circuit.qaoa(4, [(0, 1), (1, 0)], 1)
    circ = q.Circuit.qaoa(4, [(0, 1), (1, 2), (2, 3)], 1)
    with pytest.raises(q.QtcError, match="INVALID"):
        q.Network(circ, "zz", edge=(0, 9))
    with pytest.raises(q.QtcError, match="INVALID"):
        q.Network(circ, "identity", lightcone=True)
    with pytest.raises(q.QtcError, match="INVALID"):
        circ.add_gate("rx", (0,), 7, 1.0)


def test_library_exports_every_declared_symbol():
    import ctypes
    import os
    from paper_1709_03636_gb300 import _lib
    header = open(os.path.join(os.path.dirname(__file__), "..", "include", "qtc.h")).read()
    names = set(re.findall(r"\b(qtc_[a-z0-9_]+)\s*\(", header))
    assert len(names) > 20
    so = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(so, n)]
    assert not missing, missing


def _leaf_cases():
    rng = np.random.default_rng(11)
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
    out = []
    circ = q.Circuit.qaoa(4, edges, 2)
    out.append((q.Network(circ, edge=(0, 1)), 4))
    out.append((q.Network(circ, edge=(0, 1), diag=False), 4))
    for ch in ("depolarize", "dephase", "ampdamp"):
        out.append((q.Network(q.Circuit.qaoa(4, edges, 1, noise=(ch, 0.13)), edge=(1, 2)), 2))
    out.append((q.Network(circ, "pauli", pauli="XYZI", lightcone=False), 4))
    out.append((q.Network(circ, "amplitude", bits=[1, 0, 1, 1], lightcone=False), 4))
    out.append((q.Network(circ, "projector", bits=[1, 0, 2, 2], lightcone=False), 4))
    # generic gates, with parameters: slot, coefficient and constant angle
    cn = q.Circuit(4, 3)
    for g, qs, t in random_cnot_circuit(4, 12, 3) + [("h", (1,), 0.0), ("x", (2,), 0.0),
                                                    ("y", (3,), 0.0), ("z", (0,), 0.0),
                                                    ("zz", (0, 3), 0.4)]:
        slot = int(rng.integers(3)) if g in ("rx", "rz", "zz") else -1
        cn.add_gate(g, list(qs), slot, float(rng.uniform(-2, 2)) if slot >= 0 else 0.0, t)
    out.append((q.Network(cn, "pauli", pauli="ZZXY", lightcone=False), 3))
    out.append((q.Network(cn, "pauli", pauli="ZIZI", lightcone=False, diag=False), 3))
    return out, rng


def test_leaf_values_match_closed_forms():
    """Every leaf kind as the executors build it (coefficients A cos(t/2) +
    B sin(t/2) + C) against the closed forms above; derivatives against
    central differences of those closed forms."""
    cases, rng = _leaf_cases()
    kinds = set()
    for net, n_params in cases:
        params = rng.uniform(-2, 2, size=max(n_params, 1))
        leaves, _ = net.leaves()
        for i, l in enumerate(leaves):
            kinds.add(l["kind"])
            val, der = net.leaf_values(i, params)
            ref = leaf_tensor(l["kind"], l["conj"], l["slot"], l["coeff"], l["constant"], params)
            ref = np.asarray(ref, dtype=complex).flatten(order="F")
            assert np.max(np.abs(val - ref)) < 1e-14, (l, val, ref)
            if l["slot"] >= 0:
                h = 1e-5
                pp, pm = params.copy(), params.copy()
                pp[l["slot"]] += h
                pm[l["slot"]] -= h
                fd = (np.asarray(leaf_tensor(l["kind"], l["conj"], l["slot"], l["coeff"],
                                             l["constant"], pp), complex).flatten(order="F")
                      - np.asarray(leaf_tensor(l["kind"], l["conj"], l["slot"], l["coeff"],
                                               l["constant"], pm), complex).flatten(order="F"))
                assert np.max(np.abs(der - fd / (2 * h))) < 1e-8
            else:
                assert np.max(np.abs(der)) == 0
    assert len(kinds) >= 15, sorted(kinds)


def test_leaf_values_rejects_bad_leaf():
    net = q.Network(q.Circuit.qaoa(4, [(0, 1), (1, 2)], 1), edge=(0, 1))
    with pytest.raises(q.QtcError):
        net.leaf_values(10 ** 6, [0.1, 0.2])


DEGENERATE = {
    "ring8": (8, [(i, (i + 1) % 8) for i in range(8)]),
    "star8": (8, [(0, k) for k in range(1, 8)]),
    "path7": (7, [(i, i + 1) for i in range(6)]),
    "isolated6": (6, [(0, 1), (2, 3)]),
    "single2": (2, [(0, 1)]),
}


@pytest.mark.parametrize("name", sorted(DEGENERATE))
@pytest.mark.parametrize("p", [1, 2])
def test_degenerate_graph_shapes(name, p):
    """Graphs away from the random-regular workloads: a ring (every light cone
    a path), a star (one vertex of degree 7), a path (degree-1 ends), isolated
    vertices and a single edge.  Every edge network and its plan match the
    state vector, with and without the light cone, dense or diagonal; the
    batch lowers to warp programs that pass the host validator, and, forced
    into the graph form (small subtree ranks push steps to global memory), to
    waves that pass the wave validator."""
    n, edges = DEGENERATE[name]
    gammas = [0.3 + 0.4 * k for k in range(p)]
    betas = [0.9 - 0.3 * k for k in range(p)]
    ref = sv.edge_zz(n, edges, gammas, betas)
    circ = q.Circuit.qaoa(n, edges, p)
    for lightcone in (True, False):
        for diag in (True, False):
            for i, e in enumerate(edges):
                net = q.Network(circ, "zz", edge=e, lightcone=lightcone, diag=diag)
                val = run_plan(net, q.Plan(net, "lg", seed=3), gammas + betas)
                assert abs(val.real - ref[i]) < 1e-12 and abs(val.imag) < 1e-12
    for diag in (True, False):
        batch = q.Batch(circ, ordering="lg", diag=diag)
        info = batch.program_info("c64", True)
        assert info["graph"] == 0 and info["warp_teams"] == 1
        assert info["n_tasks"] == len(edges)
        for small_rank in (0, 4):
            for dtype in ("c64", "c128"):
                info = batch.program_info(dtype, True, force_graph=True, small_rank=small_rank,
                                          max_wave_bytes=1 << 22)
                assert info["graph"] == 1 and info["n_tasks"] >= len(edges)


def test_global_buffers_reuse_memory_by_live_range():
    """Graph-executor intermediates and adjoints are placed by live range,
    sharing memory only where every use of one tensor already precedes the
    writes of the other in the dependency order: for p=3 n=60 the networks'
    placed peaks sum to well under their tensors' total (the placement and
    that ordering are checked on the host when the program is built), and
    the whole graph with its gradient fits one launch under the default
    8 GiB limit."""
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    batch = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), ordering="lg")
    fwd = batch.program_info("c64", False)
    grad = batch.program_info("c64", True)
    for info in (fwd, grad):
        assert info["graph"] == 1
        # with the gradient most forward values stay live until the sweep
        assert 0 < info["net_global_bytes"] < 0.85 * info["net_global_bytes_unshared"]
        assert info["work_bytes"] <= info["net_global_bytes"]
    assert grad["n_waves"] == 1 and grad["work_bytes"] <= 8 << 30
    # forward only, a tensor is dead after the step that consumes it
    assert fwd["net_global_bytes"] < 0.6 * fwd["net_global_bytes_unshared"]


def checkpoint_cap(batch):
    """A wave limit under which the batch's gradient program needs checkpoint
    segments (None if none of the tried limits does)."""
    base = batch.program_info("c64", True)["net_global_bytes"]
    for frac in (0.7, 0.6, 0.55, 0.5, 0.45, 0.4):
        cap = max(1 << 20, int(frac * base))
        try:
            info = batch.program_info("c64", True, max_wave_bytes=cap)
        except q.QtcError:
            continue
        if info["checkpoint_segments"] > 1:
            return cap
    return None


def test_checkpoint_segments_when_one_network_exceeds_the_limit():
    """With the gradient, a network whose stored values alone exceed the wave
    limit first shares memory also where that adds write-after-read
    dependencies; below that it is lowered with checkpoint segments: values
    used only inside one segment are dropped after their forward use and
    recomputed by the adjoint sweep.  The peak then fits the limit, every
    reuse of memory is ordered (checked when the program is built), and a
    limit below what any segmentation reaches is refused with QTC_ERR_ARENA."""
    w = WORKLOADS["qaoa_p3_n60_d4"]
    edges = w.graph()
    full = q.Batch(q.Circuit.qaoa(w.n, edges, w.p), ordering="lg")
    for i in (9, 60):
        one = full.subset([i])
        base = one.program_info("c64", True)
        assert base["checkpoint_segments"] == 1
        cap = checkpoint_cap(one)
        assert cap is not None
        info = one.program_info("c64", True, max_wave_bytes=cap)
        assert info["checkpoint_segments"] > 1
        assert info["net_global_bytes"] <= cap < base["net_global_bytes"]
        # the recomputed forward steps are extra tasks
        assert info["n_tasks"] > base["n_tasks"]
        fwd = one.program_info("c64", False)
        with pytest.raises(q.QtcError, match="ARENA"):
            one.program_info("c64", True, max_wave_bytes=max(1 << 20, int(0.3 * fwd[
                "net_global_bytes"])))


@pytest.mark.parametrize("tile_mode", [0, 1, 2, 3, 4])
def test_tile_steps_emulated_against_the_plain_contraction(tile_mode):
    """The tile form of global steps (footprints copied through shared memory,
    lanes/warps/registers over the tile, reductions over summed lane and warp
    bits, split chunks) emulated on the host on random operands equals the
    plain contraction over each step's bit maps, for forward and adjoint
    programs of dense, diagonal and full networks.  Mode 0 (no tiles) checks
    the row steps taken four rows at a time along output labels one operand
    lacks (row order, each group's distinct operand elements)."""
    import ctypes
    from paper_1709_03636_gb300 import _lib
    checked = 0
    edges = random_regular_graph(12, 3, 6)
    circ = q.Circuit.qaoa(12, edges, 2)
    for kw in (dict(), dict(lightcone=False), dict(diag=False)):
        batch = q.Batch(circ, ordering="lg", **kw)
        for small, grad, dtype in ((2, 1, "c64"), (4, 0, "c128"), (6, 1, "c64")):
            err, cnt = ctypes.c_double(), ctypes.c_int32()
            _lib.check(_lib.lib.qtc_selftest_tile_steps(
                batch.ptr, q.DTYPES[dtype], grad, 1, small, tile_mode, 16,
                ctypes.byref(err), ctypes.byref(cnt)))
            assert err.value < 1e-11, (kw, small, grad, dtype)
            checked += cnt.value
    assert checked > {0: 20, 3: 20}.get(tile_mode, 500)
