"""O-TN: the QAOA circuit as a closed tensor network, contracted in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network (Section 2, built with bond dimension 2 as a ket/bra sandwich):
<psi|O|psi> = sum_{i,j} conj(psi_i) O_ij psi_j, where the ket network is the
circuit of Section 4.1 (|+> states, exp(-i gamma Z Z / 2) phase gates, RX
mixers) and the bra network is its element-wise complex conjugate with the
same index roles.  Output wires of unobserved qubits join ket to bra (a
trace); observed qubits get a Z tensor between them.

Two gate forms:
* dense: every gate is a tensor with its own input and output wires (the
  paper's form: rank-4 ZZ gates, every index shared by exactly two tensors);
* diagonal: a diagonal gate keeps the wire label, so a wire through several
  diagonal gates is one index shared by all of them (a hyperedge).

Contraction: plain variable elimination.  Repeatedly pick the index whose
elimination produces the smallest tensor (greedy minimum degree on the index
interaction graph, ties to the lowest label), multiply every tensor holding
it (Eq. 1 with batch indices, evaluated by numpy einsum) and sum the index
out.  Any elimination order gives the same scalar (exact contraction).

Gradient: each tensor carries, beside its value, its derivative with respect
to every circuit parameter (forward-mode dual tensors); a product of tensors
gets the product rule.  Parameters are ordered (gamma_1..p, beta_1..p).
"""

from __future__ import annotations

import math

import numpy as np

from .lightcone import ball

_SQRT_HALF = 1.0 / math.sqrt(2.0)


class Factor:
    __slots__ = ("value", "labels", "tangent")

    def __init__(self, value, labels, tangent=None):
        self.value = np.asarray(value, dtype=np.complex128)
        self.labels = tuple(labels)
        self.tangent = tangent  # None, or array of shape (P,) + value.shape
        if self.value.ndim != len(self.labels):
            raise ValueError("rank does not match the label list")


# ---- gate tensors (ket side; the bra uses the complex conjugates) ---------

def _zz_diag(gamma):
    z = np.array([1.0, -1.0])
    zz = np.outer(z, z)
    val = np.exp(-0.5j * gamma * zz)
    return val, (-0.5j * zz) * val


def _zz_dense(gamma):
    diag, ddiag = _zz_diag(gamma)
    val = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    dval = np.zeros_like(val)
    for a in range(2):
        for b in range(2):
            val[a, b, a, b] = diag[a, b]        # [a_out, b_out, a_in, b_in]
            dval[a, b, a, b] = ddiag[a, b]
    return val, dval


def _rx(beta):
    c, s = math.cos(beta), math.sin(beta)
    val = np.array([[c, -1j * s], [-1j * s, c]])          # [out, in]
    dval = np.array([[-s, -1j * c], [-1j * c, -s]])
    return val, dval


_H = np.array([[1.0, 1.0], [1.0, -1.0]]) * _SQRT_HALF   # [out, in]


def layer_sets(n, edges, p, edge, lightcone):
    """Per-layer kept edges and RX qubits, and the qubits of the network.

    Light cone: layer k (1-based) keeps the edges that touch B_{p-k} and RX on
    B_{p-k}; the qubits are B_p.  Without it every gate and qubit is kept.
    """
    if not lightcone:
        return [list(edges)] * p, [list(range(n))] * p, list(range(n))
    balls = [ball(n, edges, edge, r) for r in range(p + 1)]
    kept_edges, kept_rx = [], []
    for k in range(1, p + 1):
        core = set(balls[p - k])
        kept_edges.append([e for e in edges if e[0] in core or e[1] in core])
        kept_rx.append(sorted(core))
    return kept_edges, kept_rx, balls[p]


def build_network(n, edges, gammas, betas, edge=None, *, lightcone=True,
                  dense=False, observable="zz", bits=None, with_grad=False,
                  hadamard=False):
    """Factors of <psi|O|psi> (or of <x|psi> for observable='amplitude').

    observable: 'zz' (Z_u Z_v on ``edge``), 'identity', or 'amplitude' (ket
    only, closed with the basis state ``bits``; needs lightcone=False).
    """
    p = len(gammas)
    P = 2 * p
    if observable == "amplitude" and lightcone:
        raise ValueError("the amplitude network has no light cone")
    if observable in ("zz",) and edge is None:
        raise ValueError("the ZZ observable needs an edge")
    kept_edges, kept_rx, qubits = layer_sets(
        n, edges, p, edge if edge is not None else (0, 0), lightcone)

    counter = [0]

    def new_label():
        counter[0] += 1
        return counter[0] - 1

    def tangent_for(slot, dval, conj):
        if not with_grad:
            return None
        t = np.zeros((P,) + dval.shape, dtype=np.complex128)
        t[slot] = np.conj(dval) if conj else dval
        return t

    def side(conj):
        fs = []
        cur = {}
        for q in qubits:
            if hadamard:
                l0, l1 = new_label(), new_label()
                fs.append(Factor([1.0, 0.0], (l0,)))
                fs.append(Factor(_H, (l1, l0)))
                cur[q] = l1
            else:
                cur[q] = new_label()
                fs.append(Factor([_SQRT_HALF, _SQRT_HALF], (cur[q],)))
        for k in range(p):
            if dense:
                val, dval = _zz_dense(gammas[k])
            else:
                val, dval = _zz_diag(gammas[k])
            if conj:
                val = np.conj(val)
            for a, b in kept_edges[k]:
                if dense:
                    na, nb = new_label(), new_label()
                    fs.append(Factor(val, (na, nb, cur[a], cur[b]),
                                     tangent_for(k, dval, conj)))
                    cur[a], cur[b] = na, nb
                else:
                    fs.append(Factor(val, (cur[a], cur[b]),
                                     tangent_for(k, dval, conj)))
            val, dval = _rx(betas[k])
            if conj:
                val = np.conj(val)
            for q in kept_rx[k]:
                nq = new_label()
                fs.append(Factor(val, (nq, cur[q]), tangent_for(p + k, dval, conj)))
                cur[q] = nq
        return fs, cur

    ket, ket_out = side(conj=False)
    if observable == "amplitude":
        for q in qubits:
            e = np.zeros(2)
            e[int(bits[q])] = 1.0
            ket.append(Factor(e, (ket_out[q],)))
        return ket, P

    bra, bra_out = side(conj=True)
    observed = set(edge) if observable == "zz" else set()
    z = np.array([[1.0, 0.0], [0.0, -1.0]])
    rename = {}
    extra = []
    for q in qubits:
        if q in observed and dense:
            extra.append(Factor(z, (bra_out[q], ket_out[q])))     # O[i(bra), j(ket)]
        else:
            rename[bra_out[q]] = ket_out[q]
            if q in observed:
                extra.append(Factor([1.0, -1.0], (ket_out[q],)))
    bra = [Factor(f.value, tuple(rename.get(l, l) for l in f.labels), f.tangent)
           for f in bra]
    return ket + bra + extra, P


# ---- contraction -----------------------------------------------------------

def _einsum(values, labelsets, out_labels):
    letters = {}
    for ls in labelsets:
        for l in ls:
            letters.setdefault(l, len(letters))
    for l in out_labels:
        letters.setdefault(l, len(letters))
    if len(letters) > 51:
        raise ValueError("too many indices in one elimination")
    args = []
    for v, ls in zip(values, labelsets):
        args.append(v)
        args.append([letters[l] for l in ls])
    args.append([letters[l] for l in out_labels])
    return np.einsum(*args, optimize=False)


_TANGENT_AXIS = ("tangent-axis",)


def contract(factors, n_params=0, max_rank=40):
    """Variable elimination of a closed network; returns (value, tangent).

    ``tangent`` is None when no factor carries one, else an array of the
    derivative of the scalar with respect to each of the ``n_params``
    parameters.
    """
    live = {i: f for i, f in enumerate(factors)}
    holders = {}
    for i, f in live.items():
        for l in f.labels:
            holders.setdefault(l, set()).add(i)
    next_id = len(factors)
    while holders:
        best = None
        for l, hs in holders.items():
            union = set()
            for i in hs:
                union.update(live[i].labels)
            key = (len(union) - 1, l)
            if best is None or key < best[0]:
                best = (key, l, union)
        label, union = best[1], best[2]
        group_ids = sorted(holders[label])
        group = [live[i] for i in group_ids]
        out = tuple(sorted(union - {label}))
        if len(out) > max_rank:
            raise ValueError(f"intermediate of rank {len(out)} exceeds {max_rank}")
        vals = [f.value for f in group]
        lsets = [f.labels for f in group]
        value = _einsum(vals, lsets, out)
        tangent = None
        for j, f in enumerate(group):
            if f.tangent is None:
                continue
            tv = list(vals)
            tv[j] = f.tangent
            tl = list(lsets)
            tl[j] = _TANGENT_AXIS + f.labels
            term = _einsum(tv, tl, _TANGENT_AXIS + out)
            tangent = term if tangent is None else tangent + term
        for i in group_ids:
            for l in live[i].labels:
                holders[l].discard(i)
            del live[i]
        for l in [l for l, hs in holders.items() if not hs]:
            del holders[l]
        live[next_id] = Factor(value, out, tangent)
        for l in out:
            holders.setdefault(l, set()).add(next_id)
        next_id += 1
    # only scalars remain: multiply them, product rule for the tangent
    total = 1.0 + 0.0j
    scalars = list(live.values())
    for f in scalars:
        total *= complex(f.value)
    tangent = None
    for j, f in enumerate(scalars):
        if f.tangent is None:
            continue
        rest = 1.0 + 0.0j
        for k, g in enumerate(scalars):
            if k != j:
                rest *= complex(g.value)
        term = np.asarray(f.tangent, dtype=np.complex128).reshape(-1) * rest
        tangent = term if tangent is None else tangent + term
    if tangent is None and n_params:
        tangent = np.zeros(n_params, dtype=np.complex128)
    return total, tangent


def max_elimination_rank(factors):
    """Largest intermediate rank the elimination order above produces."""
    live = {i: set(f.labels) for i, f in enumerate(factors)}
    holders = {}
    for i, ls in live.items():
        for l in ls:
            holders.setdefault(l, set()).add(i)
    worst = 0
    nid = len(factors)
    while holders:
        best = None
        for l, hs in holders.items():
            union = set().union(*(live[i] for i in hs))
            key = (len(union) - 1, l)
            if best is None or key < best[0]:
                best = (key, l, union)
        label, union = best[1], best[2]
        worst = max(worst, len(union) - 1)
        for i in list(holders[label]):
            for l in live[i]:
                holders[l].discard(i)
            del live[i]
        for l in [l for l, hs in holders.items() if not hs]:
            del holders[l]
        live[nid] = union - {label}
        for l in live[nid]:
            holders.setdefault(l, set()).add(nid)
        nid += 1
    return worst


# ---- QAOA quantities -------------------------------------------------------

def edge_value(n, edges, gammas, betas, edge, **kw):
    """Complex scalar s = <psi|Z_u Z_v|psi> of one edge network."""
    fs, P = build_network(n, edges, gammas, betas, edge, **kw)
    value, _ = contract(fs)
    return value


def edge_value_grad(n, edges, gammas, betas, edge, **kw):
    """(s, ds/d(gamma, beta)) of one edge network, forward mode."""
    fs, P = build_network(n, edges, gammas, betas, edge, with_grad=True, **kw)
    return contract(fs, n_params=P)


def edge_grad_fd(n, edges, gammas, betas, edge, h=1e-4, **kw):
    """d Re s / d(gamma, beta) of one edge network by central differences
    with step h: (s(theta + h e_i) - s(theta - h e_i)) / 2h per parameter."""
    x = np.array(list(gammas) + list(betas), dtype=np.float64)
    p = len(gammas)
    out = np.zeros(len(x))
    for i in range(len(x)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        out[i] = (edge_value(n, edges, xp[:p], xp[p:], edge, **kw).real
                  - edge_value(n, edges, xm[:p], xm[p:], edge, **kw).real) / (2 * h)
    return out


def maxcut(n, edges, gammas, betas, **kw):
    """<C> = sum_e (1 - Re s_e) / 2 over every edge network."""
    return float(sum((1.0 - edge_value(n, edges, gammas, betas, e, **kw).real) / 2.0
                     for e in edges))


def maxcut_grad(n, edges, gammas, betas, **kw):
    """(<C>, d<C>/d(gamma, beta)) summed over the edge networks."""
    total = 0.0
    grad = np.zeros(2 * len(gammas))
    for e in edges:
        s, ds = edge_value_grad(n, edges, gammas, betas, e, **kw)
        total += (1.0 - s.real) / 2.0
        grad -= 0.5 * ds.real
    return total, grad


def identity_value(n, edges, gammas, betas, edge=(0, 1), **kw):
    """<psi|psi> through the network with the identity observable."""
    kw = dict(kw)
    kw["observable"] = "identity"
    return edge_value(n, edges, gammas, betas, edge, **kw)


def amplitude(n, edges, gammas, betas, bits, **kw):
    """<x|psi> from the ket-only network closed with the basis state x."""
    fs, _ = build_network(n, edges, gammas, betas, None, lightcone=False,
                          observable="amplitude", bits=bits, **kw)
    value, _ = contract(fs)
    return value
