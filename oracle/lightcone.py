"""O-LC: per-edge <Z_u Z_v> from the state vector of the radius-p ball.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For depth p, <Z_u Z_v> depends only on gates inside the reverse light cone
of {u, v}: B_0 = {u, v}, B_j = B_{j-1} plus its neighbours.  The circuit on
the induced subgraph G[B_p] has the same light cone (every ball of radius
<= p lies in B_p together with all its edges), so running the state vector
on G[B_p] gives the exact value with only |B_p| qubits.
"""

from __future__ import annotations

from . import statevector as sv


def ball(n: int, edges, centre, radius: int):
    """Vertices within graph distance ``radius`` of the set ``centre``."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = set(centre)
    frontier = list(centre)
    for _ in range(radius):
        nxt = []
        for a in frontier:
            for b in adj[a]:
                if b not in seen:
                    seen.add(b)
                    nxt.append(b)
        frontier = nxt
    return sorted(seen)


def induced(edges, verts):
    """Edges of G[verts] relabelled to 0..len(verts)-1, plus the map."""
    index = {v: i for i, v in enumerate(verts)}
    sub = [(index[a], index[b]) for a, b in edges if a in index and b in index]
    return sub, index


def edge_zz(n: int, edges, gammas, betas, edge, max_qubits: int = 26) -> float:
    """<Z_u Z_v> for one edge from the light-cone state vector."""
    u, v = edge
    verts = ball(n, edges, (u, v), len(gammas))
    if len(verts) > max_qubits:
        raise ValueError(f"light cone of {edge} has {len(verts)} qubits")
    sub, index = induced(edges, verts)
    psi = sv.qaoa_state(len(verts), sub, gammas, betas)
    return float(sv.zz_expectations(psi, [(index[u], index[v])])[0])


def edge_gradient(n: int, edges, gammas, betas, edge, max_qubits: int = 26):
    """(<Z_u Z_v>, d<Z_u Z_v>/d(gamma, beta)) from the light-cone state vector."""
    u, v = edge
    verts = ball(n, edges, (u, v), len(gammas))
    if len(verts) > max_qubits:
        raise ValueError(f"light cone of {edge} has {len(verts)} qubits")
    sub, index = induced(edges, verts)
    return sv.gradient(len(verts), sub, gammas, betas,
                       observable=(index[u], index[v]))


def all_edges_zz(n: int, edges, gammas, betas, max_qubits: int = 26):
    return [edge_zz(n, edges, gammas, betas, e, max_qubits) for e in edges]
