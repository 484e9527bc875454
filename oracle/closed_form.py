"""Closed form of <Z_u Z_v> for depth-1 QAOA on any graph.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For p = 1 the Heisenberg-picture expansion of Z_u Z_v truncates after the
neighbours of u and v and gives (Wang, Hadfield, Jiang and Rieffel, Phys.
Rev. A 97, 022304 (2018), Theorem 1, restated for the phase gate
exp(-i gamma Z Z / 2) and mixer exp(-i beta X) of Section 4.1; their
exp(-i gamma C) convention is gamma -> -gamma here):

  <Z_u Z_v> = 1/2 sin(4 beta) sin(gamma) (cos^{d_u-1} gamma + cos^{d_v-1} gamma)
            + 1/2 sin^2(2 beta) cos^{d_u+d_v-2-2 lam} gamma (1 - cos^{lam}(2 gamma))

with d_u, d_v the degrees of u and v and lam the number of triangles that
contain the edge (u, v).  The derivatives below are those of this
expression, written out term by term.
"""

from __future__ import annotations

import math


def edge_params(n, edges, edge):
    """(d_u, d_v, lam) of one edge."""
    nbr = [set() for _ in range(n)]
    for a, b in edges:
        nbr[a].add(b)
        nbr[b].add(a)
    u, v = edge
    return len(nbr[u]), len(nbr[v]), len((nbr[u] & nbr[v]) - {u, v})


def _pow(x, k):
    return x ** k if k != 0 else 1.0


def zz_p1(gamma, beta, du, dv, lam):
    cg, sg = math.cos(gamma), math.sin(gamma)
    e = du + dv - 2 - 2 * lam
    a = _pow(cg, du - 1) + _pow(cg, dv - 1)
    f = _pow(cg, e) * (1.0 - _pow(math.cos(2 * gamma), lam))
    return 0.5 * math.sin(4 * beta) * sg * a + 0.5 * math.sin(2 * beta) ** 2 * f


def zz_p1_grad(gamma, beta, du, dv, lam):
    """(d/d gamma, d/d beta) of zz_p1."""
    cg, sg = math.cos(gamma), math.sin(gamma)
    c2 = math.cos(2 * gamma)
    e = du + dv - 2 - 2 * lam
    a = _pow(cg, du - 1) + _pow(cg, dv - 1)
    da = -((du - 1) * _pow(cg, du - 2) + (dv - 1) * _pow(cg, dv - 2)) * sg
    f = _pow(cg, e) * (1.0 - _pow(c2, lam))
    df = (-e * _pow(cg, e - 1) * sg * (1.0 - _pow(c2, lam))
          + _pow(cg, e) * lam * _pow(c2, lam - 1) * 2.0 * math.sin(2 * gamma))
    s4, s2 = math.sin(4 * beta), math.sin(2 * beta)
    d_gamma = 0.5 * s4 * (cg * a + sg * da) + 0.5 * s2 * s2 * df
    d_beta = 2.0 * math.cos(4 * beta) * sg * a + s4 * f
    return d_gamma, d_beta


def maxcut_p1(n, edges, gamma, beta):
    """<C> = sum_e (1 - <Z_u Z_v>)/2 at p = 1."""
    return sum((1.0 - zz_p1(gamma, beta, *edge_params(n, edges, e))) / 2.0
               for e in edges)


def maxcut_p1_grad(n, edges, gamma, beta):
    """(d<C>/d gamma, d<C>/d beta) at p = 1."""
    g = b = 0.0
    for e in edges:
        dg, db = zz_p1_grad(gamma, beta, *edge_params(n, edges, e))
        g -= 0.5 * dg
        b -= 0.5 * db
    return g, b
