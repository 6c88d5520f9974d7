"""Exact optima of the paper's graph LPs on small inputs (pins for the MWU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  None of these routines
uses MWU: they are library LP / matching / flow solvers or brute force, so
they pin the oracle to something other than itself.

* LP optimum of any explicit LP ........................ scipy.optimize.linprog (HiGHS)
* bipartite matching LP = maximum matching ............. no integrality gap on bipartite graphs (Sec. 3, match)
* b-matching LP = max flow ............................. totally unimodular incidence matrix (Appendix A.1 with lb = 0)
* densest-subgraph LP = max density .................... Charikar's LP is exact (Sec. 3, dense-sub)
* vertex cover LP of a general graph = half the maximum matching of its bipartite double cover
* a certified lower bound on the max density of large graphs: the density of
  the best subgraph met while peeling (Bahmani, Kumar and Vassilvitskii's
  parallel peeling: each round removes every vertex of degree at most
  2 (1 + delta) times the current density; the best round is within a factor
  2 (1 + delta) of the optimum)
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog
from scipy.sparse.csgraph import maximum_bipartite_matching, maximum_flow


def _np(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(a)


def lp_packing_opt(A, c):
    """max c^T x s.t. A x <= 1, x >= 0 (HiGHS)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    r = linprog(-np.asarray(c, dtype=np.float64), A_ub=A, b_ub=np.ones(A.shape[0]),
                bounds=(0, None), method="highs")
    assert r.status == 0, r.message
    return -r.fun


def lp_covering_opt(A, c):
    """min c^T x s.t. A x >= 1, x >= 0 (HiGHS)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    r = linprog(np.asarray(c, dtype=np.float64), A_ub=-A, b_ub=-np.ones(A.shape[0]),
                bounds=(0, None), method="highs")
    assert r.status == 0, r.message
    return r.fun


def lp_densest_opt(n, u, v):
    """min D s.t. Wz >= 1, Oz <= D, z >= 0 as one LP in (z, D) (HiGHS)."""
    from . import lp as lpm
    O = lpm.pair_matrix(n, u, v)
    W = lpm.interweave(O.shape[1] // 2)
    k = O.shape[1]
    A_ub = sp.vstack([sp.hstack([-W, sp.csr_matrix((W.shape[0], 1))]),
                      sp.hstack([O, -sp.csr_matrix(np.ones((n, 1)))])]).tocsr()
    b_ub = np.concatenate([-np.ones(W.shape[0]), np.zeros(n)])
    cost = np.zeros(k + 1)
    cost[-1] = 1.0
    r = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=(0, None), method="highs")
    assert r.status == 0, r.message
    return r.fun


def bipartite_matching_size(n_left, n, u, v):
    """Maximum cardinality matching of a bipartite graph (scipy Hopcroft-Karp)."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    B = sp.csr_matrix((np.ones(u.size), (u, v - n_left)), shape=(n_left, n - n_left))
    match = maximum_bipartite_matching(B, perm_type="column")
    return int((match >= 0).sum())


def vertex_cover_lp_double_cover(n, u, v):
    """Fractional vertex cover optimum of a general graph as half the maximum
    matching of its bipartite double cover G x K2 (vertices w and w'; edges
    (u, v') and (v, u') for every edge (u, v)): the LP is half-integral, and
    this equality is a classical result (Nemhauser and Trotter)."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    uu = np.concatenate([u, v])
    vv = np.concatenate([v, u]) + n
    return bipartite_matching_size(n, 2 * n, uu, vv) / 2.0


def b_matching_size(n_left, n, u, v, b, edge_cap=None):
    """Maximum b-matching of a bipartite graph as a max flow (s -> left, left -> right, right -> t).

    The LP of Appendix A.1 bounds only the vertex sums (x >= 0, no x_e <= 1),
    so by default an edge may carry up to min(b_u, b_v), which leaves it
    unconstrained; ``edge_cap=1`` gives the simple b-matching instead.
    """
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    b = _np(b).astype(np.int64)
    s, t = n, n + 1
    rows = np.concatenate([np.full(n_left, s), u, np.arange(n_left, n)])
    cols = np.concatenate([np.arange(n_left), v, np.full(n - n_left, t)])
    ecap = np.minimum(b[u], b[v]) if edge_cap is None else np.full(u.size, edge_cap, dtype=np.int64)
    cap = np.concatenate([b[:n_left], ecap, b[n_left:]])
    G = sp.csr_matrix((cap.astype(np.int32), (rows, cols)), shape=(n + 2, n + 2))
    return int(maximum_flow(G, s, t).flow_value)


def max_density_bruteforce(n, u, v):
    """max over nonempty S of |E(S)| / |S| by enumerating all 2^n - 1 subsets (n <= 20)."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    assert n <= 20
    best = 0.0
    masks = np.arange(1, 1 << n, dtype=np.int64)
    size = np.zeros_like(masks)
    for w in range(n):
        size += (masks >> w) & 1
    inside = np.zeros_like(masks)
    for a, b in zip(u.tolist(), v.tolist()):
        inside += ((masks >> a) & 1) & ((masks >> b) & 1)
    best = float((inside / size).max())
    return best


def densest_peel_lower_bound(n, u, v, delta=0.1):
    """Density |E(S)|/|S| of the densest subgraph S met by parallel peeling: a
    lower bound on the max density (S is a real subgraph) and at least
    max density / (2 (1 + delta)).  Vectorised rounds over the edge list."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    alive = np.ones(n, dtype=bool)
    eu, ev = u, v
    best = 0.0
    while alive.any():
        nv = int(alive.sum())
        dens = eu.size / nv
        best = max(best, dens)
        if eu.size == 0:
            break
        deg = np.bincount(eu, minlength=n) + np.bincount(ev, minlength=n)
        drop = alive & (deg <= 2.0 * (1.0 + delta) * dens)
        alive &= ~drop
        keep = alive[eu] & alive[ev]
        eu, ev = eu[keep], ev[keep]
    return best


def vertex_cover_bruteforce(n, u, v, c=None):
    """Minimum-weight integral vertex cover by enumeration (n <= 20); an upper bound on the LP."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    c = np.ones(n) if c is None else _np(c).astype(np.float64)
    best = np.inf
    for mask in range(1 << n):
        ok = all(((mask >> a) & 1) or ((mask >> b) & 1) for a, b in zip(u.tolist(), v.tolist()))
        if ok:
            best = min(best, sum(c[w] for w in range(n) if (mask >> w) & 1))
    return best


def subsets(n):
    for k in range(1, n + 1):
        yield from itertools.combinations(range(n), k)


def lp_mixed_feasible(P, C):
    """Whether {x >= 0 : P x <= 1, C x >= 1} is non-empty (HiGHS, zero objective)."""
    P = sp.csr_matrix(P, dtype=np.float64)
    C = sp.csr_matrix(C, dtype=np.float64)
    A = sp.vstack([P, -C]).tocsr()
    b = np.concatenate([np.ones(P.shape[0]), -np.ones(C.shape[0])])
    r = linprog(np.zeros(P.shape[1]), A_ub=A, b_ub=b, bounds=(0, None), method="highs")
    return r.status == 0
