"""Marshalling of the paper's graph LPs (Sec. 3) into mwu_create arguments.

Each function returns ``(kind, P, C, objective)`` for ``mwu.mwu_create``; the
matrices are descriptors over the caller's arrays (implicit incidence/pair/
interweave views over an int32 edge list, Sec. 5.1.2, or an explicit CSR).
"""
from __future__ import annotations

from . import mwu as M


def _edges(edges):
    return edges.contiguous()


def bmatch_lp(n_vertices, edges, bounds=None):
    """max <1, x> s.t. M x <= b (b = 1 unless given): matching / b-matching (Sec. 3, Appendix A.1)."""
    P = M.implicit_matrix(M.MAT_INCIDENCE, _edges(edges), n_vertices, row_bound=bounds)
    return M.PACKING, P, None, None


def vcover_lp(n_vertices, edges, objective=None):
    """min <c, x> s.t. M^T x >= 1 (Sec. 3, vcover)."""
    C = M.implicit_matrix(M.MAT_INCIDENCE_T, _edges(edges), n_vertices)
    return M.COVERING, None, C, objective


def domset_lp(n_vertices, rowptr, colidx, objective=None, val=None):
    """min <c, x> s.t. (I + A) x >= 1 with I + A an explicit CSR (Sec. 3, dom-set)."""
    C = M.csr_matrix(rowptr.contiguous(), colidx.contiguous(), val, n_vertices, n_vertices)
    return M.COVERING, None, C, objective


def gmatch_lp(n_vertices, edges, upper, lower, n_left):
    """Generalized matching (Appendix A.1): find x >= 0 with diag(1/ub) M x <= 1 and
    diag(1/lb) M_L x >= 1, M the vertex-edge incidence and M_L its rows of the
    left vertices 0..n_left-1 (those with a lower bound).  The edges must be
    sorted with the left endpoint first (graphgen's canonical order), so that
    left vertex u's edges are contiguous: M_L is a CSR over edge ids."""
    import torch
    e = _edges(edges)
    P = M.implicit_matrix(M.MAT_INCIDENCE, e, n_vertices, row_bound=upper)
    left = e[:, 0].long()
    counts = torch.bincount(left, minlength=n_left)
    rowptr = torch.zeros(n_left + 1, dtype=torch.int64, device=e.device)
    rowptr[1:] = torch.cumsum(counts, 0)
    colidx = torch.arange(e.shape[0], dtype=torch.int32, device=e.device)
    C = M.csr_matrix(rowptr.to(torch.int32), colidx, None, n_left, e.shape[0], row_bound=lower)
    return M.MIXED, P, C, None


def densest_lp(n_vertices, edges):
    """min D s.t. W z >= 1, O z <= D (Sec. 3, Eq. densest_linalg)."""
    e = _edges(edges)
    P = M.implicit_matrix(M.MAT_PAIR, e, n_vertices)
    C = M.implicit_matrix(M.MAT_INTERWEAVE, e, n_vertices)
    return M.DENSEST, P, C, None


def from_workload(wl, device=None):
    """(kind, P, C, objective) of a graphgen workload; arrays moved to ``device`` if given."""
    g = wl.graph
    mv = (lambda t: t.to(device)) if device is not None else (lambda t: t)
    e = mv(wl.edges)
    if wl.lp in ("bmatch", "bmatching", "matching"):
        return bmatch_lp(g.n, e, None if wl.bounds is None else mv(wl.bounds))
    if wl.lp == "vcover":
        return vcover_lp(g.n, e, None if wl.objective is None else mv(wl.objective))
    if wl.lp == "domset":
        rp, ci = wl.csr
        return domset_lp(g.n, mv(rp), mv(ci), None if wl.objective is None else mv(wl.objective))
    if wl.lp == "densest":
        return densest_lp(g.n, e)
    if wl.lp == "gmatch":
        return gmatch_lp(g.n, e, mv(wl.bounds), mv(wl.lower), g.n_left)
    raise ValueError(wl.lp)
