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
    if wl.lp in ("bmatch", "bmatching"):
        return bmatch_lp(g.n, e, None if wl.bounds is None else mv(wl.bounds))
    if wl.lp == "vcover":
        return vcover_lp(g.n, e, None if wl.objective is None else mv(wl.objective))
    if wl.lp == "domset":
        rp, ci = wl.csr
        return domset_lp(g.n, mv(rp), mv(ci), None if wl.objective is None else mv(wl.objective))
    if wl.lp == "densest":
        return densest_lp(g.n, e)
    raise ValueError(wl.lp)
