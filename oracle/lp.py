"""Graph -> positive LP matrices, written out explicitly from the paper's Sec. 3.

TEST INFRASTRUCTURE ONLY.  This package is the plain FP64 CPU oracle that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the library never does.

Every matrix here is a scipy CSR matrix in float64 built entry by entry from
its definition in the paper (no implicit representation): the incidence matrix
M (Eq. "incidence"), the dominating-set matrix I+A, the vertex-cover matrix
M^T, the interweaved identity W (Eq. "interweaved") and the vertex-edge pair
matrix O (Eq. "oddshifted_incidence").  Edges are given as (u[e], v[e]) with
u < v; "endpoint b" of edge e is u for b = 0 and v for b = 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _np(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(a)


def incidence(n, u, v):
    """M in {0,1}^{n x m}: M[w, e] = 1 iff vertex w is an endpoint of edge e (Sec. 3, Eq. incidence)."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    m = u.size
    rows = np.concatenate([u, v])
    cols = np.concatenate([np.arange(m), np.arange(m)])
    return sp.csr_matrix((np.ones(2 * m), (rows, cols)), shape=(n, m))


def adjacency(n, u, v):
    """Symmetric adjacency A in {0,1}^{n x n} of the simple graph."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    return sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(n, n))


def dominating(n, u, v):
    """I + A, the covering matrix of the dominating-set LP (Sec. 3, dom-set)."""
    return (sp.identity(n, format="csr") + adjacency(n, u, v)).tocsr()


def interweave(m):
    """W in {0,1}^{m x 2m}: W[e, 2e] = W[e, 2e+1] = 1 (Sec. 3, Eq. interweaved).

    The paper prints the shape as n x 2m; one row per edge makes it m x 2m.
    """
    rows = np.repeat(np.arange(m), 2)
    cols = np.arange(2 * m)
    return sp.csr_matrix((np.ones(2 * m), (rows, cols)), shape=(m, 2 * m))


def pair_matrix(n, u, v):
    """O in {0,1}^{n x 2m}: O[w, 2e+b] = 1 iff w is endpoint b of e (Sec. 3, Eq. oddshifted_incidence)."""
    u, v = _np(u).astype(np.int64), _np(v).astype(np.int64)
    m = u.size
    rows = np.empty(2 * m, dtype=np.int64)
    rows[0::2] = u
    rows[1::2] = v
    cols = np.arange(2 * m)
    return sp.csr_matrix((np.ones(2 * m), (rows, cols)), shape=(n, 2 * m))


def objective_row(c, M):
    """The single row (1/M) c^T that embeds an objective as a constraint (Sec. 2.2, pure packing/covering)."""
    c = _np(c).astype(np.float64)
    return sp.csr_matrix(c.reshape(1, -1) / float(M))


def row_scaled(A, b):
    """diag(1/b) A: turns A x <= b into a <= 1 constraint (Appendix A.1 upper bounds)."""
    b = _np(b).astype(np.float64)
    return sp.diags(1.0 / b).dot(A).tocsr()


def csr_from_arrays(rowptr, colidx, val, shape):
    """Explicit CSR given by arrays (values None means all ones), as float64."""
    rowptr = _np(rowptr).astype(np.int64)
    colidx = _np(colidx).astype(np.int64)
    vals = np.ones(colidx.size) if val is None else _np(val).astype(np.float64)
    return sp.csr_matrix((vals, colidx, rowptr), shape=shape)
