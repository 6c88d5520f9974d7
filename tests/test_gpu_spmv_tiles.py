"""The staged forward SpMV (tiles of rows whose input window sits in shared
memory, the CSB-like tiles of Sec. 5.1) against the oracle's products and
against the row-binned gather kernel, on the small workloads (every window
fits), on a random geometric graph (banded: tiled) and an R-MAT graph of the
same size (not banded: binned), and on a banded matrix with a few wide rows
(tiles that do not fit gather from global memory)."""
import numpy as np
import pytest
import torch

from graphgen import workloads as W
from oracle import lp as olp
from oracle import mwu as om
from tests import _helpers as H
from tests.test_gpu_parity import M, wls, make_ctx, probe_target, vec  # noqa: F401

pytestmark = pytest.mark.gpu

PRECS = ["f32", "fp64"]


def _x_for(P, C, n, prec, seed=3):
    """A positive x at which the probe still runs (max Px and min Cx below 1)."""
    rng = np.random.default_rng(seed)
    x = om.x_init(P, 0.1) * rng.uniform(1.0, 40.0, n)
    x *= min(1.0, 0.8 / max(float((P @ x).max()), float((C @ x).min())))
    return x.astype(np.float32 if prec == "f32" else np.float64)


def _check_products(M, ctx, P, C, x, prec):
    """y = Px, z = Cx on the GPU against the oracle's products of the same x."""
    M.mwu_set_x(ctx, torch.from_numpy(x).cuda())
    xo = x.astype(np.float64)
    out = {}
    for which, A, name in [(M.VEC_Y, P, "y"), (M.VEC_Z, C, "z")]:
        if A.shape[0] > 1:
            got = vec(M, ctx, which, A.shape[0])
            H.assert_rel(got, A @ xo, 2 * H.REL[prec], what=f"{name} = A x")
            out[name] = got
    return out


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["bmatch", "bmatching", "densest", "domset", "vcover", "gmatch"])
def test_tiled_equals_oracle_and_binned_on_small_workloads(M, wls, kind, prec):
    wl = wls[kind]
    T = probe_target(wl)
    P, C, _ = H.oracle_matrices(wl, T)
    x = _x_for(P, C, H.n_vars(wl), prec)
    res = {}
    for mode in [0, -1]:
        ctx = make_ctx(M, wl, prec, spmv_tiles=mode)
        try:
            tiles = M.mwu_spmv_tiles(ctx)
            csr = [wl.lp in ("bmatch", "bmatching", "densest", "gmatch"), wl.lp in ("domset", "gmatch")]
            for s in range(2):
                assert tiles[s] == 0 or (csr[s] and mode == 0), (kind, mode, tiles)
            if mode == 0 and wl.lp in ("bmatch", "bmatching", "domset"):
                assert max(tiles) > 0          # every window of these small matrices fits
            M.mwu_set_target(ctx, T)
            res[mode] = _check_products(M, ctx, P, C, x, prec)
            # dv = A d from the same x: the direction kernel is the same in both modes
            M.mwu_set_x(ctx, torch.from_numpy(x).cuda())
            M.mwu_direction(ctx)
            if P.shape[0] > 1:
                res[mode]["dy"] = vec(M, ctx, M.VEC_DY, P.shape[0])
            if C.shape[0] > 1:
                res[mode]["dz"] = vec(M, ctx, M.VEC_DZ, C.shape[0])
        finally:
            M.mwu_destroy(ctx)
    for k in res[0]:
        H.assert_rel(res[0][k], res[-1][k], 4 * H.REL[prec], floor=H.UNDERFLOW[prec], what=f"{k}: tiled vs binned")


@pytest.mark.parametrize("prec", PRECS)
def test_tiles_follow_locality(M, prec):
    """Dominating set on rgg-14 (banded: tiled) and on R-MAT 14 (not: binned)."""
    for wl, tiled in [(W.rgg_lp("domset", scale=14, seed=7), True), (W.domset(14, seed=3), False)]:
        T = 0.3 * float(wl.objective.sum())
        P, C, _ = H.oracle_matrices(wl, T)
        x = _x_for(P, C, H.n_vars(wl), prec)
        ctx = make_ctx(M, wl, prec)
        try:
            assert (M.mwu_spmv_tiles(ctx)[1] > 0) == tiled, wl.lp
            M.mwu_set_target(ctx, T)
            _check_products(M, ctx, P, C, x, prec)
        finally:
            M.mwu_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_tiles_that_do_not_fit_gather_from_global(M, prec):
    """A banded covering matrix (rows j: columns j-3..j+3) with one wide row per
    10000 (an extra column 20000 away): the tiles holding a wide row span more
    than a window, the rest fit, so the side is tiled with a few unstaged tiles."""
    n = 40000
    rows, cols = [], []
    for j in range(n):
        cs = list(range(max(0, j - 3), min(n, j + 4)))
        if j % 10000 == 0:
            cs.append((j + 20000) % n)
        cs = sorted(set(cs))
        rows.append(len(cs))
        cols.extend(cs)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(rows)
    colidx = np.array(cols, dtype=np.int32)
    from paper_2307_03307_gb300 import lpspec
    kind, P_, C_, obj = lpspec.domset_lp(n, torch.from_numpy(rowptr.astype(np.int32)).cuda(),
                                         torch.from_numpy(colidx).cuda())
    Cm = olp.csr_from_arrays(rowptr, colidx, None, (n, n))
    T = 0.3 * n
    Pm = olp.objective_row(np.ones(n), T)
    x = _x_for(Pm, Cm, n, prec)
    ctx = M.mwu_create(kind, P_, C_, obj, precision=M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64, eps=0.1)
    try:
        tiles = M.mwu_spmv_tiles(ctx)[1]
        assert tiles > 0
        M.mwu_set_target(ctx, T)
        _check_products(M, ctx, Pm, Cm, x, prec)
    finally:
        M.mwu_destroy(ctx)
