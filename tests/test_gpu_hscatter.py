"""The scatter forms against the oracle: h = C^T w_c by one pass over C's rows
with atomic adds (option h_scatter; vertex cover's edge rows, the explicit CSR
rows of dominating set and of generalized matching's lower bounds), and
dz = C d by a scatter over the columns of the moving variables (option
dv_scatter; explicit CSR covering sides).  One
iteration's quantities from the oracle chain, and whole solves against the
exact LP and the oracle's solve.  The sums' order varies, so the bounds are
those of the gather form (propagated FP32 error), not bit equality."""
import numpy as np
import pytest

from oracle import mwu as om
from tests import _helpers as H
from tests.test_gpu_parity import (M, wls, make_ctx, probe_target, vec, run_direction_checks,  # noqa: F401
                                   Chain, check_step_decision, certificate_from_x, exact_opt)

pytestmark = pytest.mark.gpu


SCATTER = {"h": dict(h_scatter=1), "dv": dict(dv_scatter=1), "h+dv": dict(h_scatter=1, dv_scatter=1)}


@pytest.mark.parametrize("prec", ["f32", "fp64"])
@pytest.mark.parametrize("kind,opts", [("vcover", "h"), ("domset", "h"), ("gmatch", "h"),
                                       ("domset", "dv"), ("gmatch", "dv"), ("domset", "h+dv")])
def test_h_scatter_iteration_matches_oracle(M, wls, kind, opts, prec):
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec, **SCATTER[opts])
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        ch = Chain(wl, prec, T)
        for _ in range(2):   # twice: k_dir clears the sums for the next direction
            e = run_direction_checks(M, ctx, wl, prec, ch)
        rc, alpha, ev = M.mwu_search(ctx)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_kary(ch.evaluate, wl.eps, K=K, max_passes=6 if K == 8 else 64)
        check_step_decision(ch, e, prec, alpha, ao)
    finally:
        M.mwu_destroy(ctx)


@pytest.mark.parametrize("step", ["kary", "newton"])
@pytest.mark.parametrize("prec", ["f32", "fp64"])
@pytest.mark.parametrize("kind,opts", [("vcover", "h"), ("domset", "h"), ("domset", "h+dv")])
def test_h_scatter_solve_matches_oracle_and_exact(M, wls, kind, opts, prec, step):
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY, **SCATTER[opts])
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, H.n_vars(wl))
    finally:
        M.mwu_destroy(ctx)
    cert = certificate_from_x(wl, x)
    assert cert == pytest.approx(res["objective"], rel=1e-4)
    opt = exact_opt(wl)
    assert opt * (1 - 1e-9) <= cert <= opt * (1 + wl.eps) ** 2
    ores = H.oracle_solve(wl, step=step)
    assert 1 / (1 + wl.eps) <= cert / ores.objective <= 1 + wl.eps
