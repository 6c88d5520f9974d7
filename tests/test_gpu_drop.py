"""Active-set dropping of satisfied covering rows on the GPU against the oracle.

Alg. 1 and Alg. 2 end each iteration with C <- {c_j : c_j^T x < 1}; the
option ``drop_covered`` runs that step (rows with z_j >= 1 leave smin, h, Phi,
Phi' and the early exit).  The chain below starts from an x at which a good
share of the covering rows is already satisfied while the probe still runs,
and every quantity of one iteration is compared with the oracle's, which
restricts C to the active rows itself.
"""
import math

import numpy as np
import pytest
import torch

from tests import _helpers as H
from oracle import exact, mwu as om
from tests.test_gpu_parity import (M, wls, make_ctx, probe_target, vec, run_direction_checks, cand_bounds,  # noqa: F401
                             check_step_decision, certificate_from_x, exact_opt, GRAD_TOL)

pytestmark = pytest.mark.gpu

DROP_KINDS = ["densest", "domset", "vcover", "gmatch"]
PRECS = ["f32", "fp64"]


def drop_target(wl):
    """A feasible probe target (the densest probe of the other tests is infeasible)."""
    return probe_target(wl) * (2.0 if wl.lp == "densest" else 1.0)


class DropChain:
    """One oracle iteration with dropped rows, from an x the oracle itself
    reaches: the iterate of an oracle run with dropping (K-candidate steps)
    at which the dropped rows carry the largest share of the smin weights
    while the probe still runs.  Dropping changes h and Phi most there.  x is
    scaled by 1 +- a few 1e-5 until no row lies within 2e-5 of 1, so that
    both sides classify every row alike."""

    def __init__(self, wl, prec, T):
        P, C, _ = H.oracle_matrices(wl, T)
        self.P, self.C = P, C
        self.mP, self.mC = P.shape[0], C.shape[0]
        self.n = H.n_vars(wl)
        self.eta = om.eta_of(self.mP + self.mC, wl.eps)
        self.c_d = om.step_coefficient(self.mP, self.mC, self.eta)
        best = [-1.0, None]

        def on_iter(it, x, y, z, a):
            act = z < 1.0
            if act.any() and (~act).any() and y.max() <= 1 + wl.eps:
                w = np.exp(-self.eta * (z - z.min()))
                share = float(w[~act].sum() / w.sum())
                if share > best[0]:
                    best[0], best[1] = share, x.copy()

        om.mwu(P, C, wl.eps, step="kary", drop_covered=True, on_iter=on_iter)
        assert best[1] is not None, "no running iterate with dropped rows"
        self.share = best[0]
        dt = np.float32 if prec == "f32" else np.float64
        for f in [1.0, 1 - 3e-5, 1 + 3e-5, 1 - 9e-5, 1 + 9e-5, 1 - 2.7e-4, 1 + 2.7e-4]:
            x = (best[1] * f).astype(dt)
            z = C @ x.astype(np.float64)
            if np.abs(z - 1.0).min() > 2e-5 and (P @ x.astype(np.float64)).max() <= 1 + wl.eps and z.min() < 1:
                break
        else:
            pytest.skip("every scaled iterate has a row within 2e-5 of 1")
        self.x = x
        xo = self.x.astype(np.float64)
        self.xo = xo
        self.y, self.z = P @ xo, C @ xo
        self.act = self.z < 1.0
        Ca = C[np.flatnonzero(self.act)]
        self.za = self.z[self.act]
        self.g, self.h = om.gradients(P, Ca, self.y, self.za, self.eta)
        self.d = om.direction(self.g, self.h, xo, self.c_d, GRAD_TOL[prec])
        self.dy, self.dz = P @ self.d, C @ self.d
        self.dza = self.dz[self.act]
        self.evaluate = om.make_evaluator(self.y, self.dy, self.za, self.dza, self.eta)
        self.evaluate_nd = om.make_newton_evaluator(self.y, self.dy, self.za, self.dza, self.eta)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", DROP_KINDS)
def test_drop_iteration_matches_oracle(M, wls, kind, prec):
    wl = wls[kind]
    rel = H.REL[prec]
    ctx = make_ctx(M, wl, prec, drop_covered=1)
    try:
        T = drop_target(wl)
        M.mwu_set_target(ctx, T)
        ch = DropChain(wl, prec, T)
        assert ch.share > 1e-9 and (~ch.act).any()
        e = run_direction_checks(M, ctx, wl, prec, ch)
        # the stopping test reads min z over every row
        assert M.mwu_get_scalars(ctx)["zmin"] == pytest.approx(float(ch.z.min()), rel=rel)
        # variables whose covering rows are all dropped do not move
        frozen = ch.h == 0.0
        assert (e["d"][frozen] == 0.0).all()
        # Phi over the active rows; min z + alpha dz over them
        alphas = [1.0, 2.0, 4.0, 16.0, 128.0, 1000.0, 3.0e4, 1.5]
        psi, phi, zmn = M.mwu_eval_candidates(ctx, alphas)
        ez = float(np.abs(e["z"] - ch.z).max())
        for k, a in enumerate(alphas):
            bpsi, bphi = cand_bounds(ch, e, a, prec)
            H.assert_rel([psi[k]], [om.Psi(ch.y, ch.dy, a, ch.eta)], rel, abs_=bpsi, what=f"Psi({a})")
            H.assert_rel([phi[k]], [om.Phi(ch.za, ch.dza, a, ch.eta)], rel, abs_=bphi, what=f"Phi({a})")
            H.assert_rel([zmn[k]], [float((ch.za + a * ch.dza).min())], rel,
                         abs_=1.05 * (ez + a * e["edz"]), what=f"min z({a})")
        rc, alpha, ev = M.mwu_search(ctx)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_kary(ch.evaluate, wl.eps, K=K, max_passes=6 if K == 8 else 64)
        check_step_decision(ch, e, prec, alpha, ao)
    finally:
        M.mwu_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", DROP_KINDS)
def test_drop_newton_search_matches_oracle(M, wls, kind, prec):
    """The Newton search over the active rows, including its early exit with
    the smallest covering step when a warm start covers every row."""
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec, drop_covered=1, step=M.STEP_NEWTON)
    try:
        T = drop_target(wl)
        M.mwu_set_target(ctx, T)
        ch = DropChain(wl, prec, T)
        e = run_direction_checks(M, ctx, wl, prec, ch)
        rc, alpha, ev = M.mwu_search(ctx)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_newton(ch.evaluate_nd, ch.evaluate, wl.eps, K=K, alpha0=None,
                                    max_passes=16 if K == 8 else 64)
        if info.early and ao == max(1.0, ch.evaluate_nd.alpha_cover()):
            # the covering step alpha_c: continuous in z and dz
            ac = ch.evaluate_nd.alpha_cover()
            bd = 1.05 * (e["ez"] + ac * e["edz"]) / max(float(ch.dza[ch.dza > 0].min()), 1e-300)
            assert abs(alpha - ao) <= 4 * H.REL[prec] * ao + bd, (alpha, ao)
        else:
            check_step_decision(ch, e, prec, alpha, ao, rel_gap=2 * wl.eps / 20 + 1e-3)
    finally:
        M.mwu_destroy(ctx)


@pytest.mark.parametrize("step", ["kary", "newton"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["densest", "domset", "vcover"])
def test_drop_solve_matches_oracle_and_exact(M, wls, kind, prec, step):
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec, drop_covered=1, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, H.n_vars(wl))
    finally:
        M.mwu_destroy(ctx)
    assert (x >= 0).all()
    cert = certificate_from_x(wl, x)
    assert cert == pytest.approx(res["objective"], rel=1e-4)
    opt = exact_opt(wl)
    assert opt * (1 - 1e-9) <= cert <= opt * (1 + wl.eps) ** 2
    ores = H.oracle_solve(wl, step=step, drop_covered=True)
    assert 1 / (1 + wl.eps) <= cert / ores.objective <= 1 + wl.eps, (cert, ores.objective)


def test_drop_potential_takes_every_row(M, wls):
    """The potential is that of Sec. 4.1 over all rows whatever the option says,
    and the context's sums return to the active rows after it."""
    wl = wls["densest"]
    T = drop_target(wl)
    ch = DropChain(wl, "f32", T)
    assert ch.share > 0.1
    vals = []
    for drop in [0, 1]:
        ctx = make_ctx(M, wl, "f32", drop_covered=drop)
        try:
            M.mwu_set_target(ctx, T)
            xs = torch.from_numpy(ch.x).cuda()
            gx = torch.empty_like(xs)
            vals.append(M.mwu_potential(ctx, xs, gx, None, None))
            sc = M.mwu_get_scalars(ctx)
            z = ch.za if drop else ch.z
            s_c, S_c = om.lse_shift_sum(z, ch.eta, -1)
            assert sc["S_c"] == pytest.approx(S_c, rel=1e-3)
            assert sc["zmin"] == pytest.approx(float(ch.z.min()), rel=1e-6)
        finally:
            M.mwu_destroy(ctx)
    assert vals[0] == pytest.approx(vals[1], rel=1e-12)
    S_all = om.lse_shift_sum(ch.z, ch.eta, -1)[1]
    S_act = om.lse_shift_sum(ch.za, ch.eta, -1)[1]
    assert S_all > 1.1 * S_act            # the two sums differ: the check above is not vacuous


@pytest.mark.parametrize("step", ["kary", "newton"])
@pytest.mark.parametrize("prec", PRECS)
def test_compacted_probe_restores_the_rows(M, prec, step):
    """drop_covered = 1 on the vertex-cover split view compacts the unsatisfied
    edges inside mwu_iterate (the last step of Alg. 1/2 as a stream
    compaction).  On return every z equals x_u + x_v in the form's precision,
    the rows dropped earlier included, zmin is the minimum over every row, and
    the probe ends as the masked form (drop_covered = 2) ends it."""
    from graphgen import workloads as W
    wl = W.vcover(12, seed=21)
    g = wl.graph
    u, v = g.u.numpy().astype(np.int64), g.v.numpy().astype(np.int64)
    T = 1.03 * exact_opt(wl)        # feasible, near the optimum: a long probe in which most edges are met
    out = {}
    for drop in (1, 2):
        ctx = make_ctx(M, wl, prec, drop_covered=drop, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY)
        try:
            M.mwu_set_target(ctx, T)
            rc, st = M.mwu_iterate(ctx, 5000)
            x = vec(M, ctx, M.VEC_X, g.n)
            z = vec(M, ctx, M.VEC_Z, g.m)
            out[drop] = (rc, st, x, z, M.mwu_get_scalars(ctx), M.mwu_get_timing(ctx))
        finally:
            M.mwu_destroy(ctx)
    rc, st, x, z, sc, tim = out[1]
    assert tim["compactions"] >= 1 and out[2][5]["compactions"] == 0
    dt = np.float32 if prec == "f32" else np.float64
    xs = x.astype(dt)
    zx = (xs[u] + xs[v]).astype(np.float64)
    assert np.array_equal(np.sort(z), np.sort(zx))           # the context's row order is its own
    assert sc["zmin"] == float(zx.min())
    assert rc == out[2][0] == M.FEASIBLE
    if sc["zmin"] >= 1.0:                                   # the stopping test on the exact rows
        assert sc["ymax"] <= (1 + wl.eps) * sc["zmin"]
    it1, it2 = st["iters"], out[2][1]["iters"]
    assert abs(it1 - it2) <= 0.1 * max(it1, it2) + 2, (it1, it2)


@pytest.mark.parametrize("prec", PRECS)
def test_compacted_solve_matches_oracle_and_exact(M, prec):
    from graphgen import workloads as W
    wl = W.vcover(12, seed=21)
    ctx = make_ctx(M, wl, prec, drop_covered=1)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, H.n_vars(wl))
        assert M.mwu_get_timing(ctx)["compactions"] >= 1
    finally:
        M.mwu_destroy(ctx)
    cert = certificate_from_x(wl, x)
    assert cert == pytest.approx(res["objective"], rel=1e-4)
    opt = exact_opt(wl)
    assert opt * (1 - 1e-9) <= cert <= opt * (1 + wl.eps) ** 2
    ores = H.oracle_solve(wl, drop_covered=True)
    assert 1 / (1 + wl.eps) <= cert / ores.objective <= 1 + wl.eps, (cert, ores.objective)


def test_drop_covered_rejects_other_values(M, wls):
    with pytest.raises(M.MWUError) as e:
        make_ctx(M, wls["vcover"], "f32", drop_covered=3)
    assert e.value.code == M.ERR_INVALID


def test_compacted_probe_eager_launches(M):
    """The compaction between host-launched iterations (use_graph = 0) follows
    the captured-graph form: the same iterates, status and restored rows."""
    from graphgen import workloads as W
    wl = W.vcover(12, seed=21)
    g = wl.graph
    u, v = g.u.numpy().astype(np.int64), g.v.numpy().astype(np.int64)
    T = 1.03 * exact_opt(wl)
    out = {}
    for graph in (0, 1):
        ctx = make_ctx(M, wl, "f32", drop_covered=1, use_graph=graph)
        try:
            M.mwu_set_target(ctx, T)
            rc, st = M.mwu_iterate(ctx, 5000)
            out[graph] = (rc, st["iters"], vec(M, ctx, M.VEC_X, g.n), vec(M, ctx, M.VEC_Z, g.m),
                          M.mwu_get_timing(ctx)["compactions"])
        finally:
            M.mwu_destroy(ctx)
    rc, it, x, z, nc = out[0]
    assert nc >= 1 and rc == out[1][0] and it == out[1][1]
    assert np.array_equal(x, out[1][2])
    xs = x.astype(np.float32)
    assert np.array_equal(np.sort(z), np.sort((xs[u] + xs[v]).astype(np.float64)))
