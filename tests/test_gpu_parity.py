"""Parity of every hot-path step of the CUDA library with the FP64 CPU oracle.

Each step is fed the same inputs on both sides (the FP32 vectors the GPU
produced, widened to FP64 for the oracle) and compared element by element:
relative 1e-5 for the FP32 form and 1e-12 for the FP64 form, with the
allowances for gradient-test flips and step decisions derived in the design doc.
"""
import math

import numpy as np
import pytest
import torch

from oracle import exact
from oracle import lp as olp
from oracle import mwu as om
from tests import _helpers as H

pytestmark = pytest.mark.gpu

KINDS = ["bmatch", "bmatching", "densest", "domset", "vcover"]
PRECS = ["f32", "fp64"]


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03307_gb300 import _build
    _build.build()
    from paper_2307_03307_gb300 import mwu
    mwu.load()
    return mwu


@pytest.fixture(scope="module")
def wls():
    return H.small_workloads()


def make_ctx(M, wl, prec, **opts):
    from paper_2307_03307_gb300 import lpspec
    kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
    p = M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64
    return M.mwu_create(kind, P, C, obj, precision=p, eps=wl.eps, **opts)


def probe_target(wl):
    g = wl.graph
    if wl.lp == "bmatch":
        return 0.6 * g.n_left
    if wl.lp == "bmatching":
        return 0.6 * float(wl.bounds[: g.n_left].sum())
    if wl.lp == "densest":
        return 1.5 * g.m / g.n
    if wl.lp == "vcover":
        return 0.55 * g.n
    if wl.lp == "domset":
        return 0.3 * float(wl.objective.sum())


def vec(M, ctx, which, n):
    return M.mwu_get_vector(ctx, which, n, fp64=True).numpy()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", KINDS)
def test_iteration_steps_match_oracle(M, wls, kind, prec):
    wl = wls[kind]
    rel = H.REL[prec]
    ctx = make_ctx(M, wl, prec)
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        P, C, c = H.oracle_matrices(wl, T)
        n = H.n_vars(wl)
        sc = M.mwu_get_scalars(ctx)
        mP, mC = P.shape[0], C.shape[0]
        eta = om.eta_of(mP + mC, wl.eps)
        assert sc["eta"] == pytest.approx(eta, rel=1e-15)
        assert sc["c_d"] == pytest.approx(om.step_coefficient(mP, mC, eta), rel=1e-15)
        # a0: initial x
        x0 = vec(M, ctx, M.VEC_X, n)
        H.assert_rel(x0, om.x_init(P, wl.eps), 1e-7 if prec == "f32" else 1e-15, what="x0")
        # a state away from x0 so that the weights are not uniform
        rng = np.random.default_rng(7)
        dt = np.float32 if prec == "f32" else np.float64
        x = x0 * rng.uniform(1.0, 40.0, n)
        # keep the probe running: max(Px) and min(Cx) below 1
        f = 0.8 / max(float((P @ x).max()), float((C @ x).min()))
        x = (x * min(1.0, f)).astype(dt)
        M.mwu_set_x(ctx, torch.from_numpy(x).cuda())
        xo = x.astype(np.float64)
        # a1: y = Px, z = Cx
        y = vec(M, ctx, M.VEC_Y, mP)
        z = vec(M, ctx, M.VEC_Z, mC)
        H.assert_rel(y, P @ xo, rel, what="y=Px")
        H.assert_rel(z, C @ xo, rel, what="z=Cx")
        # a2, a3: shifted LSE of the same y, z
        sc = M.mwu_get_scalars(ctx)
        s_p, S_p = om.lse_shift_sum(y, eta, +1)
        s_c, S_c = om.lse_shift_sum(z, eta, -1)
        assert sc["s_p"] == s_p and sc["s_c"] == s_c
        H.assert_rel([sc["S_p"], sc["S_c"]], [S_p, S_c], rel, what="S")
        # a4, a5: gradients and direction
        rc, npos = M.mwu_direction(ctx)
        assert rc == M.OK
        g = vec(M, ctx, M.VEC_G, n)
        h = vec(M, ctx, M.VEC_H, n)
        d = vec(M, ctx, M.VEC_D, n)
        go, ho = om.gradients(P, C, y, z, eta)
        H.assert_rel(g, go, rel, what="g=P^T w_p", floor=H.UNDERFLOW[prec])
        H.assert_rel(h, ho, rel, what="h=C^T w_c", floor=H.UNDERFLOW[prec])
        c_d = sc["c_d"]
        do = om.direction(go, ho, xo, c_d)
        r = np.where(ho > 0, go / np.where(ho > 0, ho, 1), np.inf)
        band = np.abs(1.0 - r) < 10 * rel
        # variables whose g and h are both below the representable range carry no decision
        tiny = (ho <= H.UNDERFLOW[prec] * ho.max()) & (go <= H.UNDERFLOW[prec] * max(go.max(), 1e-300))
        band |= tiny
        flips = (d > 0) != (do > 0)
        assert not (flips & ~band).any(), "gradient test differs outside the rounding band"
        agree = ~flips
        tol = c_d * xo * (4 * rel * np.minimum(r, 1e6)) + rel * np.abs(do) + 1e-300
        assert (np.abs(d - do)[agree] <= tol[agree]).all(), "d magnitude"
        assert npos == int((d > 0).sum())
        assert np.dot(ho, d) >= np.dot(go, d) * (1 - 10 * rel)   # Lagrangian condition on the GPU's d
        # a6: dy = Pd, dz = Cd on the same d
        dy = vec(M, ctx, M.VEC_DY, mP)
        dz = vec(M, ctx, M.VEC_DZ, mC)
        H.assert_rel(dy, P @ d, rel, abs_=1e-300, what="dy=Pd")
        H.assert_rel(dz, C @ d, rel, abs_=1e-300, what="dz=Cd")
        # a7: candidates on the same y, dy, z, dz
        alphas = [1.0, 2.0, 4.0, 16.0, 128.0, 1000.0, 3.0e4, 1.5]
        psi, phi, zmn = M.mwu_eval_candidates(ctx, alphas)
        for k, a in enumerate(alphas):
            pw = om.Psi(y, dy, a, eta)
            pf = om.Phi(z, dz, a, eta)
            # the oracle's own FP64 cancellation error in a difference of two LSEs
            fl = 1e-14 * (1 + abs(om.smax(y, eta)) + abs(om.smin(z, eta)))
            H.assert_rel([psi[k]], [pw], rel, abs_=fl + (1e-8 / eta if prec == "f32" else 0), what=f"Psi({a})")
            H.assert_rel([phi[k]], [pf], rel, abs_=fl + (1e-8 / eta if prec == "f32" else 0), what=f"Phi({a})")
            H.assert_rel([zmn[k]], [float((z + a * dz).min())], rel, what=f"min z({a})")
        # the step-size search on the same vectors
        rc, alpha, ev = M.mwu_search(ctx)
        evaluate = om.make_evaluator(y, dy, z, dz, eta)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_kary(evaluate, wl.eps, K=K, max_passes=6 if K == 8 else 64)
        if alpha != ao:
            # only a decision inside the rounding band may differ: check f at both
            for a in (alpha, ao):
                if a >= 1:
                    f = om.Phi(z, dz, a, eta) / om.Psi(y, dy, a, eta)
                    assert abs(f - 1) < 1e-3 or (a == alpha and f >= 1 - 1e-4), (alpha, ao, f)
        # a8: one full iteration from the same x reproduces x + alpha d, y + alpha dy, z + alpha dz
        M.mwu_set_x(ctx, torch.from_numpy(x).cuda())
        rc, st = M.mwu_iterate(ctx, 1)
        a1 = st["alpha"]
        if st["iters"] == 1:
            x1 = vec(M, ctx, M.VEC_X, n)
            y1 = vec(M, ctx, M.VEC_Y, mP)
            z1 = vec(M, ctx, M.VEC_Z, mC)
            H.assert_rel(x1, xo + a1 * d, 4 * rel, abs_=1e-300, what="x update")
            if mP > 1:
                H.assert_rel(y1, y + a1 * dy, 4 * rel, what="y update")
            if mC > 1:
                H.assert_rel(z1, z + a1 * dz, 4 * rel, what="z update")
    finally:
        M.mwu_destroy(ctx)


def exact_opt(wl):
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    if wl.lp == "bmatch":
        return exact.bipartite_matching_size(g.n_left, g.n, u, v)
    if wl.lp == "bmatching":
        return exact.b_matching_size(g.n_left, g.n, u, v, wl.bounds.numpy())
    if wl.lp == "vcover":
        return exact.lp_covering_opt(olp.incidence(g.n, u, v).T.tocsr(), np.ones(g.n))
    if wl.lp == "domset":
        return exact.lp_covering_opt(olp.dominating(g.n, u, v), wl.objective.numpy().astype(np.float64))
    if wl.lp == "densest":
        return exact.lp_densest_opt(g.n, u, v)


def certificate_from_x(wl, x):
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    if wl.lp in ("bmatch", "bmatching"):
        A = olp.incidence(g.n, u, v)
        if wl.bounds is not None:
            A = olp.row_scaled(A, wl.bounds.numpy())
        return om.certified_packing(A, np.ones(g.m), x)
    if wl.lp == "vcover":
        return om.certified_covering(olp.incidence(g.n, u, v).T.tocsr(), np.ones(g.n), x)
    if wl.lp == "domset":
        return om.certified_covering(olp.dominating(g.n, u, v), wl.objective.numpy().astype(np.float64), x)
    if wl.lp == "densest":
        return om.certified_densest(olp.pair_matrix(g.n, u, v), olp.interweave(g.m), x)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", KINDS)
def test_solve_matches_oracle_and_exact(M, wls, kind, prec):
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, H.n_vars(wl))
    finally:
        M.mwu_destroy(ctx)
    assert (x >= 0).all()
    cert = certificate_from_x(wl, x)
    assert cert == pytest.approx(res["objective"], rel=1e-4)
    opt = exact_opt(wl)
    tol2 = (1 + wl.eps) ** 2
    if wl.lp in ("bmatch", "bmatching"):
        assert opt / tol2 <= cert <= opt * (1 + 1e-9)
    else:
        assert opt * (1 - 1e-9) <= cert <= opt * tol2
    ores = H.oracle_solve(wl)
    ratio = cert / ores.objective
    assert 1 / (1 + wl.eps) <= ratio <= 1 + wl.eps, (cert, ores.objective)


def test_invalid_inputs_are_rejected(M):
    from paper_2307_03307_gb300 import lpspec
    e = torch.tensor([[0, 1], [1, 2], [2, 2]], dtype=torch.int32)      # self loop
    kind, P, C, obj = lpspec.bmatch_lp(3, e)
    with pytest.raises(M.MWUError) as ei:
        M.mwu_create(kind, P, C, obj)
    assert ei.value.code == M.ERR_INVALID and "self loop" in str(ei.value)
    e = torch.tensor([[0, 1], [1, 7]], dtype=torch.int32)              # out of range
    kind, P, C, obj = lpspec.vcover_lp(3, e)
    with pytest.raises(M.MWUError):
        M.mwu_create(kind, P, C, obj)
    rp = torch.tensor([0, 2, 3, 3], dtype=torch.int32)                 # empty covering row
    ci = torch.tensor([0, 1, 1], dtype=torch.int32)
    kind, P, C, obj = lpspec.domset_lp(3, rp, ci)
    with pytest.raises(M.MWUError) as ei:
        M.mwu_create(kind, P, C, obj)
    assert "empty covering row" in str(ei.value)
    rp = torch.tensor([0, 2, 3, 4], dtype=torch.int32)
    ci = torch.tensor([0, 1, 1, 2], dtype=torch.int32)
    val = torch.tensor([1.0, -1.0, 1.0, 1.0])                          # negative value
    kind, P, C, obj = lpspec.domset_lp(3, rp, ci, val=val)
    with pytest.raises(M.MWUError):
        M.mwu_create(kind, P, C, obj)
    val = torch.tensor([1.0, float("nan"), 1.0, 1.0])
    kind, P, C, obj = lpspec.domset_lp(3, rp, ci, val=val)
    with pytest.raises(M.MWUError):
        M.mwu_create(kind, P, C, obj)
    e = torch.tensor([[0, 1]], dtype=torch.int32)
    kind, P, C, obj = lpspec.bmatch_lp(2, e)
    with pytest.raises(M.MWUError):
        M.mwu_create(kind, P, C, obj, eps=1.5)
    with pytest.raises(M.MWUError):
        M.mwu_create(kind, P, C, obj, K=9)


def test_degenerate_single_edge(M):
    """One edge: matching = 1, vertex cover = 1, densest = 1/2."""
    from paper_2307_03307_gb300 import lpspec
    e = torch.tensor([[0, 1]], dtype=torch.int32)
    for lp, want in [("bmatch", 1.0), ("vcover", 1.0), ("densest", 0.5)]:
        fn = {"bmatch": lpspec.bmatch_lp, "vcover": lpspec.vcover_lp, "densest": lpspec.densest_lp}[lp]
        kind, P, C, obj = fn(2, e)
        ctx = M.mwu_create(kind, P, C, obj)
        try:
            r = M.mwu_solve(ctx)
        finally:
            M.mwu_destroy(ctx)
        if lp == "bmatch":
            assert want / 1.21 <= r["objective"] <= want * (1 + 1e-6)
        else:
            assert want * (1 - 1e-6) <= r["objective"] <= want * 1.21


def test_host_and_device_inputs_agree(M, wls):
    """The same problem from host arrays and from device arrays gives bitwise the same x."""
    from paper_2307_03307_gb300 import lpspec
    wl = wls["densest"]
    xs = []
    for dev in ("cpu", "cuda"):
        kind, P, C, obj = lpspec.from_workload(wl, device=dev)
        ctx = M.mwu_create(kind, P, C, obj)
        try:
            M.mwu_set_target(ctx, probe_target(wl))
            M.mwu_iterate(ctx, 5)
            xs.append(vec(M, ctx, M.VEC_X, H.n_vars(wl)))
        finally:
            M.mwu_destroy(ctx)
    assert np.array_equal(xs[0], xs[1])
