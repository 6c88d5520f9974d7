"""Parity at the configurations' full sizes, in the launch configuration the
benchmark uses.

* densest subgraph on R-MAT 18 (the benchmark workload) and dominating set on
  R-MAT 20 (explicit CSR, with the autograd gradients): the oracle runs its own
  chain on the whole graph from the same host-seeded x, and every step is
  compared element by element with the propagated bounds of test_gpu_parity;
* vertex cover on R-MAT 24 (260M edges): sampled outputs the oracle computes one
  by one from their definitions (z_e = x_u + x_v, the log-sum-exp of z, h_i over
  the edges at vertex i, d_i, dz_e = d_u + d_v), plus the whole solve's
  certificate against its own definition.
"""
import math

import numpy as np
import pytest
import torch

from graphgen import workloads as W
from oracle import lp as olp
from oracle import mwu as om
from tests import _helpers as H
from tests.test_gpu_parity import Chain, cand_bounds, check_step_decision, make_ctx, probe_target, run_direction_checks, vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03307_gb300 import _build
    _build.build()
    from paper_2307_03307_gb300 import mwu
    mwu.load()
    return mwu


def _chain_checks(M, wl, step):
    ctx = make_ctx(M, wl, "f32", step=step)
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        ch = Chain(wl, "f32", T)
        x0 = vec(M, ctx, M.VEC_X, ch.n)
        H.assert_rel(x0, om.x_init(ch.P, wl.eps), 1e-7, what="x0")
        e = run_direction_checks(M, ctx, wl, "f32", ch)
        alphas = [1.0, 8.0, 64.0, 512.0]
        psi, phi, zmn = M.mwu_eval_candidates(ctx, alphas)
        for k, a in enumerate(alphas):
            bpsi, bphi = cand_bounds(ch, e, a, "f32")
            H.assert_rel([psi[k]], [om.Psi(ch.y, ch.dy, a, ch.eta)], 1e-5, abs_=bpsi, what=f"Psi({a})")
            H.assert_rel([phi[k]], [om.Phi(ch.z, ch.dz, a, ch.eta)], 1e-5, abs_=bphi, what=f"Phi({a})")
        rc, alpha, ev = M.mwu_search(ctx)
        if step == M.STEP_NEWTON:
            ao, _ = om.search_newton(ch.evaluate_nd, ch.evaluate, wl.eps, K=8, alpha0=None, max_passes=16)
            check_step_decision(ch, e, "f32", alpha, ao, rel_gap=2 * wl.eps / 20 + 1e-3)
        else:
            ao, _ = om.search_kary(ch.evaluate, wl.eps, K=8, max_passes=6)
            check_step_decision(ch, e, "f32", alpha, ao)
        return ch
    finally:
        M.mwu_destroy(ctx)


def test_fullsize_densest_rmat18_steps(M):
    wl = W.densest(18, seed=2)
    _chain_checks(M, wl, M.STEP_NEWTON)


def test_fullsize_domset_rmat20_steps_and_autograd(M):
    from paper_2307_03307_gb300 import lpspec
    from paper_2307_03307_gb300.autograd import potential
    wl = W.domset(20, seed=3)
    _chain_checks(M, wl, M.STEP_NEWTON)
    # the potential and its gradients at full size
    g = wl.graph
    rp, ci = wl.csr
    values = torch.ones(int(ci.numel()), dtype=torch.float32, device="cuda", requires_grad=True)
    kind, P, C, obj = lpspec.domset_lp(g.n, rp.cuda(), ci.cuda(), wl.objective.cuda(), val=values.detach())
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps)
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        Pm, Cm, _ = H.oracle_matrices(wl, T)
        eta = om.eta_of(Pm.shape[0] + Cm.shape[0], wl.eps)
        rng = np.random.default_rng(5)
        x_np = (om.x_init(Pm, wl.eps) * rng.uniform(1.0, 40.0, g.n)).astype(np.float32)
        x = torch.from_numpy(x_np).cuda().requires_grad_(True)
        c = obj.detach().clone().requires_grad_(True)
        pot = potential(ctx, x, c, values)
        pot.backward()
        xo = x_np.astype(np.float64)
        po = om.potential(Pm, Cm, xo, eta)
        scale_abs = abs(om.smax(Pm @ xo, eta)) + abs(om.smin(Cm @ xo, eta))
        assert abs(float(pot) - po) <= 2e-6 * (1 + scale_abs)
        gxo = om.potential_grad_x(Pm, Cm, xo, eta)
        H.assert_rel(x.grad.double().cpu().numpy(), gxo, 1e-4, abs_=1e-4 * np.abs(gxo).max(), what="d pot/dx")
        H.assert_rel(c.grad.double().cpu().numpy(), xo / T, 1e-4, what="d pot/dc")
        wc = om.grad_smin(Cm @ xo, eta)
        gvo = om.potential_grad_values(Cm, xo, wc, -1)
        H.assert_rel(values.grad.double().cpu().numpy(), gvo, 1e-4, abs_=1e-4 * np.abs(gvo).max(),
                     what="d pot/dval")
    finally:
        M.mwu_destroy(ctx)


def test_fullsize_vcover_rmat24_sampled(M):
    from paper_2307_03307_gb300 import lpspec
    wl = W.vcover(24, seed=5, device="cuda")
    g = wl.graph
    n, E = g.n, g.m
    kind, P, C, obj = lpspec.from_workload(wl)
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps)
    try:
        T = 0.55 * n
        M.mwu_set_target(ctx, T)
        eta = om.eta_of(1 + E, wl.eps)
        sc = M.mwu_get_scalars(ctx)
        assert sc["eta"] == pytest.approx(eta, rel=1e-15)
        # x0 = eps / (n / T) for the objective row (1/T) 1^T, then a seeded spread
        x0 = vec(M, ctx, M.VEC_X, n)
        H.assert_rel(x0[:1000], np.full(1000, wl.eps / (n / T)), 1e-7, what="x0")
        rng = np.random.default_rng(11)
        x_np = (x0 * rng.uniform(1.0, 3.0, n)).astype(np.float32)
        xo = x_np.astype(np.float64)
        u = g.u.cpu().numpy().astype(np.int64)
        v = g.v.cpu().numpy().astype(np.int64)
        zo = xo[u] + xo[v]                                   # z = M^T x, by definition
        f = 0.8 / max(float(xo.sum() / T), float(zo.min()))   # keep max(Px), min(Cx) below 1
        x_np = (xo * min(1.0, f)).astype(np.float32)
        xo = x_np.astype(np.float64)
        zo = xo[u] + xo[v]
        M.mwu_set_x(ctx, torch.from_numpy(x_np).cuda())
        z = vec(M, ctx, M.VEC_Z, E)
        samp = rng.integers(0, E, 20000)
        H.assert_rel(z[samp], zo[samp], 1e-6, what="z = M^T x (sampled)")
        y = vec(M, ctx, M.VEC_Y, 1)
        H.assert_rel(y, [xo.sum() / T], 1e-5, what="y = (1/T) 1^T x")
        # log-sum-exp of z: shift and sum over all edges (chunked FP64)
        s_c = float(zo.min())
        S_c = 0.0
        for lo in range(0, E, 1 << 26):
            S_c += float(np.exp(-eta * (zo[lo:lo + (1 << 26)] - s_c)).sum())
        sc = M.mwu_get_scalars(ctx)
        ez = float(np.abs(z[samp] - zo[samp]).max())
        assert sc["s_c"] == pytest.approx(s_c, abs=1e-6 * s_c)
        assert sc["S_c"] == pytest.approx(S_c, rel=1e-5 + 2.2 * math.expm1(2 * eta * 1e-6 * max(1.0, zo.max())))
        # h_i = sum over the edges at i of w_c[e] (= e^{-eta (z_e - s_c)} / S_c), at sampled vertices
        rc, npos = M.mwu_direction(ctx)
        h = vec(M, ctx, M.VEC_H, n)
        d = vec(M, ctx, M.VEC_D, n)
        se = rng.integers(0, E, 150)                        # sampled edges; their endpoints are the sampled vertices
        vs = np.unique(np.concatenate([u[se], v[se]]))
        mask = np.isin(u, vs) | np.isin(v, vs)
        ue, ve, ze = u[mask], v[mask], zo[mask]
        we = np.exp(-eta * (ze - s_c)) / S_c
        ho = np.zeros(n)
        np.add.at(ho, ue, we)
        np.add.at(ho, ve, we)
        tol_h = 1e-4 + 2.2 * math.expm1(2 * eta * 1e-6 * max(1.0, zo.max()))
        H.assert_rel(h[vs], ho[vs], tol_h, abs_=1e-35 * ho[vs].max(), what="h (sampled vertices)")
        # d_i = c_d max(0, 1 - g_i / h_i) x_i with g_i = 1/T (objective row, single packing row: smax exact)
        c_d = sc["c_d"]
        go = 1.0 / T
        ro = go / np.maximum(ho[vs], 1e-300)
        do = np.where(ro < 1 - 2.0 ** -16, c_d * (1 - ro) * xo[vs], 0.0)
        bd = c_d * xo[vs] * (1.1 * 2 * tol_h * ro + 2.0 ** -16) + 1e-5 * do + 1e-300
        assert (np.abs(d[vs] - do) <= bd).all(), "d at sampled vertices"
        assert npos == int((d > 0).sum())
        # dz_e = d_u + d_v on the sampled edges, against the oracle's d at their endpoints
        dz = vec(M, ctx, M.VEC_DZ, E)
        pos = {int(w): k for k, w in enumerate(vs)}
        iu = np.array([pos[int(a)] for a in u[se]])
        iv = np.array([pos[int(b)] for b in v[se]])
        dzo = do[iu] + do[iv]
        assert (np.abs(dz[se] - dzo) <= bd[iu] + bd[iv] + 1e-6 * dzo).all(), "dz (sampled edges)"
        # whole solve: the certificate equals its definition c^T x / min(M^T x) at the returned x
        res = M.mwu_solve(ctx)
        xs = vec(M, ctx, M.VEC_X, n)
        cert = xs.sum() / (xs[u] + xs[v]).min()
        assert res["objective"] == pytest.approx(cert, rel=1e-4)
        assert (xs >= 0).all()
    finally:
        M.mwu_destroy(ctx)


def test_fullsize_vcover_rmat24_duality_bracket(M):
    """C5 whole solve at full size through weak LP duality.  The fractional
    vertex cover LP (min 1^T x, M^T x >= 1) and the fractional matching LP on
    the same graph (max 1^T y, M y <= 1) are dual, so any certified matching
    value is a lower bound and any certified cover value an upper bound on the
    common optimum.  Both solves run on the GPU (K = 8 search); both
    certificates are computed here, in FP64 on the host, from the returned x
    and y alone.  Each certified value lies within (1+eps)^2 of the optimum,
    so the bracket is at most (1+eps)^4 wide."""
    from paper_2307_03307_gb300 import lpspec
    wl = W.vcover(24, seed=5, device="cuda")
    g = wl.graph
    n, E = g.n, g.m
    kind, P, C, obj = lpspec.from_workload(wl)
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, K=8)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, n)
    finally:
        M.mwu_destroy(ctx)
    kind_m, Pm, Cm, objm = lpspec.bmatch_lp(n, g.edge_pairs())
    ctx = M.mwu_create(kind_m, Pm, Cm, objm, eps=wl.eps, K=8)
    try:
        resm = M.mwu_solve(ctx)
        y = vec(M, ctx, M.VEC_X, E)
    finally:
        M.mwu_destroy(ctx)
    u = g.u.cpu().numpy()
    v = g.v.cpu().numpy()
    assert (x >= 0).all() and (y >= 0).all()
    cover_min = float((x[u] + x[v]).min())
    cert_vc = float(x.sum()) / cover_min
    load = np.bincount(u, weights=y, minlength=n) + np.bincount(v, weights=y, minlength=n)
    cert_m = float(y.sum()) / float(load.max())
    assert cert_vc == pytest.approx(res["objective"], rel=1e-4)
    assert cert_m == pytest.approx(resm["objective"], rel=1e-4)
    assert cert_m <= cert_vc * (1 + 1e-9), (cert_m, cert_vc)          # weak duality
    assert cert_vc <= (1 + wl.eps) ** 4 * cert_m, (cert_m, cert_vc)


def test_fullsize_domset_rmat20_duality_bracket(M):
    """C3 whole solve at full size through weak LP duality: the weighted
    dominating-set LP (min c^T x, (I + A) x >= 1) and its dual packing LP
    (max 1^T y, (I + A) y <= c, as diag(1/c)(I + A) y <= 1) are solved on the
    GPU; their certified values, recomputed here in FP64 from the returned x
    and y, bracket the common optimum, at most (1 + eps)^4 apart."""
    import scipy.sparse as sp
    from paper_2307_03307_gb300 import lpspec
    wl = W.domset(20, seed=3, device="cuda")
    g = wl.graph
    n = g.n
    kind, P, C, obj = lpspec.from_workload(wl)
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, n)
    finally:
        M.mwu_destroy(ctx)
    rowptr, col = wl.csr
    c = wl.objective
    Pd = M.csr_matrix(rowptr.int().contiguous(), col.int().contiguous(), None, n, n, row_bound=c.float().contiguous())
    ctx = M.mwu_create(M.PACKING, Pd, None, None, eps=wl.eps)
    try:
        resp = M.mwu_solve(ctx)
        y = vec(M, ctx, M.VEC_X, n)
    finally:
        M.mwu_destroy(ctx)
    rp = rowptr.cpu().numpy().astype(np.int64)
    ci = col.cpu().numpy().astype(np.int64)
    A = sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(n, n))
    cw = c.cpu().numpy().astype(np.float64)
    assert (x >= 0).all() and (y >= 0).all()
    cert_c = float(cw @ x) / float((A @ x).min())
    cert_p = float(y.sum()) / float(((A @ y) / cw).max())
    assert cert_c == pytest.approx(res["objective"], rel=1e-4)
    assert cert_p == pytest.approx(resp["objective"], rel=1e-4)
    assert cert_p <= cert_c * (1 + 1e-9), (cert_p, cert_c)          # weak duality
    assert cert_c <= (1 + wl.eps) ** 4 * cert_p, (cert_p, cert_c)
