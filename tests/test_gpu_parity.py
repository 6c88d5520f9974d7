"""Parity of every hot-path step of the CUDA library with the FP64 CPU oracle.

Both sides start from the same host-seeded x (drawn from the oracle's x0,
rounded once to the form's precision); the oracle then runs its own chain of
one iteration and no GPU value enters it.  Each GPU step is compared element
by element with a bound propagated from the measured error of that step's
inputs: relative 1e-5 (FP32 form) or 1e-12 (FP64 form) on the products, the
softmax bound e^{2 eta e} - 1 on weights and sums, the cost of a gradient test
decided differently on d, and the band around f = 1 for step decisions.
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

KINDS = ["bmatch", "bmatching", "densest", "domset", "vcover", "gmatch"]
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
    if wl.lp == "gmatch":
        return 1.0                      # a feasibility LP: the target is unused


def vec(M, ctx, which, n):
    return M.mwu_get_vector(ctx, which, n, fp64=True).numpy()


GRAD_TOL = {"f32": 2.0 ** -16, "fp64": 0.0}


class Chain:
    """The oracle's own chain of one MWU iteration from a host-seeded x.

    Nothing here comes from the GPU: x is drawn on the host from the oracle's
    x_init, rounded to the form's precision and handed to both sides; every
    later oracle quantity follows from it by the oracle's functions alone.
    """

    def __init__(self, wl, prec, T, seed=7):
        P, C, _ = H.oracle_matrices(wl, T)
        self.P, self.C = P, C
        self.mP, self.mC = P.shape[0], C.shape[0]
        self.n = H.n_vars(wl)
        self.eta = om.eta_of(self.mP + self.mC, wl.eps)
        self.c_d = om.step_coefficient(self.mP, self.mC, self.eta)
        rng = np.random.default_rng(seed)
        dt = np.float32 if prec == "f32" else np.float64
        x = om.x_init(P, wl.eps) * rng.uniform(1.0, 40.0, self.n)
        # keep the probe running: max(Px) and min(Cx) below 1
        f = 0.8 / max(float((P @ x).max()), float((C @ x).min()))
        self.x = (x * min(1.0, f)).astype(dt)
        xo = self.x.astype(np.float64)
        self.xo = xo
        self.y, self.z = P @ xo, C @ xo
        self.g, self.h = om.gradients(P, C, self.y, self.z, self.eta)
        self.d = om.direction(self.g, self.h, xo, self.c_d, GRAD_TOL[prec])
        self.dy, self.dz = P @ self.d, C @ self.d
        self.evaluate = om.make_evaluator(self.y, self.dy, self.z, self.dz, self.eta)
        self.evaluate_nd = om.make_newton_evaluator(self.y, self.dy, self.z, self.dz, self.eta)


def _softmax_l1(e_logit, eta):
    """Bound on ||softmax(eta u') - softmax(eta u)||_1 when ||u' - u||_inf <= e_logit."""
    return math.expm1(2.0 * eta * e_logit)


def run_direction_checks(M, ctx, wl, prec, ch):
    """a1-a6 on the GPU from the chain's x against the chain, with error bounds
    propagated from the measured error of each step's inputs."""
    rel = H.REL[prec]
    eta = ch.eta
    M.mwu_set_x(ctx, torch.from_numpy(ch.x).cuda())
    # a1: y = Px, z = Cx
    y = vec(M, ctx, M.VEC_Y, ch.mP)
    z = vec(M, ctx, M.VEC_Z, ch.mC)
    H.assert_rel(y, ch.y, rel, what="y=Px")
    H.assert_rel(z, ch.z, rel, what="z=Cx")
    ey = float(np.abs(y - ch.y).max())
    ez = float(np.abs(z - ch.z).max())
    # a2, a3: shifts and shifted sums; each weight e^{eta(v - s)} moves by a
    # factor of at most e^{2 eta e_v} (v and its shift both move by <= e_v)
    sc = M.mwu_get_scalars(ctx)
    s_p, S_p = om.lse_shift_sum(ch.y, eta, +1)
    s_c, S_c = om.lse_shift_sum(getattr(ch, "za", ch.z), eta, -1)   # the active covering rows
    assert abs(sc["s_p"] - s_p) <= ey and abs(sc["s_c"] - s_c) <= ez
    tw_p = rel + 1.1 * math.expm1(2 * eta * ey)
    tw_c = rel + 1.1 * math.expm1(2 * eta * ez)
    H.assert_rel([sc["S_p"]], [S_p], tw_p, what="S_p")
    H.assert_rel([sc["S_c"]], [S_c], tw_c, what="S_c")
    # a4: normalised weights move by twice that; g, h are positive sums of them
    rc, npos = M.mwu_direction(ctx)
    assert rc == M.OK
    g = vec(M, ctx, M.VEC_G, ch.n)
    h = vec(M, ctx, M.VEC_H, ch.n)
    d = vec(M, ctx, M.VEC_D, ch.n)
    tg, th = rel + 2.2 * math.expm1(2 * eta * ey), rel + 2.2 * math.expm1(2 * eta * ez)
    H.assert_rel(g, ch.g, tg, what="g=P^T w_p", floor=H.UNDERFLOW[prec])
    H.assert_rel(h, ch.h, th, what="h=C^T w_c", floor=H.UNDERFLOW[prec])
    # a5: d_i = c_d max(0, 1 - g_i/h_i) x_i; g/h moves by <= (tg + th) r, and a
    # gradient test decided differently costs at most c_d x (grad_tol + that)
    go, ho, xo = ch.g, ch.h, ch.xo
    r = np.where(ho > 0, go / np.where(ho > 0, ho, 1), 0.0)
    tiny = (ho <= H.UNDERFLOW[prec] * ho.max()) & (go <= H.UNDERFLOW[prec] * max(go.max(), 1e-300))
    bd = ch.c_d * xo * (1.1 * (tg + th) * r + GRAD_TOL[prec]) + rel * np.abs(ch.d) + 1e-300
    bad = (np.abs(d - ch.d) > bd) & ~tiny
    assert not bad.any(), f"d: {int(bad.sum())} entries outside the propagated bound"
    assert npos == int((d > 0).sum())
    assert np.dot(ch.h, d) >= np.dot(ch.g, d) * (1 - 10 * (tg + th))   # Lagrangian condition on the GPU's d
    # a6: dy = Pd, dz = Cd
    dy = vec(M, ctx, M.VEC_DY, ch.mP)
    dz = vec(M, ctx, M.VEC_DZ, ch.mC)
    bd_t = np.where(tiny, ch.c_d * xo, bd)
    bdy = ch.P @ bd_t + rel * (ch.P @ np.abs(ch.d)) + 1e-300
    bdz = ch.C @ bd_t + rel * (ch.C @ np.abs(ch.d)) + 1e-300
    assert (np.abs(dy - ch.dy) <= bdy).all(), "dy=Pd outside the propagated bound"
    assert (np.abs(dz - ch.dz) <= bdz).all(), "dz=Cd outside the propagated bound"
    edy = float(np.abs(dy - ch.dy).max())
    edz = float(np.abs(dz - ch.dz).max())
    return dict(ey=ey, ez=ez, edy=edy, edz=edz, d=d, y=y, z=z, dy=dy, dz=dz)


def cand_bounds(ch, e, a, prec):
    """|Psi' - Psi| and |Phi' - Phi| at alpha = a: smax and smin are 1-Lipschitz
    in the max norm, plus the GPU's own evaluation error of the difference."""
    rel = H.REL[prec]
    fl = 1e-14 * (1 + abs(om.smax(ch.y, ch.eta)) + abs(om.smin(ch.z, ch.eta)))
    own = fl + (1e-8 / ch.eta if prec == "f32" else 0.0)
    bpsi = 1.05 * (2 * e["ey"] + a * e["edy"]) + own
    bphi = 1.05 * (2 * e["ez"] + a * e["edz"]) + own
    return bpsi, bphi


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", KINDS)
def test_iteration_steps_match_oracle(M, wls, kind, prec):
    wl = wls[kind]
    rel = H.REL[prec]
    ctx = make_ctx(M, wl, prec)
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        ch = Chain(wl, prec, T)
        sc = M.mwu_get_scalars(ctx)
        assert sc["eta"] == pytest.approx(ch.eta, rel=1e-15)
        assert sc["c_d"] == pytest.approx(ch.c_d, rel=1e-15)
        # a0: initial x
        x0 = vec(M, ctx, M.VEC_X, ch.n)
        H.assert_rel(x0, om.x_init(ch.P, wl.eps), 1e-7 if prec == "f32" else 1e-15, what="x0")
        e = run_direction_checks(M, ctx, wl, prec, ch)
        # a7: candidates
        alphas = [1.0, 2.0, 4.0, 16.0, 128.0, 1000.0, 3.0e4, 1.5]
        psi, phi, zmn = M.mwu_eval_candidates(ctx, alphas)
        for k, a in enumerate(alphas):
            bpsi, bphi = cand_bounds(ch, e, a, prec)
            H.assert_rel([psi[k]], [om.Psi(ch.y, ch.dy, a, ch.eta)], rel, abs_=bpsi, what=f"Psi({a})")
            H.assert_rel([phi[k]], [om.Phi(ch.z, ch.dz, a, ch.eta)], rel, abs_=bphi, what=f"Phi({a})")
            H.assert_rel([zmn[k]], [float((ch.z + a * ch.dz).min())], rel,
                         abs_=1.05 * (e["ez"] + a * e["edz"]), what=f"min z({a})")
        # the K-candidate search
        rc, alpha, ev = M.mwu_search(ctx)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_kary(ch.evaluate, wl.eps, K=K, max_passes=6 if K == 8 else 64)
        check_step_decision(ch, e, prec, alpha, ao)
        # a8: one full iteration from the same x
        M.mwu_set_x(ctx, torch.from_numpy(ch.x).cuda())
        rc, st = M.mwu_iterate(ctx, 1)
        if st["iters"] == 1 and st["alpha"] == ao:
            bd = np.abs(e["d"] - ch.d)
            x1 = vec(M, ctx, M.VEC_X, ch.n)
            H.assert_rel(x1, ch.xo + ao * ch.d, 4 * rel, abs_=1.05 * ao * bd + 1e-300, what="x update")
            if ch.mP > 1:
                y1 = vec(M, ctx, M.VEC_Y, ch.mP)
                H.assert_rel(y1, ch.y + ao * ch.dy, 4 * rel, abs_=1.05 * (e["ey"] + ao * e["edy"]), what="y update")
            if ch.mC > 1:
                z1 = vec(M, ctx, M.VEC_Z, ch.mC)
                H.assert_rel(z1, ch.z + ao * ch.dz, 4 * rel, abs_=1.05 * (e["ez"] + ao * e["edz"]), what="z update")
    finally:
        M.mwu_destroy(ctx)


def check_step_decision(ch, e, prec, alpha, ao, rel_gap=0.0):
    """The GPU's step equals the oracle's, or both lie where f = Phi/Psi is
    within the propagated evaluation error of 1 (a decision in the rounding band)."""
    if alpha == ao or (rel_gap > 0 and ao > 0 and abs(alpha / ao - 1) <= rel_gap):
        return
    for a in (alpha, ao):
        if a >= 1:
            ps = om.Psi(ch.y, ch.dy, a, ch.eta)
            ph = om.Phi(ch.z, ch.dz, a, ch.eta)
            bpsi, bphi = cand_bounds(ch, e, a, prec)
            band = (bpsi + bphi) / ps + 10 * H.REL[prec]
            f = ph / ps
            assert f >= 1 - band, (alpha, ao, f, band)
            if rel_gap == 0:
                assert abs(f - 1) <= band or a == alpha, (alpha, ao, f, band)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", KINDS)
def test_newton_search_matches_oracle(M, wls, kind, prec):
    """Newton's method (Sec. 4.2): Psi', Phi' and the search from a cold start."""
    wl = wls[kind]
    rel = H.REL[prec]
    ctx = make_ctx(M, wl, prec, step=M.STEP_NEWTON)
    try:
        T = probe_target(wl)
        M.mwu_set_target(ctx, T)
        ch = Chain(wl, prec, T)
        e = run_direction_checks(M, ctx, wl, prec, ch)
        for a in [1.0, 7.0, 150.0, 4000.0]:
            psi, phi, dpsi, dphi = M.mwu_eval_newton(ctx, a)
            bpsi, bphi = cand_bounds(ch, e, a, prec)
            H.assert_rel([psi], [om.Psi(ch.y, ch.dy, a, ch.eta)], rel, abs_=bpsi, what=f"Psi({a})")
            H.assert_rel([phi], [om.Phi(ch.z, ch.dz, a, ch.eta)], rel, abs_=bphi, what=f"Phi({a})")
            # Psi' = <dy, softmax(eta (y + a dy))>: the weights move by the
            # softmax bound of the logits' error, dy by its own error
            wp = _softmax_l1(e["ey"] + a * e["edy"], ch.eta)
            wc = _softmax_l1(e["ez"] + a * e["edz"], ch.eta)
            H.assert_rel([dpsi], [om.dPsi(ch.y, ch.dy, a, ch.eta)], 4 * rel,
                         abs_=1.1 * (e["edy"] + np.abs(ch.dy).max() * wp) + 1e-300, what=f"Psi'({a})")
            H.assert_rel([dphi], [om.dPhi(ch.z, ch.dz, a, ch.eta)], 4 * rel,
                         abs_=1.1 * (e["edz"] + np.abs(ch.dz).max() * wc) + 1e-300, what=f"Phi'({a})")
        rc, alpha, ev = M.mwu_search(ctx)
        K = 1 if prec == "fp64" else 8
        ao, info = om.search_newton(ch.evaluate_nd, ch.evaluate, wl.eps, K=K, alpha0=None,
                                    max_passes=16 if K == 8 else 64)
        # Newton iterates are continuous in Psi, Phi: the two searches may end a
        # Newton tolerance apart; decisions must otherwise be valid
        check_step_decision(ch, e, prec, alpha, ao, rel_gap=2 * wl.eps / 20 + 1e-3)
        ok, _ = ch.evaluate([alpha])
        if alpha >= 1 and not ok[0]:
            bpsi, bphi = cand_bounds(ch, e, alpha, prec)
            ps = om.Psi(ch.y, ch.dy, alpha, ch.eta)
            assert om.Phi(ch.z, ch.dz, alpha, ch.eta) >= ps - bpsi - bphi
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
    """The certified objective of a returned x (R13: the LP is homogeneous, so
    x rescaled to exact feasibility), written out here in FP64 rather than by
    the oracle's function, so that no GPU value enters the oracle."""
    g = wl.graph
    u, v = g.u.numpy().astype(np.int64), g.v.numpy().astype(np.int64)
    x = np.asarray(x, dtype=np.float64)
    if wl.lp in ("bmatch", "bmatching"):
        load = np.bincount(u, weights=x, minlength=g.n) + np.bincount(v, weights=x, minlength=g.n)
        if wl.bounds is not None:
            load = load / wl.bounds.numpy().astype(np.float64)
        return float(x.sum() / load.max())
    if wl.lp == "vcover":
        return float(x.sum() / (x[u] + x[v]).min())
    if wl.lp == "domset":
        nb = x + np.bincount(u, weights=x[v], minlength=g.n) + np.bincount(v, weights=x[u], minlength=g.n)
        return float(wl.objective.numpy().astype(np.float64) @ x / nb.min())
    if wl.lp == "densest":
        oz = np.bincount(u, weights=x[0::2], minlength=g.n) + np.bincount(v, weights=x[1::2], minlength=g.n)
        return float(oz.max() / (x[0::2] + x[1::2]).min())


@pytest.mark.parametrize("step", ["kary", "newton"])
@pytest.mark.parametrize("prec", PRECS)
def test_gmatch_solve_feasible(M, wls, prec, step):
    """Generalized matching (Appendix A.1): the mixed feasibility LP is solved to a
    (1+eps)-relative feasible x, as the oracle's solve is, and the LP is feasible
    by the exact solver."""
    wl = wls["gmatch"]
    ctx = make_ctx(M, wl, prec, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY)
    try:
        res = M.mwu_solve(ctx)
        x = vec(M, ctx, M.VEC_X, H.n_vars(wl))
    finally:
        M.mwu_destroy(ctx)
    P, C, _ = H.oracle_matrices(wl, 1.0)
    assert exact.lp_mixed_feasible(P, C)
    assert res["status"] == M.OK and (x >= 0).all()
    xs = x / (C @ x).min()
    assert (P @ xs).max() <= 1 + wl.eps + 1e-6
    assert res["objective"] == pytest.approx((P @ x).max() / (C @ x).min(), rel=1e-4)
    r = om.mwu(P, C, wl.eps, step=step)
    assert r.status == om.FEASIBLE


@pytest.mark.parametrize("step", ["kary", "newton"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", [k for k in KINDS if k != "gmatch"])
def test_solve_matches_oracle_and_exact(M, wls, kind, prec, step):
    wl = wls[kind]
    ctx = make_ctx(M, wl, prec, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY)
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
    ores = H.oracle_solve(wl, step=step)
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


def test_one_minus_exp_neg_against_cuda_expm1(M):
    """The candidate passes' own 1 - e^{-b} (Taylor series below 1/4, the fast
    exponential above) against FP64 expm1 and CUDA's FP32 expm1f (via torch):
    relative error below 2^-20 over b in [0, 100]."""
    b = torch.cat([torch.zeros(1), torch.logspace(-12, 2, 200001), torch.linspace(0.2, 0.3, 100001)]).float().cuda()
    u = M.mwu_diag_one_minus_exp_neg(b)
    want = -torch.expm1(-b.double())
    rel = ((u.double() - want).abs() / want.clamp_min(1e-300))[1:]
    assert float(u[0]) == 0.0
    assert float(rel.max()) < 2.0 ** -20, float(rel.max())
    f32 = -torch.expm1(-b)
    rel32 = ((u - f32).abs() / f32.clamp_min(1e-38))[1:]
    assert float(rel32.max()) < 2.0 ** -20


@pytest.mark.parametrize("kind", ["matching", "domset", "vcover", "densest"])
def test_rgg_solves_match_exact_lp(M, kind):
    """The LPs on a random geometric graph (banded, planar-like structure of the
    rgg family): certified objective within (1+eps)^2 of the HiGHS optimum."""
    from graphgen import workloads as W
    wl = W.rgg_lp(kind, scale=9, seed=4)
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    ctx = make_ctx(M, wl, "f32", step=M.STEP_NEWTON)
    try:
        res = M.mwu_solve(ctx)
    finally:
        M.mwu_destroy(ctx)
    tol2 = (1 + wl.eps) ** 2
    if kind == "matching":
        opt = exact.lp_packing_opt(olp.incidence(g.n, u, v), np.ones(g.m))
        assert opt / tol2 <= res["objective"] <= opt * (1 + 1e-6)
    elif kind == "densest":
        opt = exact.lp_densest_opt(g.n, u, v)
        assert opt * (1 - 1e-6) <= res["objective"] <= opt * tol2
    else:
        A = olp.dominating(g.n, u, v) if kind == "domset" else olp.incidence(g.n, u, v).T.tocsr()
        opt = exact.lp_covering_opt(A, np.ones(g.n))
        assert opt * (1 - 1e-6) <= res["objective"] <= opt * tol2
