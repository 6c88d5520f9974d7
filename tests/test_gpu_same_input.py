"""Parity of each kernel of one iteration with the FP64 oracle on identical inputs.

The stage hooks mwu_set_x, mwu_set_state and mwu_set_direction load
host-seeded x, y, z, d, dy, dz (rounded once to the form's precision) into the
library; the oracle receives the same rounded values in float64.  Nothing the
GPU computes enters the oracle.  Each kernel's output is then compared with
the oracle's function of the same inputs at the stated tolerance: relative
1e-5 in the FP32 form, 1e-12 in the FP64 form.

* a6 forward products dy = Pd, dz = Cd (row-binned / staged SpMV, column
  scatter)                                       -> oracle P @ d, C @ d
* a2, a3 shifts and shifted sums of y and z      -> oracle lse_shift_sum (Sec. 2.2)
* a4 gradients g = P^T grad smax(y), h = C^T grad smin(z) -> oracle gradients
* a5 direction d = c_d max(0, 1 - g/h) x          -> oracle direction, with the
  gradient test allowed to differ only inside the band its inputs' tolerance leaves
* a7 Psi, Phi, min(z + alpha dz) at candidates (Sec. 4.1), Psi', Phi' (Sec. 4.2)
                                                  -> oracle Psi, Phi, dPsi, dPhi
* the step decision of the K-candidate search     -> oracle search_kary

Sums whose every term underflows in the form's precision (weights below
e^-87 in FP32) have no relative accuracy; they are compared with a floor of
1e-12 of the largest entry.  Entries above that floor have exponents
|eta (v - s)| < 28, whose FP32 rounding moves a weight by less than 6e-6.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mwu as om
from tests import _helpers as H
from tests.test_gpu_parity import GRAD_TOL, KINDS, PRECS, make_ctx, probe_target, vec

pytestmark = pytest.mark.gpu

FLOOR = {"f32": 1e-12, "fp64": 1e-280}
ALPHAS = [1.0, 3.0, 16.0, 100.0]


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


def seed_rows(rng, m, eta, edge, sign, lo, hi):
    """Half the rows within 40/eta of the extreme value `edge` (weights that
    matter), the rest spread over [lo, hi] (weights down to underflow)."""
    v = rng.uniform(lo, hi, m)
    near = rng.random(m) < 0.5
    v[near] = edge - sign * rng.uniform(0.0, 40.0 / eta, int(near.sum()))
    if m > 0:
        v[0] = edge
    return v


class Inputs:
    """Host-seeded inputs of one kernel chain and the oracle's results on them."""

    def __init__(self, wl, prec, T, seed=101, z_from_x=False):
        P, C, _ = H.oracle_matrices(wl, T)
        self.P, self.C = P, C
        self.mP, self.mC = P.shape[0], C.shape[0]
        self.n = H.n_vars(wl)
        self.eta = om.eta_of(self.mP + self.mC, wl.eps)
        self.c_d = om.step_coefficient(self.mP, self.mC, self.eta)
        self.tol = GRAD_TOL[prec]
        dt = np.float32 if prec == "f32" else np.float64
        rng = np.random.default_rng(seed)
        x = om.x_init(P, wl.eps) * rng.uniform(1.0, 40.0, self.n)
        f = 0.5 / max(float((P @ x).max()), float((C @ x).min()))
        self.x = (x * min(1.0, f)).astype(dt)
        eta = self.eta
        self.y = seed_rows(rng, self.mP, eta, 0.9, +1, 0.1, 0.9).astype(dt)
        self.z = seed_rows(rng, self.mC, eta, 0.2, -1, 0.2, 0.95).astype(dt)
        if z_from_x:
            # the split form of an edge-row covering side keeps z_e = x_u + x_v
            # exactly: load x near 0.1 (weights spread over e^0 .. e^-40) and z
            # as the rounded sums in the form's precision
            g = wl.graph
            self.x = (0.1 + rng.uniform(0.0, 20.0 / eta, self.n)).astype(dt)
            self.z = (self.x[g.u.numpy()] + self.x[g.v.numpy()]).astype(dt)

        self.dy = (rng.uniform(0.0, 3.0 / eta, self.mP)).astype(dt)
        self.dz = (rng.uniform(0.0, 3.0 / eta, self.mC)).astype(dt)
        d = rng.uniform(0.0, 1.0, self.n) * self.x.astype(np.float64)
        d[rng.random(self.n) < 0.3] = 0.0
        self.d = d.astype(dt)
        # the oracle on the same values, in float64
        o = {k: getattr(self, k).astype(np.float64) for k in ("x", "y", "z", "dy", "dz", "d")}
        self.o = o
        self.Pd, self.Cd = P @ o["d"], C @ o["d"]
        self.lse_p = om.lse_shift_sum(o["y"], eta, +1)
        self.lse_c = om.lse_shift_sum(o["z"], eta, -1)
        self.g, self.h = om.gradients(P, C, o["y"], o["z"], eta)
        self.dir = om.direction(self.g, self.h, o["x"], self.c_d, self.tol)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_direction(d, inp, rel, e_gh, what="d"):
    """d against the oracle's direction at the same x, y, z.

    With g and h within relative e_gh of the oracle's, the ratio g/h moves by
    at most 2.2 e_gh (g/h), so where both sides take the gradient test the same
    way d_i differs by at most c_d x_i (g/h) 2.2 e_gh plus rel |d_i|; the test
    may differ only for ratios inside that band around the threshold 1 - tol.
    Where h underflows in the form's precision the GPU's d_i must still be a
    valid step, in [0, c_d x_i]."""
    x, g, h, c_d = inp.o["x"], inp.g, inp.h, inp.c_d
    thr = 1.0 - inp.tol
    hmax = float(np.max(h)) if h.size else 0.0
    live = h > FLOOR_ACTIVE[0] * hmax
    r = np.where(h > 0, g / np.where(h > 0, h, 1.0), np.inf)
    band = 2.2 * e_gh * r
    on_o = inp.dir > 0
    on_g = d > 0
    agree = on_o == on_g
    flip_ok = np.abs(r - thr) <= band
    bad_flip = live & ~agree & ~flip_ok
    assert not bad_flip.any(), (f"{what}: gradient test differs outside its band at "
                                f"{np.flatnonzero(bad_flip)[:5]}, ratios {r[bad_flip][:5]}")
    tol_d = rel * np.abs(inp.dir) + c_d * x * np.minimum(r, 1.0) * 2.2 * e_gh
    both = live & agree
    H.assert_rel(d[both], inp.dir[both], 0.0, abs_=tol_d[both], what=what)
    assert (d >= 0).all() and (d <= c_d * x * (1 + 1e-6) + 1e-300).all(), f"{what}: outside [0, c_d x]"


FLOOR_ACTIVE = [1e-12]


def check_decision(o, eta, alpha, ao):
    """The K-candidate search's step on the GPU equals the oracle's on the same
    inputs, or the searches parted at a candidate whose f = Phi/Psi lies within
    1e-4 of 1 (the decision band): then the GPU's step still passes the
    oracle's test up to that band, and the larger of the two steps sits in it
    (or covers every row, the early exit)."""
    if alpha == pytest.approx(ao, rel=1e-12):
        return

    def f_of(a):
        return om.Phi(o["z"], o["dz"], a, eta) / om.Psi(o["y"], o["dy"], a, eta)

    if alpha >= 1.0:
        assert f_of(alpha) >= 1.0 - 1e-4, (alpha, ao, f_of(alpha))
    big, small = max(alpha, ao), min(alpha, ao)
    covers = small >= 1.0 and float(np.min(o["z"] + small * o["dz"])) >= 1.0 - 1e-6
    assert abs(f_of(big) - 1.0) <= 1e-4 or covers, (alpha, ao, f_of(big))


def run_same_input(M, wl, prec, **opts):
    rel = H.REL[prec]
    fl = FLOOR[prec]
    FLOOR_ACTIVE[0] = fl
    T = probe_target(wl)
    split = wl.lp == "vcover" and opts.get("col_split", 0) >= 0 and not opts.get("h_scatter", 0)
    inp = Inputs(wl, prec, T, z_from_x=split)
    ctx = make_ctx(M, wl, prec, **opts)
    try:
        M.mwu_set_target(ctx, T)
        sc = M.mwu_get_scalars(ctx)
        assert sc["eta"] == pytest.approx(inp.eta, rel=1e-15)
        M.mwu_set_x(ctx, cuda(inp.x))
        # a6: forward products of a loaded d
        M.mwu_set_direction(ctx, cuda(inp.d))
        H.assert_rel(vec(M, ctx, M.VEC_DY, inp.mP), inp.Pd, rel, what="dy=Pd")
        H.assert_rel(vec(M, ctx, M.VEC_DZ, inp.mC), inp.Cd, rel, what="dz=Cd")
        # a2, a3: shifts and shifted sums of loaded y, z
        M.mwu_set_state(ctx, y=cuda(inp.y), z=cuda(inp.z))
        sc = M.mwu_get_scalars(ctx)
        assert sc["s_p"] == inp.lse_p[0] and sc["s_c"] == inp.lse_c[0], (sc, inp.lse_p, inp.lse_c)
        H.assert_rel([sc["S_p"]], [inp.lse_p[1]], rel, what="S_p")
        H.assert_rel([sc["S_c"]], [inp.lse_c[1]], rel, what="S_c")
        # a4, a5: gradients and direction at the loaded y, z and x
        rc, npos = M.mwu_direction(ctx)
        g = vec(M, ctx, M.VEC_G, inp.n)
        h = vec(M, ctx, M.VEC_H, inp.n)
        H.assert_rel(g, inp.g, rel, what="g", floor=fl)
        H.assert_rel(h, inp.h, rel, what="h", floor=fl)
        check_direction(vec(M, ctx, M.VEC_D, inp.n), inp, rel, rel)
        # a7: candidates, Newton sums and the search on loaded dy, dz
        M.mwu_set_state(ctx, dy=cuda(inp.dy), dz=cuda(inp.dz))
        o = inp.o
        psi, phi, zmn = M.mwu_eval_candidates(ctx, ALPHAS)
        for k, a in enumerate(ALPHAS):
            want_psi = om.Psi(o["y"], o["dy"], a, inp.eta)
            want_phi = om.Phi(o["z"], o["dz"], a, inp.eta)
            absf = (1e-8 if prec == "f32" else 1e-15) / inp.eta
            H.assert_rel([psi[k]], [want_psi], rel, abs_=absf, what=f"Psi({a})")
            H.assert_rel([phi[k]], [want_phi], rel, abs_=absf, what=f"Phi({a})")
            H.assert_rel([zmn[k]], [float(np.min(o["z"] + a * o["dz"]))], 1e-6 if prec == "f32" else 1e-14,
                         what=f"min(z + {a} dz)")
        for a in (1.0, 16.0):
            out = M.mwu_eval_newton(ctx, a)
            H.assert_rel([out[2]], [om.dPsi(o["y"], o["dy"], a, inp.eta)], rel, what=f"Psi'({a})")
            H.assert_rel([out[3]], [om.dPhi(o["z"], o["dz"], a, inp.eta)], rel, what=f"Phi'({a})")
        ev = om.make_evaluator(o["y"], o["dy"], o["z"], o["dz"], inp.eta)
        rc, alpha, _ = M.mwu_search(ctx)
        # the FP64 form searches one candidate per pass (K = 1: Alg. 3), the FP32 form K = 8
        ao, _ = om.search_kary(ev, wl.eps, K=8 if prec == "f32" else 1, max_passes=6 if prec == "f32" else 64)
        check_decision(o, inp.eta, alpha, ao)
        return inp, ctx
    except BaseException:
        M.mwu_destroy(ctx)
        raise


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", KINDS)
def test_kernels_on_identical_inputs(M, wls, kind, prec):
    inp, ctx = run_same_input(M, wls[kind], prec)
    M.mwu_destroy(ctx)


@pytest.mark.parametrize("kind,opts", [("vcover", {"h_scatter": 1}), ("domset", {"h_scatter": 1}),
                                       ("domset", {"dv_scatter": 1}), ("gmatch", {"dv_scatter": 1}),
                                       ("domset", {"spmv_tiles": -1}), ("vcover", {"drop_covered": 1}),
                                       ("vcover", {"col_split": -1})])
def test_kernel_options_on_identical_inputs(M, wls, kind, opts):
    inp, ctx = run_same_input(M, wls[kind], "f32", **opts)
    M.mwu_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_vertex_cover_hub_segments_on_identical_inputs(M, prec):
    """Vertex cover on R-MAT 15 (seed 17): one vertex with 5983 incident edges,
    above the 4096 entries from which the split form's direction cuts a column
    into segments summed by separate warps, and 121 columns above 1024."""
    from graphgen import workloads as W
    inp, ctx = run_same_input(M, W.vcover(15, seed=17), prec)
    M.mwu_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_fused_pair_direction_on_identical_inputs(M, wls, prec):
    """The densest LP's hot-path direction kernel (one thread per edge: the
    two slot variables, the deferred x update, and dz = W d in the same pass)
    runs inside mwu_iterate; its d and dz after one iteration from loaded x, y,
    z are checked against the oracle's direction and W d on the same inputs."""
    wl = wls["densest"]
    rel = H.REL[prec]
    FLOOR_ACTIVE[0] = FLOOR[prec]
    T = probe_target(wl)
    inp = Inputs(wl, prec, T, seed=202)
    ctx = make_ctx(M, wl, prec)
    try:
        M.mwu_set_target(ctx, T)
        M.mwu_set_x(ctx, cuda(inp.x))
        M.mwu_set_state(ctx, y=cuda(inp.y), z=cuda(inp.z))
        M.mwu_iterate(ctx, 1)
        d = vec(M, ctx, M.VEC_D, inp.n)
        check_direction(d, inp, rel, rel, what="d (fused pair kernel)")
        dz = vec(M, ctx, M.VEC_DZ, inp.mC)
        want = inp.C @ inp.dir
        # dz_e = d_2e + d_2e+1: the d bound above, summed over the pair
        x, r = inp.o["x"], np.where(inp.h > 0, inp.g / np.where(inp.h > 0, inp.h, 1.0), 0.0)
        bd = rel * np.abs(inp.dir) + inp.c_d * x * np.minimum(r, 1.0) * 2.2 * rel
        flip = np.abs(r - (1.0 - inp.tol)) <= 2.2 * rel * r
        bd = np.where(flip, inp.c_d * x * 2.2 * rel * r + np.abs(inp.dir), bd)
        H.assert_rel(dz, want, rel, abs_=inp.C @ bd, what="dz = W d (fused)")
    finally:
        M.mwu_destroy(ctx)
