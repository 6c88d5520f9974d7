"""The smoothed potential (Sec. 4.1) as a torch.autograd.Function on the device:
value and gradients (x, objective weights, explicit CSR values) against the FP64
oracle on the same host-seeded x, and directional central differences.

The difference check compares f(x+) - f(x-) with <grad f(x), x+ - x-> where
x+ and x- are the FP32 points actually evaluated, so rounding of the step does
not enter; the step moves the exponents eta (Px, Cx) by at most h = 1e-3 (FP64
form) or 1e-2 (FP32 form, whose potential resolves about 1e-7 absolute), which
keeps the O(h^2) curvature term below the tolerance.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lp as olp
from oracle import mwu as om
from tests import _helpers as H

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


def domset_ctx(M, wl, prec, values):
    from paper_2307_03307_gb300 import lpspec
    g = wl.graph
    rp, ci = wl.csr
    kind, P, C, obj = lpspec.domset_lp(g.n, rp.cuda(), ci.cuda(), wl.objective.cuda(), val=values)
    p = M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64
    return M.mwu_create(kind, P, C, obj, precision=p, eps=wl.eps), obj


@pytest.mark.parametrize("prec", ["f32", "fp64"])
def test_potential_autograd_matches_oracle_and_differences(M, prec):
    from paper_2307_03307_gb300.autograd import potential
    wl = H.small_workloads()["domset"]
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    rp, ci = wl.csr
    nnz = int(ci.numel())
    values = torch.ones(nnz, dtype=torch.float32, device="cuda", requires_grad=True)
    ctx, obj = domset_ctx(M, wl, prec, values.detach())
    try:
        T = 0.3 * float(wl.objective.sum())
        M.mwu_set_target(ctx, T)
        c = obj.detach().clone().float().requires_grad_(True)      # same values as the context's objective
        Pm, Cm, cvec = H.oracle_matrices(wl, T)
        eta = om.eta_of(Pm.shape[0] + Cm.shape[0], wl.eps)
        rng = np.random.default_rng(3)
        x_np = (om.x_init(Pm, wl.eps) * rng.uniform(1.0, 40.0, g.n)).astype(np.float32)
        x = torch.from_numpy(x_np).cuda().requires_grad_(True)
        pot = potential(ctx, x, c, values)
        pot.backward()
        xo = x_np.astype(np.float64)
        # value: a difference of two LSEs of FP32-accumulated rows
        po = om.potential(Pm, Cm, xo, eta)
        scale_abs = abs(om.smax(Pm @ xo, eta)) + abs(om.smin(Cm @ xo, eta))
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert abs(float(pot) - po) <= tol * (1 + scale_abs), (float(pot), po)
        # d/dx = g - h
        gxo = om.potential_grad_x(Pm, Cm, xo, eta)
        # the gradients come back as FP32 arrays in both forms
        rel = 2.5e-7 if prec == "fp64" else 1e-4
        H.assert_rel(x.grad.double().cpu().numpy(), gxo, rel, abs_=rel * np.abs(gxo).max(), what="d pot/dx")
        # d/dc_i of smax((1/T) c^T x) for the single objective row = x_i / T
        H.assert_rel(c.grad.double().cpu().numpy(), xo / T, rel, what="d pot/dc")
        # d/dval of -smin(Cx): -w_j x_i per stored entry (CSR order)
        wc = om.grad_smin(Cm @ xo, eta)
        gvo = om.potential_grad_values(olp.dominating(g.n, u, v), xo, wc, -1)
        H.assert_rel(values.grad.double().cpu().numpy(), gvo, rel, abs_=rel * np.abs(gvo).max(), what="d pot/dval")

        # directional central differences at the FP32 points actually evaluated
        h = 1e-3 if prec == "fp64" else 1e-2
        grad = x.grad.double().cpu().numpy()
        for k in range(3):
            dvec = rng.standard_normal(g.n) * xo
            step = h / (eta * max(np.abs(Pm @ dvec).max(), np.abs(Cm @ dvec).max()))
            xp = (xo + step * dvec).astype(np.float32)
            xm = (xo - step * dvec).astype(np.float32)
            fp = M.mwu_potential(ctx, torch.from_numpy(xp).cuda())
            fm = M.mwu_potential(ctx, torch.from_numpy(xm).cuda())
            lin = float(grad @ (xp.astype(np.float64) - xm.astype(np.float64)))
            tolfd = 1e-5 if prec == "fp64" else 2e-2
            assert abs((fp - fm) - lin) <= tolfd * abs(lin), (k, fp - fm, lin)
    finally:
        M.mwu_destroy(ctx)
