"""Failure paths of the library, made on the host (no GPU fault is raised):

* MWU_FAULT_ALLOC_AT=k makes the k-th device allocation of a context fail:
  mwu_create returns MWU_ERR_OOM and gives back every byte it had taken;
* MWU_SEARCH_GUARD=1 lowers the bound on the turns of the step search's
  device-side loop (and of the FP64 form's host-driven one) below what a
  search needs: mwu_iterate returns MWU_ERR_TIMEOUT, and the context still
  answers afterwards;
* an x that passes validation but overflows Px: MWU_ERR_NUMERIC; a NaN loaded
  into z: MWU_ERR_INVALID;
* the autograd wrapper refuses objective values that differ from the
  context's copy (an in-place update after mwu_create).
"""
import os

import numpy as np
import pytest
import torch

from graphgen import workloads as W

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


def _spec(wl):
    from paper_2307_03307_gb300 import lpspec
    return lpspec.from_workload(wl, device="cuda")


@pytest.mark.parametrize("k", [1, 2, 7, 15, 40])
def test_allocation_failure_returns_oom_and_leaks_nothing(M, k, monkeypatch):
    wl = W.vcover(10, seed=3)
    spec = _spec(wl)
    ctx = M.mwu_create(*spec)          # warm: the driver's own allocations settle first
    M.mwu_destroy(ctx)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("MWU_FAULT_ALLOC_AT", str(k))
    with pytest.raises(M.MWUError) as e:
        M.mwu_create(*spec)
    assert e.value.code == M.ERR_OOM
    monkeypatch.delenv("MWU_FAULT_ALLOC_AT")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx = M.mwu_create(*spec)          # and the next context is fine
    M.mwu_destroy(ctx)


@pytest.mark.parametrize("prec", ["f32", "fp64"])
def test_search_loop_bound_returns_timeout(M, prec, monkeypatch):
    wl = W.densest(9, seed=5)
    spec = _spec(wl)
    monkeypatch.setenv("MWU_SEARCH_GUARD", "1")
    p = M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64
    ctx = M.mwu_create(*spec, precision=p, step=M.STEP_KARY)
    try:
        M.mwu_set_target(ctx, 1.5 * wl.graph.m / wl.graph.n)
        with pytest.raises(M.MWUError) as e:
            M.mwu_iterate(ctx, 20)
        assert e.value.code == M.ERR_TIMEOUT
        assert "step search" in M.mwu_last_error(ctx)
        # the context still answers
        M.mwu_set_target(ctx, 1.5 * wl.graph.m / wl.graph.n)
        assert M.mwu_get_scalars(ctx)["n"] == 2 * wl.graph.m
    finally:
        M.mwu_destroy(ctx)


def test_overflowing_x_returns_numeric_and_nan_rows_are_invalid(M):
    """x = 3e38 passes validation (finite, >= 0) but x_u + x_v overflows FP32:
    the log-sum-exp reduction of z meets Inf (MWU_ERR_NUMERIC, also from the
    next mwu_iterate); a NaN loaded into z is refused (MWU_ERR_INVALID)."""
    wl = W.vcover(9, seed=3)
    ctx = M.mwu_create(*_spec(wl))
    try:
        M.mwu_set_target(ctx, 0.55 * wl.graph.n)
        x = torch.full((wl.graph.n,), 3.0e38, device="cuda")
        with pytest.raises(M.MWUError) as e:
            M.mwu_set_x(ctx, x)
        assert e.value.code == M.ERR_NUMERIC
        with pytest.raises(M.MWUError) as e:
            M.mwu_iterate(ctx, 1)
        assert e.value.code == M.ERR_NUMERIC
        M.mwu_set_target(ctx, 0.55 * wl.graph.n)
        z = torch.full((wl.graph.m,), 0.5, device="cuda")
        z[7] = float("nan")
        with pytest.raises(M.MWUError) as e:
            M.mwu_set_state(ctx, z=z)
        assert e.value.code == M.ERR_INVALID
    finally:
        M.mwu_destroy(ctx)


def test_autograd_refuses_changed_objective(M):
    from paper_2307_03307_gb300 import lpspec
    from paper_2307_03307_gb300.autograd import potential
    wl = W.domset(9, seed=4)
    g = wl.graph
    rp, ci = wl.csr
    c = wl.objective.cuda().clone().requires_grad_(True)
    kind, P, C, obj = lpspec.domset_lp(g.n, rp.cuda(), ci.cuda(), c.detach())
    ctx = M.mwu_create(kind, P, C, obj)
    try:
        M.mwu_set_target(ctx, 0.3 * float(c.sum()))
        x = torch.full((g.n,), 0.2, device="cuda", requires_grad=True)
        potential(ctx, x, objective=c).backward()
        with torch.no_grad():
            c.mul_(1.5)                 # an in-place update the context does not see
        with pytest.raises(ValueError):
            potential(ctx, x, objective=c)
    finally:
        M.mwu_destroy(ctx)
