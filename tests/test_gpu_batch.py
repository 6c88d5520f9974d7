"""Batched b-matching (many independent packing LPs, Appendix A.1 with lb = 0):
the concurrent batch solve gives every instance the same certified objective as
solving it alone, and each is within (1+eps)^2 of the exact b-matching LP
optimum (max flow) and within 1+eps of the FP64 oracle's solve."""
import numpy as np
import pytest
import torch

from graphgen import workloads as W
from oracle import exact
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


@pytest.mark.parametrize("workers", [0, 3])
def test_batch_equals_single_and_exact(M, workers):
    from paper_2307_03307_gb300 import lpspec
    insts = W.bmatching_batch(count=10, seed=4, lo=1e3, hi=1.2e4)
    mats = []
    for wl in insts:
        kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
        mats.append(P)
    ctx = M.mwu_create_batch(mats, batch_workers=workers)
    try:
        obj_b, it_b, tot = M.mwu_solve_batch(ctx, len(mats))
    finally:
        M.mwu_destroy(ctx)
    assert tot["iters"] == sum(it_b)
    for k, wl in enumerate(insts):
        kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
        c1 = M.mwu_create(kind, P, C, obj, eps=wl.eps)
        try:
            r1 = M.mwu_solve(c1)
        finally:
            M.mwu_destroy(c1)
        assert obj_b[k] == r1["objective"] and it_b[k] == r1["iters"], k   # concurrency changes nothing
        g = wl.graph
        opt = exact.b_matching_size(g.n_left, g.n, g.u.numpy(), g.v.numpy(), wl.bounds.numpy())
        assert opt / (1 + wl.eps) ** 2 <= obj_b[k] <= opt * (1 + 1e-6), (k, obj_b[k], opt)
        if k < 3:
            ores = H.oracle_solve(wl)
            assert 1 / (1 + wl.eps) <= obj_b[k] / ores.objective <= 1 + wl.eps
