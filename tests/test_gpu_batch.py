"""Batched b-matching (many independent packing LPs, Appendix A.1 with lb = 0)
in one persistent launch: every instance's certified objective is the same
whether it is solved in the batch or alone (one block or one cluster per
instance, a fixed order of every sum), lies within (1+eps)^2 of the exact b-matching LP optimum
(max flow), and within 1+eps of the FP64 oracle's solve; the autotuner keeps
the fastest block size it timed."""
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


def _mats(insts, device="cuda"):
    from paper_2307_03307_gb300 import lpspec
    return [lpspec.from_workload(wl, device=device)[1] for wl in insts]


@pytest.mark.parametrize("nt,step", [(256, "kary"), (512, "newton"), (1024, "kary"), (1024, "newton")])
def test_batch_equals_alone_and_exact(M, nt, step):
    insts = W.bmatching_batch(count=10, seed=4, lo=1e3, hi=1.2e4)
    st = M.STEP_NEWTON if step == "newton" else M.STEP_KARY
    ctx = M.mwu_create_batch(_mats(insts), batch_workers=nt, step=st)
    try:
        obj_b, it_b, tot = M.mwu_solve_batch(ctx, len(insts))
        obj_2, it_2, _ = M.mwu_solve_batch(ctx, len(insts))     # a second solve of the same context
    finally:
        M.mwu_destroy(ctx)
    assert tot["iters"] == sum(it_b) and tot["launches"] == 1
    assert obj_b == obj_2 and it_b == it_2
    for k, wl in enumerate(insts):
        c1 = M.mwu_create_batch(_mats([wl]), batch_workers=nt, step=st)
        try:
            o1, i1, _ = M.mwu_solve_batch(c1, 1)
        finally:
            M.mwu_destroy(c1)
        assert obj_b[k] == o1[0] and it_b[k] == i1[0], k   # the batch changes nothing
        g = wl.graph
        opt = exact.b_matching_size(g.n_left, g.n, g.u.numpy(), g.v.numpy(), wl.bounds.numpy())
        assert opt / (1 + wl.eps) ** 2 <= obj_b[k] <= opt * (1 + 1e-6), (k, obj_b[k], opt)
        if k < 3:
            ores = H.oracle_solve(wl, step=step)
            assert 1 / (1 + wl.eps) <= obj_b[k] / ores.objective <= 1 + wl.eps


def test_batch_from_host_arrays_and_autotuner(M):
    insts = W.bmatching_batch(count=12, seed=9, lo=1e3, hi=3e4)
    ctx = M.mwu_create_batch(_mats(insts, device="cpu"))
    try:
        nt0, cl0, _ = M.mwu_batch_tuning(ctx)
        assert nt0 == 0 and cl0 == 0
        obj, it, tot = M.mwu_solve_batch(ctx, len(insts))
        nt, cl, ms = M.mwu_batch_tuning(ctx)
        assert (nt, cl) in M.BATCH_TUNE_CONFIGS and ms[:3] and all(t > 0 for t in ms[:3])
        timed = [t for t in ms if t > 0]
        assert ms[M.BATCH_TUNE_CONFIGS.index((nt, cl))] == min(timed)   # the fastest configuration it timed
        passes, probes = M.mwu_batch_stats(ctx, len(insts))
        assert sum(passes) == tot["passes"] and sum(probes) == tot["probes"]
    finally:
        M.mwu_destroy(ctx)
    ctx = M.mwu_create_batch(_mats(insts), batch_workers=nt, batch_cluster=cl)
    try:
        obj2, it2, _ = M.mwu_solve_batch(ctx, len(insts))
    finally:
        M.mwu_destroy(ctx)
    assert obj == obj2 and it == it2                         # host or device inputs, same solve


@pytest.mark.parametrize("nt,cl,step", [(256, 4, "kary"), (512, 8, "newton"), (256, 8, "kary"), (512, 16, "newton")])
def test_cluster_batch_equals_alone_and_exact(M, nt, cl, step):
    """Instances of at least batch_cluster_edges edges are solved by a whole
    cluster (sums combined across its blocks in a fixed tree), the rest by one
    block; either way the batch changes nothing and the objective is certified."""
    insts = W.bmatching_batch(count=8, seed=11, lo=2e3, hi=8e4)
    thr = 16384
    assert any(w.graph.m >= thr for w in insts) and any(w.graph.m < thr for w in insts)
    st = M.STEP_NEWTON if step == "newton" else M.STEP_KARY
    opts = dict(batch_workers=nt, batch_cluster=cl, batch_cluster_edges=thr, step=st)
    ctx = M.mwu_create_batch(_mats(insts), **opts)
    try:
        obj_b, it_b, tot = M.mwu_solve_batch(ctx, len(insts))
        obj_2, it_2, _ = M.mwu_solve_batch(ctx, len(insts))
        assert M.mwu_batch_tuning(ctx)[:2] == (nt, cl)
    finally:
        M.mwu_destroy(ctx)
    assert obj_b == obj_2 and it_b == it_2 and tot["launches"] == 1
    for k, wl in enumerate(insts):
        c1 = M.mwu_create_batch(_mats([wl]), **opts)
        try:
            o1, i1, _ = M.mwu_solve_batch(c1, 1)
        finally:
            M.mwu_destroy(c1)
        assert obj_b[k] == o1[0] and it_b[k] == i1[0], k
        g = wl.graph
        opt = exact.b_matching_size(g.n_left, g.n, g.u.numpy(), g.v.numpy(), wl.bounds.numpy())
        assert opt / (1 + wl.eps) ** 2 <= obj_b[k] <= opt * (1 + 1e-6), (k, obj_b[k], opt)
    # a clustered instance against the FP64 oracle's solve
    big = max(range(len(insts)), key=lambda k: insts[k].graph.m)
    ores = H.oracle_solve(insts[big], step=step)
    assert 1 / (1 + insts[big].eps) <= obj_b[big] / ores.objective <= 1 + insts[big].eps


def test_batch_rejects_bad_cluster(M):
    insts = W.bmatching_batch(count=2, seed=4, lo=1e3, hi=2e3)
    for kw in ({"batch_workers": 256, "batch_cluster": 3}, {"batch_workers": 1024, "batch_cluster": 4}):
        with pytest.raises(M.MWUError) as e:
            M.mwu_create_batch(_mats(insts), **kw)
        assert e.value.code == M.ERR_INVALID


def test_batch_rejects_other_matrices(M):
    from paper_2307_03307_gb300 import lpspec
    wl = W.vcover(8, seed=3)
    kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
    with pytest.raises(M.MWUError) as e:
        M.mwu_create_batch([C])
    assert e.value.code == M.ERR_INVALID
