"""Whole solves of the benchmark configurations at their stated sizes.

* bipartite matching, 2,000 + 2,000 vertices, 20,000 uniform edges (seed 1),
  plain FP64 form and FP32 form: the certified objective (an exactly feasible
  matching's value, Sec. 2.2) lies in [OPT / (1 + eps)^2, OPT] with OPT the
  maximum matching by Hopcroft-Karp (the LP has no integrality gap on
  bipartite graphs, Sec. 3), and within (1 + eps) of the FP64 oracle's solve;
* 256 b-matching instances (edges log-uniform in [1e3, 2e5], capacities 1..5,
  seed 4) in one batch: every instance in [OPT / (1 + eps)^2, OPT] of its exact
  LP optimum by max flow, and a sample within (1 + eps) of the oracle's solve;
* densest subgraph on R-MAT 18 (seed 2) and dominating set on R-MAT 20
  (seed 3): within (1 + eps) of the FP64 oracle's certified objective of the
  same whole solve, stored in tests/golden/fullsize_objectives.json by
  tests/golden/make_fullsize_objectives.py (which calls only the oracle).
"""
import json
import os

import numpy as np
import pytest
import torch

from graphgen import workloads as W
from oracle import exact
from tests import _helpers as H

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_objectives.json")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03307_gb300 import _build
    _build.build()
    from paper_2307_03307_gb300 import mwu
    mwu.load()
    return mwu


def _solve(M, wl, **opts):
    from paper_2307_03307_gb300 import lpspec
    kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, **opts)
    try:
        return M.mwu_solve(ctx)
    finally:
        M.mwu_destroy(ctx)


@pytest.fixture(scope="module")
def bmatch2k():
    wl = W.bmatch()
    g = wl.graph
    assert (g.n_left, g.n - g.n_left, g.m) == (2000, 2000, 20000)
    opt = exact.bipartite_matching_size(g.n_left, g.n, g.u.numpy(), g.v.numpy())
    ores = H.oracle_solve(wl, step="kary")
    return wl, opt, ores


@pytest.mark.parametrize("prec", ["fp64", "f32"])
def test_bmatch_2k_against_hopcroft_karp_and_oracle(M, bmatch2k, prec):
    wl, opt, ores = bmatch2k
    r = _solve(M, wl, precision=M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64)
    assert r["status"] == M.OK
    assert opt / (1 + wl.eps) ** 2 <= r["objective"] <= opt * (1 + 1e-9), (r["objective"], opt)
    assert 1 / (1 + wl.eps) <= r["objective"] / ores.objective <= 1 + wl.eps, (r["objective"], ores.objective)


def test_bmatching_batch256_against_max_flow_and_oracle(M):
    from paper_2307_03307_gb300 import lpspec
    insts = W.bmatching_batch(count=256, seed=4)
    sizes = [wl.graph.m for wl in insts]
    assert min(sizes) >= 1000 and max(sizes) <= 200_000
    mats = [lpspec.from_workload(wl, device="cuda")[1] for wl in insts]
    ctx = M.mwu_create_batch(mats)
    try:
        obj, iters, tot = M.mwu_solve_batch(ctx, len(mats))
    finally:
        M.mwu_destroy(ctx)
    assert tot["status"] == M.OK
    for k, wl in enumerate(insts):
        g = wl.graph
        opt = exact.b_matching_size(g.n_left, g.n, g.u.numpy(), g.v.numpy(), wl.bounds.numpy())
        assert opt / (1 + wl.eps) ** 2 <= obj[k] <= opt * (1 + 1e-6), (k, obj[k], opt)
    # the oracle's whole solve on a sample across the size range
    order = np.argsort(sizes)
    for k in [int(order[0]), int(order[len(order) // 2]), int(order[-1])]:
        ores = H.oracle_solve(insts[k], step="kary")
        assert 1 / (1 + insts[k].eps) <= obj[k] / ores.objective <= 1 + insts[k].eps, (k, obj[k], ores.objective)


def _golden(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]


@pytest.mark.parametrize("step", ["newton", "kary"])
def test_densest_rmat18_against_oracle_objective(M, step):
    gold = _golden("densest-rmat18")
    wl = W.densest(18, seed=2, device="cuda")
    assert (wl.graph.n, wl.graph.m) == (gold["vertices"], gold["edges"])
    r = _solve(M, wl, step=M.STEP_NEWTON if step == "newton" else M.STEP_KARY)
    assert r["status"] == M.OK
    assert 1 / (1 + wl.eps) <= r["objective"] / gold["objective"] <= 1 + wl.eps, (r["objective"], gold)


@pytest.mark.parametrize("opts", [{}, {"h_scatter": 1}])
def test_domset_rmat20_against_oracle_objective(M, opts):
    gold = _golden("domset-rmat20")
    wl = W.domset(20, seed=3, device="cuda")
    assert (wl.graph.n, wl.graph.m) == (gold["vertices"], gold["edges"])
    r = _solve(M, wl, step=M.STEP_NEWTON, **opts)
    assert r["status"] == M.OK
    assert 1 / (1 + wl.eps) <= r["objective"] / gold["objective"] <= 1 + wl.eps, (r["objective"], gold)
