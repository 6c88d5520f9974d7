"""The allocation-free entry point mwu_candidates_static (collected last).

Callers that must not allocate device memory (a custom allocator's own hooks,
processes whose memory a caching allocator holds to a fixed budget, runtimes
that forbid cudaMalloc after start-up) evaluate step candidates with it; its
scratch is a static device array.  Its values must equal those of the
context-based mwu_eval_candidates on the same vectors and the oracle's Psi and
Phi on host-seeded vectors, on two calls in a row (the array keeps the
previous call's contents), also over many blocks with a ragged last block
followed by a smaller grid, and it must refuse sizes beyond its fixed capacity.
"""
import numpy as np
import pytest
import torch

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


def test_static_candidates_match_eval_candidates(M):
    from graphgen import workloads as W
    from paper_2307_03307_gb300 import lpspec
    wl = W.densest(11, seed=31)
    g = wl.graph
    kind, P, C, obj = lpspec.from_workload(wl, device="cuda")
    ctx = M.mwu_create(kind, P, C, obj)
    try:
        M.mwu_set_target(ctx, 1.5 * g.m / g.n)
        M.mwu_iterate(ctx, 3)
        rc, _ = M.mwu_direction(ctx)
        assert rc == M.OK
        alphas = [1.0, 3.0, 8.0, 40.0, 200.0, 1.0e3, 7.5e3, 6.0e4]
        psi, phi, zmin = M.mwu_eval_candidates(ctx, alphas)
        sc = M.mwu_get_scalars(ctx)
        y = M.mwu_get_vector(ctx, M.VEC_Y, g.n, fp64=False, device="cuda")
        dy = M.mwu_get_vector(ctx, M.VEC_DY, g.n, fp64=False, device="cuda")
        z = M.mwu_get_vector(ctx, M.VEC_Z, g.m, fp64=False, device="cuda")
        dz = M.mwu_get_vector(ctx, M.VEC_DZ, g.m, fp64=False, device="cuda")
        for _call in range(2):
            vp, _ = M.mwu_candidates_static(y, dy, +1, sc["eta"], sc["s_p"], sc["S_p"], alphas)
            vc, mc = M.mwu_candidates_static(z, dz, -1, sc["eta"], sc["s_c"], sc["S_c"], alphas)
            H.assert_rel(vp, psi, 1e-5, abs_=1e-12, what="Psi")
            H.assert_rel(vc, phi, 1e-5, abs_=1e-12, what="Phi")
            H.assert_rel(mc, zmin, 1e-6, what="min(z + a dz)")
    finally:
        M.mwu_destroy(ctx)


def test_static_candidates_many_blocks_against_oracle(M):
    """Host-seeded v, dv over 43 blocks of 16384 rows (the last one ragged),
    then over 2 blocks: the cross-block merge of the static records and the
    ticket's reset between grids of different sizes.  Psi / Phi against the
    oracle's definitions on the same float32 values in float64."""
    from oracle import mwu as om
    rng = np.random.default_rng(77)
    eta = 1200.0
    alphas = [1.0, 2.0, 5.0, 30.0, 250.0]
    for m in (700_001, 20_000):
        for sign in (+1, -1):
            edge = 0.9 if sign > 0 else 0.2
            v = rng.uniform(0.2, 0.9, m)
            near = rng.random(m) < 0.5
            v[near] = edge - sign * rng.uniform(0.0, 40.0 / eta, int(near.sum()))
            v = v.astype(np.float32)
            dv = rng.uniform(0.0, 3.0 / eta, m).astype(np.float32)
            vo, dvo = v.astype(np.float64), dv.astype(np.float64)
            shift, S = om.lse_shift_sum(vo, eta, sign)
            fn = om.Psi if sign > 0 else om.Phi
            want = [fn(vo, dvo, a, eta) for a in alphas]
            wmin = [float(np.min(vo + a * dvo)) for a in alphas]
            vt, dvt = torch.from_numpy(v).cuda(), torch.from_numpy(dv).cuda()
            for _call in range(2):
                got, gmin = M.mwu_candidates_static(vt, dvt, sign, eta, shift, S, alphas)
                H.assert_rel(got, want, 1e-5, abs_=1e-8 / eta, what=f"m={m} sign={sign}")
                if sign < 0:   # the minimum is that of the covering side (Alg. 3's early exit)
                    H.assert_rel(gmin, wmin, 1e-6, what=f"min m={m} sign={sign}")
                else:
                    assert all(v == float("inf") for v in gmin)


def test_static_candidates_reject_sizes_beyond_capacity(M):
    import ctypes as C
    lib = M.load()
    max_rows = 1024 * 16384
    a = (C.c_double * 1)(1.0)
    out = (C.c_double * 1)()
    x = torch.zeros(4, device="cuda")
    rc = lib.mwu_candidates_static(x.data_ptr(), x.data_ptr(), max_rows + 1, 1, 10.0, 0.0, 1.0, a, 1, out, None, None)
    assert rc == M.ERR_INVALID
    assert "MWU_STATIC_MAX_ROWS" in M.mwu_last_error(None)
    rc = lib.mwu_candidates_static(x.data_ptr(), x.data_ptr(), 4, 1, 10.0, 0.0, 1.0, a, 9, out, None, None)
    assert rc == M.ERR_INVALID
