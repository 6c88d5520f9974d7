"""Pins of the FP64 CPU oracle to facts other than itself (no GPU).

Each test checks the oracle against a closed form, an invariant the paper
proves, an exact optimum from an independent solver (HiGHS LP, Hopcroft-Karp,
max flow) or brute force, or central finite differences.  The last group
plants mistakes in the oracle and checks that a pin catches each one.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
from oracle import exact, lp, mwu

EPS = 0.1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ----------------------------------------------------------------------------
# smax / smin (Sec. 2.2)
# ----------------------------------------------------------------------------


def check_smax_closed_forms(o=mwu):
    eta = 37.0
    for m, c in [(1, 0.3), (7, 0.25), (1000, -2.0)]:
        v = np.full(m, c)
        assert o.smax(v, eta) == pytest.approx(c + math.log(m) / eta, rel=1e-13, abs=1e-13)
        assert o.smin(v, eta) == pytest.approx(c - math.log(m) / eta, rel=1e-13, abs=1e-13)
        assert np.allclose(o.grad_smax(v, eta), 1.0 / m, rtol=1e-13)
        assert np.allclose(o.grad_smin(v, eta), 1.0 / m, rtol=1e-13)
    for t in [-3.0, -0.01, 0.0, 0.2, 5.0]:
        # (1/eta) ln(1 + e^{eta t}) written with log1p / max to avoid overflow
        want = max(t, 0.0) + math.log1p(math.exp(-eta * abs(t))) / eta
        assert o.smax(np.array([0.0, t]), eta) == pytest.approx(want, rel=1e-13, abs=1e-15)
        wmin = min(t, 0.0) - math.log1p(math.exp(-eta * abs(t))) / eta
        assert o.smin(np.array([0.0, t]), eta) == pytest.approx(wmin, rel=1e-13, abs=1e-15)


def test_smax_closed_forms():
    check_smax_closed_forms()


def test_smax_bounds_shift_and_gradient_fd():
    rng = np.random.default_rng(0)
    eta = 50.0
    for _ in range(5):
        v = rng.uniform(0, 1, size=40)
        s = mwu.smax(v, eta)
        assert v.max() <= s <= v.max() + math.log(v.size) / eta + 1e-15
        t = mwu.smin(v, eta)
        assert v.min() - math.log(v.size) / eta - 1e-15 <= t <= v.min()
        assert mwu.smax(v + 0.7, eta) == pytest.approx(s + 0.7, rel=1e-13)
        assert mwu.smin(v - 0.4, eta) == pytest.approx(t - 0.4, rel=1e-13, abs=1e-14)
        # central finite differences of smax / smin against the closed-form gradients
        h = 1e-6
        gs, gm = mwu.grad_smax(v, eta), mwu.grad_smin(v, eta)
        for i in rng.choice(v.size, 6, replace=False):
            e = np.zeros_like(v)
            e[i] = h
            assert (mwu.smax(v + e, eta) - mwu.smax(v - e, eta)) / (2 * h) == pytest.approx(gs[i], rel=1e-5, abs=1e-9)
            assert (mwu.smin(v + e, eta) - mwu.smin(v - e, eta)) / (2 * h) == pytest.approx(gm[i], rel=1e-5, abs=1e-9)
        assert gs.sum() == pytest.approx(1.0) and gm.sum() == pytest.approx(1.0)


# ----------------------------------------------------------------------------
# matrices of Sec. 3
# ----------------------------------------------------------------------------


def test_matrices_from_definitions():
    g = gg.rmat(6, seed=11)
    n, m = g.n, g.m
    u, v = g.u.numpy(), g.v.numpy()
    M = lp.incidence(n, u, v).toarray()
    Md = np.zeros((n, m))
    for e in range(m):
        Md[u[e], e] = 1
        Md[v[e], e] = 1
    assert np.array_equal(M, Md)
    O = lp.pair_matrix(n, u, v)
    W = lp.interweave(m)
    assert W.shape == (m, 2 * m) and O.shape == (n, 2 * m)
    # each pair variable z_{w,e} sits in exactly one vertex row and one edge row
    assert np.array_equal(np.asarray(O.sum(axis=0)).ravel(), np.ones(2 * m))
    assert np.array_equal(np.asarray(W.sum(axis=0)).ravel(), np.ones(2 * m))
    # O W^T is the incidence matrix: vertex w meets edge e iff one of e's slots is w's
    assert np.array_equal((O @ W.T).toarray(), M)
    deg = np.bincount(np.concatenate([u, v]), minlength=n)
    assert np.array_equal(np.asarray(O.sum(axis=1)).ravel(), deg)
    D = lp.dominating(n, u, v).toarray()
    assert np.array_equal(np.diag(D), np.ones(n))
    assert np.array_equal(D - np.eye(n), (D - np.eye(n)).T)
    assert D.sum() == n + 2 * m
    rowptr, col = gg.symmetric_csr(g, with_self=True)
    Dc = lp.csr_from_arrays(rowptr, col, None, (n, n)).toarray()
    assert np.array_equal(Dc, D)


# ----------------------------------------------------------------------------
# one iteration: d, Phi, Psi (Alg. 2, Sec. 4.1, Prop. 4.2)
# ----------------------------------------------------------------------------


def _mixed_instance(seed=3):
    g = gg.rmat(7, seed=seed)
    O = lp.pair_matrix(g.n, g.u, g.v)
    W = lp.interweave(g.m)
    D = 0.8 * g.m / g.n + 1.0
    P, C = O / D, W
    eta = mwu.eta_of(P.shape[0] + C.shape[0], EPS)
    rng = np.random.default_rng(seed)
    x = mwu.x_init(P, EPS) * rng.uniform(1, 40, size=P.shape[1])
    return P, C, x, eta


def check_direction_invariants(o=mwu, seed=3):
    P, C, x, eta = _mixed_instance(seed)
    y, z = P @ x, C @ x
    g, h = o.gradients(P, C, y, z, eta)
    c_d = o.step_coefficient(P.shape[0], C.shape[0], eta)
    d = o.direction(g, h, x, c_d)
    assert (d >= 0).all()
    assert (d <= c_d * x + 1e-300).all()
    assert np.array_equal(d > 0, g < h)
    assert np.dot(h, d) >= np.dot(g, d)          # Lagrangian relaxation, Eq. LagrangianRelax
    # Psi'(0) = <g, d> and Phi'(0) = <h, d> (chain rule through smax/smin)
    dy, dz = P @ d, C @ d
    a = 1e-4 / max(1e-30, np.abs(dy).max() * eta)
    assert (o.Psi(y, dy, a, eta) - o.Psi(y, dy, -a, eta)) / (2 * a) == pytest.approx(np.dot(g, d), rel=1e-5)
    assert (o.Phi(z, dz, a, eta) - o.Phi(z, dz, -a, eta)) / (2 * a) == pytest.approx(np.dot(h, d), rel=1e-5)
    return P, C, x, eta, y, z, d, dy, dz


def test_direction_invariants():
    check_direction_invariants()


def check_phi_psi(o=mwu, seed=3):
    P, C, x, eta, y, z, d, dy, dz = check_direction_invariants(o, seed)
    assert o.Psi(y, dy, 0.0, eta) == 0.0 and o.Phi(z, dz, 0.0, eta) == 0.0
    # grid from Psi ~ 1e-6 (Psi'(0) = <g, d>) to eta * alpha * max(dy) ~ 1e4
    gd = np.dot(g_of(o, P, C, y, z, eta), d)
    alphas = np.geomspace(1e-6 / gd, 1e4 / (eta * dy.max()), 60)
    psi = np.array([o.Psi(y, dy, a, eta) for a in alphas])
    phi = np.array([o.Phi(z, dz, a, eta) for a in alphas])
    assert (psi > 0).all() and (phi > 0).all()
    # Prop. 4.2: f = Phi/Psi decreasing in alpha.  Psi and Phi are differences of
    # two O(1) log-sum-exps, so FP64 cancellation leaves ~1e-16/Psi relative
    # noise; the check uses the grid points where that noise is below 1e-8.
    f = phi / psi
    good = (psi > 1e-8) & (phi > 1e-8)
    fg = f[good]
    assert good.sum() > 30
    assert (np.diff(fg) <= 1e-7 * fg[:-1]).all()
    # f(0+) = <h,d>/<g,d> > 1 whenever d != 0, and f stays below it
    f0 = np.dot(h_of(o, P, C, y, z, eta), d) / np.dot(g_of(o, P, C, y, z, eta), d)
    assert f0 > 1 and (fg <= f0 * (1 + 1e-6)).all()
    # Psi convex, Phi concave on a uniform grid
    lin = np.linspace(0, 50 / (eta * dy.max()), 61)
    ps = np.array([o.Psi(y, dy, a, eta) for a in lin])
    ph = np.array([o.Phi(z, dz, a, eta) for a in lin])
    assert (np.diff(ps, 2) >= -1e-12).all()
    assert (np.diff(ph, 2) <= 1e-12).all()
    # weighted forms: Psi = (1/eta) ln sum w_p e^{eta a dy}, Phi = -(1/eta) ln sum w_c e^{-eta a dz}
    wp, wc = mwu.grad_smax(y, eta), mwu.grad_smin(z, eta)
    for a in [0.5, 7.0, 90.0]:
        assert o.Psi(y, dy, a, eta) == pytest.approx(np.log(np.sum(wp * np.exp(eta * a * dy))) / eta, rel=1e-10)
        assert o.Phi(z, dz, a, eta) == pytest.approx(-np.log(np.sum(wc * np.exp(-eta * a * dz))) / eta, rel=1e-10)


def g_of(o, P, C, y, z, eta):
    return o.gradients(P, C, y, z, eta)[0]


def h_of(o, P, C, y, z, eta):
    return o.gradients(P, C, y, z, eta)[1]


def test_phi_psi_properties():
    check_phi_psi()


# ----------------------------------------------------------------------------
# step-size search (Alg. 3 and its K-candidate form)
# ----------------------------------------------------------------------------


def _threshold_eval(t, zmin_at=None):
    """A monotone f: passes iff alpha <= t; min(z + alpha dz) >= 1 iff alpha >= zmin_at."""
    def ev(alphas):
        ok = [a <= t for a in alphas]
        mins = [1.0 if (zmin_at is not None and a >= zmin_at) else 0.0 for a in alphas]
        return ok, mins
    return ev


def test_search_brackets_threshold():
    rng = np.random.default_rng(1)
    for t in list(rng.uniform(1, 5000, 40)) + [1.0, 2.0, 1024.0, 3.5, 0.7]:
        for K in [1, 2, 4, 8]:
            a, info = mwu.search_kary(_threshold_eval(t), EPS, K=K)
            if t < 1:
                assert a == 0.0
                continue
            assert a <= t < a * (1 + EPS) + 1e-12
        ab, _ = mwu.search_binary(_threshold_eval(t), EPS)
        a1, _ = mwu.search_kary(_threshold_eval(t), EPS, K=1)
        if t >= 1:
            assert ab == a1


def test_search_k1_equals_alg3_on_real_instance():
    P, C, x, eta, y, z, d, dy, dz = check_direction_invariants(mwu, 5)
    ev = mwu.make_evaluator(y, dy, z, dz, eta)
    ab, ib = mwu.search_binary(ev, EPS)
    a1, i1 = mwu.search_kary(ev, EPS, K=1)
    assert ab == a1 and ib.evals == i1.evals
    a8, _ = mwu.search_kary(ev, EPS, K=8)
    ok, _ = ev([a8])
    assert ok[0] and a8 >= 1.0


def test_search_early_exit():
    a, info = mwu.search_kary(_threshold_eval(1000.0, zmin_at=5.0), EPS, K=8)
    assert a == 8.0 and info.early
    a, info = mwu.search_binary(_threshold_eval(1000.0, zmin_at=5.0), EPS)
    assert a == 8.0 and info.early


def test_standard_step_admissible_on_feasible_probe():
    """A feasible probe never has f(1) < 1 along its trajectory (alpha = 1 is the standard step)."""
    g = gg.bipartite_uniform(30, 30, 120, seed=2)
    A = lp.incidence(g.n, g.u, g.v)
    opt = exact.bipartite_matching_size(30, g.n, g.u, g.v)
    M = 0.6 * opt
    res = mwu.mwu(A, lp.objective_row(np.ones(g.m), M), EPS, step="standard", max_iter=400)
    assert res.status in (mwu.FEASIBLE, mwu.MAX_ITER)


def _root_of_b4b(o, y, dy, z, dz, eta):
    """alpha* with Phi(alpha*) = Psi(alpha*), by Brent's method on a bracket found by doubling."""
    from scipy.optimize import brentq
    F = lambda a: o.Phi(z, dz, a, eta) - o.Psi(y, dy, a, eta)
    lo = 1.0
    while F(2 * lo) >= 0:
        lo *= 2
    return brentq(F, lo, 2 * lo, xtol=1e-15 * lo, rtol=1e-15)


def check_newton(o=mwu, seed=3):
    """Newton's method of Sec. 4.2: closed-form derivatives, the step, the search."""
    P, C, x, eta, y, z, d, dy, dz = check_direction_invariants(o, seed)
    ast = _root_of_b4b(o, y, dy, z, dz, eta)
    assert ast > 4.0
    # Psi', Phi' (closed forms) against central differences of Psi, Phi
    for a in [0.3 * ast, ast, 2.0 * ast]:
        h = 1e-5 * a
        assert o.dPsi(y, dy, a, eta) == pytest.approx(
            (o.Psi(y, dy, a + h, eta) - o.Psi(y, dy, a - h, eta)) / (2 * h), rel=1e-4)
        assert o.dPhi(z, dz, a, eta) == pytest.approx(
            (o.Phi(z, dz, a + h, eta) - o.Phi(z, dz, a - h, eta)) / (2 * h), rel=1e-4)
    evn = o.make_newton_evaluator(y, dy, z, dz, eta)
    # one step from each side of the root moves toward it (a contraction here)
    a0 = 0.95 * ast
    ps, ph, dps, dph, _ = evn(a0)
    assert ph >= ps
    a1 = o.newton_update(a0, ps, ph, dps, dph, a0, math.inf)
    assert a0 < a1 <= ast * (1 + 1e-12) and ast - a1 < 0.5 * (ast - a0)
    a0 = 1.05 * ast
    ps, ph, dps, dph, _ = evn(a0)
    assert ph < ps
    a1 = o.newton_update(a0, ps, ph, dps, dph, 0.0, a0)
    assert a1 < a0 and abs(a1 - ast) < 0.75 * (a0 - ast)
    # the search: warm (near the root) and cold (exponential phase first)
    ev = o.make_evaluator(y, dy, z, dz, eta)
    for a0 in [0.95 * ast, 1.05 * ast, None]:
        a, info = o.search_newton(evn, ev, EPS, K=8, alpha0=a0)
        ok, _ = ev([a])
        assert ok[0] and a <= ast * (1 + 1e-12) and a >= 0.99 * ast
        if a0 is not None:
            assert info.newton <= 4
    return ast


def test_newton_step_search():
    for seed in [3, 5, 7]:
        check_newton(mwu, seed)


def test_newton_far_warm_start_stays_within_budget():
    """After a large step the warm start can sit orders of magnitude above the
    new root (or below it): the safeguard's jumps reach a passing step within
    the pass budget of the FP32 form (16)."""
    for seed in [3, 5, 7]:
        P, C, x, eta, y, z, d, dy, dz = check_direction_invariants(mwu, seed)
        ast = _root_of_b4b(mwu, y, dy, z, dz, eta)
        evn = mwu.make_newton_evaluator(y, dy, z, dz, eta)
        ev = mwu.make_evaluator(y, dy, z, dz, eta)
        for f0 in [3000.0, 0.001]:
            a, info = mwu.search_newton(evn, ev, EPS, K=8, alpha0=f0 * ast, max_passes=16)
            ok, _ = ev([a])
            assert ok[0] and 0.3 * ast <= a <= ast * (1 + 1e-12), (seed, f0, a / ast)
            assert info.passes <= 16


def test_newton_search_backoff_and_floor():
    """The (1 - eps)^p backoff on a threshold f, and alpha < 1 -> 0."""
    # f >= 1 iff alpha <= t, with Psi, Phi, and derivatives that make Newton
    # converge at once to 1.3 t (g' undefined -> the safeguard doubles, then bisects)
    for t in [3.0, 50.0, 1000.0]:
        ev = _threshold_eval(t)
        evn = lambda a: (1.0, 1.0 if a <= t else 0.5, 0.0, 0.0)
        a, info = mwu.search_newton(evn, ev, EPS, K=8, alpha0=1.3 * t, max_newton=1)
        p = math.ceil(math.log(t / (1.3 * t)) / math.log(1 - EPS) - 1e-12)
        assert a == pytest.approx(1.3 * t * (1 - EPS) ** p, rel=1e-14) and a <= t
    ev = _threshold_eval(0.5)
    evn = lambda a: (1.0, 1.0 if a <= 0.5 else 0.5, 0.0, 0.0)
    a, _ = mwu.search_newton(evn, ev, EPS, K=8, alpha0=4.0, max_newton=1)
    assert a == 0.0


# ----------------------------------------------------------------------------
# whole solves against exact optima (Theorem 4.1 + the objective embedding)
# ----------------------------------------------------------------------------

TOL2 = (1 + EPS) ** 2


def _packing_within(cert, opt):
    assert cert <= opt * (1 + 1e-9)
    assert cert >= opt / TOL2


def _covering_within(cert, opt):
    assert cert >= opt * (1 - 1e-9)
    assert cert <= opt * TOL2


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bipartite_matching_equals_max_matching(seed):
    g = gg.bipartite_uniform(40, 40, 160, seed=seed)
    A = lp.incidence(g.n, g.u, g.v)
    opt = exact.bipartite_matching_size(40, g.n, g.u, g.v)
    assert exact.lp_packing_opt(A, np.ones(g.m)) == pytest.approx(opt)
    r = mwu.solve_packing(A, np.ones(g.m), EPS)
    _packing_within(r.objective, opt)
    assert (r.x >= 0).all()


def test_b_matching_equals_max_flow():
    g = gg.bipartite_uniform(30, 30, 150, seed=4)
    b = gg.capacities(g.n, seed=4).numpy()
    A = lp.row_scaled(lp.incidence(g.n, g.u, g.v), b)
    opt = exact.b_matching_size(30, g.n, g.u, g.v, b)
    assert exact.lp_packing_opt(A, np.ones(g.m)) == pytest.approx(opt)
    r = mwu.solve_packing(A, np.ones(g.m), EPS)
    _packing_within(r.objective, opt)


def test_vertex_cover_koenig_and_lp():
    g = gg.bipartite_uniform(25, 25, 90, seed=6)
    A = lp.incidence(g.n, g.u, g.v).T.tocsr()
    nu = exact.bipartite_matching_size(25, g.n, g.u, g.v)
    assert exact.lp_covering_opt(A, np.ones(g.n)) == pytest.approx(nu)   # Koenig
    r = mwu.solve_covering(A, np.ones(g.n), EPS)
    _covering_within(r.objective, nu)
    gr = gg.rmat(7, seed=5)
    A = lp.incidence(gr.n, gr.u, gr.v).T.tocsr()
    keep = np.asarray(A.sum(axis=0)).ravel() >= 0
    opt = exact.lp_covering_opt(A, np.ones(gr.n))
    r = mwu.solve_covering(A, np.ones(gr.n), EPS)
    _covering_within(r.objective, opt)
    assert keep.all()


def _graph(n, edges):
    u = np.array([min(a, b) for a, b in edges])
    v = np.array([max(a, b) for a, b in edges])
    return n, u, v


def _complete(n):
    return _graph(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def _cycle(n):
    return _graph(n, [(i, (i + 1) % n) for i in range(n)])


def _star(k):
    return _graph(k + 1, [(0, i) for i in range(1, k + 1)])


def _path(n):
    return _graph(n, [(i, i + 1) for i in range(n - 1)])


@pytest.mark.parametrize("name,graph,opt", [
    ("K5", _complete(5), 1.0), ("C9", _cycle(9), 3.0), ("star6", _star(6), 1.0)])
def test_domset_closed_forms(name, graph, opt):
    n, u, v = graph
    A = lp.dominating(n, u, v)
    assert exact.lp_covering_opt(A, np.ones(n)) == pytest.approx(opt)
    r = mwu.solve_covering(A, np.ones(n), EPS)
    _covering_within(r.objective, opt)


def test_domset_weighted_rmat_against_lp():
    g = gg.rmat(7, seed=3)
    c = gg.vertex_weights(g.n, seed=3).numpy().astype(np.float64)
    A = lp.dominating(g.n, g.u, g.v)
    opt = exact.lp_covering_opt(A, c)
    r = mwu.solve_covering(A, c, EPS)
    _covering_within(r.objective, opt)
    # weighted K_n: the cheapest vertex dominates everything
    n, u, v = _complete(6)
    cw = np.array([3.0, 2.5, 9.0, 1.5, 4.0, 7.0])
    r = mwu.solve_covering(lp.dominating(n, u, v), cw, EPS)
    _covering_within(r.objective, 1.5)


@pytest.mark.parametrize("name,graph,opt", [
    ("K6", _complete(6), 2.5), ("C8", _cycle(8), 1.0), ("star5", _star(5), 5.0 / 6.0),
    ("edge", _graph(2, [(0, 1)]), 0.5)])
def test_densest_closed_forms(name, graph, opt):
    n, u, v = graph
    assert exact.max_density_bruteforce(n, u, v) == pytest.approx(opt)
    assert exact.lp_densest_opt(n, u, v) == pytest.approx(opt)
    r = mwu.solve_densest(n, u, v, EPS)
    _covering_within(r.objective, opt)


def test_densest_bruteforce_random():
    rng = np.random.default_rng(7)
    for trial in range(3):
        n = 12
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.uniform() < 0.3]
        n, u, v = _graph(n, pairs)
        opt = exact.max_density_bruteforce(n, u, v)
        assert exact.lp_densest_opt(n, u, v) == pytest.approx(opt)
        r = mwu.solve_densest(n, u, v, EPS)
        _covering_within(r.objective, opt)
        r = mwu.solve_densest(n, u, v, EPS, step="newton")
        _covering_within(r.objective, opt)


def test_fig1_example():
    with open(os.path.join(GOLDEN, "fig1_example.json")) as f:
        ex = json.load(f)
    n, u, v = ex["graph"]["n"], np.array(ex["graph"]["u"]), np.array(ex["graph"]["v"])
    assert exact.max_density_bruteforce(n, u, v) == pytest.approx(ex["densest_lp"])
    r = mwu.solve_densest(n, u, v, EPS)
    _covering_within(r.objective, ex["densest_lp"])
    r = mwu.solve_covering(lp.dominating(n, u, v), np.ones(n), EPS)
    _covering_within(r.objective, ex["domset_lp"])


@pytest.mark.parametrize("name,graph,opt", [
    ("P7", _path(7), 3.0), ("C10", _cycle(10), 5.0), ("K5", _complete(5), 2.5)])
def test_matching_closed_forms(name, graph, opt):
    n, u, v = graph
    A = lp.incidence(n, u, v)
    assert exact.lp_packing_opt(A, np.ones(u.size)) == pytest.approx(opt)
    r = mwu.solve_packing(A, np.ones(u.size), EPS)
    _packing_within(r.objective, opt)
    r = mwu.solve_packing(A, np.ones(u.size), EPS, step="newton")
    _packing_within(r.objective, opt)


def test_feasible_probe_meets_relative_conditions():
    g = gg.rmat(7, seed=9)
    A = lp.incidence(g.n, g.u, g.v).T.tocsr()
    opt = exact.lp_covering_opt(A, np.ones(g.n))
    r = mwu.mwu(lp.objective_row(np.ones(g.n), 1.3 * opt), A, EPS)
    assert r.status == mwu.FEASIBLE
    xs = r.x / r.z.min()
    assert (A @ xs).min() >= 1 - 1e-12
    assert (np.ones(g.n) @ xs) / (1.3 * opt) <= 1 + EPS + 1e-12
    assert np.allclose(r.z, A @ r.x, rtol=1e-9)      # incremental z equals Cx


# ----------------------------------------------------------------------------
# potential gradients (autograd checks of the library use these)
# ----------------------------------------------------------------------------


def test_potential_gradients_central_fd():
    g = gg.rmat(6, seed=3)
    c = gg.vertex_weights(g.n, seed=3).numpy().astype(np.float64)
    A = lp.dominating(g.n, g.u, g.v)
    M = 0.5 * c.sum()
    P = lp.objective_row(c, M)
    eta = mwu.eta_of(1 + g.n, EPS)
    rng = np.random.default_rng(0)
    x = rng.uniform(0.2, 1.0, g.n) / 10
    gx = mwu.potential_grad_x(P, A, x, eta)
    for i in rng.choice(g.n, 12, replace=False):
        h = 1e-3 * x[i]
        e = np.zeros(g.n)
        e[i] = h
        fd = (mwu.potential(P, A, x + e, eta) - mwu.potential(P, A, x - e, eta)) / (2 * h)
        assert fd == pytest.approx(gx[i], rel=1e-4, abs=1e-8)
    # d/dc_v: P = c^T / M (one row) -> x_v / M
    for i in rng.choice(g.n, 6, replace=False):
        cp, cm = c.copy(), c.copy()
        cp[i] += 1e-3
        cm[i] -= 1e-3
        fd = (mwu.potential(lp.objective_row(cp, M), A, x, eta) - mwu.potential(lp.objective_row(cm, M), A, x, eta)) / 2e-3
        assert fd == pytest.approx(x[i] / M, rel=1e-4)
    # d/d C_ji for the stored values of I + A
    wc = mwu.grad_smin(A @ x, eta)
    gv = mwu.potential_grad_values(A, x, wc, -1.0)
    for k in rng.choice(A.nnz, 10, replace=False):
        Ap, Am = A.copy(), A.copy()
        Ap.data[k] += 1e-3
        Am.data[k] -= 1e-3
        fd = (mwu.potential(P, Ap, x, eta) - mwu.potential(P, Am, x, eta)) / 2e-3
        assert fd == pytest.approx(gv[k], rel=1e-4, abs=1e-9)


# ----------------------------------------------------------------------------
# set-up of a probe (Alg. 1 / Alg. 2 before the loop, Sec. 2.2): eta, x0, c_d
# ----------------------------------------------------------------------------

# 3 x 4 packing matrix with an empty last column.  Column maxima by hand:
# (1, 4, 2, -) -> x0 = eps / (n * colmax) with n = 4 and the empty column's
# norm read as 1; its row maxima (2, 1, 4) differ from every column maximum.
_P34 = np.array([[0.5, 0.0, 2.0, 0.0],
                 [1.0, 0.25, 0.0, 0.0],
                 [0.0, 4.0, 1.0, 0.0]])
# 4 x 4 with row maxima (3, 5, 0.5, 2) and column maxima (2, 5, 3, 0.5):
# same shape either way, so a row/column slip shows in the values
_P44 = np.array([[2.0, 0.0, 3.0, 0.0],
                 [0.0, 5.0, 0.0, 0.0],
                 [0.0, 0.0, 0.0, 0.5],
                 [1.0, 2.0, 0.0, 0.0]])


def check_setup_hand_values(o=mwu):
    # eta = 10 ln(m) / eps (Alg. 1) with m = m_P + m_C: m = 4 -> 100 ln 4
    assert o.eta_of(4, 0.1) == pytest.approx(138.62943611198906, rel=1e-14)
    # m = 3 + 1 + 1000 rows, eps = 0.25 -> 40 ln(1004) = 40 (3 ln 10 + ln 1.004)
    #   = 40 (6.907755278982137 + 0.003992021269537453)
    assert o.eta_of(1004, 0.25) == pytest.approx(276.46989201006697, rel=1e-14)
    assert o.eta_of(4, 0.1, eta_factor=1.0) == pytest.approx(13.862943611198906, rel=1e-14)
    # x0_i = eps / (n ||P_{:,i}||_inf)
    x = o.x_init(sp.csr_matrix(_P34), 0.1)
    np.testing.assert_allclose(x, [0.025, 0.00625, 0.0125, 0.025], rtol=1e-15)
    x = o.x_init(sp.csr_matrix(_P44), 0.2)
    np.testing.assert_allclose(x, [0.025, 0.01, 0.2 / 12, 0.1], rtol=1e-15)
    # c_d = 1/(2 eta) (Alg. 2); 1/eta when one side is the single objective row (Sec. 2.2)
    assert o.step_coefficient(3, 5, 100.0) == pytest.approx(0.005, rel=1e-15)
    assert o.step_coefficient(3, 1, 100.0) == pytest.approx(0.01, rel=1e-15)
    assert o.step_coefficient(1, 7, 100.0) == pytest.approx(0.01, rel=1e-15)
    assert o.step_coefficient(3, 1, 100.0, double_single=False) == pytest.approx(0.005, rel=1e-15)


def test_setup_hand_values():
    check_setup_hand_values()


# ----------------------------------------------------------------------------
# planted mistakes: each pin above must catch a plausible slip in the oracle
# ----------------------------------------------------------------------------


class _Mutant:
    """A copy of the oracle's namespace with one function replaced."""

    def __init__(self, **over):
        self.__dict__.update({k: getattr(mwu, k) for k in dir(mwu) if not k.startswith("__")})
        self.__dict__.update(over)


def _smin_wrong_sign(v, eta):
    s, S = mwu.lse_shift_sum(v, eta, -1)
    return s + math.log(S) / eta


def _smax_no_eta(v, eta):
    s, S = mwu.lse_shift_sum(v, eta, +1)
    return s + math.log(S)


def _direction_swapped(g, h, x, c_d):
    return mwu.direction(h, g, x, c_d)


def _direction_no_x(g, h, x, c_d):
    return mwu.direction(g, h, np.ones_like(x), c_d)


def _gradients_transposed_weight(P, C, y, z, eta):
    return P.T @ mwu.grad_smin(y, eta), C.T @ mwu.grad_smin(z, eta)


def _psi_dropped_shift(y, dy, alpha, eta):
    return mwu.smax(y + alpha * dy, eta)


def _newton_wrong_sign(alpha, psi, phi, dpsi, dphi, lb, ub):
    return mwu.newton_update(alpha, psi, -phi + 2 * psi, dpsi, -dphi + 2 * dpsi, lb, ub)


def _dphi_unweighted(z, dz, alpha, eta):
    return float(np.mean(dz))


def _eta_log10(m, eps, eta_factor=10.0):
    return eta_factor * math.log10(m) / eps


def _x_init_rowmax(P, eps):
    P = sp.csr_matrix(P)
    rowmax = np.asarray(abs(P).max(axis=1).todense()).ravel()
    rowmax[rowmax == 0] = 1.0
    return eps / (P.shape[1] * rowmax)


def _x_init_rows_as_n(P, eps):
    return mwu.x_init(P, eps) * P.shape[1] / P.shape[0]


def _step_coefficient_never_doubled(m_P, m_C, eta, double_single=True):
    return 1.0 / (2.0 * eta)


def _step_coefficient_halved(m_P, m_C, eta, double_single=True):
    return 0.5 * mwu.step_coefficient(m_P, m_C, eta, double_single)


@pytest.mark.parametrize("mutant,check", [
    (_Mutant(smin=_smin_wrong_sign), check_smax_closed_forms),
    (_Mutant(smax=_smax_no_eta), check_smax_closed_forms),
    (_Mutant(direction=_direction_swapped), check_direction_invariants),
    (_Mutant(direction=_direction_no_x), check_direction_invariants),
    (_Mutant(gradients=_gradients_transposed_weight), check_direction_invariants),
    (_Mutant(Psi=_psi_dropped_shift), check_phi_psi),
    (_Mutant(newton_update=_newton_wrong_sign), check_newton),
    (_Mutant(dPhi=_dphi_unweighted), check_newton),
    (_Mutant(eta_of=_eta_log10), check_setup_hand_values),
    (_Mutant(x_init=_x_init_rowmax), check_setup_hand_values),
    (_Mutant(x_init=_x_init_rows_as_n), check_setup_hand_values),
    (_Mutant(step_coefficient=_step_coefficient_never_doubled), check_setup_hand_values),
    (_Mutant(step_coefficient=_step_coefficient_halved), check_setup_hand_values),
])
def test_planted_mistake_is_caught(mutant, check):
    with pytest.raises(AssertionError):
        check(mutant)


# ----------------------------------------------------------------------------
# generalized matching (Appendix A.1): a mixed packing/covering feasibility LP
# ----------------------------------------------------------------------------


def _gmatch_matrices(wl, lower=None):
    g = wl.graph
    Mi = lp.incidence(g.n, g.u.numpy(), g.v.numpy())
    P = lp.row_scaled(Mi, wl.bounds.numpy())
    low = wl.lower.numpy() if lower is None else lower
    C = lp.row_scaled(Mi[: g.n_left], low)
    return P, C


@pytest.mark.parametrize("step", ["kary", "newton"])
def test_gmatch_feasible_against_exact_lp(step):
    from graphgen import workloads as W
    wl = W.gmatch(60, 20, seed=6, min_deg=6, mean_extra=4.0)
    P, C = _gmatch_matrices(wl)
    assert exact.lp_mixed_feasible(P, C)
    r = mwu.mwu(P, C, EPS, step=step)
    assert r.status == mwu.FEASIBLE
    xs = r.x / r.z.min()                       # homogeneous: the (1+eps)-relative solution
    assert (C @ xs).min() >= 1 - 1e-12
    assert (P @ xs).max() <= 1 + EPS + 1e-12


def test_gmatch_infeasible_lower_above_upper():
    from graphgen import workloads as W
    wl = W.gmatch(60, 20, seed=6, min_deg=6, mean_extra=4.0)
    low = wl.lower.numpy().copy()
    low[0] = 7.0                                # user 0: lb 7 > ub 5
    P, C = _gmatch_matrices(wl, low)
    assert not exact.lp_mixed_feasible(P, C)
    r = mwu.mwu(P, C, EPS, step="newton")
    assert r.status == mwu.INFEASIBLE


# ----------------------------------------------------------------------------
# active-set dropping of satisfied covering rows (the last step of the loop of
# Alg. 1 and Alg. 2: C <- {c_j : c_j^T x < 1})
# ----------------------------------------------------------------------------


def test_drop_equals_keep_on_vertex_transitive_graph():
    """On a cycle every covering row has the same value at every iteration (x0
    is uniform and the graph is vertex-transitive), so the active set is all
    rows until the stop: dropping must reproduce keeping bit for bit (the
    standard step, alpha = 1, gives many iterations)."""
    n, u, v = _cycle(12)
    C = lp.incidence(n, u, v).T.tocsr()
    P = lp.objective_row(np.ones(n), 0.6 * n)
    r0 = mwu.mwu(P, C, EPS, step="standard")
    r1 = mwu.mwu(P, C, EPS, step="standard", drop_covered=True)
    assert r0.status == r1.status and r0.iters == r1.iters > 100
    assert np.array_equal(r0.x, r1.x)


def test_drop_gradient_special_case():
    """Covering rows x_1 >= 1 (z_1 = 1: satisfied) and x_2 >= 1 (z_2 = 0.999),
    packing row (x_1 + x_2)/M <= 1.  With dropping only row 2 is active: smin
    of one row is exact, so h = (0, 1), g = (1/M, 1/M), and d = (0, c_d (1 -
    1/M) x_2): x_1 stays and x_2 moves by alpha c_d (1 - 1/M) x_2.  Keeping
    row 1 gives h_1 = e^{-eta}/(e^{-eta} + e^{-0.999 eta}) > 1/M: x_1 moves."""
    M = 10.0
    C = sp.identity(2, format="csr")
    P = lp.objective_row(np.ones(2), M)
    x0 = np.array([1.0, 0.999])
    for drop in [True, False]:
        seen = []
        mwu.mwu(P, C, EPS, step="kary", x0=x0, max_iter=1, drop_covered=drop,
                on_iter=lambda it, x, y, z, a: seen.append((x.copy(), a)))
        (x1, a), = seen
        if drop:
            eta = mwu.eta_of(3, EPS)
            c_d = mwu.step_coefficient(1, 2, eta)
            assert x1[0] == x0[0]
            assert x1[1] == pytest.approx(x0[1] + a * c_d * (1.0 - 1.0 / M) * x0[1], rel=1e-12)
        else:
            assert x1[0] > x0[0]


@pytest.mark.parametrize("step", ["kary", "newton"])
def test_drop_solves_within_bound(step):
    """Whole solves with dropping still give (1 + eps)-relative objectives
    (Theorem 4.1 with the outer search's tolerance) against the exact LP."""
    gr = gg.rmat(7, seed=5)
    A = lp.incidence(gr.n, gr.u, gr.v).T.tocsr()
    opt = exact.lp_covering_opt(A, np.ones(gr.n))
    r = mwu.solve_covering(A, np.ones(gr.n), EPS, step=step, drop_covered=True)
    _covering_within(r.objective, opt)
    g = gg.rmat(7, seed=3)
    c = gg.vertex_weights(g.n, seed=3).numpy().astype(np.float64)
    A = lp.dominating(g.n, g.u, g.v)
    opt = exact.lp_covering_opt(A, c)
    r = mwu.solve_covering(A, c, EPS, step=step, drop_covered=True)
    _covering_within(r.objective, opt)
    n, u, v = gr.n, gr.u.numpy(), gr.v.numpy()
    opt = exact.lp_densest_opt(n, u, v)
    r = mwu.solve_densest(n, u, v, EPS, step=step, drop_covered=True)
    _covering_within(r.objective, opt)


def test_newton_early_exit_when_step_covers():
    """A passing Newton value that covers every row ends the search with the
    smallest covering step alpha_c (Alg. 3's early exit; alpha_c passes by
    Prop. 4.2), and never below 1."""
    t = 50.0
    ev = _threshold_eval(1e9)
    evn = lambda a: (1.0, 2.0, 0.0, 0.0, a / t)     # f >= 1 everywhere, covers from alpha = t
    evn.alpha_cover = lambda: t
    a, info = mwu.search_newton(evn, ev, EPS, K=8, alpha0=3.0 * t, max_passes=16)
    assert a == t and info.early and info.passes == 2
    evn.alpha_cover = lambda: 0.25
    a, info = mwu.search_newton(evn, ev, EPS, K=8, alpha0=3.0 * t, max_passes=16)
    assert a == 1.0 and info.early
    # the covering step of an instance: (1 - z_j)/dz_j over the open rows
    z, dz = np.array([0.5, 1.2, 0.9]), np.array([0.1, 0.0, 0.4])
    evr = mwu.make_newton_evaluator(np.zeros(1), np.zeros(1), z, dz, 10.0)
    assert evr.alpha_cover() == pytest.approx(5.0, rel=1e-15)
    assert mwu.make_newton_evaluator(np.zeros(1), np.zeros(1), z, np.array([0.1, 0.0, 0.0]),
                                     10.0).alpha_cover() == math.inf
    # without a covering value, f >= 1 everywhere drives the safeguard's jumps to the budget
    evn4 = lambda a: (1.0, 2.0, 0.0, 0.0)
    a, info = mwu.search_newton(evn4, ev, EPS, K=8, alpha0=3.0 * t, max_passes=4)
    assert a == 3.0 * t * 256.0 ** 3 and info.passes == 4


def test_incremental_y_z_drift_is_rounding_only():
    """Alg. 2 updates y and z by alpha dy and alpha dz instead of recomputing
    Px and Cx; the oracle logs the drift every 64 iterations: FP64 rounding
    only (a wrong dy, dz or update would show at once)."""
    n, u, v = _cycle(30)
    A = lp.incidence(n, u, v).T.tocsr()
    r = mwu.mwu(lp.objective_row(np.ones(n), 0.6 * n), A, EPS, step="standard", drift_every=16)
    assert r.iters > 64 and len(r.drift) >= 4
    assert max(max(dy, dz) for _, dy, dz in r.drift) < 1e-12
    g = gg.rmat(7, seed=5)
    A = lp.incidence(g.n, g.u, g.v).T.tocsr()
    r = mwu.mwu(lp.objective_row(np.ones(g.n), 0.6 * g.n), A, EPS, step="kary", drift_every=4)
    assert len(r.drift) >= 2 and max(max(dy, dz) for _, dy, dz in r.drift) < 1e-12


def test_densest_peel_lower_bound_brackets_the_optimum():
    """The peeling bound is a real subgraph's density (<= the max density) and
    within 2 (1 + delta) of it, on graphs with brute-force optima."""
    rng = np.random.default_rng(3)
    for trial in range(6):
        n = 12
        pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.35]
        if not pairs:
            continue
        u = np.array([p[0] for p in pairs])
        v = np.array([p[1] for p in pairs])
        opt = exact.max_density_bruteforce(n, u, v)
        lb = exact.densest_peel_lower_bound(n, u, v, delta=0.1)
        assert lb <= opt * (1 + 1e-12) and lb >= opt / (2 * 1.1) - 1e-12
    n, u, v = _complete(7)                       # K_7: density 3, peeling keeps it whole
    assert exact.densest_peel_lower_bound(n, np.asarray(u), np.asarray(v)) == pytest.approx(3.0)


def test_vertex_cover_lp_by_bipartite_double_cover():
    """Fractional vertex cover of non-bipartite graphs: the LP solver, the
    matching of the bipartite double cover, closed forms (odd cycle n/2,
    K_n n/2) and the oracle's MWU solve agree."""
    for n, u, v, closed in [(*_cycle(9), 4.5), (*_complete(6), 3.0)]:
        u, v = np.asarray(u), np.asarray(v)
        A = lp.incidence(n, u, v).T.tocsr()
        assert exact.lp_covering_opt(A, np.ones(n)) == pytest.approx(closed)
        assert exact.vertex_cover_lp_double_cover(n, u, v) == pytest.approx(closed)
    g = gg.rmat(7, seed=11)
    A = lp.incidence(g.n, g.u, g.v).T.tocsr()
    opt = exact.vertex_cover_lp_double_cover(g.n, g.u.numpy(), g.v.numpy())
    assert exact.lp_covering_opt(A, np.ones(g.n)) == pytest.approx(opt)
    r = mwu.solve_covering(A, np.ones(g.n), EPS, step="newton")
    _covering_within(r.objective, opt)
