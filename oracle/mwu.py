"""Plain FP64 CPU oracle of the paper's MWU solver for positive LPs.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the library never does, and it shares no
code with the library.

Everything is float64 numpy/scipy.  The matrices P (packing, m_P x n) and C
(covering, m_C x n) are explicit scipy CSR matrices (see ``oracle.lp``); the
sparse products are scipy's.  Functions follow the paper's notation:

* smax / smin and their gradients .................... Sec. 2.2 (definitions after Eq. NormFeasibleLP)
* eta, x initialisation, g, h, d, max(d) = 0 test ...... Alg. 1 / Alg. 2 (Sec. 2.2, Sec. 4)
* y = Px, z = Cx, d^(y) = Pd, d^(z) = Cd, updates ..... Alg. 2
* Psi, Phi, bang-for-buck f = Phi / Psi >= 1 ........... Sec. 4.1, Eq. b4b_conv
* BinSearch step size .................................. Alg. 3, Sec. 4.2
* K-candidate search (this library's generalisation of Alg. 3, defined here
  so that both sides compute the same alpha) ........... Sec. 4.2 + Prop. 4.2
* Newton's method on f(alpha) = 1, Psi', Phi', the
  (1 - eps)^p backoff and the covering step ............ Sec. 4.2 (+ Alg. 3's early exit)
* dropping of satisfied covering rows (option) ......... Alg. 1 / Alg. 2, last step of the loop
* objective embedding and the search over M or D ...... Sec. 2.2 (pure packing / covering), Sec. 3 (dense-sub)
* the smoothed potential and its gradients ............. Sec. 4.1

Readings of places where the paper is silent or inconsistent are marked
"Reading:" in the docstrings.  Every function above is pinned by
``tests/test_oracle_pins.py`` to closed forms, exact optima, brute force or
invariants; only the iterate trajectory as a whole is not (the GPU and the
oracle iterate independently, and tests compare single steps and results).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import lp as lpm

FEASIBLE = 0
INFEASIBLE = 1
MAX_ITER = 2

# ----------------------------------------------------------------------------
# smoothed max / min (Sec. 2.2)
# ----------------------------------------------------------------------------


def lse_shift_sum(v, eta, sign):
    """Shift and shifted sum of the log-sum-exp of sign*eta*v.

    sign = +1: s = max(v), S = sum_i exp(eta (v_i - s))      (smax = s + ln(S)/eta)
    sign = -1: s = min(v), S = sum_i exp(-eta (v_i - s))     (smin = s - ln(S)/eta)
    """
    v = np.asarray(v, dtype=np.float64)
    s = v.max() if sign > 0 else v.min()
    S = np.exp(sign * eta * (v - s)).sum()
    return float(s), float(S)


def smax(v, eta):
    """smax_eta(v) = (1/eta) log sum_i exp(eta v_i), evaluated with the max shift."""
    s, S = lse_shift_sum(v, eta, +1)
    return s + math.log(S) / eta


def smin(v, eta):
    """smin_eta(v) = -(1/eta) log sum_i exp(-eta v_i), evaluated with the min shift."""
    s, S = lse_shift_sum(v, eta, -1)
    return s - math.log(S) / eta


def grad_smax(v, eta):
    """nabla smax_eta(v) = exp(eta v) / <1, exp(eta v)>."""
    v = np.asarray(v, dtype=np.float64)
    e = np.exp(eta * (v - v.max()))
    return e / e.sum()


def grad_smin(v, eta):
    """nabla smin_eta(v) = exp(-eta v) / <1, exp(-eta v)>."""
    v = np.asarray(v, dtype=np.float64)
    e = np.exp(-eta * (v - v.min()))
    return e / e.sum()


# ----------------------------------------------------------------------------
# one MWU iteration, step by step (Alg. 1 / Alg. 2)
# ----------------------------------------------------------------------------


def eta_of(m, eps, eta_factor=10.0):
    """eta = 10 log(m) / eps with m = m_P + m_C (Alg. 1).  Reading: natural log."""
    return eta_factor * math.log(m) / eps


def x_init(P, eps):
    """x_i = eps / (n ||P_{:,i}||_inf) (Alg. 1).  Reading: an empty column uses norm 1."""
    n = P.shape[1]
    colmax = np.asarray(abs(P).max(axis=0).todense()).ravel()
    colmax[colmax == 0] = 1.0
    return eps / (n * colmax)


def step_coefficient(m_P, m_C, eta, double_single=True):
    """The factor c_d of d_i = c_d max{0, 1 - g_i/h_i} x_i.

    Alg. 1/2 print 1/(2 eta).  Sec. 2.2 notes that when one side is the single
    objective row, smin (or smax) of it is exact and the step may be doubled;
    Reading: c_d = 1/eta when m_C == 1 or m_P == 1 (and the option is on).
    """
    if double_single and (m_P == 1 or m_C == 1):
        return 1.0 / eta
    return 1.0 / (2.0 * eta)


def gradients(P, C, y, z, eta):
    """g = P^T nabla smax(y), h = C^T nabla smin(z) (Alg. 2, packing and covering gradients)."""
    return P.T @ grad_smax(y, eta), C.T @ grad_smin(z, eta)


def direction(g, h, x, c_d, tol=0.0):
    """d_i = c_d max{0, 1 - g_i/h_i} x_i (Alg. 2, new step direction).

    Reading: h_i = 0 gives d_i = 0 (the variable cannot help any covering row).
    ``tol`` > 0 makes the gradient test g_i < (1 - tol) h_i: the test d = 0 of
    Alg. 2 is then decided at the resolution of the arithmetic (0 is exact).
    """
    g = np.asarray(g, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    d = np.zeros_like(np.asarray(x, dtype=np.float64))
    ok = (h > 0) & (g < (1.0 - tol) * h)
    d[ok] = c_d * (1.0 - g[ok] / h[ok]) * np.asarray(x, dtype=np.float64)[ok]
    return d


def Psi(y, dy, alpha, eta):
    """Psi(alpha) = smax(P(x + alpha d)) - smax(Px) = smax(y + alpha dy) - smax(y) (Sec. 4.1)."""
    y = np.asarray(y, dtype=np.float64)
    return smax(y + alpha * np.asarray(dy, dtype=np.float64), eta) - smax(y, eta)


def Phi(z, dz, alpha, eta):
    """Phi(alpha) = smin(C(x + alpha d)) - smin(Cx) = smin(z + alpha dz) - smin(z) (Sec. 4.1)."""
    z = np.asarray(z, dtype=np.float64)
    return smin(z + alpha * np.asarray(dz, dtype=np.float64), eta) - smin(z, eta)


def bang_for_buck_ok(psi, phi):
    """f(alpha) = Phi/Psi >= 1 (Eq. b4b_conv), written without the division: Phi >= Psi."""
    return phi >= psi


# ----------------------------------------------------------------------------
# step-size search (Sec. 4.2)
# ----------------------------------------------------------------------------


@dataclass
class SearchInfo:
    evals: int = 0          # number of f(alpha) evaluations
    passes: int = 0         # number of candidate sets evaluated
    early: bool = False     # returned by the early-exit rule
    newton: int = 0         # Newton evaluations (f and f' at one alpha)
    candidates: list = field(default_factory=list)


def make_evaluator(y, dy, z, dz, eta):
    """Candidate evaluator over stored y, dy, z, dz: returns (f >= 1 flags, min(z + alpha dz))."""
    y = np.asarray(y, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    dz = np.asarray(dz, dtype=np.float64)
    smax0 = smax(y, eta)
    smin0 = smin(z, eta)

    def evaluate(alphas):
        ok, mins = [], []
        for a in alphas:
            psi = smax(y + a * dy, eta) - smax0
            zz = z + a * dz
            phi = smin(zz, eta) - smin0
            ok.append(bang_for_buck_ok(psi, phi))
            mins.append(float(zz.min()))
        return ok, mins

    return evaluate


def search_binary(evaluate, eps, max_evals=256):
    """Alg. 3 (BinSearch): exponential search from alpha = 1, then bisection.

    Reading: bisection continues while (ub - lb)/lb > eps, the stopping rule
    the text of Sec. 4.2 gives for returning l; the loop condition printed in
    Alg. 3, ub - lb > (1 - eps) lb, would stop after a single halving.
    The early exit returns alpha when f(alpha) >= 1 and min(z + alpha dz) >= 1
    (Reading: min, all covering rows satisfied; the prose says max).
    Returns (alpha, info); alpha < 1 signals INFEASIBLE to Alg. 2.
    """
    info = SearchInfo()
    alpha = 1.0
    while info.evals < max_evals:
        ok, mins = evaluate([alpha])
        info.evals += 1
        info.passes += 1
        info.candidates.append([alpha])
        if not ok[0]:
            break
        if mins[0] >= 1.0:
            info.early = True
            return alpha, info
        alpha *= 2.0
    lb, ub = alpha / 2.0, alpha
    while (ub - lb) > eps * lb and info.evals < max_evals:
        beta = 0.5 * (lb + ub)
        ok, _ = evaluate([beta])
        info.evals += 1
        info.passes += 1
        info.candidates.append([beta])
        if ok[0]:
            lb = beta
        else:
            ub = beta
    return lb, info


def _leading(flags):
    p = 0
    for f in flags:
        if not f:
            break
        p += 1
    return p


def search_kary(evaluate, eps, K=8, b0=0, max_passes=64):
    """K-candidate step-size search: Alg. 3 with K values of f per pass.

    Exponential phase: candidates alpha_k = 2^(b+k), k = 0..K-1 (b starts at
    b0, 0 unless warm-started).  By Prop. 4.2 f is decreasing, so the passing
    candidates form a prefix; p = length of the leading run of passes.  Early
    exit: the smallest alpha_k, k < p, with min(z + alpha_k dz) >= 1.  If all K
    pass, b += K; if none passes at b = 0, alpha < 1 (INFEASIBLE); if none
    passes at b > 0, b = max(0, b - K).  Refinement on [lb, ub]: candidates
    lb + j (ub - lb)/(K + 1), j = 1..K, new lb = last of the leading passes,
    new ub = the first failure, until (ub - lb)/lb <= eps.  Returns lb.
    With K = 1 this is exactly ``search_binary`` (midpoints coincide).
    When ``max_passes`` is exhausted the current lb is returned.
    """
    info = SearchInfo()
    lb, ub = 0.0, math.inf
    b = int(b0)
    refine = False
    while info.passes < max_passes:
        if refine:
            if (ub - lb) <= eps * lb:
                return lb, info
            cands = [lb + j * (ub - lb) / (K + 1) for j in range(1, K + 1)]
        else:
            cands = [2.0 ** (b + k) for k in range(K)]
        ok, mins = evaluate(cands)
        info.evals += K
        info.passes += 1
        info.candidates.append(cands)
        p = _leading(ok)
        if refine:
            if p > 0:
                lb = cands[p - 1]
            if p < K:
                ub = cands[p]
            continue
        for k in range(p):
            if mins[k] >= 1.0:
                info.early = True
                return cands[k], info
        if p > 0:
            lb = max(lb, cands[p - 1])
        if p < K:
            ub = min(ub, cands[p])
        if lb > 0.0 and ub < math.inf:
            refine = True
        elif lb == 0.0:
            if b == 0:
                return 0.0, info
            b = max(0, b - K)
        else:
            b += K
    return lb, info


def dPsi(y, dy, alpha, eta):
    """Psi'(alpha) = <dy, exp(eta (y + alpha dy))> / <1, exp(eta (y + alpha dy))> (Sec. 4.2, Newton's method)."""
    y = np.asarray(y, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    return float(dy @ grad_smax(y + alpha * dy, eta))


def dPhi(z, dz, alpha, eta):
    """Phi'(alpha) = <dz, exp(-eta (z + alpha dz))> / <1, exp(-eta (z + alpha dz))> (Sec. 4.2, Newton's method)."""
    z = np.asarray(z, dtype=np.float64)
    dz = np.asarray(dz, dtype=np.float64)
    return float(dz @ grad_smin(z + alpha * dz, eta))


def make_newton_evaluator(y, dy, z, dz, eta):
    """Single-candidate evaluator for Newton's method: (Psi, Phi, Psi', Phi', min(z + alpha dz)) at alpha."""
    y = np.asarray(y, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    dz = np.asarray(dz, dtype=np.float64)

    def evaluate(alpha):
        return (Psi(y, dy, alpha, eta), Phi(z, dz, alpha, eta), dPsi(y, dy, alpha, eta), dPhi(z, dz, alpha, eta),
                float((z + alpha * dz).min()))

    def alpha_cover():
        """The smallest alpha with min(z + alpha dz) >= 1: max over z_j < 1 of (1 - z_j)/dz_j."""
        open_ = z < 1.0
        if not open_.any():
            return 0.0
        if (dz[open_] <= 0.0).any():
            return math.inf
        return float(((1.0 - z[open_]) / dz[open_]).max())

    evaluate.alpha_cover = alpha_cover
    return evaluate


NEWTON_JUMP = 256.0   # the exponential phase's reach in one pass of K = 8 candidates


def newton_update(alpha, psi, phi, dpsi, dphi, lb, ub):
    """One Newton step on g(alpha) = f(alpha) - 1 with f = Phi/Psi (Sec. 4.2).

    alpha' = alpha - g/g' with g' = (Psi Phi' - Phi Psi') / Psi^2, i.e.
    alpha' = alpha - (Phi - Psi) Psi / (Psi Phi' - Phi Psi').
    Reading (safeguard; the paper gives none): [lb, ub] brackets the root by
    Prop. 4.2 (f(lb) >= 1 > f(ub)).  A step that is undefined (Psi <= 0,
    g' >= 0, not finite) or leaves the open bracket is replaced by the
    geometric midpoint sqrt(lb ub) when both ends are known, and otherwise
    moves toward the root by the exponential search's reach of one pass,
    a factor NEWTON_JUMP = 2^8 (down from ub while no passing value is known,
    up from alpha while no failing one is).  A warm start far above the new
    root (after a large previous step) then needs a few passes, not one
    halving per pass.
    """
    den = psi * dphi - phi * dpsi
    nxt = math.nan
    if psi > 0.0 and den < 0.0 and math.isfinite(den):
        nxt = alpha - (phi - psi) * psi / den
    if not (math.isfinite(nxt) and lb < nxt < ub):
        if lb > 0.0 and math.isfinite(ub):
            nxt = math.sqrt(lb * ub)
        elif math.isfinite(ub):
            nxt = ub / NEWTON_JUMP
        else:
            nxt = alpha * NEWTON_JUMP
    return nxt


def search_newton(evaluate_nd, evaluate, eps, K=8, alpha0=None, max_newton=8, max_passes=64, tol=None):
    """Step size by Newton's method on f(alpha) = 1 (Sec. 4.2), warm-started.

    * Start: alpha_0 = the previous iteration's step size when given (warm
      start); otherwise the exponential phase of the K-candidate search
      (candidates 2^(b+k), early exit on min(z + alpha dz) >= 1) brackets the
      root in [2^p, 2^(p+1)] and alpha_0 = 2^p.
    * Newton: alpha_{k+1} = alpha_k - g(alpha_k)/g'(alpha_k), g = f - 1 (see
      ``newton_update`` for the safeguard).  Reading (the paper gives no rule):
      the iteration has converged at alpha_k once |alpha_{k+1} - alpha_k| <=
      tol alpha_k (default tol = eps/20), or after ``max_newton`` evaluations.
      A loose tol returns alpha_k up to a factor 1 + tol below the root and
      costs MWU iterations; eps/20 keeps the iteration count of the bisection
      at about three Newton evaluations per step.
    * Backoff: the converged alpha_k may miss Eq. b4b_conv, so alpha_k (1 -
      eps)^p is taken for the smallest p >= 0 with f >= 1.  Reading: a value
      below 1 ends the backoff with 0 (alpha < 1 is INFEASIBLE in Alg. 2).
    * Budget: every Newton evaluation and every backoff value is one pass
      (the first backoff value nearly always passes: Newton converges to
      within tol of the root), and ``max_passes`` bounds the passes of the
      whole search (a spent budget ends Newton as converged, and the backoff
      with the largest passing value seen).
    * Early exit (reading: Alg. 3's rule, which the Newton search of Sec. 4.2
      does not restate): a Newton value alpha with f >= 1 and min(z + alpha
      dz) >= 1 completes MWU.  A warm start can sit far above the smallest
      such step, so one more pass computes alpha_c = max over the rows with
      z_j < 1 of (1 - z_j)/dz_j (the smallest step covering every row) and
      the search returns max(1, min(alpha, alpha_c)), which passes by Prop.
      4.2 (f decreases) as 1 <= alpha.  Without the rule f >= 1 can hold for
      every alpha once few covering rows are left (with dropped rows), and the
      search climbs by the safeguard's jumps until its budget is spent; with
      alpha itself instead of alpha_c the overshoot pushed max y past 1 + eps.
    ``evaluate_nd(alpha)`` -> (Psi, Phi, Psi', Phi'[, min(z + alpha dz)]),
    with an optional attribute ``alpha_cover()`` -> alpha_c;
    ``evaluate(alphas)`` -> (f >= 1 flags, min(z + alpha dz)) as for the other
    searches.
    Returns (alpha, info); info.evals counts f evaluations, info.newton the
    Newton evaluations.
    """
    info = SearchInfo()
    tol = eps / 20.0 if tol is None else tol
    lb, ub = 0.0, math.inf
    if alpha0 is None or not alpha0 >= 1.0:
        b = 0
        while True:
            if info.passes >= max_passes:
                return lb, info
            cands = [2.0 ** (b + k) for k in range(K)]
            ok, mins = evaluate(cands)
            info.evals += K
            info.passes += 1
            info.candidates.append(cands)
            p = _leading(ok)
            for k in range(p):
                if mins[k] >= 1.0:
                    info.early = True
                    return cands[k], info
            if p > 0:
                lb = max(lb, cands[p - 1])
            if p < K:
                ub = min(ub, cands[p])
            if lb > 0.0 and ub < math.inf:
                if info.passes >= max_passes:
                    return lb, info
                break
            if lb == 0.0:
                if b == 0:
                    return 0.0, info
                b = max(0, b - K)
            else:
                b += K
        alpha = lb
    else:
        alpha = float(alpha0)
    steps = 0
    while True:
        r = evaluate_nd(alpha)
        psi, phi, dpsi, dphi = r[:4]
        zmin = r[4] if len(r) > 4 else -math.inf
        info.evals += 1
        info.passes += 1
        info.newton += 1
        info.candidates.append([alpha])
        steps += 1
        ok = bang_for_buck_ok(psi, phi)
        if ok and zmin >= 1.0 and alpha >= 1.0:
            info.early = True
            cover = getattr(evaluate_nd, "alpha_cover", None)
            if cover is None:
                return alpha, info
            info.passes += 1                  # the pass that computes alpha_c
            return max(1.0, min(alpha, cover())), info
        if ok:
            lb = max(lb, alpha)
        else:
            ub = min(ub, alpha)
        nxt = newton_update(alpha, psi, phi, dpsi, dphi, lb, ub)
        if abs(nxt - alpha) <= tol * alpha or steps >= max_newton or info.passes >= max_passes:
            break
        alpha = nxt
    if ok:
        return alpha, info
    # backoff alpha (1 - eps)^p, p = 1, 2, ... (the running product), one value
    # per pass; when the pass budget is spent the largest passing value seen is
    # returned (0 if there is none or it is below 1)
    q = 1.0 - eps
    a = alpha
    while True:
        if info.passes >= max_passes:
            return (lb if lb >= 1.0 else 0.0), info
        info.passes += 1
        a = a * q
        if a < 1.0:
            return 0.0, info
        okp, _ = evaluate([a])
        info.evals += 1
        info.candidates.append([a])
        if okp[0]:
            return a, info


# ----------------------------------------------------------------------------
# Alg. 2: MWU with step-size search
# ----------------------------------------------------------------------------


@dataclass
class MWUResult:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    status: int
    reason: str
    iters: int
    evals: int
    passes: int
    eta: float
    c_d: float
    alphas: list
    drift: list = field(default_factory=list)   # (iteration, max rel. |y - Px|, max rel. |z - Cx|)


def mwu(P, C, eps, *, eta_factor=10.0, step="kary", K=8, max_iter=5000, max_passes=64,
        double_single=True, warm_start=False, x0=None, on_iter=None, stop_rule=0, grad_tol=0.0, max_newton=8,
        newton_tol=None, ratio_stop=0.0, drop_covered=False, drift_every=64):
    """MWU_STEPSIZE_SEARCH (Alg. 2) on explicit P (m_P x n) and C (m_C x n).

    Per iteration: test, g and h, d, max(d) = 0 -> INFEASIBLE, dy = Pd and
    dz = Cd, alpha = StepSize, alpha < 1 -> INFEASIBLE, then x, y, z updated
    by alpha times d, dy, dz.  Satisfied covering rows are kept (Sec. 4: the
    implementation keeps them).

    Reading of the stopping rule (Alg. 2 loops until the constraints are
    approximately met; the text after it ends MWU once a step pushes the
    packing rows past 1, with a y/z typo in that formula).  The LP is
    homogeneous: whenever max(y) <= (1 + eps) min(z) with min(z) > 0, x / min(z)
    meets Px <= (1 + eps) 1 and Cx >= 1, the (1 + eps)-relative solution of
    Theorem 4.1.  Before each iteration:
      stop_rule = 0 (default, Alg. 2): min(z) >= 1 or max(y) > 1 + eps ends it,
      FEASIBLE when the ratio test holds, INFEASIBLE otherwise;
      stop_rule = 1: the ratio test alone already ends the probe FEASIBLE.
    ``ratio_stop`` > 0 adds the exit max(y) <= ratio_stop min(z) (FEASIBLE);
    the outer search uses it to stop a probe whose certificate closes the
    bracket.
    ``max_iter`` (5000 in Sec. 6) ends it as MAX_ITER.  ``step`` is "kary" (K
    candidates per pass), "binary" (Alg. 3), "newton" (Newton's method of
    Sec. 4.2, warm-started from the previous alpha, at most ``max_newton``
    Newton evaluations, relative tolerance ``newton_tol``) or "standard"
    (alpha = 1, Alg. 1).
    ``grad_tol`` is the tolerance of the gradient test (see ``direction``).

    ``drift_every``: every that many iterations y and z are recomputed from x
    and the largest relative difference to the incrementally updated ones is
    logged in ``drift`` (a diagnostic: the iterates keep the incremental
    values, as Alg. 2 updates y and z by alpha dy and alpha dz).

    ``drop_covered`` keeps only the unsatisfied covering rows, the last step
    of the loop of Alg. 1 and Alg. 2 (C <- {c_j : c_j^T x < 1}), where the
    default keeps every row as the paper's own implementation does (Sec. 4).
    Reading: x never decreases (d >= 0, alpha >= 0, C >= 0), so a dropped row
    stays satisfied and the active set before an iteration is exactly the
    rows with z_j < 1.  The active rows alone enter smin and its gradient h,
    Phi, Phi' and the early exit of the search; the stopping tests read all of
    z, which is the same since dropped rows have z_j >= 1 (min z >= 1 is
    "C is empty").
    """
    P = sp.csr_matrix(P, dtype=np.float64)
    C = sp.csr_matrix(C, dtype=np.float64)
    m_P, n = P.shape
    m_C = C.shape[0]
    eta = eta_of(m_P + m_C, eps, eta_factor)
    c_d = step_coefficient(m_P, m_C, eta, double_single)
    x = x_init(P, eps) if x0 is None else np.array(x0, dtype=np.float64)
    y = P @ x
    z = C @ x
    it = evals = passes = 0
    alphas = []
    drift = []
    alpha_prev = None
    reason = ""
    while True:
        ymax, zmin = y.max(), z.min()
        rho = max(ratio_stop, (1.0 + eps) if stop_rule == 1 else 0.0)
        if rho > 0.0 and zmin > 0.0 and ymax <= rho * zmin:
            status, reason = FEASIBLE, "ratio"
            break
        if zmin >= 1.0 or ymax > 1.0 + eps:
            if ymax <= (1.0 + eps) * zmin:
                status, reason = FEASIBLE, "covered"
            else:
                status, reason = INFEASIBLE, "packing"
            break
        if it >= max_iter:
            status, reason = MAX_ITER, "max_iter"
            break
        if drop_covered:
            act = z < 1.0                   # the active covering rows (Alg. 2, keep unsatisfied)
            Ca, za = C[np.flatnonzero(act)], z[act]
        else:
            Ca, za = C, z
        g, h = gradients(P, Ca, y, za, eta)
        d = direction(g, h, x, c_d, grad_tol)
        if d.max() <= 0.0:
            status, reason = INFEASIBLE, "d=0"
            break
        dy = P @ d
        dz = C @ d
        dza = dz[act] if drop_covered else dz
        ev = make_evaluator(y, dy, za, dza, eta)
        if step == "standard":
            alpha = 1.0
            ok, _ = ev([1.0])
            evals += 1
            passes += 1
        elif step == "binary":
            alpha, info = search_binary(ev, eps)
            evals += info.evals
            passes += info.passes
        elif step == "newton":
            evn = make_newton_evaluator(y, dy, za, dza, eta)
            alpha, info = search_newton(evn, ev, eps, K=K, alpha0=alpha_prev, max_newton=max_newton,
                                        max_passes=max_passes, tol=newton_tol)
            evals += info.evals
            passes += info.passes
        else:
            b0 = 0
            if warm_start and alpha_prev is not None and alpha_prev >= 1.0:
                b0 = int(math.floor(math.log2(alpha_prev)))
            alpha, info = search_kary(ev, eps, K=K, b0=b0, max_passes=max_passes)
            evals += info.evals
            passes += info.passes
        if alpha < 1.0:
            status, reason = INFEASIBLE, "alpha<1"
            break
        x = x + alpha * d
        y = y + alpha * dy
        z = z + alpha * dz
        alphas.append(alpha)
        alpha_prev = alpha
        it += 1
        if drift_every and it % drift_every == 0:
            yx, zx = P @ x, C @ x
            drift.append((it, float(np.max(np.abs(y - yx) / np.maximum(np.abs(yx), 1e-300))),
                          float(np.max(np.abs(z - zx) / np.maximum(np.abs(zx), 1e-300)))))
        if on_iter is not None:
            on_iter(it, x, y, z, alpha)
    return MWUResult(x, y, z, status, reason, it, evals, passes, eta, c_d, alphas, drift)


# ----------------------------------------------------------------------------
# certified objectives and the outer search over M or D (Sec. 2.2, Sec. 3)
# ----------------------------------------------------------------------------


def certified_packing(A, c, x):
    """Objective of the exactly feasible point x / max(Ax) for max c^T x, Ax <= 1 (LP is homogeneous)."""
    mx = float((A @ x).max())
    if mx <= 0.0:
        return 0.0
    return float(np.dot(c, x) / mx)


def certified_covering(A, c, x):
    """Objective of the exactly feasible point x / min(Ax) for min c^T x, Ax >= 1 (LP is homogeneous)."""
    mn = float((A @ x).min())
    if mn <= 0.0:
        return math.inf
    return float(np.dot(c, x) / mn)


def certified_densest(O, W, z):
    """D of the feasible dual point z / min(Wz): max_v (Oz)_v / min_e (Wz)_e (Sec. 3, Eq. densest_linalg)."""
    mn = float((W @ z).min())
    if mn <= 0.0:
        return math.inf
    return float((O @ z).max() / mn)


@dataclass
class SolveResult:
    objective: float          # best certified objective over all probes
    lo: float
    hi: float
    probes: int
    iters: int
    evals: int
    history: list
    x: np.ndarray


def _probe_loop(lo, hi, tol, probe, max_probes=64):
    history = []
    while hi > (1.0 + tol) * lo and len(history) < max_probes:
        M = math.sqrt(lo * hi)
        r, cert, lo, hi = probe(M, lo, hi)
        history.append((M, r.status, r.iters, cert))
    return lo, hi, history


def solve_packing(A, c, eps, *, tol=None, **kw):
    """max c^T x s.t. Ax <= 1, x >= 0 via the objective row (1/M) c^T x >= 1 and a search on M.

    Bracket: hi = sum_i c_i max_{j: a_ji > 0} 1/a_ji (the paper's estimate of M)
    and lo = the objective of the feasible point x_i = 1/(n max_j a_ji).
    Reading (the paper gives no bracket or tolerance): geometric bisection
    M = sqrt(lo hi) until hi <= (1 + tol) lo, tol = eps by default.  A FEASIBLE
    probe raises lo to M, any other lowers hi to M; every probe's certified
    objective also raises lo.  A probe also stops (FEASIBLE) as soon as its
    certificate M min(z)/max(y) reaches hi/(1 + tol), which ends the search.
    The answer is the best certified objective.
    """
    tol = eps if tol is None else tol
    A = sp.csc_matrix(A, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    n = A.shape[1]
    colmax = np.asarray(A.max(axis=0).todense()).ravel()
    colmax[colmax == 0] = 1.0
    colmin = _colmin_fast(A)
    hi = float(np.sum(c / colmin))
    lo = float(np.sum(c / colmax) / n)
    A = A.tocsr()
    best = [lo, None]
    tot = {"iters": 0, "evals": 0}

    def probe(M, lo, hi):
        r = mwu(A, lpm.objective_row(c, M), eps, ratio_stop=(1 + tol) * M / hi, **kw)
        cert = certified_packing(A, c, r.x)
        tot["iters"] += r.iters
        tot["evals"] += r.evals
        if cert > best[0]:
            best[0], best[1] = cert, r.x
        lo = max(lo, cert)
        if r.status == FEASIBLE:
            lo = max(lo, M)
        else:
            hi = min(hi, M)
        return r, cert, lo, hi

    lo, hi, hist = _probe_loop(lo, hi, tol, probe)
    return SolveResult(best[0], lo, hi, len(hist), tot["iters"], tot["evals"], hist, best[1])


def _colmin_fast(A):
    A = sp.csc_matrix(A)
    out = np.ones(A.shape[1])
    nz = np.diff(A.indptr) > 0
    out[nz] = np.minimum.reduceat(A.data, A.indptr[:-1][nz])
    return out


def solve_covering(A, c, eps, *, tol=None, **kw):
    """min c^T x s.t. Ax >= 1, x >= 0 via the objective row (1/M) c^T x <= 1 and a search on M.

    Bracket: hi = c^T x for the feasible x_i = 1 / min_{j: a_ji > 0} a_ji, and
    lo = max_j min_{i: a_ji > 0} c_i / a_ji (each row alone needs that much).
    A FEASIBLE probe lowers hi to M, any other raises lo to M; every probe's
    certified objective also lowers hi.  Same bisection reading as
    ``solve_packing``.
    """
    tol = eps if tol is None else tol
    A = sp.csr_matrix(A, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    colmin = _colmin_fast(A)
    hi = float(np.sum(c / colmin))
    # row j: min over its nonzeros of c_i / a_ji
    ratio = A.copy()
    ratio.data = c[A.indices] / A.data
    nzr = np.diff(A.indptr) > 0
    rowmin = np.minimum.reduceat(ratio.data, A.indptr[:-1][nzr]) if ratio.nnz else np.array([0.0])
    lo = float(rowmin.max())
    best = [hi, 1.0 / colmin]
    tot = {"iters": 0, "evals": 0}

    def probe(M, lo, hi):
        r = mwu(lpm.objective_row(c, M), A, eps, ratio_stop=(1 + tol) * lo / M, **kw)
        cert = certified_covering(A, c, r.x)
        tot["iters"] += r.iters
        tot["evals"] += r.evals
        if cert < best[0]:
            best[0], best[1] = cert, r.x
        hi = min(hi, cert)
        if r.status == FEASIBLE:
            hi = min(hi, M)
        else:
            lo = max(lo, M)
        return r, cert, lo, hi

    lo, hi, hist = _probe_loop(lo, hi, tol, probe)
    return SolveResult(best[0], lo, hi, len(hist), tot["iters"], tot["evals"], hist, best[1])


def solve_densest(n, u, v, eps, *, tol=None, **kw):
    """min D s.t. Wz >= 1, Oz <= D 1, z >= 0 (Sec. 3, Eq. densest_linalg), by search on D.

    Each probe is the mixed LP with P = O/D and C = W.  Bracket: lo = m/n
    (the whole graph's density, a lower bound on the optimum) and hi =
    d_max/2 (the certified D of z = 1/2 everywhere).  A FEASIBLE probe lowers
    hi to D, any other raises lo to D; certified D values also lower hi.
    """
    tol = eps if tol is None else tol
    O = lpm.pair_matrix(n, u, v)
    W = lpm.interweave(O.shape[1] // 2)
    m = W.shape[0]
    deg = np.asarray(O.sum(axis=1)).ravel()
    lo = m / n
    hi = float(deg.max()) / 2.0
    best = [hi, np.full(2 * m, 0.5)]
    tot = {"iters": 0, "evals": 0}

    def probe(D, lo, hi):
        r = mwu(O / D, W, eps, ratio_stop=(1 + tol) * lo / D, **kw)
        cert = certified_densest(O, W, r.x)
        tot["iters"] += r.iters
        tot["evals"] += r.evals
        if cert < best[0]:
            best[0], best[1] = cert, r.x
        hi = min(hi, cert)
        if r.status == FEASIBLE:
            hi = min(hi, D)
        else:
            lo = max(lo, D)
        return r, cert, lo, hi

    lo, hi, hist = _probe_loop(lo, hi, tol, probe)
    return SolveResult(best[0], lo, hi, len(hist), tot["iters"], tot["evals"], hist, best[1])


# ----------------------------------------------------------------------------
# the smoothed potential and its gradients (used by the autograd checks)
# ----------------------------------------------------------------------------


def potential(P, C, x, eta):
    """smax_eta(Px) - smin_eta(Cx): the potential of Sec. 4.1 without its 1/eta factor.

    Reading: Sec. 4.1 writes f(x) = (1/eta)(smax - smin) while the proof
    sketch of Theorem 4.1 uses smax - smin; the step test is unaffected and
    the unscaled form is the one differentiated here.
    """
    return smax(P @ x, eta) - smin(C @ x, eta)


def potential_grad_x(P, C, x, eta):
    """d potential / dx = P^T nabla smax(Px) - C^T nabla smin(Cx) = g - h."""
    g, h = gradients(P, C, P @ x, C @ x, eta)
    return g - h


def potential_grad_values(A, x, w, sign):
    """d potential / d A_ji = sign * w_j x_i for every stored entry of A (CSR order).

    sign = +1 with w = nabla smax(Px) for packing values, -1 with nabla smin(Cx) for covering values.
    """
    A = sp.csr_matrix(A)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    return sign * w[rows] * x[A.indices]
