"""Shared helpers of the parity tests: small workloads, the oracle's explicit
matrices for a workload, and tolerance checks."""
import math

import numpy as np
import scipy.sparse as sp
import torch

import graphgen as gg
from graphgen import workloads as W
from oracle import lp as olp
from oracle import mwu as om

EPS = 0.1

# Relative tolerance of a product computed from identical inputs: a few FP32
# roundings (FP32 form) or FP64 roundings (FP64 form).
REL = {"f32": 1e-5, "fp64": 1e-12}


def small_workloads():
    """Workloads the oracle finishes in seconds that still span many blocks and ragged tails."""
    return {
        "bmatch": W.bmatch(300, 300, 3001, seed=11),
        "bmatching": W.bmatching_instance(2999, seed=12),
        "densest": W.densest(10, seed=13),
        "gmatch": W.gmatch(600, 60, seed=16, min_deg=6, mean_extra=8.0),
        "domset": W.domset(10, seed=14),
        "vcover": W.vcover(11, seed=15),
    }


def oracle_matrices(wl, target):
    """Explicit (P, C, objective c or None) of a workload at probe target M (or D)."""
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    if wl.lp in ("bmatch", "bmatching", "matching"):
        A = olp.incidence(g.n, u, v)
        if wl.bounds is not None:
            A = olp.row_scaled(A, wl.bounds.numpy())
        c = np.ones(g.m)
        return A, olp.objective_row(c, target), c
    if wl.lp == "vcover":
        A = olp.incidence(g.n, u, v).T.tocsr()
        c = np.ones(g.n)
        return olp.objective_row(c, target), A, c
    if wl.lp == "domset":
        A = olp.dominating(g.n, u, v)
        c = wl.objective.numpy().astype(np.float64)
        return olp.objective_row(c, target), A, c
    if wl.lp == "densest":
        O = olp.pair_matrix(g.n, u, v)
        Wm = olp.interweave(g.m)
        return (O / target).tocsr(), Wm, None
    if wl.lp == "gmatch":
        Mi = olp.incidence(g.n, u, v)
        return olp.row_scaled(Mi, wl.bounds.numpy()), olp.row_scaled(Mi[: g.n_left], wl.lower.numpy()), None
    raise ValueError(wl.lp)


def oracle_solve(wl, **kw):
    g = wl.graph
    u, v = g.u.numpy(), g.v.numpy()
    if wl.lp in ("bmatch", "bmatching", "matching"):
        A = olp.incidence(g.n, u, v)
        if wl.bounds is not None:
            A = olp.row_scaled(A, wl.bounds.numpy())
        return om.solve_packing(A, np.ones(g.m), wl.eps, **kw)
    if wl.lp == "vcover":
        return om.solve_covering(olp.incidence(g.n, u, v).T.tocsr(), np.ones(g.n), wl.eps, **kw)
    if wl.lp == "domset":
        return om.solve_covering(olp.dominating(g.n, u, v), wl.objective.numpy().astype(np.float64), wl.eps, **kw)
    if wl.lp == "densest":
        return om.solve_densest(g.n, u, v, wl.eps, **kw)
    raise ValueError(wl.lp)


def n_vars(wl):
    g = wl.graph
    if wl.lp in ("bmatch", "bmatching", "matching"):
        return g.m
    if wl.lp == "densest":
        return 2 * g.m
    if wl.lp == "gmatch":
        return g.m
    return g.n


# Weights exp(+-eta (v - s)) below these fractions of the largest one are not
# representable (FP32: e^-87 ~ 1.6e-38 underflows; FP64: e^-708), so sums made
# only of such weights are compared with an absolute floor at that level.
UNDERFLOW = {"f32": 1e-35, "fp64": 1e-295}


def assert_rel(got, want, rel, abs_=0.0, what="", floor=0.0):
    """|got - want| <= rel |want| + abs_ + floor * max|want| elementwise."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    err = np.abs(got - want)
    scale = float(np.max(np.abs(want))) if want.size else 0.0
    tol = rel * np.abs(want) + abs_ + floor * scale
    bad = err > tol
    if bad.any():
        idx = np.flatnonzero(bad.ravel())
        ratio = err.ravel()[idx] / np.maximum(tol.ravel()[idx], 1e-320)
        i = int(idx[int(np.argmax(ratio))])
        raise AssertionError(f"{what}: {int(bad.sum())}/{bad.size} outside tolerance; worst i={i} "
                             f"got={got.flat[i]!r} want={want.flat[i]!r} "
                             f"rel={err.flat[i] / max(abs(want.flat[i]), 1e-320):.3e}")
