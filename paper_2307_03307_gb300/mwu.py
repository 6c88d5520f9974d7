"""Thin Python binding of libmwu (include/mwu.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays may be
torch tensors (host or CUDA) or numpy arrays; they are passed by pointer and
the library copies what it keeps during ``mwu_create``.  All compute runs in
the CUDA library; if the library is missing this module raises ImportError
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmwu.so")

# ---------------------------------------------------------------- constants
OK = FEASIBLE = 0
INFEASIBLE, MAX_ITER, RUNNING = 1, 2, 3
ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6
PACKING, COVERING, MIXED, DENSEST = 0, 1, 2, 3
MAT_CSR, MAT_INCIDENCE, MAT_INCIDENCE_T, MAT_PAIR, MAT_INTERWEAVE, MAT_NONE = 0, 1, 2, 3, 4, 5
STEP_KARY, STEP_BINARY, STEP_STANDARD, STEP_NEWTON = 0, 1, 2, 3
PREC_F32_R64, PREC_FP64 = 0, 1
VEC_X, VEC_Y, VEC_Z, VEC_D, VEC_DY, VEC_DZ, VEC_G, VEC_H = range(8)
REASONS = {0: "none", 1: "covered", 2: "packing", 3: "d=0", 4: "alpha<1", 5: "max_iter", 6: "ratio"}


class mwu_matrix(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("val", C.c_void_p),
                ("edges", C.c_void_p), ("n_vertices", C.c_int32), ("n_edges", C.c_int64),
                ("row_bound", C.c_void_p)]


class mwu_options(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_iter", C.c_int32), ("eta_factor", C.c_double),
                ("step", C.c_int32), ("K", C.c_int32), ("max_passes", C.c_int32),
                ("warm_start", C.c_int32), ("double_single", C.c_int32), ("precision", C.c_int32),
                ("outer_tol", C.c_double), ("max_probes", C.c_int32), ("use_graph", C.c_int32),
                ("check_every", C.c_int32), ("group", C.c_int32), ("timing", C.c_int32),
                ("stop_rule", C.c_int32), ("grad_tol", C.c_double), ("stream", C.c_void_p),
                ("max_newton", C.c_int32), ("newton_tol", C.c_double), ("batch_workers", C.c_int32),
                ("drop_covered", C.c_int32), ("spmv_tiles", C.c_int32), ("h_scatter", C.c_int32),
                ("dv_scatter", C.c_int32), ("col_split", C.c_int32), ("batch_cluster", C.c_int32),
                ("batch_cluster_edges", C.c_int32)]


class mwu_iter_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("reason", C.c_int32), ("iters", C.c_int32),
                ("last_passes", C.c_int32), ("evals", C.c_int64), ("passes", C.c_int64),
                ("alpha", C.c_double), ("ymax", C.c_double), ("zmin", C.c_double)]


class mwu_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("objective", C.c_double), ("lo", C.c_double), ("hi", C.c_double),
                ("probes", C.c_int32), ("iters", C.c_int64), ("evals", C.c_int64), ("passes", C.c_int64),
                ("seconds", C.c_double), ("launches", C.c_int64)]


class mwu_timing(C.Structure):
    _fields_ = [("dir_ms", C.c_double), ("spmv_ms", C.c_double), ("cand_ms", C.c_double),
                ("update_ms", C.c_double), ("iters", C.c_int64), ("cand_passes", C.c_int64),
                ("compactions", C.c_int64)]


class mwu_scalars(C.Structure):
    _fields_ = [("eta", C.c_double), ("c_d", C.c_double), ("eps", C.c_double), ("target", C.c_double),
                ("s_p", C.c_double), ("S_p", C.c_double), ("s_c", C.c_double), ("S_c", C.c_double),
                ("ymax", C.c_double), ("zmin", C.c_double), ("alpha", C.c_double),
                ("n_positive", C.c_int64), ("n", C.c_int64), ("m_P", C.c_int64), ("m_C", C.c_int64),
                ("K", C.c_int32), ("iters", C.c_int32)]


def _as_dict(st):
    return {k: getattr(st, k) for k, _ in st._fields_}


class MWUError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmwu error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libmwu.so (built by ``__graft_entry__.build()``); ImportError if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmwu.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    V, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "mwu_default_options": (C.c_int, [P(mwu_options)]),
        "mwu_create": (C.c_int, [I32, P(mwu_matrix), P(mwu_matrix), V, P(mwu_options), P(V)]),
        "mwu_destroy": (None, [V]),
        "mwu_last_error": (C.c_char_p, [V]),
        "mwu_set_target": (C.c_int, [V, D]),
        "mwu_set_x": (C.c_int, [V, V, I32]),
        "mwu_set_state": (C.c_int, [V, V, V, V, V, I32]),
        "mwu_set_direction": (C.c_int, [V, V, I32]),
        "mwu_iterate": (C.c_int, [V, I32, P(mwu_iter_stats)]),
        "mwu_direction": (C.c_int, [V, P(I64)]),
        "mwu_eval_candidates": (C.c_int, [V, P(D), I32, P(D), P(D), P(D)]),
        "mwu_eval_newton": (C.c_int, [V, D, P(D)]),
        "mwu_search": (C.c_int, [V, P(D), P(I64)]),
        "mwu_solve": (C.c_int, [V, D, D, P(mwu_result)]),
        "mwu_get_vector": (C.c_int, [V, I32, V, I64, I32]),
        "mwu_get_scalars": (C.c_int, [V, P(mwu_scalars)]),
        "mwu_get_timing": (C.c_int, [V, P(mwu_timing), I32]),
        "mwu_spmv_tiles": (C.c_int, [V, P(I32), P(I32)]),
        "mwu_potential": (C.c_int, [V, V, P(D), V, V, V]),
        "mwu_check_values": (C.c_int, [V, V, V, P(I32)]),
        "mwu_candidates_static": (C.c_int, [V, V, I64, I32, D, D, D, P(D), I32, P(D), P(D), V]),
        "mwu_create_batch": (C.c_int, [I32, P(mwu_matrix), P(mwu_options), P(V)]),
        "mwu_diag_one_minus_exp_neg": (C.c_int, [V, V, I64, V]),
        "mwu_solve_batch": (C.c_int, [V, P(D), P(I64), P(mwu_result)]),
        "mwu_batch_tuning": (C.c_int, [V, P(I32), P(I32), P(D)]),
        "mwu_batch_stats": (C.c_int, [V, P(I64), P(I32)]),
        "mwu_batch_timeline": (C.c_int, [V, P(D), P(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return ["mwu_default_options", "mwu_create", "mwu_destroy", "mwu_last_error", "mwu_set_target",
            "mwu_set_x", "mwu_set_state", "mwu_set_direction", "mwu_iterate", "mwu_direction", "mwu_eval_candidates", "mwu_eval_newton", "mwu_search",
            "mwu_solve",
            "mwu_get_vector", "mwu_get_scalars", "mwu_get_timing", "mwu_spmv_tiles", "mwu_potential", "mwu_check_values",
            "mwu_candidates_static", "mwu_create_batch", "mwu_solve_batch", "mwu_batch_tuning", "mwu_batch_stats",
            "mwu_batch_timeline",
            "mwu_diag_one_minus_exp_neg"]


# ---------------------------------------------------------------- marshalling
def _ptr(a):
    """Data pointer of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _check(ctx, rc):
    if rc < 0:
        msg = load().mwu_last_error(ctx)
        raise MWUError(rc, msg.decode() if msg else "")
    return rc


class Matrix:
    """A mwu_matrix plus references keeping its arrays alive during mwu_create."""

    def __init__(self, kind, keep, **fields):
        self.kind = kind
        self.keep = keep
        self.s = mwu_matrix()
        self.s.kind = kind
        for k, v in fields.items():
            setattr(self.s, k, v)


def csr_matrix(rowptr, colidx, val, rows, cols, row_bound=None):
    """Explicit CSR (int32 rowptr/colidx, float32 val or None = ones)."""
    return Matrix(MAT_CSR, (rowptr, colidx, val, row_bound), rows=int(rows), cols=int(cols),
                  nnz=int(colidx.shape[0]), rowptr=_ptr(rowptr), colidx=_ptr(colidx), val=_ptr(val),
                  row_bound=_ptr(row_bound))


def implicit_matrix(kind, edges, n_vertices, row_bound=None):
    """Implicit graph matrix over an [E, 2] int32 edge list (INCIDENCE, INCIDENCE_T, PAIR, INTERWEAVE)."""
    return Matrix(kind, (edges, row_bound), edges=_ptr(edges), n_vertices=int(n_vertices),
                  n_edges=int(edges.shape[0]), row_bound=_ptr(row_bound))


def none_matrix():
    return Matrix(MAT_NONE, ())


def mwu_default_options(**kw):
    o = mwu_options()
    load().mwu_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _current_stream():
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


def mwu_create(kind, P=None, C_=None, objective=None, options=None, **kw):
    """Create a context; returns an opaque handle (int).  ``options`` or keyword options."""
    lib = load()
    o = options if options is not None else mwu_default_options(**kw)
    if o.stream is None:
        o.stream = _current_stream()
    ctx = C.c_void_p()
    Ps = C.byref(P.s) if P is not None else None
    Cs = C.byref(C_.s) if C_ is not None else None
    rc = lib.mwu_create(int(kind), Ps, Cs, _ptr(objective), C.byref(o), C.byref(ctx))
    _check(None, rc)
    return ctx.value


def mwu_destroy(ctx):
    if ctx:
        load().mwu_destroy(ctx)


def mwu_last_error(ctx=None):
    m = load().mwu_last_error(ctx)
    return m.decode() if m else ""


def mwu_set_target(ctx, target):
    return _check(ctx, load().mwu_set_target(ctx, float(target)))


def mwu_set_x(ctx, x):
    fp64 = 1 if str(getattr(x, "dtype", "")).endswith("float64") else 0
    return _check(ctx, load().mwu_set_x(ctx, _ptr(x), fp64))


def _fp64_of(*arrays):
    kinds = {str(getattr(a, "dtype", "")).endswith("float64") for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("arrays of one call must share a dtype (float32 or float64)")
    return 1 if kinds == {True} else 0


def mwu_set_state(ctx, y=None, z=None, dy=None, dz=None):
    """Load y, z, dy, dz (None keeps a vector); see mwu.h."""
    fp64 = _fp64_of(y, z, dy, dz)
    return _check(ctx, load().mwu_set_state(ctx, _ptr(y), _ptr(z), _ptr(dy), _ptr(dz), fp64))


def mwu_set_direction(ctx, d):
    """Load d and compute dy = Pd, dz = Cd on the device."""
    return _check(ctx, load().mwu_set_direction(ctx, _ptr(d), _fp64_of(d)))


def mwu_iterate(ctx, n_iters):
    st = mwu_iter_stats()
    rc = _check(ctx, load().mwu_iterate(ctx, int(n_iters), C.byref(st)))
    return rc, _as_dict(st)


def mwu_direction(ctx):
    npos = C.c_int64()
    rc = _check(ctx, load().mwu_direction(ctx, C.byref(npos)))
    return rc, npos.value


def mwu_eval_candidates(ctx, alphas):
    K = len(alphas)
    a = (C.c_double * K)(*[float(v) for v in alphas])
    psi, phi, zm = (C.c_double * K)(), (C.c_double * K)(), (C.c_double * K)()
    _check(ctx, load().mwu_eval_candidates(ctx, a, K, psi, phi, zm))
    return list(psi), list(phi), list(zm)


def mwu_eval_newton(ctx, alpha):
    """(Psi, Phi, Psi', Phi') of the last direction at one step size."""
    out = (C.c_double * 4)()
    _check(ctx, load().mwu_eval_newton(ctx, float(alpha), out))
    return tuple(out)


def mwu_diag_one_minus_exp_neg(b, stream=None):
    """1 - exp(-b) on the device by the library's candidate-pass function (b: CUDA float32 tensor)."""
    import torch
    u = torch.empty_like(b)
    if stream is None:
        stream = _current_stream()
    _check(None, load().mwu_diag_one_minus_exp_neg(_ptr(b), _ptr(u), b.numel(), stream))
    return u


def mwu_search(ctx):
    a = C.c_double()
    ev = C.c_int64()
    rc = _check(ctx, load().mwu_search(ctx, C.byref(a), C.byref(ev)))
    return rc, a.value, ev.value


def mwu_solve(ctx, lo=0.0, hi=0.0):
    r = mwu_result()
    _check(ctx, load().mwu_solve(ctx, float(lo), float(hi), C.byref(r)))
    return _as_dict(r)


def mwu_get_scalars(ctx):
    s = mwu_scalars()
    _check(ctx, load().mwu_get_scalars(ctx, C.byref(s)))
    return _as_dict(s)


def mwu_spmv_tiles(ctx):
    """(tiles of P, tiles of C) of the staged SpMV; 0 = the row-binned kernel."""
    tp, tc = C.c_int32(), C.c_int32()
    _check(ctx, load().mwu_spmv_tiles(ctx, C.byref(tp), C.byref(tc)))
    return tp.value, tc.value


def mwu_get_timing(ctx, reset=False):
    t = mwu_timing()
    _check(ctx, load().mwu_get_timing(ctx, C.byref(t), 1 if reset else 0))
    return _as_dict(t)


def mwu_get_vector(ctx, which, n, fp64=True, device=None):
    """Vector ``which`` (VEC_*) as a torch tensor on ``device`` (default: host)."""
    import torch
    t = torch.empty(int(n), dtype=torch.float64 if fp64 else torch.float32,
                    device=device if device is not None else "cpu")
    _check(ctx, load().mwu_get_vector(ctx, int(which), t.data_ptr(), int(n), 1 if fp64 else 0))
    return t


def mwu_potential(ctx, x, grad_x=None, grad_obj=None, grad_vals=None):
    pot = C.c_double()
    _check(ctx, load().mwu_potential(ctx, _ptr(x), C.byref(pot), _ptr(grad_x), _ptr(grad_obj), _ptr(grad_vals)))
    return pot.value


def mwu_check_values(ctx, objective=None, values=None):
    """True when objective / values equal the copies the context was created from."""
    def f32(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            return np.ascontiguousarray(a, dtype=np.float32)
        return a.detach().float().contiguous()

    same = C.c_int32()
    ob, va = f32(objective), f32(values)
    _check(ctx, load().mwu_check_values(ctx, _ptr(ob), _ptr(va), C.byref(same)))
    return bool(same.value)


def mwu_candidates_static(v, dv, sign, eta, shift, S, alphas, stream=None):
    """Allocation-free candidate evaluation of one side (see mwu.h); returns (val, vmin) lists."""
    K = len(alphas)
    a = (C.c_double * K)(*[float(x) for x in alphas])
    val, vmin = (C.c_double * K)(), (C.c_double * K)()
    if stream is None:
        stream = _current_stream()
    rc = load().mwu_candidates_static(_ptr(v), _ptr(dv), int(v.numel()), int(sign), float(eta), float(shift),
                                      float(S), a, K, val, vmin, stream)
    _check(None, rc)
    return list(val), list(vmin)


def mwu_create_batch(matrices, options=None, **kw):
    lib = load()
    o = options if options is not None else mwu_default_options(**kw)
    if o.stream is None:
        o.stream = _current_stream()
    arr = (mwu_matrix * len(matrices))(*[m.s for m in matrices])
    ctx = C.c_void_p()
    _check(None, lib.mwu_create_batch(len(matrices), arr, C.byref(o), C.byref(ctx)))
    return ctx.value


def mwu_solve_batch(ctx, count):
    obj = (C.c_double * count)()
    it = (C.c_int64 * count)()
    r = mwu_result()
    _check(ctx, load().mwu_solve_batch(ctx, obj, it, C.byref(r)))
    return list(obj), list(it), _as_dict(r)


# the autotuner's (threads per block, blocks per cluster), in mwu_batch_tuning's order
BATCH_TUNE_CONFIGS = ((256, 1), (512, 1), (1024, 1), (256, 4), (512, 4), (256, 8), (512, 8), (256, 16), (512, 16))


def mwu_batch_tuning(ctx):
    """(threads per block, blocks per cluster, [ms per BATCH_TUNE_CONFIGS entry])
    of the batch autotuner."""
    nt, cl = C.c_int32(), C.c_int32()
    ms = (C.c_double * len(BATCH_TUNE_CONFIGS))()
    _check(ctx, load().mwu_batch_tuning(ctx, C.byref(nt), C.byref(cl), ms))
    return nt.value, cl.value, list(ms)


def mwu_batch_timeline(ctx, count):
    """Per-instance (start ms, end ms) of the last batch solve, after the earliest start."""
    a = (C.c_double * count)()
    b = (C.c_double * count)()
    _check(ctx, load().mwu_batch_timeline(ctx, a, b))
    return list(a), list(b)


def mwu_batch_stats(ctx, count):
    """Per-instance candidate passes and probes of the last batch solve."""
    pa = (C.c_int64 * count)()
    pr = (C.c_int32 * count)()
    _check(ctx, load().mwu_batch_stats(ctx, pa, pr))
    return list(pa), list(pr)
