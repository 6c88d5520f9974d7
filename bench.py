#!/usr/bin/env python
"""Benchmark of the MWU solver on one GB300 (or N independent replicas).

Workload (default, the headline line): the vertex-cover covering LP
(min 1^T x, M^T x >= 1, Sec. 3) on a synthetic R-MAT graph of scale 24, edge
factor 16, (a,b,c) = (.57,.19,.19), seed 5 (260,382,634 undirected edges after
merging), eps = 0.1, FP32 vectors with FP64 reductions, the step-size search
with K = 8 candidates per pass over the rows (Alg. 3 generalised).  One step
is one complete solve (search on M, every probe's MWU iterations with their
step-size searches) to a (1+0.1)-relative certified objective, with the
problem already resident in HBM.

Metric: edges * MWU iterations / second over the timed steps (undirected
edges E, iterations summed over all probes).  Also reported: time to the
(1+0.1) approximation, the same solve in the plain FP64 GPU form and with
Newton's step search (Sec. 4.2), the e2e number through the C ABI with host
buffers, the roofline of the dominant kernel class against the measured HBM
bandwidth, and the FP64 oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--step kary|newton]

--workload selects the other configurations (each with the same fields):
densest-rmat18, domset-rmat20, bmatch-2k (plain FP64 form), bmatching-batch256,
gmatch-200kx8k, and the rgg-18 lines; --step-table prints the step-rule
comparison of Table 2 instead of a bench line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges·iters/sec and time-to-(1+0.1)-approx vs plain FP64 GPU form; HBM GB/s % of peak"
UNIT = "edges*iters/s"

# workload -> (LP, description, default step rule, precision)
WORKLOADS = {
    "vcover-rmat24": ("vcover", "vertex cover, M^T x >= 1 implicit (R-MAT 24, seed 5), K = 8 candidates per pass",
                      "kary", "f32"),
    "vcover-rmat21": ("vcover", "vertex cover, M^T x >= 1 implicit (R-MAT 21, seed 5), K = 8 candidates per pass; "
                                "the profiling-size case of the same kernels", "kary", "f32"),
    "densest-rmat18": ("densest", "densest subgraph, Charikar dual W z >= 1, O z <= D (R-MAT 18, seed 2)",
                       "newton", "f32"),
    "domset-rmat20": ("domset", "weighted dominating set, (I + A) x >= 1 explicit CSR (R-MAT 20, seed 3)",
                      "newton", "f32"),
    "bmatch-2k": ("bmatch", "bipartite matching, M x <= 1 implicit (2,000 + 2,000 vertices, 20,000 edges, seed 1), "
                            "plain FP64 form", "kary", "fp64"),
    "bmatching-batch256": ("bmatching", "256 independent b-matching LPs (Appendix A.1, lb = 0), edges log-uniform "
                                        "in [1e3, 2e5], b in 1..5 (seed 4)", "newton", "f32"),
    "gmatch-200kx8k": ("gmatch", "generalized matching, lb <= M x <= ub (users lb 3 ub 5, items ub 200), "
                                 "feasibility", "newton", "f32"),
    "matching-rgg18": ("matching", "fractional matching M x <= 1 on a random geometric graph (rgg-18, seed 7)",
                       "newton", "f32"),
    "domset-rgg18": ("domset", "dominating set on a random geometric graph (rgg-18, seed 7)", "newton", "f32"),
    "vcover-rgg18": ("vcover", "vertex cover on a random geometric graph (rgg-18, seed 7)", "newton", "f32"),
    "densest-rgg18": ("densest", "densest subgraph on a random geometric graph (rgg-18, seed 7)", "newton", "f32"),
}
HEADLINE = "vcover-rmat24"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--step", default=None, choices=["kary", "newton"],
                    help="step-size search: K candidates per pass (Alg. 3 generalised) or Newton (Sec. 4.2); "
                         "default per workload")
    ap.add_argument("--scale", type=int, default=18, help="--step-table: rgg scale")
    ap.add_argument("--rules", default="",
                    help="--step-table: comma-separated subset of the step rules (default: all)")
    ap.add_argument("--step-table", action="store_true",
                    help="the step-rule comparison of Table 2 on rgg-18 (a whole solve per LP and rule) instead of a bench line")
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel from the host instead of replaying captured iterations (for "
                         "profilers that cannot see the kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--drop", action="store_true",
                    help="drop satisfied covering rows (the last step of Alg. 1/2's loop)")
    ap.add_argument("--h-scatter", action="store_true",
                    help="vertex cover, dominating set: h by a scatter over C's rows with atomic adds "
                         "(not bit-reproducible)")
    ap.add_argument("--dv-scatter", action="store_true",
                    help="dominating set: dz = C d by a scatter over the columns of the moving variables "
                         "(not bit-reproducible)")
    ap.add_argument("--no-split", action="store_true",
                    help="vertex cover: gather z over every vertex's incident edge ids instead of the split view")
    ap.add_argument("--warm-start", type=int, default=-1,
                    help="K-candidate search: 1 starts the exponential phase at the previous step size (the "
                         "start Table 2 of the paper uses), 0 at alpha = 1 (Alg. 3 as printed); -1: per workload")
    ap.add_argument("--no-tiles", action="store_true",
                    help="row-binned gather SpMV everywhere (no staged tiles for banded CSR sides)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--fp64-full", action="store_true",
                    help="the FP64 comparison as a whole solve also on graphs above 5e7 edges (many minutes)")
    ap.add_argument("--fp64-iters", type=int, default=20, help="FP64 sample iterations on large graphs")
    ap.add_argument("--no-alt", action="store_true", help="skip the comparison solve with the other step rule")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes (0: one per host core)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def aggregate(dist, seconds, units, device):
    """Whole-job throughput over N independent replicas: the slowest rank's time
    and the work units of all ranks (no data-path collective; one all-reduce of
    two numbers after the timed region).  dist = None: one process."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds, units], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ byte models
def algorithmic_bytes(lp, N, E, n_left=0, split=True, fused_pairs=True):
    """Algorithmic bytes per launch of each kernel class: FP32 values, int32
    indices, every referenced array element counted once per launch (a vector
    gathered at random counts its length once, like one streamed through).

      dir     the direction kernel(s): variables x, d; the column views of both
              sides and the constraint vectors their weights come from
      spmv    dv = A d of the sides not written by the direction kernel
      cand    one candidate pass: v, dv of every side with rows
      update  v += alpha dv (v read and written, dv read) of every side

    vcover (split view, z kept equal to x_u + x_v): dir reads x, writes d,
    reads the combined column pointers (2 x 4N), z and the endpoint list (4E
    each) and gathers x (4N once); the update also steps x (x, d read, x
    written) and rebuilds z from the edge list and x.
    """
    if lp == "vcover":
        if split:
            return {"dir": 20 * N + 8 * E, "spmv": 12 * E + 4 * N, "cand": 8 * E, "update": 12 * E + 16 * N}
        return {"dir": 20 * N + 12 * E, "spmv": 12 * E + 4 * N, "cand": 8 * E, "update": 12 * E}
    if lp == "densest":   # n = 2E slot variables, P = O/D (N rows), C = W (E rows)
        n = 2 * E
        dz = 4 * E if fused_pairs else 0
        return {"dir": 16 * n + 4 * n + 4 * N + 4 * E + dz,
                "spmv": 4 * (N + 1) + 4 * n + 4 * n + 4 * N + (0 if fused_pairs else 8 * E + 4 * E),
                "cand": 8 * N + 8 * E, "update": 12 * N + 12 * E}
    if lp == "domset":    # n = N, P = objective row c, C = I + A (N rows, N + 2E entries)
        nnz = N + 2 * E
        return {"dir": 16 * N + 4 * N + 4 * (N + 1) + 4 * nnz + 4 * N, "spmv": 4 * (N + 1) + 4 * nnz + 4 * N + 4 * N,
                "cand": 8 * N, "update": 12 * N}
    if lp in ("bmatch", "bmatching", "matching"):   # n = E, P = M (N rows), C = objective row
        bounds = 4 * N if lp == "bmatching" else 0
        return {"dir": 16 * E + 8 * E + 4 * N + bounds, "spmv": 4 * (N + 1) + 8 * E + 4 * E + 4 * N + bounds,
                "cand": 8 * N, "update": 12 * N}
    if lp == "gmatch":    # n = E, P = diag(1/ub) M (N rows), C = diag(1/lb) M_L (n_left rows over edge ids)
        nl = n_left
        return {"dir": 16 * E + 8 * E + 4 * N + 4 * N + 4 * (E + 1) + 4 * E + 4 * nl + 4 * nl,
                "spmv": 4 * (N + 1) + 8 * E + 4 * E + 4 * N + 4 * N + 4 * (nl + 1) + 4 * E + 4 * nl + 4 * nl,
                "cand": 8 * N + 8 * nl, "update": 12 * N + 12 * nl}
    raise ValueError(lp)


def batch_roofline(M, ctx, insts, last, step_ms):
    """The persistent batch solve is one kernel: its algorithmic bytes are the
    per-instance sums of every iteration's direction, SpMV and update bytes and
    every candidate pass's bytes (the byte model of one instance), over the
    kernel's time (the step's CUDA events: one graph launch)."""
    passes, _ = M.mwu_batch_stats(ctx, len(insts))
    total = 0.0
    for w, it, pa in zip(insts, last["iters_k"], passes):
        ab = algorithmic_bytes("bmatching", w.graph.n, w.graph.m)
        total += it * (ab["dir"] + ab["spmv"] + ab["update"]) + pa * ab["cand"]
    peak, src = measured_peaks()
    nt, cl, ms = M.mwu_batch_tuning(ctx)
    achieved = total / (step_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": "k_batch_solve (one persistent launch)", "class": "batch",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "algorithmic_bytes_per_launch": total, "avg_launch_ms": step_ms,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if src == "measured" else "fallback 6800 GB/s",
            "threads_per_block": nt, "blocks_per_cluster": cl,
            "autotune_ms": {f"{t}x{c}": m for (t, c), m in zip(M.BATCH_TUNE_CONFIGS, ms)},
            "note": "the instances' vectors (about 150 MB) stay largely in the 129 MB L2"}


KERNELS = {"dir": "k_dir (+ k_split_seg / k_dir_pairs / k_h_scatter)", "spmv": "k_spmv",
           "cand": "k_cand / k_cand_newton (one pass)", "update": "k_update (+ k_xstep)"}


def profiled_traffic(workload, cls):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic_<workload>.md), or None when there is none or when the
    kernel source has changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.md")
    src = os.path.join(ROOT, "paper_2307_03307_gb300", "csrc", "mwu_kernels.cu")
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if f"kernels_sha256_16: {digest}" not in text:
        return None
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) == 3 and cells[0] == cls and cells[2].isdigit():
            return int(cells[2])
    return None


def roofline(ab, tim, workload):
    """The dominant kernel class (largest device time) against the measured HBM
    bandwidth: achieved = algorithmic bytes per launch (ab, per class) / average
    launch time (CUDA events recorded in the captured iterations on the
    launching stream)."""
    per_class_ms = {k: tim[f"{k}_ms"] for k in ("dir", "spmv", "cand", "update")}
    if sum(per_class_ms.values()) <= 0.0:
        return None
    nit = max(1, tim["iters"])
    launches = {"dir": nit, "spmv": nit, "cand": max(1, tim["cand_passes"]), "update": nit}
    peak, src = measured_peaks()
    fr = {}
    for k in per_class_ms:
        avg = per_class_ms[k] / launches[k]
        fr[k] = {"ms_per_launch": avg, "launches_per_iter": launches[k] / nit,
                 "algorithmic_bytes_per_launch": ab[k], "achieved_gbs": ab[k] / (avg / 1e3) / 1e9 if avg > 0 else None}
        fr[k]["frac"] = fr[k]["achieved_gbs"] / peak if fr[k]["achieved_gbs"] else None
    dom = max(per_class_ms, key=lambda k: per_class_ms[k])
    return {"bound": "hbm", "kernel": KERNELS[dom], "class": dom, "achieved": fr[dom]["achieved_gbs"], "peak": peak,
            "unit": "GB/s", "frac": fr[dom]["frac"], "traffic": profiled_traffic(workload, dom),
            "algorithmic_bytes_per_launch": ab[dom], "avg_launch_ms": fr[dom]["ms_per_launch"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if src == "measured" else "fallback 6800 GB/s",
            "per_class_ms_per_iter": {k: v / nit for k, v in per_class_ms.items()}, "per_class": fr}


# ------------------------------------------------------------------ workloads
def make_workload(name, device):
    from graphgen import workloads as W
    return {"vcover-rmat24": lambda: W.vcover(24, seed=5, device=device),
            "vcover-rmat21": lambda: W.vcover(21, seed=5, device=device),
            "densest-rmat18": lambda: W.densest(18, seed=2, device=device),
            "domset-rmat20": lambda: W.domset(20, seed=3, device=device),
            "bmatch-2k": lambda: W.bmatch(device=device),
            "bmatching-batch256": lambda: W.bmatching_batch(count=256, seed=4, device=device),
            "gmatch-200kx8k": lambda: W.gmatch(200_000, 8_000, seed=6, device=device),
            "matching-rgg18": lambda: W.rgg_lp("matching", scale=18, seed=7, device=device),
            "domset-rgg18": lambda: W.rgg_lp("domset", scale=18, seed=7, device=device),
            "vcover-rgg18": lambda: W.rgg_lp("vcover", scale=18, seed=7, device=device),
            "densest-rgg18": lambda: W.rgg_lp("densest", scale=18, seed=7, device=device)}[name]()


def host_inputs(wl):
    """The workload's input arrays in pinned host memory (the e2e leg's H2D copies)."""
    import torch
    pin = (lambda t: t.cpu().contiguous().pin_memory()) if torch.cuda.is_available() else (lambda t: t.cpu())
    out = {"edges": pin(wl.edges)}
    if wl.csr is not None:
        out["csr"] = (pin(wl.csr[0]), pin(wl.csr[1]))
    for k in ("objective", "bounds", "lower"):
        t = getattr(wl, k)
        if t is not None:
            out[k] = pin(t)
    return out


def spec_from_host(wl, h):
    """lpspec arguments over the pinned host arrays (mwu_create copies them to the device)."""
    from paper_2307_03307_gb300 import lpspec
    g = wl.graph
    if wl.lp in ("bmatch", "bmatching", "matching"):
        return lpspec.bmatch_lp(g.n, h["edges"], h.get("bounds"))
    if wl.lp == "vcover":
        return lpspec.vcover_lp(g.n, h["edges"], h.get("objective"))
    if wl.lp == "domset":
        return lpspec.domset_lp(g.n, h["csr"][0], h["csr"][1], h.get("objective"))
    if wl.lp == "densest":
        return lpspec.densest_lp(g.n, h["edges"])
    if wl.lp == "gmatch":
        return lpspec.gmatch_lp(g.n, h["edges"], h["bounds"], h["lower"], g.n_left)
    raise ValueError(wl.lp)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2307_03307_gb300 import lpspec
    from paper_2307_03307_gb300 import mwu as M

    name = args.workload
    lp, desc, step_default, prec = WORKLOADS[name]
    step_name = args.step or step_default
    step = M.STEP_NEWTON if step_name == "newton" else M.STEP_KARY
    precision = M.PREC_FP64 if prec == "fp64" else M.PREC_F32_R64
    batch = lp == "bmatching"
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    wl = make_workload(name, "cuda")
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    warm = args.warm_start if args.warm_start >= 0 else int(step_name == "kary")
    opts = dict(step=step, precision=precision, drop_covered=int(args.drop), timing=0 if args.eager else 1,
                warm_start=warm,
                use_graph=0 if args.eager else 1, spmv_tiles=-1 if args.no_tiles else 0,
                h_scatter=int(args.h_scatter), dv_scatter=int(args.dv_scatter), col_split=-1 if args.no_split else 0)
    if batch:
        mats = [lpspec.from_workload(w)[1] for w in wl]
        edges_k = [w.graph.m for w in wl]
        E = int(sum(edges_k))
        N = int(sum(w.graph.n for w in wl))
        ctx = M.mwu_create_batch(mats, **opts)

        def solve():
            obj, it, tot = M.mwu_solve_batch(ctx, len(mats))
            return {"units": float(sum(e * i for e, i in zip(edges_k, it))), "iters": tot["iters"],
                    "probes": tot["probes"], "objective": float(sum(obj)), "launches": tot["launches"],
                    "status": tot["status"], "iters_k": list(it)}
        cfg = {"workload": name, "lp": desc, "instances": len(wl), "edges": E, "vertices": N, "eps": 0.1}
    else:
        kind, P, C, obj = lpspec.from_workload(wl)
        ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, **opts)
        N, E = wl.graph.n, wl.graph.m

        def solve():
            r = M.mwu_solve(ctx)
            return {"units": float(E) * r["iters"], "iters": r["iters"], "probes": r["probes"],
                    "objective": r["objective"], "launches": r["launches"], "status": r["status"]}
        cfg = {"workload": name, "lp": desc, "vertices": N, "edges": E, "eps": wl.eps}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        solve()
    M.mwu_get_timing(ctx, reset=True)
    clocks = ClockSampler(local_rank)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    timed = []
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()                      # evict the problem from L2 between steps
        ev0[k].record(stream)
        timed.append(solve())
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    tim = M.mwu_get_timing(ctx)
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    total_s, units = aggregate(dist, sum(step_ms) / 1e3, sum(r["units"] for r in timed), "cuda")
    iters = sum(r["iters"] for r in timed)
    split = lp == "vcover" and not args.no_split and not args.h_scatter
    if batch:
        ab = None
    else:
        ab = algorithmic_bytes(lp, N, E, wl.graph.n_left or 0, split=split, fused_pairs=lp == "densest")
    cfg.update({"step": step_name, "K": 8 if step_name == "kary" and prec == "f32" else 1, "warm_start": bool(warm),
                "covering_rows": ("dropped when satisfied (compacted rows)" if args.drop and split else
                                  "dropped when satisfied (masked in place)" if args.drop else "kept"),
                "precision": "f64 (plain form)" if prec == "fp64" else "f32 vectors, f64 reductions",
                "h": ("row scatter (atomic adds)" if args.h_scatter else
                      "split view (deterministic streams)" if split else "gather") if lp in ("vcover", "domset") else None,
                "l2": "flushed (512 MB write) between steps",
                "parallelism": "replicas" if world > 1 else "single", "graph_generation_s": t_gen})
    line = {
        "metric": METRIC, "value": units / total_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": cfg,
        "time_to_approx_s": statistics.mean(step_ms) / 1e3,
        "iters_per_solve": iters / args.steps,
        "probes_per_solve": sum(r["probes"] for r in timed) / args.steps,
        "objective": timed[-1]["objective"],
        "gpu_launches": int(sum(r["launches"] for r in timed)),
        "clocks": clk,
        "roofline": (batch_roofline(M, ctx, wl, timed[-1], statistics.mean(step_ms)) if batch else
                     roofline(ab, tim, name) if not args.eager else None),
    }
    if args.drop and line["roofline"]:
        # the byte model counts every covering row; compacted passes read only the active ones,
        # and the committed DRAM counters were taken with every row kept
        line["roofline"]["traffic"] = None
        line["roofline"]["note"] = ("algorithmic bytes count every covering row; with dropping the SpMV, "
                                    "candidate and update classes read only the active rows, so their "
                                    "fractions overstate")
    if batch:   # the e2e leg reuses the tuned block and cluster size (a fresh context would tune again)
        opts["batch_workers"], opts["batch_cluster"] = M.mwu_batch_tuning(ctx)[:2]
    M.mwu_destroy(ctx)

    if rank == 0 and not batch and not args.no_alt:
        # the same solve with the other step rule (Newton's method of Sec. 4.2 / the K-candidate search)
        alt_name = "kary" if step_name == "newton" else "newton"
        alt = dict(opts, step=M.STEP_KARY if alt_name == "kary" else M.STEP_NEWTON, timing=0)
        ctx2 = M.mwu_create(kind, P, C, obj, eps=wl.eps, **alt)
        M.mwu_solve(ctx2)   # warm
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r2 = M.mwu_solve(ctx2)
        b.record(stream)
        torch.cuda.synchronize()
        ms2 = a.elapsed_time(b)
        M.mwu_destroy(ctx2)
        line[f"{alt_name}_search"] = {"time_to_approx_s": ms2 / 1e3, "value": E * r2["iters"] / (ms2 / 1e3),
                                      "iters": r2["iters"], "probes": r2["probes"], "objective": r2["objective"]}

    if rank == 0 and not batch and prec != "fp64" and not args.no_fp64:
        ctx64 = M.mwu_create(kind, P, C, obj, eps=wl.eps, **dict(opts, precision=M.PREC_FP64, timing=0))
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.fp64_full or E < 50_000_000:
            a.record(stream)
            r64 = M.mwu_solve(ctx64)
            b.record(stream)
            torch.cuda.synchronize()
            ms64 = a.elapsed_time(b)
            line["fp64_form"] = {"time_to_approx_s": ms64 / 1e3, "value": E * r64["iters"] / (ms64 / 1e3),
                                 "iters": r64["iters"], "probes": r64["probes"], "objective": r64["objective"],
                                 "speedup_of_f32_form": (ms64 / 1e3) / line["time_to_approx_s"]}
        else:
            # a whole FP64 solve of this size takes many minutes (FP64 exponentials on
            # GB300): a bounded sample of the first probe's iterations instead
            # a probe near the optimum (the solve's longest probes sit there)
            near = 0.95 if lp in ("bmatch", "matching", "bmatching") else 1.05
            M.mwu_set_target(ctx64, near * (timed[-1]["objective"] or 1.0))
            M.mwu_iterate(ctx64, 2)
            a.record(stream)
            rc, st64 = M.mwu_iterate(ctx64, args.fp64_iters)
            b.record(stream)
            torch.cuda.synchronize()
            ms64 = a.elapsed_time(b)
            its = max(1, st64["iters"] - 2)
            f32_per_iter = line["time_to_approx_s"] / max(1.0, line["iters_per_solve"])
            line["fp64_form"] = {"value": E * its / (ms64 / 1e3), "iters_timed": its, "seconds": ms64 / 1e3,
                                 "ms_per_iter": ms64 / its, "per_iter_slowdown_vs_f32_form": (ms64 / 1e3 / its) /
                                 f32_per_iter,
                                 "sample": f"{its} MWU iterations of one probe at the F32 form's certified objective "
                                           f"x {near} (the whole solve: --fp64-full)"}
        M.mwu_destroy(ctx64)

    if not args.no_e2e:
        line["e2e"] = run_e2e(M, wl, opts, batch, dist)

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(name, wl, args.cpu_seconds, args.cpu_procs, step_name)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(M, wl, opts, batch, dist):
    """End to end through the C ABI from pinned host buffers: mwu_create (the
    H2D copies of the inputs and the setup on the device), mwu_solve, and the
    solution x read back to a host buffer (D2H), timed on the host clock."""
    import torch
    insts = wl if batch else [wl]
    hosts = [host_inputs(w) for w in insts]
    h2d = sum(sum(t.numel() * t.element_size() for t in (v if isinstance(v, tuple) else (v,)))
              for h in hosts for v in h.values())
    from paper_2307_03307_gb300 import lpspec  # noqa: F401
    esz = 8 if opts["precision"] == M.PREC_FP64 else 4
    secs, units, d2h = [], 0.0, 0
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if batch:
            mats = [spec_from_host(w, h)[1] for w, h in zip(insts, hosts)]
            cx = M.mwu_create_batch(mats, **dict(opts, timing=0))
            obj, it, tot = M.mwu_solve_batch(cx, len(mats))
            out = torch.empty(len(mats), dtype=torch.float64).pin_memory()
            out.copy_(torch.tensor(obj, dtype=torch.float64))
            M.mwu_destroy(cx)
            u = float(sum(w.graph.m * i for w, i in zip(insts, it)))
            nb = out.numel() * 8
        else:
            kd, Ph, Ch, oh = spec_from_host(wl, hosts[0])
            cx = M.mwu_create(kd, Ph, Ch, oh, eps=wl.eps, **dict(opts, timing=0))
            r = M.mwu_solve(cx)
            n = int(M.mwu_get_scalars(cx)["n"])
            x_h = torch.empty(n, dtype=torch.float64 if esz == 8 else torch.float32).pin_memory()
            M.load().mwu_get_vector(cx, M.VEC_X, x_h.data_ptr(), n, 1 if esz == 8 else 0)
            M.mwu_destroy(cx)
            u = float(wl.graph.m) * r["iters"]
            nb = n * esz
        torch.cuda.synchronize()
        secs.append(time.perf_counter() - t0)
        units += u
        d2h = nb
    tot_s, units = aggregate(dist, sum(secs), units, "cuda")
    return {"value": units / tot_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "seconds_per_step": statistics.mean(secs),
            "includes": "mwu_create from pinned host buffers (H2D + device setup), mwu_solve, x read back (D2H)"}


# ------------------------------------------------------------------ oracle (CPU)
def _oracle_lp(lp, n, u, v, target, c=None, bounds=None, lower=None, n_left=None):
    """Explicit (P, C) of one of the paper's graph LPs (Sec. 3) at probe target
    M (or D), built by the oracle's own matrix constructors."""
    import numpy as np
    from oracle import lp as olp
    if lp in ("bmatch", "bmatching", "matching"):
        A = olp.incidence(n, u, v)
        if bounds is not None:
            A = olp.row_scaled(A, bounds)
        return A, olp.objective_row(np.ones(u.size), target)
    if lp == "vcover":
        return olp.objective_row(np.ones(n), target), olp.incidence(n, u, v).T.tocsr()
    if lp == "domset":
        cc = np.ones(n) if c is None else c
        return olp.objective_row(cc, target), olp.dominating(n, u, v)
    if lp == "densest":
        return (olp.pair_matrix(n, u, v) / target).tocsr(), olp.interweave(u.size)
    if lp == "gmatch":
        Mi = olp.incidence(n, u, v)
        return olp.row_scaled(Mi, bounds), olp.row_scaled(Mi[:n_left], lower)
    raise ValueError(lp)


def _probe_target(lp, n, m, c=None, bounds=None, n_left=None):
    """A probe target inside the search bracket (the first midpoints of the search)."""
    if lp in ("bmatch", "matching"):
        return 0.6 * (n_left if n_left else n / 2)
    if lp == "bmatching":
        return 0.6 * float(bounds[:n_left].sum())
    if lp == "vcover":
        return 0.55 * n
    if lp == "domset":
        return 0.3 * (float(c.sum()) if c is not None else float(n))
    if lp == "densest":
        return 1.5 * m / n
    return 1.0


def oracle_worker(job):
    """One process of the CPU baseline: the FP64 oracle, as it stands, on one
    slice of the workload: MWU iterations of one probe, the probe restarted
    whenever it ends, until `seconds` elapse (or `iters` iterations after
    `warmup`).  Returns (edges, timed iterations, timed seconds)."""
    from oracle import mwu as om
    lp, n, u, v, extra, seconds, step, warmup, iters = job
    P, C = _oracle_lp(lp, n, u, v, _probe_target(lp, n, u.size, **{k: extra[k] for k in extra if k in
                                                                     ("c", "bounds", "n_left")}), **extra)
    state = {"g": 0, "t0": time.perf_counter() if warmup == 0 else None, "t_end": None}

    class Stop(Exception):
        pass

    def on_iter(it, x, y, z, a):
        state["g"] += 1
        g = state["g"]
        if g == warmup:
            state["t0"] = time.perf_counter()
        if state["t0"] is not None and g >= warmup:
            done = (g - warmup >= iters) if iters else (time.perf_counter() - state["t0"] > seconds)
            if done:
                state["t_end"] = time.perf_counter()
                raise Stop()

    while True:
        try:
            r = om.mwu(P, C, 0.1, on_iter=on_iter, step=step, max_iter=10 ** 6)
        except Stop:
            break
        if r.iters == 0:   # a probe that cannot take a step: nothing more to time
            break
    t_end = state["t_end"] or time.perf_counter()
    t0 = state["t0"] if state["t0"] is not None else t_end
    return u.size, max(0, state["g"] - warmup), t_end - t0


def _relabel(u, v):
    import numpy as np
    ids, inv = np.unique(np.concatenate([u, v]), return_inverse=True)
    return ids.size, inv[: u.size].astype(np.int64), inv[u.size:].astype(np.int64), ids


def oracle_jobs(name, wl, procs, seconds, step, warmup=0, iters=0):
    """Disjoint slices of the workload, one per process: consecutive blocks of
    at most 4,194,304 edges of the (sorted) edge list, vertices renumbered to
    those the block touches (a subgraph of the same graph); small workloads are
    run whole by every process (the batch: one instance per process)."""
    import numpy as np
    lp = WORKLOADS[name][0]
    jobs = []
    if lp == "bmatching":
        ws = sorted(wl, key=lambda w: w.graph.m)
        pick = [ws[int(k * (len(ws) - 1) / max(1, procs - 1))] for k in range(procs)]
        for w in pick:
            g = w.graph
            jobs.append((lp, g.n, g.u.cpu().numpy().astype(np.int64), g.v.cpu().numpy().astype(np.int64),
                         {"bounds": w.bounds.cpu().numpy().astype(np.float64), "n_left": g.n_left},
                         seconds, step, warmup, iters))
        return jobs, "one instance per process across the size range"
    g = wl.graph
    u_all = g.u.cpu().numpy().astype(np.int64)
    v_all = g.v.cpu().numpy().astype(np.int64)
    S = 4_194_304
    if lp in ("bmatch", "gmatch") or g.m <= S:
        extra = {}
        if lp == "gmatch":
            extra = {"bounds": wl.bounds.cpu().numpy().astype(np.float64),
                     "lower": wl.lower.cpu().numpy().astype(np.float64), "n_left": g.n_left}
        if lp == "domset":
            extra = {"c": wl.objective.cpu().numpy().astype(np.float64)}
        if lp == "bmatch":
            extra = {"n_left": g.n_left}
        jobs = [(lp, g.n, u_all, v_all, extra, seconds, step, warmup, iters) for _ in range(procs)]
        return jobs, "the whole workload in every process"
    nblocks = max(1, min(procs, g.m // S))
    for k in range(procs):
        b = k % nblocks
        u, v = u_all[b * S:(b + 1) * S], v_all[b * S:(b + 1) * S]
        n, uu, vv, ids = _relabel(u, v)
        extra = {}
        if lp == "domset":
            extra = {"c": wl.objective.cpu().numpy().astype(np.float64)[ids]}
        jobs.append((lp, n, uu, vv, extra, seconds, step, warmup, iters))
    return jobs, f"{nblocks} disjoint blocks of {S:,} consecutive edges of the same graph (vertices renumbered)"


def run_oracle_jobs(jobs):
    """Run the jobs in spawned processes (never forked from a CUDA process) at
    the same time; returns (edges x iterations summed, wall seconds of the
    slowest process)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        res = pool.map(oracle_worker, jobs)
    units = sum(e * it for e, it, _ in res)
    wall = max(dt for _, _, dt in res)
    return units, wall, res


def cpu_baseline(name, wl, seconds, procs, step):
    """The FP64 CPU oracle on all host cores: one single-threaded oracle
    process per core, each on its own slice of the same workload, run at the
    same time for about `seconds`; the aggregate edges x iterations per second."""
    procs = procs or os.cpu_count() or 1
    jobs, how = oracle_jobs(name, wl, procs, seconds, step)
    units, wall, res = run_oracle_jobs(jobs)
    its = [it for _, it, _ in res]
    return {"value": units / wall if wall > 0 else None, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes of the FP64 oracle (numpy/scipy, one thread each), one probe's MWU "
                      f"iterations ({step} search) for about {seconds:.0f} s each; slices: {how}; "
                      f"iterations per process {min(its)}..{max(its)}",
            "host_cpus": os.cpu_count()}


def run_reference(args):
    """The oracle arm: the FP64 oracle as it stands, on the machine's host cores
    (one process per core on its own slice of the same workload), W untimed
    iterations then K timed ones per process.  The workload's graph is
    generated on the GPU when there is one (inputs only) and copied to the host."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    name = args.workload
    lp, desc, step_default, prec = WORKLOADS[name]
    step = args.step or step_default
    dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda"
    except ImportError:
        pass
    wl = make_workload(name, dev)
    procs = args.cpu_procs or os.cpu_count() or 1
    jobs, how = oracle_jobs(name, wl, procs, 0.0, step, warmup=args.warmup, iters=args.steps)
    units, wall, res = run_oracle_jobs(jobs)
    value = units / wall if wall > 0 else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "lp": desc, "step": step, "eps": 0.1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"each step: one MWU iteration ({step} search) of one probe in each of "
                                       f"{procs} oracle processes at once; slices: {how}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ Table 2
def run_step_table(args):
    """Table 2 of Sec. 6: MWU iterations, step-size evaluations per iteration and
    time of a whole solve (bisection on M or D to a (1+0.1)-relative certified
    objective) with the standard step (alpha = 1, Alg. 1), Alg. 3's bisection
    (warm-started from the previous alpha, as in the table), the K = 8
    candidate search and Newton's method (Sec. 4.2), on the LPs of rgg-18.
    The standard step gets 30000 iterations per probe (the table's counts
    exceed the usual 5000)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2307_03307_gb300 import lpspec
    from paper_2307_03307_gb300 import mwu as M
    from graphgen import workloads as W
    rules = [("std", dict(step=M.STEP_STANDARD, max_iter=30000)), ("bin", dict(step=M.STEP_BINARY, warm_start=1)),
             ("kary8", dict(step=M.STEP_KARY, K=8)), ("newton", dict(step=M.STEP_NEWTON)),
             # the same rules with the ratio stopping test (stop_rule = 1): a probe ends as soon
             # as x / min(Cx) is a (1+eps)-relative solution
             ("bin_ratio", dict(step=M.STEP_BINARY, warm_start=1, stop_rule=1)),
             ("newton_ratio", dict(step=M.STEP_NEWTON, stop_rule=1)),
             # Newton with the satisfied covering rows dropped (Alg. 1/2's last step)
             ("newton_drop", dict(step=M.STEP_NEWTON, drop_covered=1))]
    rows = {}
    for kind in ["matching", "domset", "vcover", "densest"]:
        wl = W.rgg_lp(kind, scale=args.scale, seed=7, device="cuda")
        spec = lpspec.from_workload(wl)
        row = {"vertices": wl.graph.n, "edges": wl.graph.m}
        for name, opts in rules:
            if args.rules and name not in args.rules.split(","):
                continue
            ctx = M.mwu_create(*spec, eps=wl.eps, **opts)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = M.mwu_solve(ctx)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            M.mwu_destroy(ctx)
            row[name] = {"iters": r["iters"], "evals_per_iter": r["evals"] / max(1, r["iters"]),
                         "probes": r["probes"], "objective": r["objective"], "seconds": dt}
        rows[kind] = row
    print(json.dumps({"table": "step rules on rgg-18, whole solves", "graph": f"rgg-{args.scale} seed 7",
                      "eps": 0.1, "rows": rows}), flush=True)


def main():
    args = parse()
    if args.step_table:
        run_step_table(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
