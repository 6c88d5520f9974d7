#!/usr/bin/env python
"""Benchmark of the MWU solver on one GB300 (or N independent replicas).

Workload (default): the densest-subgraph LP (Charikar dual, W z >= 1, O z <= D)
on a synthetic R-MAT graph of scale 18, edge factor 16, (a,b,c) = (.57,.19,.19),
seed 2, eps = 0.1, FP32 vectors with FP64 reductions, Newton's step-size
search of Sec. 4.2 (--step kary: K = 8 candidates per pass).  One step is one
complete solve (search on D, every probe's MWU
iterations with their step-size searches) to a (1+0.1)-relative certified
objective, with the problem already resident in HBM.

Metric: edges * MWU iterations / second over the timed steps (undirected
edges E, iterations summed over all probes).  Also reported: time to the
(1+0.1) approximation, the same solve in the plain FP64 GPU form, the e2e
number through the C ABI with host buffers, the dominant kernel's achieved
HBM bandwidth against the measured peak, and the oracle timed on host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import os

# before torch initialises CUDA: more hardware work queues for the concurrent
# streams of the batched solve (see the package's __init__)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse  # noqa: E402
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=18)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--step", default="newton", choices=["kary", "newton"],
                    help="step-size search: K candidates per pass (Alg. 3 generalised) or Newton (Sec. 4.2)")
    ap.add_argument("--workload", default="densest-rmat18",
                    choices=["densest-rmat18", "bmatching-batch256", "domset-rmat20", "vcover-rmat24",
                             "gmatch-200kx8k", "matching-rgg18", "domset-rgg18", "vcover-rgg18", "densest-rgg18"],
                    help="densest-rmat18 is the headline line; the others measure the remaining configurations")
    ap.add_argument("--rules", default="",
                    help="--step-table: comma-separated subset of the step rules (default: all)")
    ap.add_argument("--step-table", action="store_true",
                    help="the step-rule comparison of Table 2 on rgg-18 (a whole solve per LP and rule) instead of a bench line")
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel from the host instead of replaying captured iterations (for "
                         "profilers that cannot see the kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--one-iteration", action="store_true",
                    help="profiling aid: after a warm-up solve, run 10 eager iterations of a probe at 1.1 x the "
                         "certified density and then one more inside the NVTX range 'mwu_iteration' "
                         "(ncu --nvtx --nvtx-include mwu_iteration/ captures exactly its kernels)")
    ap.add_argument("--drop", action="store_true",
                    help="drop satisfied covering rows (the last step of Alg. 1/2's loop)")
    ap.add_argument("--h-scatter", action="store_true",
                    help="vertex cover, dominating set: h by a scatter over C's rows with atomic adds "
                         "(not bit-reproducible)")
    ap.add_argument("--dv-scatter", action="store_true",
                    help="dominating set: dz = C d by a scatter over the columns of the moving variables "
                         "(not bit-reproducible)")
    ap.add_argument("--no-tiles", action="store_true",
                    help="row-binned gather SpMV everywhere (no staged tiles for banded CSR sides)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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


def algorithmic_bytes(N, E):
    """Algorithmic bytes per launch of each kernel class on the densest-subgraph LP.

    FP32 values and int32 indices, every referenced array element counted once
    (n = 2E variable slots):
      dir        x read + written, d of the previous step read (deferred update),
                 d written, endpoint pair per edge, z per edge, y per vertex,
                 dz = W d written (fused)
      spmv       dy = (O/D) d: rowptr, slot index and d per slot, dy written
      cand       y, dy, z, dz read (one candidate pass, Newton or K-candidate)
      update     y, z read + written, dy, dz read
    """
    n = 2 * E
    return {
        "dir": 8 * n + 4 * n + 4 * n + 8 * E + 4 * E + 4 * N + 4 * E,
        "spmv": 4 * (N + 1) + 4 * n + 4 * n + 4 * N,
        "cand": 8 * N + 8 * E,
        "update": 12 * N + 12 * E,
    }


def profiled_traffic(workload, cls):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic_<workload>.md), or None when there is none or when the
    kernel source has changed since the counters were taken."""
    import hashlib
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
    from graphgen import workloads as W

    wl = W.densest(args.scale, seed=args.seed, device="cuda")
    N, E = wl.graph.n, wl.graph.m
    kind, P, C, obj = lpspec.from_workload(wl)
    stream = torch.cuda.current_stream()
    step = M.STEP_NEWTON if args.step == "newton" else M.STEP_KARY
    ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, timing=0 if args.eager else 1, step=step,
                       use_graph=0 if args.eager else 1, drop_covered=int(args.drop))
    if args.one_iteration:
        r = M.mwu_solve(ctx)
        M.mwu_destroy(ctx)
        ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, step=step, use_graph=0, drop_covered=int(args.drop))
        M.mwu_set_target(ctx, 1.1 * r["objective"])
        M.mwu_iterate(ctx, 10)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("mwu_iteration")
        rc, st = M.mwu_iterate(ctx, 1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        M.mwu_destroy(ctx)
        print(json.dumps({"one_iteration": {"workload": f"densest-rmat{args.scale}", "target": 1.1 * r["objective"],
                                            "status": st["status"], "iters": st["iters"],
                                            "last_passes": st["last_passes"], "alpha": st["alpha"]}}), flush=True)
        return
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    results = []
    for _ in range(args.warmup):
        results.append(M.mwu_solve(ctx))
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
        timed.append(M.mwu_solve(ctx))
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    tim = M.mwu_get_timing(ctx)
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    iters = sum(r["iters"] for r in timed)
    units = float(E) * iters
    launches = sum(r["launches"] for r in timed)
    total_s, units = aggregate(dist, total_s, units, "cuda")
    value = units / total_s

    # roofline of the dominant kernel class (device time from the events captured in the graph)
    ab = algorithmic_bytes(N, E)
    per_class_ms = {"dir": tim["dir_ms"], "spmv": tim["spmv_ms"], "cand": tim["cand_ms"], "update": tim["update_ms"]}
    timed_classes = sum(per_class_ms.values()) > 0.0     # no event times in --eager runs
    dom = max(per_class_ms, key=lambda k: per_class_ms[k])
    nit = max(1, tim["iters"])
    # launches per iteration: one per class, the candidate passes as counted by the library
    per_launch = {"dir": nit, "spmv": nit, "cand": max(1, tim["cand_passes"]), "update": nit}
    avg_ms = per_class_ms[dom] / per_launch[dom]
    achieved = ab[dom] / (avg_ms / 1e3) / 1e9 if timed_classes else None
    peak, peak_src = measured_peaks()
    traffic = profiled_traffic(f"densest-rmat{args.scale}", dom)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"densest-rmat{args.scale}", "lp": "densest subgraph (Charikar dual)",
                   "vertices": N, "edges": E, "variables": 2 * E, "eps": wl.eps, "K": 8, "step": args.step,
                   "covering_rows": "dropped when satisfied" if args.drop else "kept",
                   "precision": "f32 vectors, f64 reductions", "l2": "flushed (512 MB write) between steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "time_to_approx_s": statistics.mean(step_ms) / 1e3,
        "iters_per_solve": iters / args.steps,
        "probes_per_solve": sum(r["probes"] for r in timed) / args.steps,
        "objective": timed[-1]["objective"],
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": {"bound": "hbm", "kernel": {"dir": "k_dir_pairs", "spmv": "k_spmv",
                                                 "cand": "k_cand / k_cand_newton (one pass)", "update": "k_update"}[dom],
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved is not None else None,
                     "traffic": traffic, "algorithmic_bytes_per_launch": ab[dom], "avg_launch_ms": avg_ms,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6800 GB/s",
                     "per_class_ms_per_iter": {k: v / nit for k, v in per_class_ms.items()},
                     "cand_passes_per_iter": tim["cand_passes"] / nit},
    }
    M.mwu_destroy(ctx)

    if rank == 0 and not args.no_fp64:
        ctx64 = M.mwu_create(kind, P, C, obj, eps=wl.eps, precision=M.PREC_FP64, step=step,
                             drop_covered=int(args.drop))
        flush.zero_()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r64 = M.mwu_solve(ctx64)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        M.mwu_destroy(ctx64)
        line["fp64_form"] = {"time_to_approx_s": ms64 / 1e3, "value": E * r64["iters"] / (ms64 / 1e3),
                             "iters": r64["iters"], "probes": r64["probes"], "objective": r64["objective"],
                             "speedup_of_f32_form": (ms64 / 1e3) / line["time_to_approx_s"]}

    if not args.no_e2e:
        # end to end through the C ABI from pinned host buffers: create (H2D copies and
        # setup), solve, read x back (D2H)
        edges_h = wl.edges.cpu().pin_memory()
        x_h = torch.empty(2 * E, dtype=torch.float32).pin_memory()
        e2e_s, e2e_units = [], 0.0
        for k in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kd, Ph, Ch, oh = lpspec.densest_lp(N, edges_h)
            cx = M.mwu_create(kd, Ph, Ch, oh, eps=wl.eps, step=step, drop_covered=int(args.drop))
            r = M.mwu_solve(cx)
            M.load().mwu_get_vector(cx, M.VEC_X, x_h.data_ptr(), 2 * E, 0)
            M.mwu_destroy(cx)
            torch.cuda.synchronize()
            e2e_s.append(time.perf_counter() - t0)
            e2e_units += E * r["iters"]
        e2e_tot, e2e_units = aggregate(dist, sum(e2e_s), e2e_units, "cuda")
        line["e2e"] = {"value": e2e_units / e2e_tot, "unit": UNIT,
                       "h2d_bytes_per_step": int(edges_h.numel() * 4), "d2h_bytes_per_step": int(x_h.numel() * 4),
                       "seconds_per_step": statistics.mean(e2e_s)}

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = oracle_sample(wl, args.cpu_seconds, args.step)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ oracle
def oracle_sample(wl, seconds, step):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same workload:
    MWU iterations of one probe (D = 1.5 |E|/|V|) run until `seconds` elapse."""
    import numpy as np
    from oracle import lp as olp
    from oracle import mwu as om
    g = wl.graph.to("cpu")
    u, v = g.u.numpy(), g.v.numpy()
    O = olp.pair_matrix(g.n, u, v)
    Wm = olp.interweave(g.m)
    D = 1.5 * g.m / g.n
    t0 = time.perf_counter()
    count = [0]

    class Stop(Exception):
        pass

    def on_iter(it, x, y, z, a):
        count[0] = it
        if time.perf_counter() - t0 > seconds:
            raise Stop()

    try:
        om.mwu((O / D).tocsr(), Wm, wl.eps, on_iter=on_iter, step=step)
    except Stop:
        pass
    dt = time.perf_counter() - t0
    its = max(count[0], 1)
    return {"value": g.m * its / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{its} MWU iterations ({step} search) of one densest probe D=1.5|E|/|V| on the same graph, "
                      f"{dt:.1f} s, numpy/scipy single thread",
            "host_cpus": os.cpu_count()}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from graphgen import workloads as W
    import numpy as np
    from oracle import lp as olp
    from oracle import mwu as om
    wl = W.densest(args.scale, seed=args.seed, device="cpu")
    g = wl.graph
    O = olp.pair_matrix(g.n, g.u.numpy(), g.v.numpy())
    Wm = olp.interweave(g.m)
    D = 1.5 * g.m / g.n
    P = (O / D).tocsr()
    # each step: one oracle MWU iteration of a probe at D (bounded sample of the solve)
    state = {"x": None}
    times = []

    def one_iter():
        r = om.mwu(P, Wm, wl.eps, max_iter=1, x0=state["x"], step=args.step)
        state["x"] = r.x
        return r.iters

    for _ in range(args.warmup):
        one_iter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one_iter()
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = g.m * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"densest-rmat{args.scale}", "vertices": g.n, "edges": g.m, "eps": wl.eps,
                       "step": args.step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one MWU iteration ({args.step} search, cold start) per step of a densest "
                                       "probe at D=1.5|E|/|V|"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_other(args):
    """Measurement line of a configuration other than the headline one: the
    256-instance b-matching batch (one step = the whole batch), dominating set
    on R-MAT 20 over an explicit CSR, or vertex cover on R-MAT 24 (one step =
    one solve).  Same timing rules; no roofline (the byte model above is the
    densest LP's)."""
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
    from graphgen import workloads as W
    step = M.STEP_NEWTON if args.step == "newton" else M.STEP_KARY
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    batch = args.workload == "bmatching-batch256"
    if batch:
        insts = W.bmatching_batch(count=256, seed=4, device="cuda")
        mats = [lpspec.from_workload(w)[1] for w in insts]
        ctx = M.mwu_create_batch(mats, step=step)
        edges = [w.graph.m for w in insts]
        cfg = {"workload": "bmatching-batch256", "lp": "b-matching (Appendix A.1, lb = 0), 256 independent instances",
               "instances": 256, "edges": int(sum(edges)), "eps": 0.1}

        def solve():
            obj, it, tot = M.mwu_solve_batch(ctx, len(mats))
            return float(sum(e * i for e, i in zip(edges, it))), tot["iters"], tot["probes"]
    else:
        wl = {"domset-rmat20": lambda: W.domset(20, seed=3, device="cuda"),
              "vcover-rmat24": lambda: W.vcover(24, seed=5, device="cuda"),
              "gmatch-200kx8k": lambda: W.gmatch(200_000, 8_000, seed=6, device="cuda"),
              "matching-rgg18": lambda: W.rgg_lp("matching", scale=18, seed=7, device="cuda"),
              "domset-rgg18": lambda: W.rgg_lp("domset", scale=18, seed=7, device="cuda"),
              "vcover-rgg18": lambda: W.rgg_lp("vcover", scale=18, seed=7, device="cuda"),
              "densest-rgg18": lambda: W.rgg_lp("densest", scale=18, seed=7, device="cuda")}[args.workload]()
        kind, P, C, obj = lpspec.from_workload(wl)
        ctx = M.mwu_create(kind, P, C, obj, eps=wl.eps, step=step, drop_covered=int(args.drop),
                           timing=0 if args.eager else 1, use_graph=0 if args.eager else 1,
                           spmv_tiles=-1 if args.no_tiles else 0, h_scatter=int(args.h_scatter),
                           dv_scatter=int(args.dv_scatter))
        E = wl.graph.m
        lp_names = {"domset-rmat20": "dominating set, (I + A) x >= 1 explicit CSR",
                    "vcover-rmat24": "vertex cover, M^T x >= 1 implicit",
                    "gmatch-200kx8k": "generalized matching, lb <= M x <= ub (users lb 3 ub 5, items ub 200), "
                                      "feasibility",
                    "matching-rgg18": "fractional matching M x <= 1 on a random geometric graph",
                    "domset-rgg18": "dominating set on a random geometric graph",
                    "vcover-rgg18": "vertex cover on a random geometric graph",
                    "densest-rgg18": "densest subgraph on a random geometric graph"}
        cfg = {"workload": args.workload, "lp": lp_names[args.workload],
               "vertices": wl.graph.n, "edges": E, "eps": wl.eps,
               "h": "row scatter (atomic adds)" if args.h_scatter else "gather",
               "dz": "column scatter of the moving variables" if args.dv_scatter else "SpMV",
               "spmv": "staged tiles (P %d, C %d)" % M.mwu_spmv_tiles(ctx) if any(M.mwu_spmv_tiles(ctx))
               else "row-binned gathers"}

        def solve():
            r = M.mwu_solve(ctx)
            return float(E) * r["iters"], r["iters"], r["probes"]
        if args.workload == "gmatch-200kx8k":
            solve_status = M.mwu_solve(ctx)
            cfg["status"] = "feasible" if solve_status["status"] == M.OK else f"status {solve_status['status']}"
            cfg["ratio_maxPx_minCx"] = solve_status["objective"]
    for _ in range(args.warmup):
        solve()
    if not batch:
        M.mwu_get_timing(ctx, reset=True)
    clocks = ClockSampler(local_rank)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    out = []
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        out.append(solve())
        ev1[k].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    total_s, units = aggregate(dist, sum(step_ms) / 1e3, sum(o[0] for o in out), "cuda")
    cfg.update({"step": args.step, "covering_rows": "dropped when satisfied" if args.drop else "kept",
                "precision": "f32 vectors, f64 reductions",
                "l2": "flushed (512 MB write) between steps", "parallelism": "replicas" if world > 1 else "single"})
    line = {"metric": METRIC, "value": units / total_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "time_to_approx_s": statistics.mean(step_ms) / 1e3,
            "iters_per_step": sum(o[1] for o in out) / args.steps,
            "probes_per_step": sum(o[2] for o in out) / args.steps,
            "clocks": clk, "roofline": None}
    if not batch and not args.eager:
        tim = M.mwu_get_timing(ctx)
        nit = max(1, tim["iters"])
        line["per_class_ms_per_iter"] = {k: tim[f"{k}_ms"] / nit for k in ("dir", "spmv", "cand", "update")}
    M.mwu_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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
    elif args.workload != "densest-rmat18":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
