"""Write the FP64 oracle's certified objectives of the full-size configurations.

    python tests/golden/make_fullsize_objectives.py [densest-rmat18] [domset-rmat20]

Calls only ``oracle/`` (and ``graphgen/`` for the seeded inputs): each
workload is solved by the oracle's whole search (bisection on D or M, one MWU
probe per midpoint, Newton's step-size search of Sec. 4.2, eps = 0.1) on the
CPU, and its best certified objective (Sec. 2.2 for covering, Sec. 3 for the
densest subgraph) lands in ``fullsize_objectives.json`` beside this script.
The GPU tests compare the library's whole solve with these values within the
factor (1 + eps).  A run takes minutes (densest) to tens of minutes
(dominating set) on one core.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "fullsize_objectives.json")


def densest_rmat18():
    from graphgen import workloads as W
    from oracle import mwu as om
    wl = W.densest(18, seed=2)
    g = wl.graph
    t0 = time.perf_counter()
    r = om.solve_densest(g.n, g.u.numpy(), g.v.numpy(), wl.eps, step="newton")
    return {"lp": "densest subgraph, min D s.t. Wz >= 1, Oz <= D (Sec. 3)", "graph": "R-MAT scale 18, seed 2",
            "vertices": g.n, "edges": g.m, "eps": wl.eps, "objective": r.objective, "lo": r.lo, "hi": r.hi,
            "probes": r.probes, "iters": r.iters, "seconds": time.perf_counter() - t0}


def domset_rmat20():
    import numpy as np
    from graphgen import workloads as W
    from oracle import lp as olp
    from oracle import mwu as om
    wl = W.domset(20, seed=3)
    g = wl.graph
    A = olp.dominating(g.n, g.u.numpy(), g.v.numpy())
    c = wl.objective.numpy().astype(np.float64)
    t0 = time.perf_counter()
    r = om.solve_covering(A, c, wl.eps, step="newton")
    return {"lp": "weighted dominating set, min c^T x s.t. (I + A) x >= 1 (Sec. 3)",
            "graph": "R-MAT scale 20, seed 3, c_v in U[1,10) seed 3", "vertices": g.n, "edges": g.m,
            "eps": wl.eps, "objective": r.objective, "lo": r.lo, "hi": r.hi, "probes": r.probes, "iters": r.iters,
            "seconds": time.perf_counter() - t0}


JOBS = {"densest-rmat18": densest_rmat18, "domset-rmat20": domset_rmat20}


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data.setdefault("_about", "FP64 oracle (oracle/mwu.py), whole solve with Newton's step search, eps = 0.1; "
                              "written by tests/golden/make_fullsize_objectives.py")
    for name in names or list(JOBS):
        res = JOBS[name]()
        data[name] = res
        print(name, json.dumps(res), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
