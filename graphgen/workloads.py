"""The five benchmark workloads and small stand-ins of the same structure.

Each workload is a graph plus the arrays that define one of the paper's graph
LPs (Sec. 3): the LP kind, an optional objective vector and optional row
bounds.  Inputs only; no solver arithmetic lives here.

  bmatch-2k        bipartite matching LP, 2,000 + 2,000 vertices, 20,000 uniform edges (seed 1)
  densest-rmat18   densest subgraph (Charikar dual, Sec. 3) on R-MAT scale 18, edge factor 16 (seed 2)
  domset-rmat20    weighted dominating set, explicit CSR of I + A, weights U[1,10) (seed 3)
  bmatching-256    256 bipartite b-matching LPs, edges log-uniform in [1e3, 2e5], b in 1..5 (seed 4)
  vcover-rmat24    vertex cover on R-MAT scale 24 (seed 5)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import torch

from . import (Graph, bipartite_ratings, bipartite_uniform, capacities, instance_seed, loguniform_sizes, rgg, rmat,
                symmetric_csr, vertex_weights)


@dataclass
class Workload:
    name: str
    lp: str                      # bmatch | bmatching | matching | densest | domset | vcover | gmatch
    graph: Graph
    eps: float = 0.1
    objective: Optional[torch.Tensor] = None   # float32 [n] (vertex weights for domset)
    bounds: Optional[torch.Tensor] = None      # float32 [n_vertices] (b-matching capacities)
    csr: Optional[tuple] = None                # (rowptr, colidx) of I + A for domset
    lower: Optional[torch.Tensor] = None       # float32 [n_left] lower bounds of the left vertices (gmatch)
    meta: dict = field(default_factory=dict)

    @property
    def edges(self) -> torch.Tensor:
        return self.graph.edge_pairs()

    @property
    def n_edges(self) -> int:
        return self.graph.m


def bmatch(n_left=2000, n_right=2000, m=20000, seed=1, device="cpu") -> Workload:
    g = bipartite_uniform(n_left, n_right, m, seed=seed, device=device)
    return Workload(f"bmatch-{n_left}+{n_right}-{m}", "bmatch", g)


def densest(scale=18, seed=2, device="cpu") -> Workload:
    g = rmat(scale, seed=seed, device=device)
    return Workload(f"densest-rmat{scale}", "densest", g)


def domset(scale=20, seed=3, device="cpu") -> Workload:
    g = rmat(scale, seed=seed, device=device)
    c = vertex_weights(g.n, seed=seed, device=device)
    rowptr, col = symmetric_csr(g, with_self=True)
    return Workload(f"domset-rmat{scale}", "domset", g, objective=c, csr=(rowptr, col))


def vcover(scale=24, seed=5, device="cpu") -> Workload:
    g = rmat(scale, seed=seed, device=device)
    return Workload(f"vcover-rmat{scale}", "vcover", g)


def gmatch(n_users=200_000, n_items=8_000, seed=6, lb=3.0, ub_user=5.0, ub_item=200.0, min_deg=10,
           mean_extra=20.0, eps=0.1, device="cpu") -> Workload:
    """Generalized matching (Appendix A.1): find x >= 0 with lb <= M x <= ub on a
    users x items graph; users lb 3, ub 5, items ub 200 as in the paper's
    Netflix setting (the datasets are not available; bipartite_ratings stands in)."""
    g = bipartite_ratings(n_users, n_items, min_deg=min_deg, mean_extra=mean_extra, seed=seed, device=device)
    ub = torch.full((g.n,), ub_item, dtype=torch.float32, device=device)
    ub[:n_users] = ub_user
    lower = torch.full((n_users,), lb, dtype=torch.float32, device=device)
    return Workload(f"gmatch-{n_users}x{n_items}", "gmatch", g, eps=eps, bounds=ub, lower=lower)


def rgg_lp(kind, scale=18, seed=7, device="cpu") -> Workload:
    """The graph LPs of Sec. 3 on a random geometric graph (the rgg-Y family of
    Sec. 6.3, Table 2): matching (incidence packing on the general graph),
    unweighted dominating set, vertex cover, densest subgraph."""
    g = rgg(scale, seed=seed, device=device)
    name = f"{kind}-rgg{scale}"
    if kind == "matching":
        return Workload(name, "matching", g)
    if kind == "domset":
        rowptr, col = symmetric_csr(g, with_self=True)
        return Workload(name, "domset", g, objective=torch.ones(g.n, dtype=torch.float32, device=device),
                        csr=(rowptr, col))
    if kind == "vcover":
        return Workload(name, "vcover", g)
    if kind == "densest":
        return Workload(name, "densest", g)
    raise ValueError(kind)


def bmatching_instance(m, seed, device="cpu") -> Workload:
    side = max(2, int(math.ceil(m / 10)))
    m = min(m, side * side)
    g = bipartite_uniform(side, side, m, seed=seed, device=device)
    b = capacities(g.n, seed=seed, device=device)
    return Workload(f"bmatching-{m}", "bmatching", g, bounds=b)


def bmatching_batch(count=256, seed=4, lo=1e3, hi=2e5, device="cpu") -> list:
    sizes = loguniform_sizes(count, seed, lo, hi)
    return [bmatching_instance(m, instance_seed(seed, k), device=device) for k, m in enumerate(sizes)]


WORKLOADS = {
    "bmatch-2k": lambda device="cpu": bmatch(device=device),
    "densest-rmat18": lambda device="cpu": densest(18, 2, device=device),
    "domset-rmat20": lambda device="cpu": domset(20, 3, device=device),
    "vcover-rmat24": lambda device="cpu": vcover(24, 5, device=device),
}
