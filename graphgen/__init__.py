"""Seeded synthetic graph generators shared by the oracle, the tests and the benchmark.

This module produces inputs only: edge lists, vertex weights, capacities and
batch sizes.  It holds none of the solver's arithmetic (no constraint matrices,
no weights, no step logic), so that the CPU oracle and the CUDA path can both
consume the same graphs without sharing any code of the method.

Randomness is counter based: every random word is SplitMix64 applied to
``seed_state + (counter + 1) * GAMMA`` (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Only 64-bit integer arithmetic
is used, so a graph is bit-identical whether it is generated on the CPU or on a
CUDA device, on x86 or on Arm.

Workload structure follows the paper's inputs: Graph500-style Kronecker/R-MAT
graphs (Sec. 6.3, Table 1) and random bipartite graphs (the ``bmatch`` LP of
Sec. 3 and the generalized matching of Appendix A.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import torch

_MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(v: int) -> int:
    """Reinterpret an unsigned 64-bit Python int as a signed int64 value."""
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor (torch's >> is arithmetic)."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 tensors (wrapping arithmetic)."""
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    return z ^ _lsr(z, 31)


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def stream_state(seed: int, stream: int) -> int:
    """Starting state of an independent counter stream (seed, stream)."""
    return _mix64_int((seed * GAMMA + _mix64_int(stream + 0x5EED)) & _MASK64)


def random_words(seed: int, stream: int, counters: torch.Tensor) -> torch.Tensor:
    """64-bit random words (as int64) for the given int64 counters."""
    base = stream_state(seed, stream)
    st = counters.to(torch.int64) * _s64(GAMMA) + _s64(base + GAMMA)
    return _mix64(st)


def random_top_bits(seed: int, stream: int, counters: torch.Tensor, bits: int) -> torch.Tensor:
    """The top ``bits`` bits (bits <= 63) of each random word, as non-negative int64."""
    return _lsr(random_words(seed, stream, counters), 64 - bits)


def uniform01(seed: int, stream: int, counters: torch.Tensor) -> torch.Tensor:
    """float64 uniforms in [0, 1) with 53 random bits."""
    return random_top_bits(seed, stream, counters, 53).to(torch.float64) * (2.0 ** -53)


# Stream ids (fixed, so that the same seed gives independent streams per purpose).
_S_RMAT, _S_PERM, _S_BIP, _S_WEIGHT, _S_CAP, _S_SIZES, _S_INST, _S_RATE, _S_GEO = 1, 2, 3, 4, 5, 6, 7, 8, 9


@dataclass
class Graph:
    """Undirected simple graph: edges (u[e], v[e]) with u < v, sorted, no duplicates.

    ``n`` is the vertex count.  For bipartite graphs ``n_left`` vertices
    0..n_left-1 form one side and n_left..n-1 the other.
    """
    n: int
    u: torch.Tensor  # int32 [E]
    v: torch.Tensor  # int32 [E]
    n_left: Optional[int] = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.u.numel())

    def to(self, device) -> "Graph":
        return Graph(self.n, self.u.to(device), self.v.to(device), self.n_left, dict(self.meta))

    def edge_pairs(self) -> torch.Tensor:
        """Edge list as an [E, 2] int32 tensor (u, v)."""
        return torch.stack([self.u, self.v], dim=1).contiguous()

    def degrees(self) -> torch.Tensor:
        deg = torch.zeros(self.n, dtype=torch.int64, device=self.u.device)
        one = torch.ones_like(self.u, dtype=torch.int64)
        deg.index_add_(0, self.u.long(), one)
        deg.index_add_(0, self.v.long(), one)
        return deg


def _canonical_unique(u: torch.Tensor, v: torch.Tensor, n: int):
    """Drop self loops, orient each edge as (min, max), deduplicate, sort by (u, v)."""
    keep = u != v
    u, v = u[keep], v[keep]
    a = torch.minimum(u, v)
    b = torch.maximum(u, v)
    key = torch.unique(a * n + b, sorted=True)
    return (key // n).to(torch.int32), (key % n).to(torch.int32)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, device="cpu", chunk: int = 1 << 25) -> Graph:
    """R-MAT / Graph500 Kronecker generator.

    Draws ``edge_factor * 2**scale`` directed samples.  Each sample picks one of
    the four quadrants per level with probabilities (a, b, c, 1-a-b-c) using a
    32-bit threshold compare on a counter-based random word; quadrant b sets
    the column bit, c the row bit, d both.  Vertex ids are then relabelled by a
    seeded random permutation (Graph500 convention), self loops are removed
    and undirected duplicates merged.
    """
    n = 1 << scale
    samples = edge_factor * n
    ta = int(a * 2 ** 32)
    tab = int((a + b) * 2 ** 32)
    tabc = int((a + b + c) * 2 ** 32)
    # relabelling permutation: vertex k gets the rank of its random key
    keys = random_top_bits(seed, _S_PERM, torch.arange(n, device=device), 62)
    order = torch.argsort(keys, stable=True)
    label = torch.empty(n, dtype=torch.int64, device=device)
    label[order] = torch.arange(n, device=device)
    us, vs = [], []
    for lo in range(0, samples, chunk):
        hi = min(samples, lo + chunk)
        idx = torch.arange(lo, hi, device=device, dtype=torch.int64)
        u = torch.zeros_like(idx)
        v = torch.zeros_like(idx)
        for lev in range(scale):
            r = random_top_bits(seed, _S_RMAT, idx * scale + lev, 32)
            ubit = (r >= tab).to(torch.int64)
            vbit = ((r >= ta) & (r < tab)) | (r >= tabc)
            u |= ubit << lev
            v |= vbit.to(torch.int64) << lev
        us.append(label[u])
        vs.append(label[v])
    u = torch.cat(us)
    v = torch.cat(vs)
    del us, vs
    uu, vv = _canonical_unique(u, v, n)
    return Graph(n, uu, vv, None, {"generator": "rmat", "scale": scale, "edge_factor": edge_factor,
                                   "a": a, "b": b, "c": c, "seed": seed, "samples": samples})


def bipartite_uniform(n_left: int, n_right: int, m: int, seed: int = 1, device="cpu") -> Graph:
    """Uniform random bipartite graph with exactly ``m`` distinct edges.

    Candidate pairs (l, r) are drawn from the counter stream in order; the first
    ``m`` distinct ones are kept.  Right vertices are numbered n_left..n-1.
    """
    total = n_left * n_right
    if m > total:
        raise ValueError("more edges requested than vertex pairs")
    draw = max(2 * m, 64)
    while True:
        idx = torch.arange(draw, device=device, dtype=torch.int64)
        key = random_top_bits(seed, _S_BIP, idx, 62) % total
        sk, perm = torch.sort(key, stable=True)
        first = torch.ones_like(sk, dtype=torch.bool)
        first[1:] = sk[1:] != sk[:-1]
        firsts = torch.sort(perm[first]).values
        if firsts.numel() >= m:
            break
        draw *= 2
    chosen = torch.sort(key[firsts[:m]]).values
    u = (chosen // n_right).to(torch.int32)
    v = (chosen % n_right + n_left).to(torch.int32)
    return Graph(n_left + n_right, u, v, n_left, {"generator": "bipartite_uniform", "n_left": n_left,
                                                 "n_right": n_right, "m": m, "seed": seed})


def rgg(scale: int, avg_deg: float = 30.0, seed: int = 1, device="cpu") -> Graph:
    """Random geometric graph (the rgg-Y family of Sec. 6.3: planar-like, |E| about
    15 |V|): n = 2**scale points uniform in the unit square, an edge between two
    points closer than r with pi r^2 n = avg_deg.  Vertices are numbered in the
    order of the r x r grid cells (row-major), which gives the banded structure
    of the paper's rgg matrices.  Exact pair test in float64; duplicates cannot
    occur (each unordered cell pair is visited once)."""
    n = 1 << scale
    r = math.sqrt(avg_deg / (math.pi * n))
    idx = torch.arange(n, device=device, dtype=torch.int64)
    px = uniform01(seed, _S_GEO, 2 * idx)
    py = uniform01(seed, _S_GEO, 2 * idx + 1)
    g = max(1, int(math.floor(1.0 / r)))
    cx = torch.clamp((px * g).to(torch.int64), max=g - 1)
    cy = torch.clamp((py * g).to(torch.int64), max=g - 1)
    cell = cy * g + cx
    order = torch.argsort(cell * n + idx)                 # cell-major numbering, stable within a cell
    px, py, cell = px[order], py[order], cell[order]
    counts = torch.bincount(cell, minlength=g * g)
    start = torch.zeros(g * g + 1, dtype=torch.int64, device=device)
    start[1:] = torch.cumsum(counts, 0)
    us, vs = [], []
    r2 = r * r
    # each unordered pair of neighbouring cells once: the cell itself and 4 of its 8 neighbours
    for dx, dy in [(0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]:
        ca = torch.arange(g * g, device=device, dtype=torch.int64)
        ax, ay = ca % g, ca // g
        bx, by = ax + dx, ay + dy
        ok = (bx >= 0) & (bx < g) & (by < g)
        ca, cb = ca[ok], (by * g + bx)[ok]
        na, nb = counts[ca], counts[cb]
        npairs = na * nb
        keep = npairs > 0
        ca, cb, na, nb, npairs = ca[keep], cb[keep], na[keep], nb[keep], npairs[keep]
        tot = int(npairs.sum().item())
        if tot == 0:
            continue
        pair_cell = torch.repeat_interleave(torch.arange(ca.numel(), device=device), npairs)
        off = torch.arange(tot, device=device, dtype=torch.int64) - torch.repeat_interleave(
            torch.cumsum(npairs, 0) - npairs, npairs)
        ia = start[ca][pair_cell] + off // nb[pair_cell]
        ib = start[cb][pair_cell] + off % nb[pair_cell]
        if dx == 0 and dy == 0:
            sel = ia < ib
            ia, ib = ia[sel], ib[sel]
        d2 = (px[ia] - px[ib]) ** 2 + (py[ia] - py[ib]) ** 2
        close = d2 < r2
        us.append(ia[close])
        vs.append(ib[close])
    u = torch.cat(us)
    v = torch.cat(vs)
    uu, vv = _canonical_unique(u, v, n)
    return Graph(n, uu, vv, None, {"generator": "rgg", "scale": scale, "avg_deg": avg_deg, "radius": r,
                                   "seed": seed})


def bipartite_ratings(n_users: int, n_items: int, min_deg: int = 10, mean_extra: float = 20.0, skew: float = 3.0,
                      seed: int = 1, device="cpu") -> Graph:
    """Users x items rating graph (the structure of the generalized-matching
    inputs of Appendix A.2: every user rates at least ``min_deg`` items, item
    popularity skewed).  User u rates min_deg + floor(Exp(mean_extra)) items;
    each rating picks item floor(n_items * U**skew) (skew > 1 favours low item
    ids); repeated (user, item) pairs are merged.  Users are 0..n_users-1,
    items n_users..n-1.
    """
    users = torch.arange(n_users, device=device, dtype=torch.int64)
    ue = uniform01(seed, _S_RATE, users)
    extra = torch.floor(-mean_extra * torch.log1p(-ue)).to(torch.int64)
    deg = min_deg + extra
    total = int(deg.sum().item())
    owner = torch.repeat_interleave(users, deg)
    r = uniform01(seed, _S_RATE, torch.arange(n_users, n_users + total, device=device, dtype=torch.int64))
    item = torch.clamp(torch.floor(n_items * r.pow(skew)).to(torch.int64), max=n_items - 1)
    key = torch.unique(owner * n_items + item, sorted=True)
    u = (key // n_items).to(torch.int32)
    v = (key % n_items + n_users).to(torch.int32)
    return Graph(n_users + n_items, u, v, n_users, {"generator": "bipartite_ratings", "n_users": n_users,
                                                   "n_items": n_items, "min_deg": min_deg, "mean_extra": mean_extra,
                                                   "skew": skew, "seed": seed})


def vertex_weights(n: int, seed: int, lo: float = 1.0, hi: float = 10.0, device="cpu") -> torch.Tensor:
    """float32 weights uniform in [lo, hi), rounded once from float64."""
    u = uniform01(seed, _S_WEIGHT, torch.arange(n, device=device))
    return (lo + (hi - lo) * u).to(torch.float32)


def capacities(n: int, seed: int, lo: int = 1, hi: int = 5, device="cpu") -> torch.Tensor:
    """Integer capacities uniform in {lo..hi}, returned as float32 (exact)."""
    r = random_top_bits(seed, _S_CAP, torch.arange(n, device=device), 32)
    return (lo + r % (hi - lo + 1)).to(torch.float32)


def loguniform_sizes(count: int, seed: int, lo: float, hi: float) -> list:
    """Integer sizes floor(10**U(log10 lo, log10 hi)), computed on the host in float64."""
    u = uniform01(seed, _S_SIZES, torch.arange(count)).tolist()
    l0, l1 = math.log10(lo), math.log10(hi)
    return [int(math.floor(10.0 ** (l0 + x * (l1 - l0)))) for x in u]


def instance_seed(seed: int, k: int) -> int:
    """Seed of the k-th instance of a batch (a word of its own counter stream)."""
    return int(random_top_bits(seed, _S_INST, torch.tensor([k]), 31).item())


def symmetric_csr(g: Graph, with_self: bool = False):
    """CSR of the symmetric adjacency (optionally with the diagonal), column-sorted rows.

    Returns (rowptr int32 [n+1], colidx int32 [nnz]).  Structure only: the
    values of any matrix built on it are the caller's business.
    """
    dev = g.u.device
    r = torch.cat([g.u, g.v]).long()
    c = torch.cat([g.v, g.u]).long()
    if with_self:
        ar = torch.arange(g.n, device=dev)
        r = torch.cat([r, ar])
        c = torch.cat([c, ar])
    key = torch.sort(r * g.n + c).values
    r = key // g.n
    c = key % g.n
    counts = torch.bincount(r, minlength=g.n)
    rowptr = torch.zeros(g.n + 1, dtype=torch.int64, device=dev)
    rowptr[1:] = torch.cumsum(counts, 0)
    return rowptr.to(torch.int32), c.to(torch.int32)
