"""Input generators: the random geometric graph against brute force, and the
counter-based streams' determinism (CPU)."""
import math

import numpy as np
import torch

import graphgen as gg


def test_rgg_equals_bruteforce():
    g = gg.rgg(9, seed=3)
    n = g.n
    idx = torch.arange(n, dtype=torch.int64)
    px = gg.uniform01(3, gg._S_GEO, 2 * idx).numpy()
    py = gg.uniform01(3, gg._S_GEO, 2 * idx + 1).numpy()
    r = g.meta["radius"]
    assert abs(math.pi * r * r * n - 30.0) < 1e-9
    d2 = (px[:, None] - px[None, :]) ** 2 + (py[:, None] - py[None, :]) ** 2
    want = {(i, j) for i in range(n) for j in range(i + 1, n) if d2[i, j] < r * r}
    gsz = max(1, int(math.floor(1 / r)))
    cx = np.minimum((px * gsz).astype(np.int64), gsz - 1)
    cy = np.minimum((py * gsz).astype(np.int64), gsz - 1)
    order = np.argsort((cy * gsz + cx) * n + np.arange(n), kind="stable")
    got = {tuple(sorted((int(order[a]), int(order[b])))) for a, b in zip(g.u.tolist(), g.v.tolist())}
    assert got == want
    assert (g.u < g.v).all()


def test_rgg_size_and_band():
    g = gg.rgg(14, seed=7)
    assert 13.5 < g.m / g.n < 16.0                      # |E| about 15 |V|
    # cell-major numbering keeps most edges near the diagonal
    span = (g.v - g.u).double()
    assert float(span.median()) < 0.02 * g.n


def test_generators_are_deterministic():
    a = gg.rgg(10, seed=5)
    b = gg.rgg(10, seed=5)
    assert torch.equal(a.u, b.u) and torch.equal(a.v, b.v)
    r1 = gg.rmat(10, seed=2)
    r2 = gg.rmat(10, seed=2)
    assert torch.equal(r1.u, r2.u) and torch.equal(r1.v, r2.v)
