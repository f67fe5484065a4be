"""The shortest-distance certificate used by the full-size GPU test accepts
the oracle's Dijkstra distances and rejects each planted mistake: a distance
one too high or too low, an unreachable vertex given a distance, a reachable
one left at INF, a wrong source distance, and a wrong weight (each found on a
uniform graph and a directed graph with unreachable vertices)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from sssp_certificate import INF, sssp_certificate


def graphs():
    yield gg.uniform(1 << 12, 8, seed=3, weights=True)
    rng = np.random.default_rng(9)
    n = 3000
    s = rng.integers(0, n, size=12000)
    d = rng.integers(0, n // 2, size=12000)  # vertices n/2.. have no in-edges
    yield gg.csr_from_edges(n, s, d, weights=rng.integers(1, 256, size=s.size), symmetrize=False,
                            name="directed-half-unreachable")


@pytest.mark.parametrize("chunk", [1, 1000, 1 << 25])
def test_certificate_accepts_dijkstra(chunk):
    for g in graphs():
        for src in (0, g.n // 3):
            dist = oracle.sssp_g(g, src)
            assert sssp_certificate(g.offsets, g.cols, g.weights, src, dist, chunk_edges=chunk) is None


def test_certificate_rejects_planted_mistakes():
    for g in graphs():
        src = 0
        exact = oracle.sssp_g(g, src)
        reach = np.flatnonzero((exact != INF) & (np.arange(g.n) != src))
        unreach = np.flatnonzero(exact == INF)
        rng = np.random.default_rng(1)
        cases = []
        for v in rng.choice(reach, size=5, replace=False):
            for delta in (1, -1):
                d = exact.copy()
                d[v] = d[v] + delta if delta > 0 else d[v] - 1
                cases.append((f"dist[{v}] {delta:+d}", d))
            d = exact.copy()
            d[v] = INF
            cases.append((f"dist[{v}] = INF", d))
        if unreach.size:
            d = exact.copy()
            d[unreach[0]] = 5
            cases.append(("unreachable given 5", d))
        d = exact.copy()
        d[src] = 1
        cases.append(("dist[src] = 1", d))
        for name, d in cases:
            assert sssp_certificate(g.offsets, g.cols, g.weights, src, d, chunk_edges=997) is not None, name
        w = g.weights.copy()
        used = np.flatnonzero(exact[g.cols.astype(np.int64)] != INF)
        w[used[len(used) // 2]] += 300  # the distances no longer fit these weights
        changed = oracle.sssp(g.n, g.offsets, g.cols, w, src)
        if not np.array_equal(changed, exact):
            assert sssp_certificate(g.offsets, g.cols, w, src, exact) is not None


def test_certificate_needs_positive_weights():
    g = gg.uniform(1 << 8, 4, seed=2, weights=True)
    w = g.weights.copy()
    w[0] = 0
    d = oracle.sssp(g.n, g.offsets, g.cols, w, 0)
    assert "positive" in sssp_certificate(g.offsets, g.cols, w, 0, d)
