"""A certificate check of single-source shortest distances, for graphs too
large for the oracle's Dijkstra to finish in a test.

With every weight at least 1, an array `dist` equals the exact shortest
distances from `src` (INF = 2^32 - 1 where no path exists) if and only if
  (1) dist[src] == 0,
  (2) every edge (v, u, w) with dist[v] finite has dist[u] <= dist[v] + w
      (the triangle inequality: dist is at most the true distance), and
  (3) every vertex other than src with dist finite has an in-edge (v, u, w)
      with dist[v] + w == dist[u] (a tight edge: following tight edges back
      strictly lowers dist, so it ends at src and spells out a path of length
      dist[u], and dist is at least the true distance).
The edges are streamed in chunks of whole lists so that the temporaries stay
a few hundred MB at any graph size.
"""
import numpy as np

INF = 0xFFFFFFFF


def sssp_certificate(offsets, cols, weights, src, dist, chunk_edges=1 << 25):
    """Returns None when `dist` is certified exact, else a one-line reason."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    n = offsets.size - 1
    dist = np.asarray(dist).view(np.uint32) if np.asarray(dist).dtype != np.uint32 else np.asarray(dist)
    if dist.size != n:
        return f"dist has {dist.size} entries for {n} vertices"
    if int(dist[src]) != 0:
        return f"dist[src] = {int(dist[src])}"
    d64 = dist.astype(np.int64)
    tight = np.zeros(n, dtype=bool)
    tight[src] = True
    v0 = 0
    while v0 < n:
        lo = int(offsets[v0])
        v1 = int(np.searchsorted(offsets, lo + chunk_edges, side="right")) - 1
        v1 = min(max(v1, v0 + 1), n)
        hi = int(offsets[v1])
        if hi > lo:
            w = np.asarray(weights[lo:hi], dtype=np.int64)
            if w.min() < 1:
                return "a weight below 1: the certificate needs positive weights"
            u = np.asarray(cols[lo:hi], dtype=np.int64)
            du = np.repeat(d64[v0:v1], np.diff(offsets[v0:v1 + 1]).astype(np.int64))
            dv = d64[u]
            fin = du != INF
            cand = du + w
            bad = np.flatnonzero(fin & (dv > cand))
            if bad.size:
                i = int(bad[0])
                return f"edge {lo + i} to {int(u[i])}: {int(dv[i])} > {int(du[i])} + {int(w[i])}"
            tight[u[fin & (dv == cand)]] = True
        v0 = v1
    loose = np.flatnonzero((dist != INF) & ~tight)
    if loose.size:
        return f"vertex {int(loose[0])} (dist {int(dist[loose[0]])}) has no tight in-edge"
    return None
