"""Pins for the CPU oracle: brute force, library routines, invariants, closed forms.

Nothing here compares the oracle with itself.  Each check comes from the
mathematics of the problem (Sec. 2.1 traversal flow; BFS, SSSP and CC as
defined in Sec. 5.1.2 / 5.4) or from values the paper prints (link model,
Sec. 3.3 / 5.3.1), and the mutation test at the end shows that plausible
mistakes planted in the oracle's C source fail at least one of them.
"""
import ctypes
import itertools
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import linkmodel

INF = oracle.INF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- brute force
def bf_bfs(n, src_list, dst_list, s):
    """Hop distance by boolean adjacency-matrix powers: level[v] is the first k
    with a length-k walk from s to v."""
    A = np.zeros((n, n), dtype=bool)
    for u, v in zip(src_list, dst_list):
        A[u, v] = True
    level = np.full(n, INF, dtype=np.uint32)
    level[s] = 0
    P = np.eye(n, dtype=bool)
    for k in range(1, n):
        P = (P.astype(np.int64) @ A.astype(np.int64)) > 0
        newly = P[s] & (level == INF)
        level[newly] = k
    return level


def bf_sssp(n, src_list, dst_list, w_list, s):
    """Floyd-Warshall over the min weight of parallel edges."""
    big = np.iinfo(np.int64).max // 4
    D = np.full((n, n), big, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for u, v, w in zip(src_list, dst_list, w_list):
        if u != v:
            D[u, v] = min(D[u, v], int(w))
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    d = D[s]
    return np.where(d >= big, INF, d).astype(np.uint32)


def bf_cc(n, src_list, dst_list):
    """Transitive closure (Warshall) of the symmetric reflexive relation;
    label = smallest vertex reachable."""
    R = np.eye(n, dtype=bool)
    for u, v in zip(src_list, dst_list):
        R[u, v] = R[v, u] = True
    for k in range(n):
        R = R | (R[:, k:k + 1] & R[k:k + 1, :])
    return np.array([int(np.nonzero(R[v])[0].min()) for v in range(n)], dtype=np.uint32)


def edge_lists(g):
    deg = np.diff(g.offsets).astype(np.int64)
    src = np.repeat(np.arange(g.n), deg)
    return src, g.cols.astype(np.int64), (None if g.weights is None else g.weights.astype(np.int64))


# ---------------------------------------------------------- oracle entry points
class Impl:
    """Calls the three oracle functions through a given shared library, so the
    same pin suite runs on the real oracle and on planted mutants."""

    def __init__(self, lib):
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        lib.oracle_bfs.argtypes = [u64, p, p, u64, p]
        lib.oracle_sssp.argtypes = [u64, p, p, p, u64, p]
        lib.oracle_cc.argtypes = [u64, p, p, p]
        lib.oracle_pagerank.argtypes = [u64, p, p, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, p, p]
        self.lib = lib

    @staticmethod
    def _p(a):
        return ctypes.c_void_p(a.ctypes.data)

    def bfs(self, g, s):
        out = np.empty(max(g.n, 1), dtype=np.uint32)
        off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
        col = np.ascontiguousarray(g.cols, dtype=np.uint64)
        assert self.lib.oracle_bfs(g.n, self._p(off), self._p(col), s, self._p(out)) == 0
        return out[:g.n]

    def sssp(self, g, s):
        out = np.empty(max(g.n, 1), dtype=np.uint32)
        off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
        col = np.ascontiguousarray(g.cols, dtype=np.uint64)
        w = np.ascontiguousarray(g.weights, dtype=np.uint32)
        assert self.lib.oracle_sssp(g.n, self._p(off), self._p(col), self._p(w), s, self._p(out)) == 0
        return out[:g.n]

    def cc(self, g):
        out = np.empty(max(g.n, 1), dtype=np.uint32)
        off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
        col = np.ascontiguousarray(g.cols, dtype=np.uint64)
        assert self.lib.oracle_cc(g.n, self._p(off), self._p(col), self._p(out)) == 0
        return out[:g.n]


    def pagerank(self, g, damping=0.85, tol=1e-15, max_iter=2000):
        out = np.empty(max(g.n, 1), dtype=np.float64)
        it = np.zeros(1, dtype=np.uint32)
        off = np.ascontiguousarray(g.offsets, dtype=np.uint64)
        col = np.ascontiguousarray(g.cols, dtype=np.uint64)
        assert self.lib.oracle_pagerank(g.n, self._p(off), self._p(col), damping, tol, max_iter, self._p(out),
                                        self._p(it)) == 0
        return out[:g.n], int(it[0])


@pytest.fixture(scope="module")
def impl():
    return Impl(oracle._lib())


# ------------------------------------------------------------------ pin suites
def all_undirected_graphs(nmax, seed=7):
    """Every simple undirected graph on n <= nmax labelled vertices, with
    seeded symmetric weights in [1, 255]."""
    rng = np.random.default_rng(seed)
    for n in range(1, nmax + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            s = np.array([e[0] for e in es], dtype=np.uint64)
            d = np.array([e[1] for e in es], dtype=np.uint64)
            w = rng.integers(1, 256, size=len(es)).astype(np.uint32)
            yield gg.csr_from_edges(n, s, d, weights=w, symmetrize=True)


def random_directed_multigraphs(count, nmax, seed=11):
    """Seeded directed graphs with duplicate edges and self-loops kept."""
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, nmax + 1))
        m = int(rng.integers(0, 3 * n + 1))
        s = rng.integers(0, n, size=m).astype(np.uint64)
        d = rng.integers(0, n, size=m).astype(np.uint64)
        w = rng.integers(1, 256, size=m).astype(np.uint32)
        yield gg.csr_from_edges(n, s, d, weights=w, symmetrize=False, dedup=False,
                                drop_self_loops=False, sort=False)


def check_bruteforce(impl, graphs, do_cc=True):
    for g in graphs:
        s, d, w = edge_lists(g)
        for src in range(g.n):
            np.testing.assert_array_equal(impl.bfs(g, src), bf_bfs(g.n, s, d, src))
            np.testing.assert_array_equal(impl.sssp(g, src), bf_sssp(g.n, s, d, w, src))
        if do_cc:
            np.testing.assert_array_equal(impl.cc(g), bf_cc(g.n, s, d))


def check_invariants(impl, g, sources):
    """Certificates that hold at any size (they characterise the answers)."""
    s, d, w = edge_lists(g)
    for src in sources:
        lv = impl.bfs(g, src).astype(np.int64)
        assert lv[src] == 0
        reached = lv != INF
        # every edge out of a reached vertex: level[v] <= level[u] + 1
        e = reached[s]
        assert np.all(lv[d[e]] <= lv[s[e]] + 1)
        # every reached v != src has an in-neighbour one level up
        par = np.zeros(g.n, dtype=bool)
        tight = e & (lv[d] == lv[s] + 1)
        par[d[tight]] = True
        rv = np.nonzero(reached)[0]
        assert np.all(par[rv[rv != src]])
        if g.undirected:
            both = reached[s] & reached[d]
            assert np.all(np.abs(lv[s[both]] - lv[d[both]]) <= 1)
        if w is not None:
            dist = impl.sssp(g, src).astype(np.int64)
            assert dist[src] == 0
            rd = dist != INF
            assert np.array_equal(rd, reached)
            e = rd[s]
            assert np.all(dist[d[e]] <= dist[s[e]] + w[e])  # triangle inequality
            tight = e & (dist[d] == dist[s] + w)
            par = np.zeros(g.n, dtype=bool)
            par[d[tight]] = True
            rv = np.nonzero(rd)[0]
            assert np.all(par[rv[rv != src]])  # a tight in-edge exists
    if g.undirected:
        lab = impl.cc(g).astype(np.int64)
        assert np.all(lab[s] == lab[d])  # every edge joins equal labels
        assert np.all(lab <= np.arange(g.n))
        assert np.all(lab[lab] == lab)
        # component count equals the number of BFS sweeps needed to cover V
        seen = np.zeros(g.n, dtype=bool)
        sweeps = 0
        for v in range(g.n):
            if not seen[v]:
                sweeps += 1
                seen |= impl.bfs(g, v) != INF
        assert sweeps == np.unique(lab).size


def check_special(impl):
    n = 50
    p = gg.path_graph(n)
    np.testing.assert_array_equal(impl.bfs(p, 0), np.arange(n, dtype=np.uint32))
    np.testing.assert_array_equal(impl.bfs(p, n - 1), np.arange(n, dtype=np.uint32)[::-1])
    gg.add_weights(p, seed=3)
    # the edge (i, i+1) is the last entry of row i (row 0 has only that edge)
    ws = np.array([p.weights[int(p.offsets[i + 1]) - 1] for i in range(n - 1)], dtype=np.int64)
    np.testing.assert_array_equal(impl.sssp(p, 0), np.concatenate([[0], np.cumsum(ws)]).astype(np.uint32))
    st = gg.star_graph(20, center=7)
    lv = impl.bfs(st, 7)
    assert lv[7] == 0 and np.all(np.delete(lv, 7) == 1)
    lv = impl.bfs(st, 3)
    assert lv[3] == 0 and lv[7] == 1 and np.all(np.delete(lv, [3, 7]) == 2)
    kn = gg.complete_graph(9)
    assert np.all(np.delete(impl.bfs(kn, 4), 4) == 1)
    assert np.all(impl.cc(kn) == 0)
    e = gg.empty_graph(6)
    lv = impl.bfs(e, 2)
    assert lv[2] == 0 and np.all(np.delete(lv, 2) == INF)
    np.testing.assert_array_equal(impl.cc(e), np.arange(6, dtype=np.uint32))
    # unit weights reduce SSSP to BFS
    g = gg.kronecker(9, 8, seed=5)
    g.weights = np.ones(g.m, dtype=np.uint32)
    src = gg.max_degree_vertex(g)
    np.testing.assert_array_equal(impl.sssp(g, src), impl.bfs(g, src))


# ------------------------------------------------------------------ the tests
def test_bruteforce_all_undirected_graphs_up_to_5(impl):
    check_bruteforce(impl, all_undirected_graphs(5))


def test_bruteforce_random_directed_multigraphs(impl):
    check_bruteforce(impl, random_directed_multigraphs(300, 12), do_cc=False)


def test_bruteforce_random_undirected_multigraphs(impl):
    rng = np.random.default_rng(5)
    gs = []
    for _ in range(150):
        n = int(rng.integers(1, 13))
        m = int(rng.integers(0, 2 * n + 1))
        s = rng.integers(0, n, size=m)
        d = rng.integers(0, n, size=m)
        w = rng.integers(1, 256, size=m)
        gs.append(gg.csr_from_edges(n, s, d, weights=w, symmetrize=True, dedup=False,
                                    drop_self_loops=False))
    check_bruteforce(impl, gs)


def test_special_cases(impl):
    check_special(impl)


@pytest.mark.parametrize("scale", [8, 11, 13])
def test_invariants_kronecker(impl, scale):
    g = gg.kronecker(scale, 16, seed=scale, weights=True)
    srcs = [gg.max_degree_vertex(g)] + [int(x) for x in gg.random_sources(g, 3, seed=2)]
    srcs.append(int(np.argmin(g.degrees())))  # possibly isolated source
    check_invariants(impl, g, srcs)


def test_invariants_uniform(impl):
    g = gg.uniform(1 << 12, 6, seed=3, weights=True)
    check_invariants(impl, g, [int(x) for x in gg.random_sources(g, 3, seed=2)])


def test_directed_invariants(impl):
    for g in random_directed_multigraphs(20, 60, seed=99):
        g.undirected = False
        check_invariants(impl, g, list(range(min(g.n, 4))))


def test_against_scipy_csgraph(impl):
    """BFS = unweighted shortest path, SSSP = Dijkstra, CC = connected
    components (relabelled to the smallest id), all from scipy."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    g = gg.kronecker(12, 16, seed=4, weights=True)
    A = sp.csr_matrix((g.weights.astype(np.float64), g.cols.astype(np.int64),
                       g.offsets.astype(np.int64)), shape=(g.n, g.n))
    for src in [gg.max_degree_vertex(g)] + [int(x) for x in gg.random_sources(g, 2, seed=2)]:
        hop = csg.shortest_path(A, method="D", unweighted=True, indices=src)
        exp = np.where(np.isinf(hop), INF, hop).astype(np.uint32)
        np.testing.assert_array_equal(impl.bfs(g, src), exp)
        dd = csg.dijkstra(A, indices=src)
        exp = np.where(np.isinf(dd), INF, dd).astype(np.uint32)
        np.testing.assert_array_equal(impl.sssp(g, src), exp)
    ncomp, lab = csg.connected_components(A, directed=False)
    first = np.full(ncomp, g.n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(g.n))
    np.testing.assert_array_equal(impl.cc(g), first[lab].astype(np.uint32))


def test_msbfs_rows_are_single_bfs():
    g = gg.kronecker(10, 8, seed=2)
    srcs = gg.random_sources(g, 5, seed=2)
    ms = oracle.msbfs(g.n, g.offsets, g.cols, srcs)
    s, d, _ = edge_lists(g)
    for k, src in enumerate(srcs):
        np.testing.assert_array_equal(ms[k], oracle.bfs_g(g, int(src)))
    # one row re-derived independently of the oracle on a small graph
    g2 = gg.kronecker(5, 4, seed=3)
    s2, d2, _ = edge_lists(g2)
    ms2 = oracle.msbfs(g2.n, g2.offsets, g2.cols, [0, 5, 31])
    for k, src in enumerate([0, 5, 31]):
        np.testing.assert_array_equal(ms2[k], bf_bfs(g2.n, s2, d2, src))


def test_sssp_overflow_detected():
    # a path whose total weight passes UINT32_MAX - 1
    n = 4
    g = gg.csr_from_edges(n, [0, 1, 2], [1, 2, 3], weights=[0x7FFFFFFF, 0x7FFFFFFF, 5])
    with pytest.raises(oracle.OracleOverflow):
        oracle.sssp_g(g, 0)


def test_bad_source_rejected():
    g = gg.path_graph(3)
    with pytest.raises(oracle.OracleError):
        oracle.bfs_g(g, 3)


def test_reached_edges_counts_out_degree_of_reached():
    g = gg.csr_from_edges(5, [0, 1, 3], [1, 2, 4])  # two components
    lv = oracle.bfs_g(g, 0)
    assert oracle.reached_edges(g.offsets, lv) == 4  # 0-1, 1-0, 1-2, 2-1


# ------------------------------------------------------------ link-model golden
def _golden_rows():
    with open(os.path.join(GOLDEN, "link_model.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield [c.strip() for c in line.split("|")]


def test_link_model_matches_printed_values():
    rows = list(_golden_rows())
    assert len(rows) == 7
    for fn, args, value, tol, cite in rows:
        kw = dict(a.split("=") for a in args.split())
        if fn == "tag_limited_bandwidth":
            got = linkmodel.tag_limited_bandwidth(float(kw["req_bytes"]), float(kw["rtt_s"]),
                                                  int(kw["tags"])) / linkmodel.GIB
        elif fn == "header_overhead":
            got = linkmodel.header_overhead(float(kw["req_bytes"]), float(kw["header_bytes"]))
        elif fn == "outstanding_needed":
            got = linkmodel.outstanding_needed(float(kw["bandwidth_gib"]) * linkmodel.GIB, float(kw["rtt_s"]),
                                               float(kw["req_bytes"]))
        elif fn == "dram_effective":
            got = linkmodel.dram_effective(float(kw["peak"]), float(kw["req_bytes"]),
                                           float(kw["burst_bytes"]))
        elif fn == "aligned_start_probability":
            got = linkmodel.aligned_start_probability(int(kw["elem_bytes"]), int(kw["line_bytes"]))
        else:
            raise AssertionError(fn)
        exp = float(value.split()[0])
        assert abs(got - exp) <= float(tol) + 1e-12, (fn, got, exp, cite)


def test_uniform_graph_alignment_statistic():
    """Sec. 5.3.1: with 8-byte ids a list starts on a 128-byte line with
    probability 1/16 when start offsets are uniform."""
    g = gg.uniform(1 << 16, 32, seed=9)
    starts = g.offsets[:-1][g.degrees() > 0]
    frac = float(np.mean(starts % 16 == 0))
    assert abs(frac - linkmodel.aligned_start_probability(8)) < 0.01


# ---------------------------------------------------------------- mutations
# ------------------------------------------------------------------ PageRank pins
def pagerank_exact(g, d):
    """The fixed point of the PageRank iteration, by a dense linear solve:
    r = (1-d)/n + d (P^T r + (dangling . r)/n), P[v,u] = edges v->u / outdeg v."""
    n = g.n
    P = np.zeros((n, n))
    dang = np.zeros(n)
    deg = np.diff(g.offsets).astype(np.int64)
    for v in range(n):
        if deg[v] == 0:
            dang[v] = 1.0
        for i in range(int(g.offsets[v]), int(g.offsets[v + 1])):
            P[v, int(g.cols[i])] += 1.0 / deg[v]
    A = np.eye(n) - d * P.T - (d / n) * np.outer(np.ones(n), dang)
    return np.linalg.solve(A, np.full(n, (1.0 - d) / n))


def check_pagerank(impl):
    # exact fixed point on small directed multigraphs (dangling vertices,
    # parallel edges, self-loops) and undirected graphs, two damping factors
    small = list(random_directed_multigraphs(40, 12)) + list(all_undirected_graphs(4))[::7]
    for g in small:
        for d in (0.85, 0.5):
            r, it = impl.pagerank(g, d)
            assert it < 2000
            assert np.allclose(r, pagerank_exact(g, d), rtol=0, atol=1e-12)
    # closed forms: a star's centre, a cycle and a complete graph (uniform)
    d, n = 0.85, 25
    r, _ = impl.pagerank(gg.star_graph(n), d)
    assert abs(r[0] - (1 + d * (n - 1)) / (n * (1 + d))) < 1e-12
    assert np.allclose(r[1:], ((1 - d) / n + d * r[0] / (n - 1)), atol=1e-12)
    ring = gg.csr_from_edges(n, np.arange(n), (np.arange(n) + 1) % n, symmetrize=True)
    assert np.allclose(impl.pagerank(ring, d)[0], 1.0 / n, atol=1e-14)
    assert np.allclose(impl.pagerank(gg.complete_graph(9), d)[0], 1.0 / 9, atol=1e-14)
    # invariants on a larger graph: a probability vector, and a fixed point
    g = gg.kronecker(10, 8, seed=4)
    r, it = impl.pagerank(g, d, tol=1e-13)
    assert abs(r.sum() - 1.0) < 1e-12 and np.all(r > 0)
    r2, _ = impl.pagerank(g, d, tol=0.0, max_iter=it + 1)
    assert np.abs(r2 - r).sum() < 1e-12


def test_pagerank_pins(impl):
    check_pagerank(impl)


def test_pagerank_against_networkx():
    """An independent implementation (networkx, dangling mass spread evenly
    as here) on simple directed and undirected graphs."""
    nx = pytest.importorskip("networkx")
    for seed, directed in ((1, True), (2, False), (3, True)):
        g = gg.random_small(60, 0.08, seed=seed, directed=directed)
        G = nx.DiGraph()
        G.add_nodes_from(range(g.n))
        deg = np.diff(g.offsets).astype(np.int64)
        G.add_edges_from(zip(np.repeat(np.arange(g.n), deg).tolist(), g.cols.astype(np.int64).tolist()))
        ref = nx.pagerank(G, alpha=0.85, tol=1e-14, max_iter=10000)
        r, _ = oracle.pagerank_g(g, 0.85, tol=1e-15, max_iter=10000)
        assert np.allclose(r, [ref[v] for v in range(g.n)], rtol=0, atol=1e-10)


MUTANTS = [
    ("bfs level step", "level[u] = level[v] + 1;", "level[u] = level[v] + 2;"),
    ("bfs stack order", "uint64_t v = queue[head++];", "uint64_t v = queue[--tail];"),
    ("bfs drops last neighbour", "for (uint64_t i = offsets[v]; i < offsets[v + 1]; i++) {\n            uint64_t u = cols[i];\n            if (level[u]",
     "for (uint64_t i = offsets[v]; i + 1 < offsets[v + 1]; i++) {\n            uint64_t u = cols[i];\n            if (level[u]"),
    ("sssp ignores weights", "uint64_t nd = x.d + (uint64_t)w[i];", "uint64_t nd = x.d + 1;"),
    ("sssp relax sign", "if (nd < d[u]) {", "if (nd > d[u]) {"),
    ("sssp heap order", "if (!hless(h[i], h[p])) break;", "if (hless(h[i], h[p])) break;"),
    ("sssp pushes wrong vertex", "hitem y = {nd, u};", "hitem y = {nd, x.v};"),
    ("cc link direction", "if (a < b) parent[b] = a; else parent[a] = b;",
     "if (a < b) parent[a] = b; else parent[b] = a;"),
    ("cc links a non-root", "b = uf_find(parent, cols[i]);", "b = cols[i];"),
    ("pagerank drops dangling mass", "if (offsets[v + 1] == offsets[v]) dangling += rank[v];",
     "if (offsets[v + 1] == offsets[v]) dangling += 0.0;"),
    ("pagerank damps the teleport", "(1.0 - damping) / (double)n + damping * dangling",
     "damping / (double)n + damping * dangling"),
    ("pagerank divides by n, not the degree", "damping * rank[v] / (double)deg;",
     "damping * rank[v] / (double)n;"),
    ("pagerank sends to the source", "next[cols[i]] += damping", "next[v] += damping"),
]


def _pin_suite_fails(lib_path):
    impl = Impl(ctypes.CDLL(lib_path))
    try:
        check_bruteforce(impl, all_undirected_graphs(5))
        check_bruteforce(impl, random_directed_multigraphs(60, 9), do_cc=False)
        check_special(impl)
        g = gg.kronecker(9, 16, seed=9, weights=True)
        check_invariants(impl, g, [gg.max_degree_vertex(g)])
        g = gg.uniform(1 << 12, 4, seed=3, weights=True)
        check_invariants(impl, g, [int(x) for x in gg.random_sources(g, 2, seed=2)])
        check_pagerank(impl)
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_the_pins(name, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, name
    tmp = tempfile.mkdtemp()
    try:
        path = os.path.join(tmp, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "mutant.so")
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, path])
        assert _pin_suite_fails(so), f"mutant '{name}' survived the pins"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
