"""GPU parity with 4-byte edge lists (emogi_load_csr32, the uint32 edge list
of Sec. 5.4): every traversal of a graph loaded with uint32 ids equals the
oracle element by element, as the same graph with uint64 ids does.

A uint32 list is read four ids per 16-byte lane load from the 128-byte line
holding its first id (32 ids per line), so the residue, split-list, borrowed
and every-variant cases of the uint64 tests are repeated here with the new
alignment.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2006_06890_gb300 import emogi as E  # noqa: E402
from test_gpu_parity import (VARIANTS, VID, check_all, graph, hub_graph, many_components_graph,  # noqa: E402
                             ms_sources, sources, uneven_graphs)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_06890_gb300 import _build
    _build.build()
    E.lib()
    yield


def load32(g, **kw):
    return E.load_graph(g, ids32=True, **kw)


def residue_graph32():
    """Rows of length 0..70 so that list starts fall on every index mod 32."""
    rng = np.random.default_rng(5)
    n = 700
    s, d = [], []
    for v in range(n):
        for u in rng.integers(0, n, size=v % 71):
            s.append(v)
            d.append(int(u))
    return gg.csr_from_edges(n, s, d, weights=rng.integers(1, 256, size=len(s)), symmetrize=False,
                             dedup=False, drop_self_loops=False, sort=False, name="residues32")


@pytest.mark.parametrize("placement", ["device", "host", "managed"])
@pytest.mark.parametrize("variant", VARIANTS, ids=VID)
def test_kron16_ids32_all_variants_and_placements(placement, variant):
    g = graph("kron16")
    with load32(g, placement=placement) as h:
        check_all(g, h, **variant)


@pytest.mark.parametrize("name", ["kron12", "urand14", "path", "hub", "directed", "empty", "single", "residues32"])
@pytest.mark.parametrize("variant", [VARIANTS[0], VARIANTS[1], VARIANTS[4], VARIANTS[5], VARIANTS[6]],
                         ids=[VID[0], VID[1], VID[4], VID[5], VID[6]])
def test_ids32_graph_set_host(name, variant):
    g = residue_graph32() if name == "residues32" else graph(name)
    with load32(g, placement="host") as h:
        check_all(g, h, **variant)


@pytest.mark.parametrize("chunk", [1, 3, 32, 500])
def test_ids32_split_chunk_sizes(chunk):
    g = graph("hub")
    with load32(g, placement="host") as h:
        check_all(g, h, access="merged_aligned", granularity=8, chunk_lines=chunk)


def test_ids32_borrowed_arrays_at_every_16_byte_offset():
    """Borrowed uint32 ids at every 16-byte slot of a 128-byte line (shifts of
    0, 4, ..., 28 ids) give exact results."""
    g = residue_graph32()
    for shift in range(0, 32, 4):
        cols = gg.aligned_empty(g.m + 32, np.uint32, 128)[shift:shift + g.m]
        cols[:] = g.cols
        w = gg.aligned_empty(g.m + 32, np.uint32, 128)[28 - shift:28 - shift + g.m]
        w[:] = g.weights
        assert cols.ctypes.data % 16 == 0 and w.ctypes.data % 16 == 0
        with E.load_csr32(g.n, g.m, g.offsets, cols, w, placement="host", borrow=True, undirected=False) as h:
            check_all(g, h)
            check_all(g, h, granularity=4)


def test_ids32_stats_count_four_bytes_per_id():
    g = graph("kron16")
    s = gg.max_degree_vertex(g)
    deg = g.degrees()
    with load32(g, placement="host", heads=False) as h:  # every entry from the edge list
        lv, st = E.bfs(h, s, top_down_only=True)
        reached = oracle.reached_edges(g.offsets, lv)
        assert st["edges_scanned"] == reached
        assert st["edge_bytes"] == 4 * reached
        _, st = E.sssp(h, s)
        assert st["edge_bytes"] == 4 * st["edges_scanned"] and st["weight_bytes"] == 4 * st["edges_scanned"]
    with load32(g, placement="host") as h:  # lists of 1..store_bound entries from the short-list store
        lv, st = E.bfs(h, s, top_down_only=True)
        assert h.store_bound in (16, 32)
        short = int(deg[(lv != E.INF) & (deg >= 1) & (deg <= h.store_bound)].sum())
        assert st["edge_bytes"] == 4 * (oracle.reached_edges(g.offsets, lv) - short)


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "directed"])
def test_ids32_sssp_loops_and_windows(name):
    g = graph(name)
    with load32(g, placement="host") as h:
        for s in sources(g):
            exp = oracle.sssp_g(g, s)
            np.testing.assert_array_equal(E.sssp(h, s)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s, host_loop=True)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s, granularity=32, delta=7)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s, delta=0xFFFFFFFF)[0], exp)


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path"])
@pytest.mark.parametrize("heads", [True, False])
def test_ids32_bfs_directions_and_heads(name, heads):
    g = graph(name)
    with load32(g, placement="host", heads=heads) as h:
        for s in sources(g):
            exp = oracle.bfs_g(g, s)
            for kw in (dict(), dict(top_down_only=True), dict(granularity=4), dict(granularity=32)):
                np.testing.assert_array_equal(E.bfs(h, s, **kw)[0], exp, err_msg=f"{kw} src={s}")
        np.testing.assert_array_equal(E.cc(h)[0], oracle.cc_g(g))


@pytest.mark.parametrize("placement", ["device", "host"])
@pytest.mark.parametrize("name", ["many", "kron16", "hub"])
def test_ids32_cc(placement, name):
    g = many_components_graph() if name == "many" else graph(name)
    exp = oracle.cc_g(g)
    with load32(g, placement=placement) as h:
        for kw in (dict(), dict(cc_full_pass=True), dict(granularity=32, chunk_lines=2), dict(access="naive")):
            np.testing.assert_array_equal(E.cc(h, **kw)[0], exp, err_msg=str(kw))


@pytest.mark.parametrize("k", [1, 17, 64])
def test_ids32_msbfs(k):
    g = graph("kron16")
    srcs = ms_sources(g, k)
    with load32(g, placement="host") as h:
        for kw in (dict(), dict(granularity=4), dict(access="merged")):
            lv, _ = E.msbfs(h, srcs, **kw)
            np.testing.assert_array_equal(lv, oracle.msbfs(g.n, g.offsets, g.cols, srcs))


def test_ids32_batch_mixed_with_ids64():
    """A batch may hold graphs of both id widths."""
    gs = uneven_graphs(24, seed=6)
    hs = [E.load_graph(g, placement="device", ids32=(i % 2 == 0)) for i, g in enumerate(gs)]
    srcs = [gg.max_degree_vertex(g) for g in gs]
    try:
        with E.Batch(hs) as b:
            for kw in (dict(), dict(granularity=4, chunk_lines=1), dict(granularity=32)):
                lv, _ = b.bfs(srcs, **kw)
                for g, s, got in zip(gs, srcs, lv):
                    np.testing.assert_array_equal(got, oracle.bfs_g(g, s))
    finally:
        for h in hs:
            h.free()


def test_ids32_server():
    g = graph("kron16")
    with load32(g, placement="host") as h:
        srcs = sources(g, 6)
        outs = [np.empty(g.n, dtype=np.uint32) for _ in range(2 * len(srcs))]
        with E.Server(max_slots=4) as srv:
            tickets = [srv.submit(h, "bfs", s, o) for s, o in zip(srcs, outs)]
            tickets += [srv.submit(h, "sssp", s, o) for s, o in zip(srcs, outs[len(srcs):])]
            for t in tickets:
                srv.wait(t)
        for s, o in zip(srcs, outs):
            np.testing.assert_array_equal(o, oracle.bfs_g(g, s))
        for s, o in zip(srcs, outs[len(srcs):]):
            np.testing.assert_array_equal(o, oracle.sssp_g(g, s))


def test_ids32_hub_larger_than_a_split_chunk():
    """A list of 300k uint32 ids is split into chunk items of 32-id lines."""
    g = hub_graph(300_000)
    with load32(g, placement="host") as h:
        exp = oracle.bfs_g(g, 0)
        np.testing.assert_array_equal(E.bfs(h, 0, top_down_only=True)[0], exp)
        np.testing.assert_array_equal(E.sssp(h, 0)[0], oracle.sssp_g(g, 0))


def array_end_graph(r, symmetric):
    """A graph whose last list ends at the end of the edge array, with
    m = r (mod 4) for a directed graph (every residue of a 16-byte load of
    uint32 ids, and of uint64 ids mod 2) and m even for a symmetric one; the
    last vertex has the longest list so that it ends in a partial load."""
    rng = np.random.default_rng(100 + r)
    n = 48
    s, d = [], []
    for v in range(n - 1):
        for u in rng.choice(n, size=int(rng.integers(0, 6)), replace=False):
            s.append(v)
            d.append(int(u))
    if symmetric:  # m is even: m = 2 (mod 4) for odd r
        k = 30
        while True:
            last = [int(u) for u in rng.choice(n - 1, size=k, replace=False)]
            g = gg.csr_from_edges(n, s + [n - 1] * k, d + last, symmetrize=True, name=f"array-end-sym{r}")
            if g.m % 4 == 2 * (r % 2):
                return gg.add_weights(g, seed=r)
            k += 1
    k = 37
    while (len(s) + k) % 4 != r:
        k += 1
    last = [int(u) for u in rng.integers(0, n, size=k)]
    s += [n - 1] * k
    d += last
    return gg.csr_from_edges(n, s, d, weights=rng.integers(1, 256, size=len(s)), symmetrize=False, dedup=False,
                             drop_self_loops=False, sort=False, name=f"array-end{r}")


@pytest.mark.parametrize("ids32", [True, False], ids=["u32", "u64"])
@pytest.mark.parametrize("placement", ["device", "host", "managed"])
@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_lists_ending_at_the_end_of_the_edge_array(r, placement, ids32):
    """The load of a list's last ids is a whole 16-byte load (ids past the
    list masked off) except where it would pass the end of the edge array;
    lists ending at every residue of m, and at m itself, stay exact."""
    for symmetric in (False, True):
        g = array_end_graph(r, symmetric)
        assert g.offsets[-2] < g.offsets[-1] == g.m
        with E.load_graph(g, placement=placement, ids32=ids32) as h:
            for kw in (dict(), dict(granularity=4), dict(granularity=32)):
                check_all(g, h, **kw)
                for s in range(0, g.n, 7):
                    np.testing.assert_array_equal(E.sssp(h, s, **kw)[0], oracle.sssp_g(g, s))
            if symmetric:
                exp, _ = oracle.pagerank_g(g, 0.85, tol=0.0, max_iter=15)
                np.testing.assert_allclose(E.pagerank(h, 0.85, tol=0.0, max_iters=15)[0], exp, rtol=1e-9, atol=1e-12)
                srcs = list(range(0, g.n, 3))
                np.testing.assert_array_equal(E.msbfs(h, srcs)[0], oracle.msbfs(g.n, g.offsets, g.cols, srcs))
