"""GPU parity: every CUDA result equals the CPU oracle element by element.

All traversal results are integers, so the bar is bit-exact.  Covered: every
access variant (naive / merged / merged+aligned at each granularity) and every
placement (device / pinned host / managed), borrowed host arrays, device
outputs, the split path for long lists, lists starting at every residue of the
128-byte line, empty / ragged / degenerate graphs, the SSSP overflow check and
host-side error paths.
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


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_06890_gb300 import _build
    _build.build()
    E.lib()
    yield


# ------------------------------------------------------------------ graphs
def residue_graph():
    """Rows of length 0..40 so list starts fall on every index mod 16."""
    rng = np.random.default_rng(1)
    n = 400
    s, d = [], []
    for v in range(n):
        deg = v % 41
        for u in rng.integers(0, n, size=deg):
            s.append(v)
            d.append(int(u))
    return gg.csr_from_edges(n, s, d, weights=rng.integers(1, 256, size=len(s)), symmetrize=False,
                             dedup=False, drop_self_loops=False, sort=False, name="residues")


def hub_graph(n=200_000):
    """A star whose centre has n-1 neighbours (the split path) plus a ring."""
    c = np.zeros(n - 1, dtype=np.uint64)
    leaves = np.arange(1, n, dtype=np.uint64)
    ring_s = np.arange(1, n, dtype=np.uint64)
    ring_d = np.concatenate([np.arange(2, n), [1]]).astype(np.uint64)
    g = gg.csr_from_edges(n, np.concatenate([c, ring_s]), np.concatenate([leaves, ring_d]), name="hub")
    return gg.add_weights(g, seed=3)


def directed_multigraph():
    rng = np.random.default_rng(7)
    n, m = 3000, 20000
    s = rng.integers(0, n, size=m)
    d = rng.integers(0, n, size=m)
    w = rng.integers(1, 256, size=m)
    g = gg.csr_from_edges(n, s, d, weights=w, symmetrize=False, dedup=False, drop_self_loops=False,
                          sort=False, name="directed-multi")
    g.undirected = False
    return g


GRAPHS = {}


def graph(name):
    if name not in GRAPHS:
        if name == "kron16":  # the 65,536-vertex Kronecker workload (edge factor 16)
            GRAPHS[name] = gg.kronecker(16, 16, seed=1, weights=True)
        elif name == "kron12":
            GRAPHS[name] = gg.kronecker(12, 16, seed=3, weights=True)
        elif name == "urand14":
            GRAPHS[name] = gg.uniform(1 << 14, 7, seed=2, weights=True)
        elif name == "path":
            GRAPHS[name] = gg.add_weights(gg.path_graph(3000), seed=1)
        elif name == "residues":
            GRAPHS[name] = residue_graph()
        elif name == "hub":
            GRAPHS[name] = hub_graph()
        elif name == "directed":
            GRAPHS[name] = directed_multigraph()
        elif name == "empty":
            GRAPHS[name] = gg.add_weights(gg.empty_graph(7), seed=1)
        elif name == "single":
            GRAPHS[name] = gg.add_weights(gg.empty_graph(1), seed=1)
        else:
            raise KeyError(name)
    return GRAPHS[name]


def sources(g, k=2):
    out = [gg.max_degree_vertex(g)]
    out += [int(x) for x in gg.random_sources(g, k, seed=2)]
    out.append(int(np.argmin(g.degrees())))  # possibly an isolated vertex
    return sorted(set(out))


def check_all(g, h, **kw):
    for s in sources(g):
        lv, st = E.bfs(h, s, **kw)
        exp = oracle.bfs_g(g, s)
        np.testing.assert_array_equal(lv, exp, err_msg=f"bfs src={s} {kw}")
        assert st["edges_reached"] == oracle.reached_edges(g.offsets, exp)
        if g.weights is not None:
            d, _ = E.sssp(h, s, **kw)
            np.testing.assert_array_equal(d, oracle.sssp_g(g, s), err_msg=f"sssp src={s} {kw}")
    if g.undirected:
        lab, st = E.cc(h, **kw)
        np.testing.assert_array_equal(lab, oracle.cc_g(g), err_msg=f"cc {kw}")
        assert st["edges_scanned"] <= g.m + 2 * g.n
        lab, st = E.cc(h, cc_full_pass=True, **kw)
        np.testing.assert_array_equal(lab, oracle.cc_g(g), err_msg=f"cc full pass {kw}")
        assert st["edges_scanned"] == g.m


VARIANTS = [dict(access="merged_aligned"), dict(access="merged_aligned", granularity=4),
            dict(access="merged_aligned", granularity=8), dict(access="merged_aligned", granularity=16),
            dict(access="merged_aligned", granularity=32), dict(access="merged"), dict(access="naive")]
VID = ["aligned-auto", "aligned-g4", "aligned-g8", "aligned-g16", "aligned-g32", "merged", "naive"]


# ------------------------------------------------------------------ parity
@pytest.mark.parametrize("placement", ["device", "host", "managed"])
@pytest.mark.parametrize("variant", VARIANTS, ids=VID)
def test_kron16_all_variants_and_placements(placement, variant):
    g = graph("kron16")
    with E.load_graph(g, placement=placement) as h:
        check_all(g, h, **variant)


@pytest.mark.parametrize("name", ["kron12", "urand14", "path", "residues", "hub", "directed", "empty", "single"])
@pytest.mark.parametrize("variant", VARIANTS, ids=VID)
def test_graph_set_host(name, variant):
    g = graph(name)
    with E.load_graph(g, placement="host") as h:
        check_all(g, h, **variant)


@pytest.mark.parametrize("chunk", [1, 3, 32, 500])
def test_split_chunk_sizes(chunk):
    g = graph("hub")
    with E.load_graph(g, placement="device") as h:
        check_all(g, h, access="merged_aligned", granularity=8, chunk_lines=chunk)


def test_borrowed_host_arrays_at_every_line_offset():
    """EMOGI_LOAD_BORROW pins the caller's arrays in place; bases that are not
    128-byte aligned (but 16-byte aligned) still give exact results."""
    g = graph("residues")
    for shift_elems in (0, 2, 4, 6, 8, 10, 12, 14):
        cols = gg.aligned_empty(g.m + 16, np.uint64, 128)[shift_elems:shift_elems + g.m]
        cols[:] = g.cols
        w_off = 2 * shift_elems  # 0, 4, ..., 28 weights: 16-byte aligned, every 16-byte slot of a line
        w = gg.aligned_empty(g.m + 32, np.uint32, 128)[w_off:w_off + g.m]
        w[:] = g.weights
        assert cols.ctypes.data % 16 == 0 and w.ctypes.data % 16 == 0
        with E.load_csr(g.n, g.m, g.offsets, cols, w, placement="host", borrow=True,
                        undirected=False) as h:
            check_all(g, h)


def test_device_outputs_with_torch_tensors():
    g = graph("kron12")
    s = gg.max_degree_vertex(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with E.load_graph(g, placement="host") as h:
        E.bfs(h, s, out=out, stream=stream)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.bfs_g(g, s))
        E.sssp(h, s, out=out)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.sssp_g(g, s))
        E.cc(h, out=out)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.cc_g(g))


def test_repeated_calls_reuse_buffers():
    g = graph("urand14")
    srcs = sources(g, 4)
    with E.load_graph(g, placement="host") as h:
        for _ in range(2):
            for s in srcs:
                np.testing.assert_array_equal(E.sssp(h, s)[0], oracle.sssp_g(g, s))
                np.testing.assert_array_equal(E.bfs(h, s)[0], oracle.bfs_g(g, s))


@pytest.mark.parametrize("delta", [1, 7, 64, 0, 0xFFFFFFFF], ids=["d1", "d7", "d64", "auto", "bellman-ford"])
@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "directed", "path"])
def test_sssp_windows(name, delta):
    """Every distance-window width gives the exact distances (the window only
    orders the work)."""
    g = graph(name)
    with E.load_graph(g, placement="device") as h:
        for s in sources(g):
            d, st = E.sssp(h, s, delta=delta)
            np.testing.assert_array_equal(d, oracle.sssp_g(g, s), err_msg=f"sssp src={s} delta={delta}")


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "directed"])
def test_sssp_device_loop_equals_host_loop(name):
    """The device-driven SSSP loop (recorded CUDA graph with a conditional
    while-node) and the host-driven loop give the oracle's distances."""
    g = graph(name)
    with E.load_graph(g, placement="host") as h:
        for s in sources(g):
            exp = oracle.sssp_g(g, s)
            d1, st1 = E.sssp(h, s)
            d2, st2 = E.sssp(h, s, host_loop=True)
            np.testing.assert_array_equal(d1, exp)
            np.testing.assert_array_equal(d2, exp)
            for G in (4, 32):  # a different granularity records a new loop graph
                np.testing.assert_array_equal(E.sssp(h, s, granularity=G)[0], exp)


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "directed", "residues"])
def test_sssp_ordered_frontier(name):
    """Near frontiers rebuilt in vertex order (flag per vertex + compaction;
    automatic for edge lists of 16 GiB or more, forced here) give the oracle's
    distances in both loops and at several window widths."""
    g = graph(name)
    with E.load_graph(g, placement="host") as h:
        for s in sources(g):
            exp = oracle.sssp_g(g, s)
            np.testing.assert_array_equal(E.sssp(h, s, ordered_frontier=True)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s, ordered_frontier=True, host_loop=True)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s, ordered_frontier=True, delta=1, granularity=4)[0], exp)
            np.testing.assert_array_equal(E.sssp(h, s)[0], exp)  # and back to the queue form


def far_then_near_multigraph(n, light):
    """Source 0 has a heavy edge (255) and then a light one (`light`) to every
    other vertex, plus a directed ring of weight 5 over vertices 1..n-1.  In
    the first sweep each neighbour is improved first to a far distance (it is
    flagged for the far pile) and then to a near one (it is queued), so the
    window's tail and the far pile hold the same vertices."""
    others = np.arange(1, n, dtype=np.uint64)
    s = np.concatenate([np.zeros(2 * (n - 1), dtype=np.uint64), others])
    d = np.concatenate([np.repeat(others, 2), np.concatenate([others[1:], others[:1]])])
    w = np.concatenate([np.tile(np.array([255, light], dtype=np.uint32), n - 1),
                        np.full(n - 1, 5, dtype=np.uint32)])
    g = gg.csr_from_edges(n, s, d, weights=w, symmetrize=False, dedup=False, drop_self_loops=False,
                          sort=False, name=f"far-then-near-{n}")
    g.undirected = False
    return g


@pytest.mark.parametrize("n", [200, 256, 3000])
@pytest.mark.parametrize("light,delta", [(0, 1), (1, 2), (1, 0)], ids=["w0-d1", "w1-d2", "w1-auto"])
def test_sssp_vertex_both_far_and_near_in_one_sweep(n, light, delta):
    """A vertex sent to the far pile and then queued near in the same sweep is
    queued once: the far split that follows a kept window tail must not append
    it behind the tail a second time (each queue holds n entries).  Host loop,
    device loop and ordered frontiers, from device and host memory."""
    g = far_then_near_multigraph(n, light)
    exp = oracle.sssp_g(g, 0)
    for placement in ("device", "host"):
        with E.load_graph(g, placement=placement) as h:
            for kw in (dict(), dict(host_loop=True), dict(ordered_frontier=True),
                       dict(ordered_frontier=True, host_loop=True), dict(granularity=32)):
                d, st = E.sssp(h, 0, delta=delta, **kw)
                np.testing.assert_array_equal(d, exp, err_msg=f"{placement} {kw}")
                assert st["edges_scanned"] <= 4 * g.m, (placement, kw, st)


def test_sssp_device_loop_time_bound():
    """The device loop checks %globaltimer at every iteration; a 1 ns bound
    stops it with EMOGI_E_TIMEOUT, and the next call is exact again."""
    g = graph("path")
    with E.load_graph(g, placement="device") as h:
        with pytest.raises(E.EmogiError) as ei:
            E.sssp(h, 0, timeout_ns=1)
        assert ei.value.status == E.E_TIMEOUT
        np.testing.assert_array_equal(E.sssp(h, 0)[0], oracle.sssp_g(g, 0))


def test_sssp_zero_and_extreme_weights():
    rng = np.random.default_rng(4)
    n, m = 2000, 12000
    s, d = rng.integers(0, n, size=m), rng.integers(0, n, size=m)
    w = rng.choice(np.array([0, 1, 2, 0xFFFF, 0x7FFFFF], dtype=np.uint32), size=m)
    g = gg.csr_from_edges(n, s, d, weights=w, symmetrize=False, dedup=False, drop_self_loops=False, sort=False)
    g.undirected = False
    with E.load_graph(g, placement="host") as h:
        for src in (0, 1, 17):
            for delta in (0, 1, 0xFFFFFFFF):
                np.testing.assert_array_equal(E.sssp(h, src, delta=delta)[0], oracle.sssp_g(g, src))


def test_unit_weights_sssp_equals_bfs():
    g = gg.kronecker(11, 16, seed=8)
    g.weights = np.ones(g.m, dtype=np.uint32)
    s = gg.max_degree_vertex(g)
    with E.load_graph(g, placement="host") as h:
        np.testing.assert_array_equal(E.sssp(h, s)[0], E.bfs(h, s)[0])


def test_sssp_overflow_is_reported():
    g = gg.csr_from_edges(4, [0, 1, 2], [1, 2, 3], weights=[0x7FFFFFFF, 0x7FFFFFFF, 5],
                          symmetrize=False)
    with E.load_graph(g, placement="device") as h:
        with pytest.raises(E.EmogiError) as ei:
            E.sssp(h, 0)
        assert ei.value.status == E.E_OVERFLOW
        # a large but representable distance is not an overflow
        d, _ = E.sssp(h, 1)
        assert d.tolist() == [E.INF, 0, 0x7FFFFFFF, 0x7FFFFFFF + 5]


def test_sssp_spurious_overflow_candidate_is_cleared():
    """A relaxation can overflow from a non-final distance while every true
    distance fits: the long detour 0->1->2 is relaxed before the short edge
    0->2 lowers dist[2]; the result must be exact and not an error."""
    big = 0xFFFFFF00
    g = gg.csr_from_edges(4, [0, 0, 1, 2], [1, 2, 2, 3], weights=[big, 3, 1000, 7], symmetrize=False)
    with E.load_graph(g, placement="device") as h:
        d, _ = E.sssp(h, 0, access="naive")
        np.testing.assert_array_equal(d, oracle.sssp_g(g, 0))


def test_errors():
    g = graph("directed")
    with E.load_graph(g, placement="host") as h:
        with pytest.raises(E.EmogiError) as ei:
            E.bfs(h, g.n)
        assert ei.value.status == E.E_ARG
        with pytest.raises(E.EmogiError) as ei:
            E.cc(h)
        assert ei.value.status == E.E_UNSUPPORTED
    with E.load_graph(g, placement="host", with_weights=False) as h:
        with pytest.raises(E.EmogiError) as ei:
            E.sssp(h, 0)
        assert ei.value.status == E.E_UNSUPPORTED


def test_budget_and_injected_alloc_failure():
    g = graph("kron12")
    base = E.device_bytes_in_use()
    E.set_device_budget(base + 1024)
    try:
        with pytest.raises(E.EmogiError) as ei:
            E.load_graph(g, placement="device")
        assert ei.value.status == E.E_BUDGET
    finally:
        E.set_device_budget(0)
    assert E.device_bytes_in_use() == base
    E.test_fail_device_alloc_after(2)
    try:
        with pytest.raises(E.EmogiError) as ei:
            E.load_graph(g, placement="device")
        assert ei.value.status == E.E_NOMEM
    finally:
        E.test_fail_device_alloc_after(0)
    assert E.device_bytes_in_use() == base
    with E.load_graph(g, placement="host") as h:  # allocations work again
        np.testing.assert_array_equal(E.cc(h)[0], oracle.cc_g(g))
    assert E.device_bytes_in_use() == base


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "kron12", "residues"])
@pytest.mark.parametrize("kw", [dict(top_down_only=True), dict(), dict(granularity=4), dict(granularity=32)],
                         ids=["top-down", "diropt", "diropt-g4", "diropt-g32"])
def test_bfs_directions(name, kw):
    """Direction-optimising BFS (bottom-up dense levels) gives the same levels as
    the push-only form, and reads no more list entries than it."""
    g = graph(name)
    with E.load_graph(g, placement="host") as h:
        for s in sources(g):
            lv, st = E.bfs(h, s, **kw)
            exp = oracle.bfs_g(g, s)
            np.testing.assert_array_equal(lv, exp)
            assert st["edges_reached"] == oracle.reached_edges(g.offsets, exp)
            if kw.get("top_down_only"):
                assert st["edges_scanned"] == st["edges_reached"]


def test_direction_optimising_reads_less_on_dense_levels():
    g = graph("kron16")
    s = gg.max_degree_vertex(g)
    with E.load_graph(g, placement="host") as h:
        _, td = E.bfs(h, s, top_down_only=True)
        _, do = E.bfs(h, s)
        assert do["edges_scanned"] < 0.5 * td["edges_scanned"]


def store_skew_graph(n=4000):
    """Most lists hold 1 to 32 entries, ten hubs hold about 94 % of the
    entries (lists of 80k to 120k entries, split across warps): the
    short-list store takes lists of up to 32 entries."""
    rng = np.random.default_rng(21)
    deg = rng.integers(1, 33, size=n)
    deg[rng.choice(n, 10, replace=False)] = rng.integers(80_000, 120_000, size=10)
    src = np.repeat(np.arange(n), deg)
    dst = rng.integers(0, n, size=src.size)
    return gg.csr_from_edges(n, src, dst, weights=rng.integers(1, 256, size=src.size), symmetrize=False,
                             dedup=False, drop_self_loops=False, sort=False, name="store-skew")


def _store_bytes(g, bound):
    deg = g.degrees()
    sel = (deg >= 1) & (deg <= bound)
    return g.n * 4 + int(((deg[sel] + 3) // 4 * 4).sum()) * 8  # index + ids + weights, 4-entry aligned


def test_store_bound_rule_and_budget():
    """The short-list store takes lists of up to 32 entries on a graph whose
    short lists hold few of its entries and up to 16 on a uniform one; with
    a device budget too small for it the bound drops to 16 and then to no
    store, the load succeeds, and every result equals the oracle's with the
    bytes read from the edge list counted by the bound."""
    g = graph("urand14")
    with E.load_graph(g, placement="host") as h:
        assert h.store_bound == expected_store_bound(g, h) == 16
    g = store_skew_graph()
    with E.load_graph(g, placement="device") as h:
        assert h.store_bound == expected_store_bound(g, h) == 0
    deg = g.degrees()
    srcs = [gg.max_degree_vertex(g), int(np.flatnonzero(deg == 20)[0])]
    exp_d = {s: oracle.sssp_g(g, s) for s in srcs}
    exp_l = {s: oracle.bfs_g(g, s) for s in srcs}
    before = E.device_bytes_in_use()
    with E.load_graph(g, placement="host") as h:
        assert h.store_bound == expected_store_bound(g, h) == 32
        base = E.device_bytes_in_use() - before - _store_bytes(g, 32)  # row offsets and list heads
    # one handle's work buffers, as the library reserves them, with room to spare
    work = 6 * g.n * 4 + (g.n // 16 + 1) * 16 + min(g.n, g.m // 497 + 1) * 20 + 4096
    budgets = {32: 0, 16: before + base + work + _store_bytes(g, 16),
               0: before + base + work + _store_bytes(g, 16) - 8192}
    assert _store_bytes(g, 32) - _store_bytes(g, 16) > 8192
    try:
        for bound, budget in budgets.items():
            E.set_device_budget(budget)
            with E.load_graph(g, placement="host") as h:
                assert h.store_bound == bound, budget
                for s in srcs:
                    d, st = E.sssp(h, s)
                    np.testing.assert_array_equal(d, exp_d[s], err_msg=f"bound={bound} src={s}")
                    lv, st = E.bfs(h, s, top_down_only=True)
                    np.testing.assert_array_equal(lv, exp_l[s], err_msg=f"bound={bound} src={s}")
                    short = int(deg[(lv != E.INF) & (deg >= 1) & (deg <= bound)].sum())
                    assert st["edges_scanned"] == oracle.reached_edges(g.offsets, lv)
                    assert st["edge_bytes"] == 8 * (st["edges_scanned"] - short)
            E.set_device_budget(0)
    finally:
        E.set_device_budget(0)
    assert E.device_bytes_in_use() == before

def test_stats_are_consistent():
    g = graph("kron16")
    s = gg.max_degree_vertex(g)
    deg = g.degrees()
    with E.load_graph(g, placement="host") as h:
        lv, st = E.bfs(h, s, time_kernels=True, top_down_only=True)
        reached = oracle.reached_edges(g.offsets, lv)
        assert st["edges_scanned"] == reached  # BFS expands each reached vertex once
        # lists of at most store_bound entries come from the short-list store in GPU memory
        assert h.store_bound == expected_store_bound(g, h)
        short = int(deg[(lv != E.INF) & (deg >= 1) & (deg <= h.store_bound)].sum())
        assert st["edge_bytes"] == 8 * (reached - short)
        assert st["iterations"] == int(lv[lv != E.INF].max()) + 1
        assert st["expand_launches"] == st["iterations"]
        assert 0 < st["expand_ms"] <= st["ms"]


# ------------------------------------------------------------------ multi-source BFS
def ms_sources(g, k, seed=2):
    srcs = [int(x) for x in gg.random_sources(g, k, seed=seed)]
    while len(srcs) < k:  # small graphs: repeat sources (allowed)
        srcs.append(srcs[len(srcs) % max(1, len(srcs))] if srcs else 0)
    if k >= 3:
        srcs[1] = srcs[0]  # a repeated source
        srcs[2] = int(np.argmin(g.degrees()))  # possibly isolated
    return srcs[:k]


@pytest.mark.parametrize("placement", ["device", "host"])
@pytest.mark.parametrize("k", [1, 5, 64])
def test_msbfs_rows_equal_oracle_bfs(placement, k):
    g = graph("kron16")
    srcs = ms_sources(g, k)
    with E.load_graph(g, placement=placement) as h:
        lv, st = E.msbfs(h, srcs)
        exp = oracle.msbfs(g.n, g.offsets, g.cols, srcs)
        np.testing.assert_array_equal(lv, exp)
        assert st["edges_reached"] == sum(oracle.reached_edges(g.offsets, exp[b]) for b in range(k))


@pytest.mark.parametrize("name", ["hub", "path", "directed", "urand14", "residues", "single"])
@pytest.mark.parametrize("variant", [dict(), dict(granularity=4), dict(granularity=32, chunk_lines=3),
                                     dict(access="merged"), dict(access="naive")],
                         ids=["auto", "g4", "g32-chunk3", "merged", "naive"])
def test_msbfs_graph_set(name, variant):
    g = graph(name)
    k = 1 if g.n == 1 else 17
    srcs = ms_sources(g, k)
    with E.load_graph(g, placement="host") as h:
        lv, _ = E.msbfs(h, srcs, **variant)
        np.testing.assert_array_equal(lv, oracle.msbfs(g.n, g.offsets, g.cols, srcs))


@pytest.mark.parametrize("placement", ["device", "host"])
@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "many"])
def test_msbfs_directions(placement, name):
    """Pulled (bottom-up) MS-BFS levels give the push-only levels, with or
    without list heads, and read fewer entries on a Kronecker graph."""
    g = many_components_graph() if name == "many" else graph(name)
    srcs = ms_sources(g, 64 if g.n > 64 else 9)
    exp = oracle.msbfs(g.n, g.offsets, g.cols, srcs)
    for heads in (True, False):
        with E.load_graph(g, placement=placement, heads=heads, with_weights=False) as h:
            lv, st = E.msbfs(h, srcs)
            np.testing.assert_array_equal(lv, exp, err_msg=f"heads={heads}")
            lv2, st2 = E.msbfs(h, srcs, top_down_only=True)
            np.testing.assert_array_equal(lv2, exp)
            np.testing.assert_array_equal(E.msbfs(h, srcs, granularity=4)[0], exp)
            if name == "kron16":
                assert st["edges_scanned"] < st2["edges_scanned"]


def test_msbfs_device_output_and_errors():
    g = graph("kron12")
    srcs = ms_sources(g, 9)
    out = torch.empty((9, g.n), dtype=torch.int32, device="cuda")
    with E.load_graph(g, placement="host") as h:
        E.msbfs(h, srcs, out=out)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.msbfs(g.n, g.offsets, g.cols, srcs))
        for bad in ([], list(range(65)), [g.n]):
            with pytest.raises(E.EmogiError) as ei:
                E.msbfs(h, bad)
            assert ei.value.status == E.E_ARG


# ------------------------------------------------------------------ batched BFS
def uneven_graphs(count, seed=4, nmin=6, nmax=12):
    """Uniform-random graphs of uneven sizes (2^nmin..2^nmax vertices, log-uniform)
    and average degrees 4..64, plus a few degenerate members."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2 ** rng.uniform(nmin, nmax))
        d = int(rng.integers(4, 65))
        out.append(gg.uniform(n, d, seed=seed * 1000 + i))
    out.append(gg.path_graph(300))
    out.append(hub_graph(5000))
    out.append(gg.empty_graph(3))
    return out


@pytest.mark.parametrize("placement", ["device", "host"])
def test_batch_bfs_equals_oracle(placement):
    gs = uneven_graphs(40)
    hs = [E.load_graph(g, placement=placement) for g in gs]
    srcs = [gg.max_degree_vertex(g) for g in gs]
    try:
        with E.Batch(hs) as b:
            for kw in (dict(), dict(granularity=4, chunk_lines=1), dict(granularity=32, chunk_lines=64)):
                lv, st = b.bfs(srcs, **kw)
                reached = 0
                for g, h, s, got in zip(gs, hs, srcs, lv):
                    exp = oracle.bfs_g(g, s)
                    np.testing.assert_array_equal(got, exp)
                    reached += oracle.reached_edges(g.offsets, exp)
                assert st["edges_reached"] == reached
            # the autotuner keeps a configuration that gives the same result
            G, claim, ms = b.autotune(srcs)
            assert G in (4, 8, 16, 32) and claim in (1, 4, 16, 64) and ms > 0
            srcs2 = [int(gg.random_sources(g, 1, seed=9)[0]) if g.m else 0 for g in gs]
            lv, _ = b.bfs(srcs2)
            for g, s, got in zip(gs, srcs2, lv):
                np.testing.assert_array_equal(got, oracle.bfs_g(g, s))
            out = torch.empty(b.total, dtype=torch.int32, device="cuda")
            lv, _ = b.bfs(srcs, out=out)
            for g, s, got in zip(gs, srcs, lv):
                np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), oracle.bfs_g(g, s))
    finally:
        for h in hs:
            h.free()


def test_bfs_batch_one_shot_and_errors():
    gs = uneven_graphs(5, seed=8)
    hs = [E.load_graph(g, placement="device") for g in gs]
    try:
        srcs = [0] * len(gs)
        lv, _ = E.bfs_batch(hs, srcs)
        for g, got in zip(gs, lv):
            np.testing.assert_array_equal(got, oracle.bfs_g(g, 0))
        with pytest.raises(E.EmogiError) as ei:
            E.bfs_batch(hs, [g.n for g in gs])
        assert ei.value.status == E.E_ARG
        with pytest.raises(E.EmogiError) as ei:
            E.bfs_batch(hs, srcs, access="naive")
        assert ei.value.status == E.E_UNSUPPORTED
    finally:
        for h in hs:
            h.free()


def test_batch_barrier_timeout_is_reported_not_hung():
    """A level barrier that waits longer than timeout_ns returns
    EMOGI_E_TIMEOUT (the wait is bounded); a 1 ns bound trips it on the first
    barrier while every block is co-resident, so nothing hangs."""
    gs = uneven_graphs(8, seed=3)
    hs = [E.load_graph(g, placement="device") for g in gs]
    try:
        with E.Batch(hs) as b:
            with pytest.raises(E.EmogiError) as ei:
                b.bfs([0] * len(gs), timeout_ns=1)
            assert ei.value.status == E.E_TIMEOUT
            lv, _ = b.bfs([0] * len(gs))  # the batch still works afterwards
            for g, got in zip(gs, lv):
                np.testing.assert_array_equal(got, oracle.bfs_g(g, 0))
    finally:
        for h in hs:
            h.free()


def many_components_graph():
    """Several components of different sizes (a big uniform block, small
    Kronecker blocks, paths, stars, isolated vertices) with ids interleaved by
    a permutation, so that the sampled giant tree is not the only one."""
    rng = np.random.default_rng(21)
    parts, n = [], 0
    for sub in [gg.uniform(3000, 6, seed=1), gg.kronecker(8, 4, seed=2), gg.path_graph(200),
                gg.star_graph(50), gg.empty_graph(30), gg.uniform(500, 3, seed=3)]:
        deg = np.diff(sub.offsets).astype(np.int64)
        src = np.repeat(np.arange(sub.n), deg) + n
        parts.append((src, sub.cols.astype(np.int64) + n))
        n += sub.n
    perm = rng.permutation(n)
    s = perm[np.concatenate([p[0] for p in parts])]
    d = perm[np.concatenate([p[1] for p in parts])]
    return gg.csr_from_edges(n, s, d, symmetrize=True, name="many-components")


@pytest.mark.parametrize("placement", ["device", "host"])
@pytest.mark.parametrize("name", ["many", "kron16", "urand14", "hub", "path", "empty", "single", "residues-sym"])
def test_cc_sampled_and_full_pass(placement, name):
    if name == "many":
        g = many_components_graph()
    elif name == "residues-sym":
        r = graph("residues")
        deg = np.diff(r.offsets).astype(np.int64)
        g = gg.csr_from_edges(r.n, np.repeat(np.arange(r.n), deg), r.cols, symmetrize=True, dedup=False,
                              drop_self_loops=False)
    else:
        g = graph(name)
    exp = oracle.cc_g(g)
    with E.load_graph(g, placement=placement) as h:
        for kw in (dict(), dict(cc_full_pass=True), dict(granularity=4), dict(granularity=32, chunk_lines=2)):
            lab, st = E.cc(h, **kw)
            np.testing.assert_array_equal(lab, exp, err_msg=str(kw))
    if name in ("urand14", "kron16"):
        with E.load_graph(g, placement=placement) as h:
            _, full = E.cc(h, cc_full_pass=True)
            _, smp = E.cc(h)
            assert smp["edges_scanned"] < 0.5 * full["edges_scanned"]


@pytest.mark.parametrize("placement", ["host", "managed"])
@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "residues-sym", "many"])
def test_list_heads_on_and_off(placement, name):
    """The first four ids of every list mirrored in GPU memory (used by sampled
    CC and bottom-up BFS) change how much is read over the host link, never
    the result."""
    if name == "many":
        g = many_components_graph()
    elif name == "residues-sym":
        r = graph("residues")
        deg = np.diff(r.offsets).astype(np.int64)
        g = gg.csr_from_edges(r.n, np.repeat(np.arange(r.n), deg), r.cols, symmetrize=True, dedup=False,
                              drop_self_loops=False)
    else:
        g = graph(name)
    exp_cc = oracle.cc_g(g)
    for heads in (True, False):
        with E.load_graph(g, placement=placement, heads=heads, with_weights=False) as h:
            for s in sources(g):
                np.testing.assert_array_equal(E.bfs(h, s)[0], oracle.bfs_g(g, s), err_msg=f"heads={heads} src={s}")
                np.testing.assert_array_equal(E.bfs(h, s, granularity=4)[0], oracle.bfs_g(g, s))
            np.testing.assert_array_equal(E.cc(h)[0], exp_cc, err_msg=f"heads={heads}")


@pytest.mark.slow
def test_host_arrays_of_a_gib_or_more():
    """An edge list of 1.3 GB takes the huge-page mapping path of the HOST
    placement (and graphgen allocates it on huge pages, which BORROW then pins
    in place); results equal the oracle's either way."""
    g = gg.uniform(1 << 22, 40, seed=11, weights=True)
    assert g.m * 8 > (1 << 30) and g.m * 4 < (1 << 30)
    s = int(gg.random_sources(g, 1, seed=5)[0])
    exp_bfs, exp_sssp, exp_cc = oracle.bfs_g(g, s), oracle.sssp_g(g, s), oracle.cc_g(g)
    for borrow in (False, True):
        with E.load_graph(g, placement="host", borrow=borrow) as h:
            np.testing.assert_array_equal(E.bfs(h, s)[0], exp_bfs)
            np.testing.assert_array_equal(E.sssp(h, s)[0], exp_sssp)
            np.testing.assert_array_equal(E.cc(h)[0], exp_cc)


def test_borrowed_managed_arrays():
    """EMOGI_PLACE_MANAGED | EMOGI_LOAD_BORROW reads the caller's managed
    arrays in place (read-mostly advice); results equal the oracle's, a
    managed list starting 16 bytes past a line included, and plain host
    memory is rejected."""
    g = graph("kron12")
    for shift in (0, 2):
        cols = E.managed_empty(g.m + 16, np.uint64)[shift:shift + g.m]
        cols[:] = g.cols
        w = E.managed_empty(g.m + 32, np.uint32)[2 * shift:2 * shift + g.m]
        w[:] = g.weights
        with E.load_csr(g.n, g.m, g.offsets, cols, w, placement="managed", borrow=True, undirected=True) as h:
            check_all(g, h)
        del cols, w
    with pytest.raises(E.EmogiError) as ei:
        E.load_csr(g.n, g.m, g.offsets, g.cols, g.weights, placement="managed", borrow=True, undirected=True)
    assert ei.value.status == E.E_ARG and "cudaMallocManaged" in str(ei.value)


def expected_store_bound(g, h):
    """The short-list store's bound for a graph loaded with heads, without a
    device budget: 32 when the lists of 1..32 entries hold at most 1/8 of
    the entries, else 16 (0 for graphs in GPU memory)."""
    if h.placement == E.PLACE_DEVICE:
        return 0
    deg = g.degrees()
    return 32 if int(deg[(deg >= 1) & (deg <= 32)].sum()) * 8 <= g.m else 16


def short_lists_graph(n=20000):
    """Lists of 0 to 19 entries (those of at most 16 are read whole from the
    short-list store in GPU memory, the others from the edge list), every
    multiplicity and order, with a few long lists among them, weights in
    [1, 255]."""
    rng = np.random.default_rng(12)
    deg = rng.integers(0, 20, size=n)
    deg[rng.integers(0, n, size=40)] = rng.integers(5, 700, size=40)
    src = np.repeat(np.arange(n), deg)
    dst = rng.integers(0, n, size=src.size)
    return gg.csr_from_edges(n, src, dst, weights=rng.integers(1, 256, size=src.size), symmetrize=False,
                             dedup=False, drop_self_loops=False, sort=False, name="short-lists")


@pytest.mark.parametrize("placement", ["host", "managed"])
@pytest.mark.parametrize("ids32", [False, True], ids=["u64", "u32"])
def test_short_lists_from_heads_sssp_bfs(placement, ids32):
    """Lists of at most sixteen entries come from the short-list store in GPU
    memory (ids, and weights for SSSP); results equal the oracle's with the
    store on and off, and the bytes reported as read from the edge list leave
    out the entries the store served."""
    g = short_lists_graph()
    g.undirected = False
    srcs = [int(s) for s in gg.random_sources(g, 3, seed=4)] + [gg.max_degree_vertex(g)]
    deg = g.degrees()
    for heads in (True, False):
        with E.load_graph(g, placement=placement, heads=heads, ids32=ids32) as h:
            for s in srcs:
                exp_d = oracle.sssp_g(g, s)
                for kw in (dict(), dict(host_loop=True), dict(granularity=4), dict(ordered_frontier=True)):
                    d, st = E.sssp(h, s, **kw)
                    np.testing.assert_array_equal(d, exp_d, err_msg=f"heads={heads} src={s} {kw}")
                    assert st["edge_bytes"] <= st["edges_scanned"] * (4 if ids32 else 8)
                    if not heads:
                        assert st["edge_bytes"] == st["edges_scanned"] * (4 if ids32 else 8)
                        assert st["weight_bytes"] == st["edges_scanned"] * 4
                lv, st = E.bfs(h, s, top_down_only=True)
                exp = oracle.bfs_g(g, s)
                np.testing.assert_array_equal(lv, exp, err_msg=f"heads={heads} src={s}")
                assert h.store_bound == (expected_store_bound(g, h) if heads else 0)
                if heads:  # every reached list of 1..store_bound entries came from the store
                    short = int(deg[(exp != E.INF) & (deg >= 1) & (deg <= h.store_bound)].sum())
                    assert st["edges_scanned"] * (4 if ids32 else 8) - st["edge_bytes"] == \
                        short * (4 if ids32 else 8)


def test_host_read_probe():
    """The zero-copy read probe times its three patterns over a borrowed edge
    list while the graph is loaded, and rejects memory that is not pinned and
    arguments whose reads would leave the range."""
    g = graph("kron16")
    cols = gg.aligned_empty(g.m, np.uint64)
    cols[:] = g.cols
    nb = cols.nbytes
    with E.load_csr(g.n, g.m, g.offsets, cols, None, placement="host", borrow=True):
        assert E.probe_host_reads(cols, "stream") > 0
        assert E.probe_host_reads(cols, "random", 512, 4096) > 0
        assert E.probe_host_reads(cols, "regions", 512, nb // 4096) > 0
        assert E.probe_host_reads(cols, "regions", 16, nb // 16) > 0  # blocks back to back
        assert E.probe_host_reads(cols, "random", nb // 16 * 16, 3) > 0  # one block spans the range
        for args in (("random", 24, 10), ("random", 0, 10), ("random", 512, 0), ("regions", 512, 0),
                     ("regions", 32, nb // 16), ("random", (nb // 16 + 1) * 16, 1)):
            with pytest.raises(E.EmogiError) as ei:
                E.probe_host_reads(cols, *args)
            assert ei.value.status == E.E_ARG, args
    with pytest.raises(E.EmogiError) as ei:  # unregistered again once the graph is freed
        E.probe_host_reads(cols, "stream")
    assert ei.value.status == E.E_ARG
    with pytest.raises(E.EmogiError) as ei:
        E.probe_host_reads(np.zeros(4096, np.uint64), "random", 512, 16)
    assert ei.value.status == E.E_ARG
