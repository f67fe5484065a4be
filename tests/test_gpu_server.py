"""The continuous-batching query server: every query's result equals the
single-call result, alone and in a mix; BFS queries of one graph are merged;
the device budget limits admission without changing results."""
import threading

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


@pytest.fixture(scope="module")
def resident():
    """Three resident graphs with mixed placements."""
    gs = [gg.kronecker(13, 16, seed=1, weights=True), gg.uniform(1 << 13, 12, seed=2, weights=True),
          gg.kronecker(11, 8, seed=3, weights=True)]
    hs = [E.load_graph(gs[0], placement="host"), E.load_graph(gs[1], placement="device"),
          E.load_graph(gs[2], placement="host")]
    yield gs, hs
    for h in hs:
        h.free()


def _queries(gs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        gi = int(rng.integers(0, len(gs)))
        kind = "bfs" if rng.random() < 0.8 else "sssp"
        src = int(rng.integers(0, gs[gi].n))
        out.append((gi, kind, src))
    return out


def _expected(gs, q):
    gi, kind, src = q
    g = gs[gi]
    return oracle.bfs_g(g, src) if kind == "bfs" else oracle.sssp_g(g, src)


def test_results_equal_alone_and_in_a_mix(resident):
    gs, hs = resident
    qs = _queries(gs, 120, seed=5)
    with E.Server(max_slots=4) as srv:
        # alone: one query at a time
        alone = []
        for gi, kind, src in qs[:10]:
            out = np.empty(gs[gi].n, dtype=np.uint32)
            t = srv.submit(hs[gi], kind, src, out)
            r = srv.wait(t)
            assert r["batch_size"] == 1
            alone.append(out)
        # in a mix: everything submitted at once from two threads
        outs = [np.empty(gs[gi].n, dtype=np.uint32) for gi, _, _ in qs]
        tickets = [None] * len(qs)

        def submitter(lo, hi):
            for i in range(lo, hi):
                gi, kind, src = qs[i]
                tickets[i] = srv.submit(hs[gi], kind, src, outs[i])

        th = [threading.Thread(target=submitter, args=(0, 60)), threading.Thread(target=submitter, args=(60, 120))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        res = [srv.wait(t) for t in tickets]
        for i, q in enumerate(qs):
            np.testing.assert_array_equal(outs[i], _expected(gs, q), err_msg=str(q))
        for i in range(10):
            np.testing.assert_array_equal(alone[i], outs[i])
        assert max(r["batch_size"] for r in res) > 1  # queued BFS queries were merged
        assert all(r["latency_ms"] >= r["run_ms"] >= 0 for r in res)


def test_bfs_queries_of_one_graph_are_batched(resident):
    gs, hs = resident
    g, h = gs[0], hs[0]
    srcs = [int(x) for x in gg.random_sources(g, 150, seed=4)]
    with E.Server(max_slots=1, max_batch=64) as srv:
        outs = [np.empty(g.n, dtype=np.uint32) for _ in srcs]
        ts = [srv.submit(h, "bfs", s, o) for s, o in zip(srcs, outs)]
        res = [srv.wait(t) for t in ts]
    assert max(r["batch_size"] for r in res) == 64
    for s, o in zip(srcs, outs):
        np.testing.assert_array_equal(o, oracle.bfs_g(g, s))


def test_budget_limits_batches_and_rejects_what_never_fits(resident):
    gs, hs = resident
    g, h = gs[1], hs[1]
    n = g.n
    # room for the buffers plus about 4 level rows: batches shrink, results stay exact
    budget = (6 * 4 * n + (n // 16 + 1) * 16 + 20 * (g.m // 497 + 1) + 3 * 8 * n + 1024) + 4 * 4 * n + 16
    srcs = [int(x) for x in gg.random_sources(g, 40, seed=6)]
    with E.Server(max_slots=2, device_budget=budget) as srv:
        outs = [np.empty(n, dtype=np.uint32) for _ in srcs]
        ts = [srv.submit(h, "bfs", s, o) for s, o in zip(srcs, outs)]
        res = [srv.wait(t) for t in ts]
        assert max(r["batch_size"] for r in res) <= 4
        assert srv.device_bytes() <= budget
    for s, o in zip(srcs, outs):
        np.testing.assert_array_equal(o, oracle.bfs_g(g, s))
    with E.Server(max_slots=1, device_budget=1024) as srv:
        t = srv.submit(h, "bfs", 0, np.empty(n, dtype=np.uint32))
        with pytest.raises(E.EmogiError) as ei:
            srv.wait(t)
        assert ei.value.status == E.E_BUDGET


def test_discarded_results_and_errors(resident):
    gs, hs = resident
    with E.Server(max_slots=2) as srv:
        ts = [srv.submit(hs[i % 3], "bfs" if i % 2 else "sssp", 0) for i in range(12)]
        res = [srv.wait(t) for t in ts]
        assert all(r["status"] == 0 for r in res)
        with pytest.raises(E.EmogiError) as ei:
            srv.submit(hs[0], "bfs", gs[0].n)
        assert ei.value.status == E.E_ARG
        with pytest.raises(E.EmogiError):
            srv.wait(123456)
