"""emogi_bfs_noalloc: BFS for callers that cannot allocate GPU memory.

Such callers (code that runs while another component owns the whole device
heap, latency-critical loops that must not block or fail on allocation, or
code sharing a context whose allocator it may not use) hand the library their
own graph and output buffers; the library keeps its frontier queues in one
fixed array per device instead of calling cudaMalloc.  This file checks,
through the C ABI, that two calls in a row give exactly what emogi_bfs and
the oracle's BFS give, at the largest size the array allows too.
It is collected after the other parity tests (only the full-size cases come
later) so that a failure here hides none of them.
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


def _device_csr(g):
    off = torch.from_numpy(np.ascontiguousarray(g.offsets).view(np.int64)).cuda()
    cols = torch.from_numpy(np.ascontiguousarray(g.cols).view(np.int64)).cuda()
    return off, cols


@pytest.mark.parametrize("edges_in", ["device", "pinned-host"])
def test_two_calls_in_a_row_match_emogi_bfs(edges_in):
    g = gg.kronecker(14, 16, seed=5)
    off, cols = _device_csr(g)
    if edges_in == "pinned-host":
        cols = torch.from_numpy(np.ascontiguousarray(g.cols).view(np.int64)).pin_memory()
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    srcs = [gg.max_degree_vertex(g), int(gg.random_sources(g, 1, seed=7)[0])]
    in_use = E.device_bytes_in_use()
    with E.load_graph(g, placement="device") as h:
        for src in srcs:  # two calls in a row share the scratch array
            E.bfs_noalloc(g.n, off, cols, src, level)
            torch.cuda.synchronize()
            got = level.cpu().numpy().view(np.uint32)
            want, _ = E.bfs(h, src)
            np.testing.assert_array_equal(got, want)
            np.testing.assert_array_equal(got, oracle.bfs_g(g, src))
    assert E.device_bytes_in_use() == in_use


def test_maximum_size_and_unaligned_edge_list():
    """n at the maximum the fixed array is sized for, on a uniform graph with
    device edges, then the same edge list seen through
    a view 16 bytes past a 128-byte boundary (list reads start at another
    offset within their line)."""
    n = E.NOALLOC_MAX_VERTICES
    g = gg.uniform(n, 8, seed=11)
    off, cols = _device_csr(g)
    padded = torch.zeros(g.m + 16, dtype=torch.int64, device="cuda")
    assert padded.data_ptr() % 128 == 0
    shifted = padded[2:2 + g.m]
    shifted.copy_(cols)
    assert shifted.data_ptr() % 128 == 16
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    srcs = [gg.max_degree_vertex(g), int(gg.random_sources(g, 1, seed=3)[0])]
    with E.load_graph(g, placement="device") as h:
        for src in srcs:
            want = oracle.bfs_g(g, src)
            np.testing.assert_array_equal(E.bfs(h, src)[0], want)
            for c in (cols, shifted):
                level.fill_(-7)
                E.bfs_noalloc(n, off, c, src, level)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(level.cpu().numpy().view(np.uint32), want)


def test_sizes_beyond_the_maximum_are_rejected():
    n = E.NOALLOC_MAX_VERTICES + 1
    with pytest.raises(E.EmogiError) as ei:
        E.bfs_noalloc(n, 0, 0, 0, 0)
    assert ei.value.status == E.E_ARG
    assert str(E.NOALLOC_MAX_VERTICES) in str(ei.value)
