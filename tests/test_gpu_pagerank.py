"""GPU parity for PageRank (the fourth application of Sec. 5.4) against the
double-precision oracle.

PageRank is floating point: the GPU adds the same terms in another order
(per-list shuffle trees, atomic adds on split lists and on directed graphs),
so each rank may differ from the oracle's by rounding.  With fixed iteration
counts (tolerance 0) both sides run the same iterations; a rank is a sum of
at most n + 2 terms of size <= 1 per iteration, each rounding contributing
at most 2^-53 relative, so the bar is |gpu - oracle| <= 1e-12 + 1e-9 * oracle
(several orders above the worst rounding drift over 30 iterations here,
and far below any algorithmic difference: a dropped dangling term or a
wrong degree moves ranks by > 1e-4 on these graphs).
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
from test_gpu_parity import graph, many_components_graph  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_06890_gb300 import _build
    _build.build()
    E.lib()
    yield


def close(got, exp):
    np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-12)


def get(name):
    return many_components_graph() if name == "many" else graph(name)


@pytest.mark.parametrize("placement", ["device", "host", "managed"])
@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "path", "directed", "residues", "many", "empty",
                                  "single"])
def test_pagerank_fixed_iterations(placement, name):
    g = get(name)
    exp, it = oracle.pagerank_g(g, 0.85, tol=0.0, max_iter=30)
    with E.load_graph(g, placement=placement, with_weights=False) as h:
        for kw in (dict(), dict(granularity=4), dict(granularity=32, chunk_lines=2)):
            r, st = E.pagerank(h, 0.85, tol=0.0, max_iters=30, **kw)
            close(r, exp)
            if g.n:
                assert st["iterations"] == it == 30
                assert st["edges_reached"] == 30 * g.m


@pytest.mark.parametrize("name", ["kron16", "urand14", "hub", "directed"])
def test_pagerank_ids32_and_damping(name):
    g = get(name)
    for d in (0.5, 0.85, 0.99):
        exp, _ = oracle.pagerank_g(g, d, tol=0.0, max_iter=20)
        with E.load_graph(g, placement="host", with_weights=False, ids32=True) as h:
            close(E.pagerank(h, d, tol=0.0, max_iters=20)[0], exp)


@pytest.mark.parametrize("name", ["kron16", "urand14", "directed"])
def test_pagerank_converges_like_the_oracle(name):
    """With a tolerance both stop once the L1 change falls below it; the
    iteration counts agree (the changes are far from the threshold's
    rounding) and the ranks are a probability vector."""
    g = get(name)
    exp, it = oracle.pagerank_g(g, 0.85, tol=1e-10, max_iter=500)
    with E.load_graph(g, placement="host", with_weights=False) as h:
        r, st = E.pagerank(h, 0.85, tol=1e-10, max_iters=500)
    assert abs(st["iterations"] - it) <= 1
    assert abs(r.sum() - 1.0) < 1e-9
    np.testing.assert_allclose(r, exp, rtol=1e-7, atol=1e-11)


def test_pagerank_device_output_and_errors():
    g = graph("kron12")
    exp, _ = oracle.pagerank_g(g, 0.85, tol=0.0, max_iter=10)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    with E.load_graph(g, placement="host", with_weights=False) as h:
        E.pagerank(h, 0.85, tol=0.0, max_iters=10, out=out)
        close(out.cpu().numpy(), exp)
        for bad in (dict(damping=1.0), dict(damping=-0.1), dict(tol=-1.0), dict(max_iters=0)):
            with pytest.raises(E.EmogiError) as ei:
                E.pagerank(h, **bad)
            assert ei.value.status == E.E_ARG
