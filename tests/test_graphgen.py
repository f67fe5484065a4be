"""The seeded input generators: structure, cleaning and determinism."""
import os
import subprocess
import sys

import numpy as np

import graphgen as gg


def _check_clean_symmetric(g):
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.uint64), deg)
    assert np.all(src != g.cols)  # no self-loops
    assert np.all(g.cols < g.n)
    # rows strictly increasing => sorted and de-duplicated
    inner = np.ones(g.m, dtype=bool)
    starts = g.offsets[:-1][deg > 0].astype(np.int64)
    inner[starts] = False
    assert np.all(np.diff(g.cols.astype(np.int64))[inner[1:]] > 0)
    # symmetric: the multiset of (u, v) equals that of (v, u)
    a = np.sort(src * np.uint64(g.n) + g.cols)
    b = np.sort(g.cols * np.uint64(g.n) + src)
    assert np.array_equal(a, b)


def test_kronecker_clean_symmetric_weighted():
    g = gg.kronecker(12, 16, seed=1, weights=True)
    assert g.n == 4096
    _check_clean_symmetric(g)
    assert 0 < g.m <= 2 * 16 * 4096
    assert g.weights.min() >= 1 and g.weights.max() <= 255
    # weight symmetry: w(u,v) == w(v,u)
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.uint64), deg)
    key_uv = src * np.uint64(g.n) + g.cols
    key_vu = g.cols * np.uint64(g.n) + src
    o1, o2 = np.argsort(key_uv), np.argsort(key_vu)
    assert np.array_equal(g.weights[o1], g.weights[o2])
    # heavy tail: the hub is far above the mean degree
    assert deg.max() > 20 * deg.mean()


def test_uniform_degree_distribution():
    g = gg.uniform(1 << 16, 32, seed=1)
    _check_clean_symmetric(g)
    deg = g.degrees()
    assert abs(deg.mean() - 32) < 0.5
    assert deg.max() < 80


def test_generation_is_deterministic_across_thread_counts():
    code = ("import graphgen as gg, hashlib;"
            "g = gg.kronecker(11, 8, seed=3, weights=True);"
            "print(hashlib.sha1(g.offsets.tobytes() + g.cols.tobytes() + g.weights.tobytes()).hexdigest())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t, PYTHONPATH=root)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=root).strip())
    assert outs[0] == outs[1]


def test_seeds_differ_and_relabelling_is_bijective():
    for scale in (1, 2, 7, 10, 16):
        p = gg.relabelling(scale, 5)
        assert np.array_equal(np.sort(p), np.arange(1 << scale, dtype=np.uint64))
    p, q = gg.relabelling(12, 5), gg.relabelling(12, 6)
    assert not np.array_equal(p, q) and not np.array_equal(p, np.arange(1 << 12, dtype=np.uint64))
    a = gg.kronecker(10, 8, seed=1)
    b = gg.kronecker(10, 8, seed=2)
    assert not np.array_equal(a.cols[:100], b.cols[:100])


def test_sources():
    g = gg.kronecker(10, 8, seed=1)
    s = gg.max_degree_vertex(g)
    assert g.degrees()[s] == g.degrees().max()
    assert s == int(np.nonzero(g.degrees() == g.degrees().max())[0][0])
    r = gg.random_sources(g, 16, seed=2)
    assert len(set(r.tolist())) == 16 and np.all(g.degrees()[r.astype(np.int64)] >= 1)


def test_csr_from_edges_keeps_duplicates_when_asked():
    g = gg.csr_from_edges(3, [0, 0, 1, 2], [1, 1, 1, 0], symmetrize=False, dedup=False,
                          drop_self_loops=False, sort=False)
    assert g.offsets.tolist() == [0, 2, 3, 4]
    assert g.cols.tolist() == [1, 1, 1, 0]


def test_aligned_allocation():
    a = gg.aligned_empty(1000, np.uint64, 4096)
    assert a.ctypes.data % 4096 == 0 and a.size == 1000


def test_builder_equals_a_plain_csr_of_the_raw_samples(monkeypatch):
    """The C builder (per-part counts, scatter, block sort-and-pack) gives the
    CSR that numpy builds from the same raw samples: self-loops dropped, both
    directions, rows sorted and de-duplicated; whatever the number of blocks
    of the pack pass (a dense graph, so that later blocks move by more than
    their own length and are copied in parallel chunks)."""
    scale, ef = 12, 64
    n = 1 << scale
    src, dst = gg.samples(gg.KRON, n, scale, seed=4, count=ef * n)
    ref = gg.csr_from_edges(n, src, dst)
    assert ref.m < 0.6 * 2 * ef * n  # many duplicates
    for blocks in (1, 2, 3, 4096):
        monkeypatch.setattr(gg, "FINISH_BLOCKS", blocks)
        g = gg.kronecker(scale, ef, seed=4)
        assert np.array_equal(g.offsets, ref.offsets), blocks
        assert np.array_equal(g.cols, ref.cols), blocks
    u = gg.uniform(5000, 9, seed=3)
    us, ud = gg.samples(gg.UNIFORM, 5000, 0, seed=3, count=int(round(5000 * 9 / 2)))
    ur = gg.csr_from_edges(5000, us, ud)
    assert np.array_equal(u.offsets, ur.offsets) and np.array_equal(u.cols, ur.cols)


def test_kronecker_quadrant_frequencies():
    """Each bit level of a raw (unrelabelled) sample picks quadrant
    (0,0), (0,1), (1,0), (1,1) with probabilities 0.57, 0.19, 0.19, 0.05."""
    scale = 10
    src, dst = gg.samples(gg.KRON, 1 << scale, scale, seed=9, count=200_000, permute=False)
    for lvl in (0, 3, 4, 9):
        bu = (src >> np.uint64(lvl)) & np.uint64(1)
        bv = (dst >> np.uint64(lvl)) & np.uint64(1)
        f = [np.mean((bu == a) & (bv == b)) for a, b in ((0, 0), (0, 1), (1, 0), (1, 1))]
        np.testing.assert_allclose(f, [0.57, 0.19, 0.19, 0.05], atol=0.005)


def test_release_host_range_frees_pages_of_a_large_array():
    a = gg.aligned_empty((1 << 30) // 8 + 1024, np.uint64)
    a[:] = 7
    released = gg.release_host_range(a, 1000, a.size - 1000)
    assert released > (1 << 29)
    assert a[0] == 7 and a[-1] == 7 and a[a.size // 2] == 0


def _same_graph(a, b):
    assert (a.n, a.m, a.undirected, a.name) == (b.n, b.m, b.undirected, b.name)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    assert (a.weights is None) == (b.weights is None)
    if a.weights is not None:
        assert np.array_equal(a.weights, b.weights)


def test_binary_cache_round_trip(tmp_path):
    """Weighted and unweighted, directed and undirected, empty graphs read
    back equal to what was written, with every array 4096-byte aligned."""
    graphs = [gg.kronecker(11, 16, seed=4, weights=True), gg.uniform(3000, 5, seed=2),
              gg.empty_graph(7),
              gg.csr_from_edges(5, np.array([0, 0, 3, 4]), np.array([1, 1, 2, 0]), weights=np.array([9, 8, 7, 6]),
                                symmetrize=False, dedup=False, drop_self_loops=False, sort=False, name="tiny")]
    graphs[-1].undirected = False
    for i, g in enumerate(graphs):
        p = str(tmp_path / f"g{i}.csr")
        gg.save(g, p)
        h = gg.load(p)
        _same_graph(g, h)
        for arr in (h.offsets, h.cols) + ((h.weights,) if h.weights is not None else ()):
            assert arr.ctypes.data % 4096 == 0
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]


def test_binary_cache_rejects_other_files(tmp_path):
    g = gg.kronecker(10, 8, seed=1, weights=True)
    p = str(tmp_path / "g.csr")
    gg.save(g, p)
    raw = open(p, "rb").read()
    for bad, what in ((raw[:-4], "bytes"), (b"NOTACSR!" + raw[8:], "not a graph cache"),
                      (raw[:8] + (9).to_bytes(4, "little") + raw[12:], "format")):
        q = str(tmp_path / "bad.csr")
        open(q, "wb").write(bad)
        try:
            gg.load(q)
        except ValueError as e:
            assert what in str(e)
        else:
            raise AssertionError(f"accepted a file with bad {what}")


def test_cached_generates_once_then_reads(tmp_path, monkeypatch):
    """The first call generates and writes, the second reads the file and
    gets the same graph; other arguments get other files."""
    d = str(tmp_path)
    a = gg.cached(d, "kron", 10, 16, seed=5, weights=True)
    _same_graph(a, gg.kronecker(10, 16, seed=5, weights=True))
    calls = []
    monkeypatch.setattr(gg, "kronecker", lambda *x, **k: calls.append(x))
    b = gg.cached(d, "kron", 10, 16, seed=5, weights=True)
    assert not calls
    _same_graph(a, b)
    monkeypatch.undo()
    gg.cached(d, "kron", 10, 16, seed=6, weights=True)
    gg.cached(d, "kron", 10, 16, seed=5)
    gg.cached(d, "urand", 1000, 4, seed=5)
    assert len(os.listdir(d)) == 4
