"""Seeded synthetic graph inputs shared by the CPU oracle and the CUDA path.

This package only makes inputs (CSR arrays, weights, sources).  It holds none
of the traversal arithmetic; the oracle and the CUDA library both consume its
output and neither is imported here.

Large graphs come from the C builder in ``graphgen.c`` (OpenMP, counter-based
SplitMix64 streams, so results do not depend on the thread count); tiny
hand-made graphs come from :func:`csr_from_edges`.
"""
from __future__ import annotations

import ctypes
import mmap
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lib_handle = None

KRON = 0
UNIFORM = 1
# vertex blocks of the final sort-and-pack pass (the result does not depend on it)
FINISH_BLOCKS = 4096


def build_lib(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build_lib())
        u64, i32 = ctypes.c_uint64, ctypes.c_int
        p = ctypes.c_void_p
        lib.gg_rand.restype = u64
        lib.gg_rand.argtypes = [u64, u64]
        lib.gg_relabel_table.argtypes = [i32, u64, p]
        lib.gg_sample.argtypes = [i32, u64, i32, u64, i32, u64, u64, p, p]
        lib.gg_count.argtypes = [i32, u64, i32, u64, i32, u64, i32, p, p]
        lib.gg_fill.argtypes = [i32, u64, i32, u64, i32, u64, i32, p, p, p]
        lib.gg_finish.argtypes = [u64, p, p, u64, p, p, p]
        lib.gg_weights.argtypes = [u64, p, p, u64, p]
        lib.gg_num_threads.restype = i32
        _lib_handle = lib
    return _lib_handle


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _huge_page_bytes() -> int:
    try:
        with open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size") as f:
            v = int(f.read().strip())
        return v if v >= 4096 and v & (v - 1) == 0 else 2 << 20
    except (OSError, ValueError):
        return 2 << 20


def aligned_empty(count: int, dtype, align: int = 4096) -> np.ndarray:
    """Uninitialised 1-D array whose data pointer is `align`-byte aligned.
    Arrays of a GiB or more come from an anonymous mapping advised to use
    transparent huge pages (aligned to the huge-page size), so that a GPU
    reading them in place (zero-copy) needs few address translations."""
    dtype = np.dtype(dtype)
    nbytes = max(1, int(count)) * dtype.itemsize
    if nbytes >= (1 << 30) and hasattr(mmap, "MADV_HUGEPAGE"):
        hp = max(_huge_page_bytes(), align)
        mm = mmap.mmap(-1, nbytes + hp, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        raw = np.frombuffer(mm, dtype=np.uint8)
        off = (-raw.ctypes.data) % hp
        try:
            mm.madvise(mmap.MADV_HUGEPAGE, off, nbytes)
        except (OSError, ValueError):
            pass  # without transparent huge pages the mapping keeps small pages
        return raw[off:off + nbytes].view(dtype)[:int(count)]
    raw = np.empty(nbytes + align, dtype=np.uint8)
    off = (-raw.ctypes.data) % align
    return raw[off:off + nbytes].view(dtype)[:int(count)]


def huge_page_report() -> dict:
    """Transparent huge page settings and this process's anonymous memory on
    huge pages (from /proc), for reports beside measurements of arrays that a
    GPU reads in place: with 64 KiB pages a tens-of-GB edge list needs far
    more address translations than the GPU holds."""
    out = {}
    for name in ("enabled", "defrag"):
        try:
            with open(f"/sys/kernel/mm/transparent_hugepage/{name}") as f:
                txt = f.read().strip()
            out[name] = txt[txt.index("[") + 1:txt.index("]")] if "[" in txt else txt
        except (OSError, ValueError):
            out[name] = None
    out["huge_page_bytes"] = _huge_page_bytes()
    try:
        with open("/proc/self/smaps_rollup") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k in ("Anonymous", "AnonHugePages"):
                    out[k.lower() + "_bytes"] = int(v.split()[0]) * 1024
    except OSError:
        pass
    return out


def numa_report(*arrays) -> dict:
    """Where the host pages of the given arrays live: for each array, the NUMA
    nodes holding its mapping's pages and the mapping's page size (from
    /proc/self/numa_maps), and the kernel's automatic NUMA balancing setting
    (which unmaps pages now and then to sample accesses)."""
    out = {}
    try:
        with open("/proc/sys/kernel/numa_balancing") as f:
            out["numa_balancing"] = f.read().strip()
    except OSError:
        out["numa_balancing"] = None
    try:
        maps = []
        with open("/proc/self/numa_maps") as f:
            for line in f:
                parts = line.split()
                maps.append((int(parts[0], 16), parts[1:]))
        maps.sort()
        for i, a in enumerate(arrays):
            addr, best = a.ctypes.data, None
            for start, fields in maps:
                if start > addr:
                    break
                best = fields
            if best is not None:
                rec = dict(f.split("=", 1) for f in best if "=" in f)
                out[f"array{i}"] = {k: v for k, v in rec.items()
                                    if k.startswith("N") or k in ("kernelpagesize_kB", "anon")}
    except (OSError, ValueError):
        pass
    return out


def release_host_range(arr: np.ndarray, lo: int, hi: int) -> int:
    """Return the physical pages wholly inside elements [lo, hi) of a 1-D
    array to the operating system (madvise MADV_DONTNEED; for anonymous
    memory those pages then read as zeros).  Lets a caller that has copied
    a large array elsewhere in pieces free each piece at once, so that the
    two copies never coexist.  Returns the bytes released."""
    item = arr.dtype.itemsize
    a = arr.ctypes.data + max(0, int(lo)) * item
    b = arr.ctypes.data + min(int(hi), arr.size) * item
    page = mmap.PAGESIZE
    a = (a + page - 1) // page * page
    b = b // page * page
    if b <= a:
        return 0
    libc = ctypes.CDLL(None, use_errno=True)
    libc.madvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    MADV_DONTNEED = 4
    if libc.madvise(ctypes.c_void_p(a), ctypes.c_size_t(b - a), MADV_DONTNEED) != 0:
        raise OSError(ctypes.get_errno(), "madvise(MADV_DONTNEED) failed")
    return b - a


@dataclass
class Graph:
    """A CSR graph: offsets uint64[n+1], cols uint64[m], optional weights uint32[m]."""
    n: int
    offsets: np.ndarray
    cols: np.ndarray
    weights: Optional[np.ndarray] = None
    undirected: bool = True
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.offsets[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


def rand(seed: int, i: int) -> int:
    """i-th output of the SplitMix64 stream seeded with `seed`."""
    return int(_lib().gg_rand(seed & (2**64 - 1), i))


def relabelling(scale: int, seed: int) -> np.ndarray:
    """The seeded bijection of [0, 2^scale) that relabels Kronecker vertex ids
    (entry x = the new id of x)."""
    perm = np.empty(1 << scale, dtype=np.uint64)
    _lib().gg_relabel_table(scale, seed, _ptr(perm))
    return perm


def samples(kind: int, n: int, scale: int, seed: int, count: int, permute: bool = True,
            k0: int = 0):
    """Raw edge samples (before cleaning) of a generated graph."""
    src = np.empty(count, dtype=np.uint64)
    dst = np.empty(count, dtype=np.uint64)
    _lib().gg_sample(kind, n, scale, seed, int(bool(permute)), k0, count, _ptr(src), _ptr(dst))
    return src, dst


def _build(kind: int, n: int, scale: int, nsamples: int, seed: int, permute: bool,
           with_weights: bool, wseed: int, name: str) -> Graph:
    lib = _lib()
    pm = int(bool(permute and kind == KRON))
    deg = aligned_empty(n, np.uint64)
    # per-part vertex counts (no atomics in either pass); more parts than
    # threads would only cost memory, fewer would idle threads.  The arrays
    # that both passes update at random sit on huge pages (aligned_empty) so
    # that those updates rarely miss the TLB.
    parts = max(1, min(num_threads(), 64, max(1, nsamples // 4096)))
    cnt = aligned_empty(parts * n, np.uint32)
    lib.gg_count(kind, n, scale, seed, pm, nsamples, parts, _ptr(cnt), _ptr(deg))
    off_raw = aligned_empty(n + 1, np.uint64)
    off_raw[0] = 0
    np.cumsum(deg, out=off_raw[1:])
    m_raw = int(off_raw[-1])
    cols = aligned_empty(m_raw, np.uint64)
    lib.gg_fill(kind, n, scale, seed, pm, nsamples, parts, _ptr(cnt), _ptr(off_raw), _ptr(cols))
    del cnt
    off = np.empty(n + 1, dtype=np.uint64)
    nblocks = max(1, min(n, FINISH_BLOCKS))
    blk = np.empty(nblocks, dtype=np.uint64)
    lib.gg_finish(n, _ptr(off_raw), _ptr(cols), nblocks, _ptr(blk), _ptr(deg), _ptr(off))
    m = int(off[-1])
    cols = cols[:m]
    w = None
    if with_weights:
        w = aligned_empty(m, np.uint32)
        lib.gg_weights(n, _ptr(off), _ptr(cols), wseed, _ptr(w))
    return Graph(n=n, offsets=off, cols=cols, weights=w, undirected=True, name=name)


def kronecker(scale: int, edge_factor: int, seed: int = 1, weights: bool = False,
              wseed: Optional[int] = None, permute: bool = True) -> Graph:
    """Undirected Kronecker graph: 2^scale vertices, edge_factor * 2^scale samples,
    initiator (0.57, 0.19, 0.19, 0.05), ids permuted by seed, cleaned, symmetric."""
    n = 1 << scale
    return _build(KRON, n, scale, edge_factor * n, seed, permute, weights,
                  seed if wseed is None else wseed, f"kron{scale}_ef{edge_factor}_s{seed}")


def uniform(n: int, avg_degree: float, seed: int = 1, weights: bool = False,
            wseed: Optional[int] = None) -> Graph:
    """Undirected uniform-random graph with n vertices and n*avg_degree/2 samples
    (so about n*avg_degree directed edges after symmetrisation)."""
    nsamples = int(round(n * avg_degree / 2))
    return _build(UNIFORM, n, 0, nsamples, seed, False, weights,
                  seed if wseed is None else wseed, f"urand_n{n}_d{avg_degree}_s{seed}")


def add_weights(g: Graph, seed: int = 1) -> Graph:
    """Attach symmetric weights in [1, 255] to an existing graph."""
    w = aligned_empty(g.m, np.uint32)
    if g.m:
        _lib().gg_weights(g.n, _ptr(np.ascontiguousarray(g.offsets, dtype=np.uint64)),
                          _ptr(np.ascontiguousarray(g.cols, dtype=np.uint64)), seed, _ptr(w))
    g.weights = w
    return g


def csr_from_edges(n: int, src, dst, weights=None, symmetrize: bool = True,
                   dedup: bool = True, drop_self_loops: bool = True, sort: bool = True,
                   name: str = "") -> Graph:
    """Build a CSR graph from an edge list with numpy (small graphs).

    With dedup, duplicate (u, v) pairs keep the smallest weight.  Without
    dedup/sort, rows keep the input order (stable), which tests use to make
    lists with duplicates and self-loops.
    """
    src = np.asarray(src, dtype=np.uint64).ravel()
    dst = np.asarray(dst, dtype=np.uint64).ravel()
    w = None if weights is None else np.asarray(weights, dtype=np.uint32).ravel()
    if drop_self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
        w = None if w is None else w[keep]
    if symmetrize:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        w = None if w is None else np.concatenate([w, w])
    if sort or dedup:
        if w is None:
            order = np.lexsort((dst, src))
        else:
            order = np.lexsort((w, dst, src))
        src, dst = src[order], dst[order]
        w = None if w is None else w[order]
    else:
        order = np.argsort(src, kind="stable")
        src, dst = src[order], dst[order]
        w = None if w is None else w[order]
    if dedup and src.size:
        keep = np.ones(src.size, dtype=bool)
        keep[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
        src, dst = src[keep], dst[keep]
        w = None if w is None else w[keep]
    deg = np.bincount(src.astype(np.int64), minlength=n).astype(np.uint64) if src.size else \
        np.zeros(n, dtype=np.uint64)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg, out=off[1:])
    cols = aligned_empty(dst.size, np.uint64)
    cols[:] = dst
    wa = None
    if w is not None:
        wa = aligned_empty(w.size, np.uint32)
        wa[:] = w
    return Graph(n=n, offsets=off, cols=cols, weights=wa, undirected=symmetrize, name=name)


def path_graph(n: int) -> Graph:
    i = np.arange(max(n - 1, 0), dtype=np.uint64)
    return csr_from_edges(n, i, i + 1, name=f"path{n}")


def star_graph(n: int, center: int = 0) -> Graph:
    leaves = np.array([v for v in range(n) if v != center], dtype=np.uint64)
    return csr_from_edges(n, np.full(leaves.size, center, dtype=np.uint64), leaves,
                          name=f"star{n}")


def complete_graph(n: int) -> Graph:
    iu = np.triu_indices(n, 1)
    return csr_from_edges(n, iu[0], iu[1], name=f"complete{n}")


def empty_graph(n: int) -> Graph:
    return csr_from_edges(n, np.zeros(0), np.zeros(0), name=f"empty{n}")


def random_small(n: int, p: float, seed: int, directed: bool = False) -> Graph:
    """Erdos-Renyi G(n, p) from the counter stream (small n only)."""
    s, d = [], []
    k = 0
    for u in range(n):
        for v in range(n):
            if u == v or (not directed and v < u):
                continue
            r = rand(seed, k) >> 11
            k += 1
            if r < int(p * 2**53):
                s.append(u)
                d.append(v)
    return csr_from_edges(n, np.array(s, dtype=np.uint64), np.array(d, dtype=np.uint64),
                          symmetrize=not directed, name=f"gnp{n}_{p}_{seed}")


def max_degree_vertex(g: Graph) -> int:
    """Highest-degree vertex; ties go to the smallest id."""
    return int(np.argmax(g.degrees())) if g.n else 0


def pick_seeded(candidates, count: int, seed: int) -> np.ndarray:
    """`count` distinct entries of `candidates` drawn by the seeded stream
    (value i of the stream picks candidate floor(r_i * size / 2^64))."""
    cand = np.asarray(candidates)
    if cand.size == 0:
        return np.zeros(0, dtype=np.uint64)
    out, seen, i = [], set(), 0
    while len(out) < min(count, cand.size):
        j = int(cand[(rand(seed, i) * cand.size) >> 64])
        i += 1
        if j not in seen:
            seen.add(j)
            out.append(j)
    return np.array(out, dtype=np.uint64)


def random_sources(g: Graph, count: int, seed: int = 2, min_degree: int = 1) -> np.ndarray:
    """`count` distinct seeded vertices with out-degree >= min_degree."""
    return pick_seeded(np.nonzero(g.degrees() >= min_degree)[0], count, seed)


def num_threads() -> int:
    return int(_lib().gg_num_threads())


# ------------------------------------------------------------ binary CSR cache
# A generated graph is written once as one binary file and read back instead of
# being generated again.  Layout (little-endian): a 64-byte header
#   magic "EMOGICSR", format version u32, flags u32 (bit 0: weights, bit 1:
#   undirected), n u64, m u64, name length u32, 28 reserved bytes,
# the name (UTF-8), zero padding to a 4096-byte boundary, then offsets
# uint64[n+1], cols uint64[m] and weights uint32[m], each starting on a
# 4096-byte boundary, so that every array is read straight into its
# (huge-page) destination.
CACHE_MAGIC = b"EMOGICSR"
CACHE_VERSION = 1
# bumped whenever the generators' output for given arguments changes, so that a
# cache written by an older builder is never read for a newer one
GENERATOR_VERSION = 1
_CACHE_ALIGN = 4096
_CACHE_CHUNK = 1 << 28


def _cache_layout(n: int, m: int, weights: bool, name: bytes):
    def up(x):
        return (x + _CACHE_ALIGN - 1) // _CACHE_ALIGN * _CACHE_ALIGN
    off_at = up(64 + len(name))
    cols_at = up(off_at + (n + 1) * 8)
    w_at = up(cols_at + m * 8)
    end = w_at + (m * 4 if weights else 0)
    return off_at, cols_at, w_at, end


def _io_ranges(start: int, nbytes: int):
    return [(start + a, min(_CACHE_CHUNK, nbytes - a)) for a in range(0, nbytes, _CACHE_CHUNK)]


def _parallel_io(fd: int, jobs, write: bool):
    """jobs: (numpy byte view, file offset); chunks of 256 MiB on a thread pool
    (the system calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(job):
        view, at = job
        done = 0
        while done < view.nbytes:
            mv = memoryview(view[done:])
            k = os.pwrite(fd, mv, at + done) if write else os.preadv(fd, [mv], at + done)
            if k <= 0:
                raise OSError(f"short {'write' if write else 'read'} at byte {at + done}")
            done += k

    pieces = []
    for arr, at in jobs:
        b = arr.view(np.uint8).reshape(-1)
        for a, k in _io_ranges(0, b.nbytes):
            pieces.append((b[a:a + k], at + a))
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(one, pieces))


def save(g: Graph, path: str) -> None:
    """Write `g` to `path` in the cache format (through a temporary file that
    is renamed into place, so a reader never sees a partial file)."""
    name = (g.name or "").encode()
    n, m, has_w = int(g.n), int(g.m), g.weights is not None
    off_at, cols_at, w_at, end = _cache_layout(n, m, has_w, name)
    head = bytearray(64)
    head[0:8] = CACHE_MAGIC
    flags = (1 if has_w else 0) | (2 if g.undirected else 0)
    head[8:36] = np.array([CACHE_VERSION, flags], "<u4").tobytes() + np.array([n, m], "<u8").tobytes() + \
        np.array([len(name)], "<u4").tobytes()
    tmp = f"{path}.tmp{os.getpid()}"
    fd = os.open(tmp, os.O_WRONLY | os.O_CREAT | os.O_TRUNC, 0o644)
    try:
        os.ftruncate(fd, end)
        os.pwrite(fd, bytes(head) + name, 0)
        jobs = [(np.ascontiguousarray(g.offsets, dtype=np.uint64), off_at),
                (np.ascontiguousarray(g.cols, dtype=np.uint64), cols_at)]
        if has_w:
            jobs.append((np.ascontiguousarray(g.weights, dtype=np.uint32), w_at))
        _parallel_io(fd, jobs, write=True)
        os.fsync(fd)
    except BaseException:
        os.close(fd)
        os.unlink(tmp)
        raise
    os.close(fd)
    os.replace(tmp, path)


def load(path: str) -> Graph:
    """Read a graph written by :func:`save`.  The edge list and weights land
    in fresh arrays from :func:`aligned_empty` (huge pages from 1 GiB up), as
    if generated.  Raises ValueError on a file that is not a cache of this
    format or whose size does not match its header."""
    fd = os.open(path, os.O_RDONLY)
    try:
        head = os.pread(fd, 64, 0)
        if len(head) != 64 or head[0:8] != CACHE_MAGIC:
            raise ValueError(f"{path}: not a graph cache file")
        version, flags = np.frombuffer(head[8:16], "<u4")
        n, m = (int(x) for x in np.frombuffer(head[16:32], "<u8"))
        name_len = int(np.frombuffer(head[32:36], "<u4")[0])
        if int(version) != CACHE_VERSION:
            raise ValueError(f"{path}: cache format {int(version)}, expected {CACHE_VERSION}")
        has_w = bool(flags & 1)
        name = os.pread(fd, name_len, 64).decode()
        off_at, cols_at, w_at, end = _cache_layout(n, m, has_w, name.encode())
        if os.fstat(fd).st_size != end:
            raise ValueError(f"{path}: {os.fstat(fd).st_size} bytes, the header describes {end}")
        off = aligned_empty(n + 1, np.uint64)
        cols = aligned_empty(m, np.uint64)
        w = aligned_empty(m, np.uint32) if has_w else None
        jobs = [(off, off_at), (cols, cols_at)] + ([(w, w_at)] if has_w else [])
        _parallel_io(fd, jobs, write=False)
    finally:
        os.close(fd)
    if int(off[0]) != 0 or int(off[-1]) != m:
        raise ValueError(f"{path}: row offsets do not run from 0 to m = {m}")
    return Graph(n=n, offsets=off, cols=cols, weights=w, undirected=bool(flags & 2), name=name)


def cache_key(kind: str, size: int, degree: float, seed: int, weights: bool, wseed: Optional[int] = None) -> str:
    """File name of a generated graph: the generator, its arguments and the
    generator version."""
    w = f"_w{seed if wseed is None else wseed}" if weights else ""
    return f"{kind}_{size}_{degree}_s{seed}{w}_g{GENERATOR_VERSION}.csr"


def cached(cache_dir: str, kind: str, size: int, degree: float, seed: int = 1, weights: bool = False,
           wseed: Optional[int] = None) -> Graph:
    """The graph `kronecker(size, degree, ...)` (kind "kron") or
    `uniform(size, degree, ...)` (kind "urand"), read from `cache_dir` when it
    holds it, else generated and written there."""
    if kind not in ("kron", "urand"):
        raise ValueError(f"unknown generator {kind!r}")
    path = os.path.join(cache_dir, cache_key(kind, size, degree, seed, weights, wseed))
    if os.path.exists(path):
        return load(path)
    if kind == "kron":
        g = kronecker(int(size), int(degree), seed=seed, weights=weights, wseed=wseed)
    else:
        g = uniform(int(size), degree, seed=seed, weights=weights, wseed=wseed)
    os.makedirs(cache_dir, exist_ok=True)
    save(g, path)
    return g
