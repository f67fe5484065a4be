"""CPU oracle for BFS / SSSP / CC / multi-source BFS / PageRank: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package.  The CUDA library never calls it
and it never calls the CUDA library: the two share nothing but the seeded
input generators in ``graphgen``.

The arithmetic lives in ``oracle.c`` (plain, single-threaded C); this module
compiles it with gcc and marshals numpy arrays.  ``linkmodel`` restates the
paper's closed-form interconnect model (Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import linkmodel  # noqa: F401

INF = 0xFFFFFFFF
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lib_handle = None


class OracleError(RuntimeError):
    pass


class OracleOverflow(OracleError):
    """A finite shortest-path distance does not fit below UINT32_MAX."""


def build_lib(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build_lib())
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        lib.oracle_bfs.argtypes = [u64, p, p, u64, p]
        lib.oracle_sssp.argtypes = [u64, p, p, p, u64, p]
        lib.oracle_cc.argtypes = [u64, p, p, p]
        lib.oracle_pagerank.argtypes = [u64, p, p, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, p, p]
        for f in (lib.oracle_bfs, lib.oracle_sssp, lib.oracle_cc, lib.oracle_pagerank):
            f.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


def bfs(n, offsets, cols, src) -> np.ndarray:
    """BFS level of every vertex from `src` (UINT32_MAX = unreachable)."""
    off, po = _arr(offsets, np.uint64)
    col, pc = _arr(cols, np.uint64)
    out = np.empty(max(n, 1), dtype=np.uint32)
    rc = _lib().oracle_bfs(n, po, pc, int(src), ctypes.c_void_p(out.ctypes.data))
    if rc:
        raise OracleError(f"oracle_bfs failed ({rc})")
    return out[:n]


def sssp(n, offsets, cols, weights, src) -> np.ndarray:
    """Shortest-path distance of every vertex from `src` (UINT32_MAX = unreachable)."""
    off, po = _arr(offsets, np.uint64)
    col, pc = _arr(cols, np.uint64)
    w, pw = _arr(weights, np.uint32)
    out = np.empty(max(n, 1), dtype=np.uint32)
    rc = _lib().oracle_sssp(n, po, pc, pw, int(src), ctypes.c_void_p(out.ctypes.data))
    if rc == 3:
        raise OracleOverflow("a shortest-path distance exceeds UINT32_MAX - 1")
    if rc:
        raise OracleError(f"oracle_sssp failed ({rc})")
    return out[:n]


def cc(n, offsets, cols) -> np.ndarray:
    """Connected-component label of every vertex = smallest vertex id in its component."""
    off, po = _arr(offsets, np.uint64)
    col, pc = _arr(cols, np.uint64)
    out = np.empty(max(n, 1), dtype=np.uint32)
    rc = _lib().oracle_cc(n, po, pc, ctypes.c_void_p(out.ctypes.data))
    if rc:
        raise OracleError(f"oracle_cc failed ({rc})")
    return out[:n]


def msbfs(n, offsets, cols, sources) -> np.ndarray:
    """Multi-source BFS: row k is the independent BFS from sources[k]."""
    srcs = [int(s) for s in np.asarray(sources).ravel()]
    out = np.empty((len(srcs), n), dtype=np.uint32)
    for k, s in enumerate(srcs):
        out[k] = bfs(n, offsets, cols, s)
    return out


def pagerank(n, offsets, cols, damping=0.85, tol=1e-10, max_iter=100):
    """(ranks float64[n], iterations) by power iteration (oracle.c)."""
    off, poff = _arr(offsets, np.uint64)
    col, pcol = _arr(cols, np.uint64)
    out = np.empty(max(n, 1), dtype=np.float64)
    it = np.zeros(1, dtype=np.uint32)
    rc = _lib().oracle_pagerank(n, poff, pcol, float(damping), float(tol), int(max_iter),
                                ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(it.ctypes.data))
    if rc != 0:
        raise OracleError(f"oracle_pagerank failed ({rc})")
    return out[:n], int(it[0])


def pagerank_g(g, damping=0.85, tol=1e-10, max_iter=100):
    return pagerank(g.n, g.offsets, g.cols, damping, tol, max_iter)


def bfs_g(g, src):
    return bfs(g.n, g.offsets, g.cols, src)


def sssp_g(g, src):
    return sssp(g.n, g.offsets, g.cols, g.weights, src)


def cc_g(g):
    return cc(g.n, g.offsets, g.cols)


def reached_edges(offsets, values) -> int:
    """Directed edges out of reached vertices (finite value): the TEPS numerator."""
    deg = np.diff(np.asarray(offsets, dtype=np.uint64)).astype(np.int64)
    return int(deg[np.asarray(values) != INF].sum())
