"""Thin Python binding of the C ABI in include/emogi.h (ctypes).

Argument marshalling only: every step of a traversal runs in libemogi.so's
CUDA kernels.  The functions carry the C names without the ``emogi_`` prefix.
If the shared library has not been built, importing works but the first call
raises :class:`LibraryNotBuilt` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libemogi.so")

INF = 0xFFFFFFFF
MAX_SOURCES = 64

# emogi_status
OK, E_ARG, E_NOMEM, E_BUDGET, E_CUDA, E_TIMEOUT, E_OVERFLOW, E_UNSUPPORTED = range(8)
# emogi_placement
PLACE_DEVICE, PLACE_HOST, PLACE_MANAGED = 0, 1, 2
PLACEMENTS = {"device": PLACE_DEVICE, "host": PLACE_HOST, "managed": PLACE_MANAGED}
# load flags
LOAD_UNDIRECTED, LOAD_BORROW, LOAD_NO_HEADS = 1, 2, 4
# emogi_access
ACCESS_MERGED_ALIGNED, ACCESS_MERGED, ACCESS_NAIVE = 0, 1, 2
ACCESS = {"merged_aligned": ACCESS_MERGED_ALIGNED, "aligned": ACCESS_MERGED_ALIGNED,
          "merged": ACCESS_MERGED, "naive": ACCESS_NAIVE}
# opts flags
OPT_TIME_KERNELS = 1
OPT_TOP_DOWN_ONLY = 2
OPT_CC_FULL_PASS = 4
OPT_HOST_LOOP = 8
OPT_BEAMER = 16
OPT_ORDERED_FRONTIER = 32


class LibraryNotBuilt(RuntimeError):
    pass


class EmogiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("access", ctypes.c_uint32),
                ("granularity", ctypes.c_uint32), ("chunk_lines", ctypes.c_uint32),
                ("timeout_ns", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("out_on_device", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("delta", ctypes.c_uint32), ("reserved0", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("edges_scanned", ctypes.c_uint64), ("edges_reached", ctypes.c_uint64),
                ("edge_bytes", ctypes.c_uint64), ("weight_bytes", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("expand_ms", ctypes.c_double),
                ("expand_launches", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# (name, restype, argtypes) of every exported entry point
_P, _U64, _U32, _I32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_SIGNATURES = [
    ("emogi_load_csr", _I32, [_U64, _U64, _P, _P, _P, _I32, _U32, ctypes.POINTER(_P)]),
    ("emogi_load_csr32", _I32, [_U64, _U64, _P, _P, _P, _I32, _U32, ctypes.POINTER(_P)]),
    ("emogi_bfs", _I32, [_P, _U64, _P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_sssp", _I32, [_P, _U64, _P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_cc", _I32, [_P, _P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_pagerank", _I32, [_P, ctypes.c_double, ctypes.c_double, _U32, _P, ctypes.POINTER(Opts),
                              ctypes.POINTER(Stats)]),
    ("emogi_msbfs", _I32, [_P, _P, _U32, _P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_set_device_budget", _I32, [_U64]),
    ("emogi_device_bytes_in_use", _U64, []),
    ("emogi_managed_alloc", _I32, [_U64, ctypes.POINTER(_P)]),
    ("emogi_managed_free", _I32, [_P]),
    ("emogi_free_graph", _I32, [_P]),
    ("emogi_graph_num_vertices", _U64, [_P]),
    ("emogi_graph_num_edges", _U64, [_P]),
    ("emogi_graph_placement", _I32, [_P]),
    ("emogi_graph_store_bound", _U32, [_P]),
    ("emogi_probe_host_reads", _I32, [_P, _U64, _U32, _U32, _U64, _P, ctypes.POINTER(ctypes.c_double)]),
    ("emogi_graph_share", _I32, [_P, ctypes.POINTER(_P)]),
    ("emogi_graph_workspace_bytes", _U64, [_P]),
    ("emogi_status_string", ctypes.c_char_p, [_I32]),
    ("emogi_last_error", ctypes.c_char_p, []),
    ("emogi_version", ctypes.c_char_p, []),
    ("emogi_test_fail_device_alloc_after", None, [_I32]),
    ("emogi_bfs_noalloc", _I32, [_U64, _P, _P, _U64, _P, _P]),
    ("emogi_batch_create", _I32, [_P, _U32, ctypes.POINTER(_P)]),
    ("emogi_batch_bfs", _I32, [_P, _P, _P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_batch_autotune", _I32, [_P, _P, ctypes.POINTER(_U32), ctypes.POINTER(_U32),
                                    ctypes.POINTER(ctypes.c_double)]),
    ("emogi_batch_offset", _U64, [_P, _U32]),
    ("emogi_batch_total_vertices", _U64, [_P]),
    ("emogi_batch_free", _I32, [_P]),
    ("emogi_bfs_batch", _I32, [_P, _P, _P, _U32, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
    ("emogi_server_create", _I32, [ctypes.c_void_p, ctypes.POINTER(_P)]),
    ("emogi_server_submit", _I32, [_P, _P, _U32, _U64, _P, ctypes.POINTER(_U64)]),
    ("emogi_server_wait", _I32, [_P, _U64, _U64, ctypes.c_void_p]),
    ("emogi_server_drain", _I32, [_P]),
    ("emogi_server_device_bytes", _U64, [_P]),
    ("emogi_server_destroy", _I32, [_P]),
]
NOALLOC_MAX_VERTICES = 1 << 21

_lib_handle = None


def lib():
    """The loaded libemogi.so (raises LibraryNotBuilt if it is missing)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryNotBuilt(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib_handle = L
    return _lib_handle


def exported_names():
    return [s[0] for s in _SIGNATURES]


def _check(status: int):
    if status != OK:
        msg = lib().emogi_last_error().decode(errors="replace")
        raise EmogiError(status, msg or status_string(status))


def status_string(status: int) -> str:
    return lib().emogi_status_string(status).decode()


def last_error() -> str:
    return lib().emogi_last_error().decode(errors="replace")


def version() -> str:
    return lib().emogi_version().decode()


def set_device_budget(nbytes: int):
    _check(lib().emogi_set_device_budget(int(nbytes)))


def device_bytes_in_use() -> int:
    return int(lib().emogi_device_bytes_in_use())


def managed_empty(count: int, dtype) -> np.ndarray:
    """An uninitialised numpy array over managed (UVM) memory from
    emogi_managed_alloc, for load_csr(..., placement="managed", borrow=True).
    The memory is freed once the array and every view of it are gone."""
    import weakref
    dtype = np.dtype(dtype)
    nbytes = max(1, int(count)) * dtype.itemsize
    p = ctypes.c_void_p()
    _check(lib().emogi_managed_alloc(nbytes, ctypes.byref(p)))
    buf = (ctypes.c_uint8 * nbytes).from_address(p.value)
    weakref.finalize(buf, lib().emogi_managed_free, ctypes.c_void_p(p.value))
    return np.frombuffer(buf, dtype=np.uint8).view(dtype)[:int(count)]


def test_fail_device_alloc_after(k: int):
    lib().emogi_test_fail_device_alloc_after(int(k))


def _host_array(a, dtype, name):
    if a is None:
        return None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr


class Graph:
    """A loaded CSR graph (owns the C handle; call free() or use `with`)."""

    def __init__(self, handle, n, m, placement, keepalive=()):
        self._h = ctypes.c_void_p(handle)
        self.n = n
        self.m = m
        self.placement = placement
        self._keepalive = keepalive  # borrowed host arrays stay alive with the handle

    @property
    def handle(self):
        if not self._h:
            raise EmogiError(E_ARG, "graph already freed")
        return self._h

    def free(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p(None)
            _check(lib().emogi_free_graph(h))
            self._keepalive = ()

    def share(self):
        """emogi_graph_share: another handle on the same arrays with its own buffers."""
        h = ctypes.c_void_p()
        _check(lib().emogi_graph_share(self.handle, ctypes.byref(h)))
        return Graph(h.value, self.n, self.m, self.placement, (self,))

    def workspace_bytes(self) -> int:
        return int(lib().emogi_graph_workspace_bytes(self.handle))

    @property
    def store_bound(self) -> int:
        """Lists of 1..store_bound entries are read from the short-list store in GPU memory (0: no store)."""
        return int(lib().emogi_graph_store_bound(self.handle))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            if self._h:
                lib().emogi_free_graph(self._h)
        except Exception:
            pass


def _load(entry, id_dtype, n, m, row_offsets, col_idx, weights, placement, flags, undirected, borrow, heads):
    place = PLACEMENTS[placement] if isinstance(placement, str) else int(placement)
    f = int(flags)
    if not heads:
        f |= LOAD_NO_HEADS
    if undirected:
        f |= LOAD_UNDIRECTED
    if borrow:
        f |= LOAD_BORROW
    off = _host_array(row_offsets, np.uint64, "row_offsets")
    col = _host_array(col_idx, id_dtype, "col_idx")
    w = _host_array(weights, np.uint32, "weights")
    h = ctypes.c_void_p()
    st = getattr(lib(), entry)(int(n), int(m), off.ctypes.data,
                               col.ctypes.data if col is not None else None,
                               w.ctypes.data if w is not None else None,
                               place, f, ctypes.byref(h))
    _check(st)
    keep = (col, w) if (f & LOAD_BORROW) else ()
    return Graph(h.value, int(n), int(m), place, keep)


def load_csr(n, m, row_offsets, col_idx, weights=None, placement="host", flags=0,
             undirected: Optional[bool] = None, borrow: bool = False, heads: bool = True) -> Graph:
    """emogi_load_csr: copy (or, with borrow, pin in place) a CSR graph with uint64 ids."""
    return _load("emogi_load_csr", np.uint64, n, m, row_offsets, col_idx, weights, placement, flags,
                 undirected, borrow, heads)


def load_csr32(n, m, row_offsets, col_idx, weights=None, placement="host", flags=0,
               undirected: Optional[bool] = None, borrow: bool = False, heads: bool = True) -> Graph:
    """emogi_load_csr32: as load_csr, with a 4-byte (uint32) edge list."""
    return _load("emogi_load_csr32", np.uint32, n, m, row_offsets, col_idx, weights, placement, flags,
                 undirected, borrow, heads)


def load_graph(g, placement="host", borrow=False, with_weights=True, heads=True, ids32=False) -> Graph:
    """Load a graphgen.Graph-like object (n, offsets, cols, weights, undirected);
    ids32 loads its edge list as uint32 ids (emogi_load_csr32)."""
    w = g.weights if with_weights else None
    fn = load_csr32 if ids32 else load_csr
    cols = g.cols.astype(np.uint32) if ids32 else g.cols
    return fn(g.n, g.m, g.offsets, cols, w, placement=placement,
              undirected=bool(getattr(g, "undirected", False)), borrow=borrow, heads=heads)


def _opts(access=None, granularity=0, chunk_lines=0, timeout_ns=0, stream=None, out_on_device=False,
          time_kernels=False, delta=0, top_down_only=False, cc_full_pass=False, host_loop=False, beamer=False,
          ordered_frontier=False):
    o = Opts()
    o.struct_size = ctypes.sizeof(Opts)
    o.access = ACCESS[access] if isinstance(access, str) else int(access or 0)
    o.granularity = int(granularity)
    o.chunk_lines = int(chunk_lines)
    o.timeout_ns = int(timeout_ns)
    if stream is not None:
        o.cuda_stream = int(getattr(stream, "cuda_stream", stream))
    o.out_on_device = 1 if out_on_device else 0
    o.flags = (OPT_TIME_KERNELS if time_kernels else 0) | (OPT_TOP_DOWN_ONLY if top_down_only else 0) | \
        (OPT_CC_FULL_PASS if cc_full_pass else 0) | (OPT_HOST_LOOP if host_loop else 0) | \
        (OPT_BEAMER if beamer else 0) | (OPT_ORDERED_FRONTIER if ordered_frontier else 0)
    o.delta = int(delta)
    return o


def _out_buffer(n, out):
    """Returns (pointer, result object, on_device)."""
    if out is None:
        arr = np.empty(max(n, 1), dtype=np.uint32)
        return arr.ctypes.data, arr[:n], False
    if hasattr(out, "data_ptr"):  # torch tensor
        if out.numel() < n or out.element_size() != 4 or not out.is_contiguous():
            raise EmogiError(E_ARG, "output tensor must be contiguous, 4-byte and hold n entries")
        return out.data_ptr(), out, bool(out.is_cuda)
    arr = out
    if arr.dtype != np.uint32 or arr.size < n or not arr.flags.c_contiguous:
        raise EmogiError(E_ARG, "output array must be contiguous uint32 with n entries")
    return arr.ctypes.data, arr, False


def _run(fn, g: Graph, args, out, kw):
    ptr, res, on_dev = _out_buffer(g.n, out)
    o = _opts(out_on_device=on_dev, **kw)
    s = Stats()
    _check(fn(g.handle, *args, ptr, ctypes.byref(o), ctypes.byref(s)))
    return res, s.as_dict()


def bfs(g: Graph, src: int, out=None, **kw):
    """emogi_bfs -> (level array, stats dict)."""
    return _run(lib().emogi_bfs, g, (int(src),), out, kw)


def sssp(g: Graph, src: int, out=None, **kw):
    """emogi_sssp -> (dist array, stats dict)."""
    return _run(lib().emogi_sssp, g, (int(src),), out, kw)


def cc(g: Graph, out=None, **kw):
    """emogi_cc -> (label array, stats dict)."""
    return _run(lib().emogi_cc, g, (), out, kw)


def pagerank(g: Graph, damping=0.85, tol=1e-10, max_iters=100, out=None, **kw):
    """emogi_pagerank -> (float64 ranks, stats dict); `out` may be a float64
    numpy array or a CUDA float64 tensor of n entries."""
    if out is None:
        arr = np.empty(max(g.n, 1), dtype=np.float64)
        ptr, res, on_dev = arr.ctypes.data, arr[:g.n], False
    elif hasattr(out, "data_ptr"):
        if out.numel() < g.n or out.element_size() != 8 or not out.is_contiguous():
            raise EmogiError(E_ARG, "output tensor must be contiguous float64 with n entries")
        ptr, res, on_dev = out.data_ptr(), out, bool(out.is_cuda)
    else:
        if out.dtype != np.float64 or out.size < g.n or not out.flags.c_contiguous:
            raise EmogiError(E_ARG, "output array must be contiguous float64 with n entries")
        ptr, res, on_dev = out.ctypes.data, out, False
    o = _opts(out_on_device=on_dev, **kw)
    s = Stats()
    _check(lib().emogi_pagerank(g.handle, float(damping), float(tol), int(max_iters), ptr, ctypes.byref(o),
                                ctypes.byref(s)))
    return res, s.as_dict()


def msbfs(g: Graph, sources, out=None, **kw):
    """emogi_msbfs -> (levels of shape (k, n), stats dict); row b is the BFS from sources[b]."""
    srcs = np.ascontiguousarray(np.asarray(sources, dtype=np.uint64).ravel())
    k = int(srcs.size)
    if out is None:
        arr = np.empty((k, max(g.n, 1)), dtype=np.uint32)
        ptr, res, on_dev = arr.ctypes.data, arr[:, :g.n], False
    elif hasattr(out, "data_ptr"):
        if out.numel() < k * g.n or out.element_size() != 4 or not out.is_contiguous():
            raise EmogiError(E_ARG, "output tensor must be contiguous, 4-byte and hold k * n entries")
        ptr, res, on_dev = out.data_ptr(), out, bool(out.is_cuda)
    else:
        if out.dtype != np.uint32 or out.size < k * g.n or not out.flags.c_contiguous:
            raise EmogiError(E_ARG, "output array must be contiguous uint32 with k * n entries")
        ptr, res, on_dev = out.ctypes.data, out, False
    o = _opts(out_on_device=on_dev, **kw)
    s = Stats()
    _check(lib().emogi_msbfs(g.handle, srcs.ctypes.data, k, ptr, ctypes.byref(o), ctypes.byref(s)))
    return res, s.as_dict()


PROBE_PATTERNS = {"stream": 0, "random": 1, "regions": 2}


def probe_host_reads(arr: np.ndarray, pattern="stream", block_bytes=0, blocks=0, nbytes=None, stream=None) -> float:
    """Milliseconds of one zero-copy read kernel over the pinned host array
    `arr` (its first `nbytes` bytes): emogi_probe_host_reads."""
    ms = ctypes.c_double()
    nb = arr.nbytes if nbytes is None else int(nbytes)
    st = int(getattr(stream, "cuda_stream", stream)) if stream is not None else None
    _check(lib().emogi_probe_host_reads(arr.ctypes.data, nb, PROBE_PATTERNS[pattern], int(block_bytes), int(blocks),
                                        st, ctypes.byref(ms)))
    return ms.value


def free_graph(g: Graph):
    g.free()


def _dptr(x):
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def bfs_noalloc(n, row_offsets, col_idx, src, level, stream=None):
    """emogi_bfs_noalloc: BFS that allocates nothing, for callers that may not
    call cudaMalloc.  `row_offsets` and `level` are device buffers (torch CUDA
    tensors or raw device addresses) the caller owns; `col_idx` is device
    memory or mapped pinned host memory.  Calls that overlap on the GPU share
    one scratch array and must be serialised."""
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().emogi_bfs_noalloc(int(n), _dptr(row_offsets), _dptr(col_idx), int(src), _dptr(level), s))
    return level


class Batch:
    """A set of loaded graphs traversed together (emogi_batch_*)."""

    def __init__(self, graphs):
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        h = ctypes.c_void_p()
        _check(lib().emogi_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.graphs), ctypes.byref(h)))
        self._h = h
        self.total = int(lib().emogi_batch_total_vertices(h))
        self.offsets = [int(lib().emogi_batch_offset(h, i)) for i in range(len(self.graphs))]

    def _srcs(self, sources):
        s = np.ascontiguousarray(np.asarray(sources, dtype=np.uint64).ravel())
        if s.size != len(self.graphs):
            raise EmogiError(E_ARG, "one source per graph")
        return s

    def bfs(self, sources, out=None, **kw):
        """emogi_batch_bfs -> (list of per-graph level arrays, stats dict)."""
        s = self._srcs(sources)
        if out is None:
            buf = np.empty(max(self.total, 1), dtype=np.uint32)
            ptr, on_dev = buf.ctypes.data, False
        else:
            buf, ptr, on_dev = out, out.data_ptr(), bool(out.is_cuda)
        o = _opts(out_on_device=on_dev, **kw)
        st = Stats()
        _check(lib().emogi_batch_bfs(self._h, s.ctypes.data, ptr, ctypes.byref(o), ctypes.byref(st)))
        views = [buf[o0:o0 + g.n] for o0, g in zip(self.offsets, self.graphs)]
        return views, st.as_dict()

    def autotune(self, sources):
        """emogi_batch_autotune -> (granularity, claim, ms)."""
        s = self._srcs(sources)
        g, c, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
        _check(lib().emogi_batch_autotune(self._h, s.ctypes.data, ctypes.byref(g), ctypes.byref(c),
                                          ctypes.byref(ms)))
        return int(g.value), int(c.value), float(ms.value)

    def free(self):
        if self._h:
            lib().emogi_batch_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def bfs_batch(graphs, sources, **kw):
    """emogi_bfs_batch (one-shot) -> (list of per-graph level arrays, stats dict)."""
    graphs = list(graphs)
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    s = np.ascontiguousarray(np.asarray(sources, dtype=np.uint64).ravel())
    total = sum(g.n for g in graphs)
    buf = np.empty(max(total, 1), dtype=np.uint32)
    o = _opts(**kw)
    st = Stats()
    _check(lib().emogi_bfs_batch(ctypes.cast(arr, ctypes.c_void_p), s.ctypes.data, buf.ctypes.data, len(graphs),
                                 ctypes.byref(o), ctypes.byref(st)))
    out, off = [], 0
    for g in graphs:
        out.append(buf[off:off + g.n])
        off += g.n
    return out, st.as_dict()


QUERY_BFS, QUERY_SSSP = 0, 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_slots", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class QueryResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_uint32), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("edges_reached", ctypes.c_uint64), ("edges_scanned", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """emogi_server_*: continuous-batching query server over loaded graphs."""

    def __init__(self, max_slots=4, device_budget=0, max_batch=0):
        cfg = ServerConfig(ctypes.sizeof(ServerConfig), int(max_slots), int(device_budget), int(max_batch), 0)
        h = ctypes.c_void_p()
        _check(lib().emogi_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, graph: Graph, kind, src, out=None) -> int:
        """Queue a query; `out` is a host uint32 array of n entries (or None)."""
        k = {"bfs": QUERY_BFS, "sssp": QUERY_SSSP}.get(kind, kind)
        ptr = None
        if out is not None:
            if out.dtype != np.uint32 or out.size < graph.n or not out.flags.c_contiguous:
                raise EmogiError(E_ARG, "output array must be contiguous uint32 with n entries")
            ptr = out.ctypes.data
        t = ctypes.c_uint64()
        _check(lib().emogi_server_submit(self._h, graph.handle, int(k), int(src), ptr, ctypes.byref(t)))
        self._keep[t.value] = out
        return int(t.value)

    def wait(self, ticket, timeout_ns=0):
        r = QueryResult()
        st = lib().emogi_server_wait(self._h, int(ticket), int(timeout_ns), ctypes.byref(r))
        if st != E_TIMEOUT:
            self._keep.pop(int(ticket), None)
        _check(st)
        return r.as_dict()

    def drain(self):
        _check(lib().emogi_server_drain(self._h))

    def device_bytes(self):
        return int(lib().emogi_server_device_bytes(self._h))

    def close(self):
        if self._h:
            lib().emogi_server_destroy(self._h)
            self._h = ctypes.c_void_p(None)
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
