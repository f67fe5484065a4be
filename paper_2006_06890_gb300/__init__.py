"""GB300-native zero-copy graph traversal (EMOGI, arxiv 2006.06890).

The compute path is the CUDA library ``libemogi.so`` (C ABI in
``include/emogi.h``); ``emogi`` is its thin ctypes binding.
"""
from . import emogi  # noqa: F401
from .emogi import (Batch, EmogiError, Graph, LibraryNotBuilt, Server, bfs, bfs_batch, bfs_noalloc,  # noqa: F401
                    cc, load_csr, load_csr32, load_graph, msbfs, pagerank, sssp)

__all__ = ["emogi", "Batch", "EmogiError", "Graph", "LibraryNotBuilt", "Server", "bfs", "bfs_batch",
           "bfs_noalloc", "cc", "load_csr", "load_csr32", "load_graph", "msbfs", "pagerank", "sssp"]
