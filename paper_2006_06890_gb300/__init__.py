"""GB300-native zero-copy graph traversal (EMOGI, arxiv 2006.06890).

The compute path is the CUDA library ``libemogi.so`` (C ABI in
``include/emogi.h``); ``emogi`` is its thin ctypes binding.
"""
from . import emogi  # noqa: F401
from .emogi import (EmogiError, Graph, LibraryNotBuilt, bfs, cc, load_csr, load_graph,  # noqa: F401
                    sssp)

__all__ = ["emogi", "EmogiError", "Graph", "LibraryNotBuilt", "bfs", "cc", "load_csr",
           "load_graph", "sssp"]
