"""The C ABI library without a GPU: it loads, exports every symbol that
include/*.h declares, and rejects bad input on the host before any CUDA call."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi
    emogi.lib()
    return emogi


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"\b(emogi_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(E):
    import ctypes
    names = declared_functions()
    assert "emogi_load_csr" in names and "emogi_bfs" in names and len(names) >= 14
    L = ctypes.CDLL(E.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding covers every declared entry point with the same names
    assert set(names) <= set(E.exported_names())


def test_status_strings(E):
    assert E.status_string(E.OK) == "EMOGI_OK"
    assert E.status_string(E.E_OVERFLOW) == "EMOGI_E_OVERFLOW"
    assert E.version().startswith("emogi-gb300")


def _bad_load(E, *args, **kw):
    with pytest.raises(E.EmogiError) as ei:
        E.load_csr(*args, **kw)
    return ei.value


def test_load_rejects_bad_csr_on_host(E):
    u = np.uint64
    e = _bad_load(E, 3, 2, np.array([0, 1, 3, 2], dtype=u), np.array([1, 0], dtype=u))
    assert e.status == E.E_ARG and "decrease" in str(e)
    e = _bad_load(E, 3, 2, np.array([0, 1, 2, 2], dtype=u), np.array([1, 5], dtype=u))
    assert e.status == E.E_ARG and "col_idx[1]" in str(e)
    e = _bad_load(E, 3, 3, np.array([0, 1, 2, 2], dtype=u), np.array([1, 0, 0], dtype=u))
    assert e.status == E.E_ARG and "row_offsets[n]" in str(e)
    e = _bad_load(E, 3, 2, np.array([1, 1, 2, 2], dtype=u), np.array([1, 0], dtype=u))
    assert e.status == E.E_ARG
    e = _bad_load(E, 2**32 - 1, 0, np.zeros(1, dtype=u), np.zeros(0, dtype=u))
    assert e.status == E.E_ARG and "2^32" in str(e)


def test_load32_rejects_bad_csr_on_host(E):
    u, u32 = np.uint64, np.uint32

    def bad(*args, **kw):
        with pytest.raises(E.EmogiError) as ei:
            E.load_csr32(*args, **kw)
        return ei.value

    e = bad(3, 2, np.array([0, 1, 3, 2], dtype=u), np.array([1, 0], dtype=u32))
    assert e.status == E.E_ARG and "decrease" in str(e)
    e = bad(3, 2, np.array([0, 1, 2, 2], dtype=u), np.array([1, 3], dtype=u32))
    assert e.status == E.E_ARG and "col_idx[1] = 3" in str(e)
    e = bad(2, 2, np.array([0, 1, 2], dtype=u), np.array([1, 0], dtype=u32), placement="device", borrow=True)
    assert e.status == E.E_ARG and "BORROW" in str(e)


def test_load_rejects_bad_flags_and_placement(E):
    u = np.uint64
    off, col = np.array([0, 1, 2], dtype=u), np.array([1, 0], dtype=u)
    assert _bad_load(E, 2, 2, off, col, placement=7).status == E.E_ARG
    assert _bad_load(E, 2, 2, off, col, flags=1 << 9).status == E.E_ARG
    e = _bad_load(E, 2, 2, off, col, placement="device", borrow=True)
    assert e.status == E.E_ARG and "BORROW" in str(e)
    assert "BORROW" in E.last_error()


def test_binding_rejects_bad_outputs_without_gpu(E):
    with pytest.raises(E.EmogiError):
        E._out_buffer(10, np.zeros(5, dtype=np.uint32))
    with pytest.raises(E.EmogiError):
        E._out_buffer(10, np.zeros(10, dtype=np.int64))


def test_budget_accounting_starts_at_zero(E):
    E.set_device_budget(0)
    assert E.device_bytes_in_use() == 0
