"""Host-side arithmetic of the bench line: the roofline object (achieved bytes
over the SSSP loop's time, traffic only from sector counts of the current
kernels) and the zero-copy probe's rates, on synthetic statistics."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(reached, edge_bytes, weight_bytes, expand_ms):
    return {"edges_reached": reached, "edge_bytes": edge_bytes, "weight_bytes": weight_bytes, "expand_ms": expand_ms}


def _per():
    # two steps of (BFS, SSSP, CC)
    step = (_stats(100, 800, 0, 1.0), _stats(100, 8000, 4000, 10.0), _stats(100, 0, 0, 0.5))
    return [step, step]


@pytest.mark.parametrize("current", [True, False, None])
def test_roofline_object(current):
    factors = None if current is None else {"sssp": 1.25, "current": current}
    r = bench.roofline(_per(), 200.0, factors, {"hbm_gbs": 6800.0}, "k")
    # 12,000 algorithmic bytes per 10 ms SSSP call = 1.2 MB/s = 1.2e-3 GB/s
    assert r["achieved"] == pytest.approx(12000 / 10e-3 / 1e9, abs=0.01)
    assert r["frac"] == pytest.approx(r["achieved"] / 200.0, abs=1e-4)
    assert r["algorithmic_bytes_per_launch"] == 12000 and r["launch_ms"] == 10.0
    assert r["step_expansion"]["algorithmic_bytes"] == 12800 and r["step_expansion"]["ms"] == 11.5
    assert r["bound"] == "host_link" and r["unit"] == "GB/s" and r["peak"] == 200.0
    if current:
        assert r["traffic"] == 15000 and "link_frac" in r
    else:
        assert r["traffic"] is None and "link_frac" not in r and r["traffic_note"]
    if current is False:
        assert r["link_frac_estimate"] == pytest.approx(15000 / 10e-3 / 1e9 / 200.0, abs=1e-4)


def test_committed_factors_are_marked_stale():
    """The sector counts behind the factors predate the current SSSP kernels."""
    for fam in ("urand", "kron"):
        assert bench.LINK_BYTES_PER_ALG_BYTE[fam]["current"] is False


class _ProbeStub:
    """emogi.probe_host_reads stand-in: 1 ms per launch, whatever the pattern."""
    def __init__(self):
        self.calls = []

    def probe_host_reads(self, arr, pattern, block_bytes=0, blocks=0, nbytes=None, stream=None):
        self.calls.append((pattern, block_bytes, blocks, nbytes))
        return 1.0


def test_link_probe_rates():
    import numpy as np
    cols = np.zeros((3 << 30) // 8 // 1024, dtype=np.uint64)  # 3 MiB stands in for the edge list
    E = _ProbeStub()
    r = bench.link_probe(E, cols, None)
    nb = cols.nbytes
    assert r["stream_all"] == round(nb // 16 * 16 / 1e-3 / 1e9, 1)
    assert r["random512_all"] == round(512 * (1 << 21) / 1e-3 / 1e9, 1)
    assert r["random4k_all"] == round(4096 * (1 << 18) / 1e-3 / 1e9, 1)
    assert r["regions512_all"] == round(512 * (nb // 32768) / 1e-3 / 1e9, 1)
    assert r["unit"] == "GB/s"
    # every case runs twice, each over at most the array
    assert len(E.calls) == 10 and all(c[3] <= nb for c in E.calls)


def test_host_cpu_reports_cores_and_model():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and isinstance(h["cpu_model"], str) and h["cpu_model"]
