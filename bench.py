"""Benchmark: BFS + SSSP + CC over an undirected Kronecker graph of scale 27
(edge factor 32) whose edge and weight arrays sit in pinned host memory and
are read zero-copy, with the device held to a 16 GiB budget.

Workload (the paper's scale, Sec. 5.2 and the 16 GB device of Sec. 5.6):
2^27 vertices, 2^32 Kronecker samples stored in both directions and cleaned
(about 8.6e9 directed uint64 edges = 69 GB, plus 34 GB of uint32 weights in
[1, 255]), generated on huge pages and pinned in place (no copy); offsets,
list heads and vertex state in HBM.  One step = BFS + SSSP from one of 16
seeded sources of the giant component (used in turn) + CC.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload kron27|urand24]

Prints one JSON line.  `value` is GTEPS over the whole step (edges out of
reached vertices for BFS and SSSP, all m edges for CC, divided by the
device-timed step), with the graph resident.  `e2e` repeats the step through
the public API with host output buffers, so every step's D2H result copy (and
the source id sent to the device) sits inside the timed region.  Beside it:
`variants.managed_capped` (the same graph in managed memory with 16 GiB of
HBM left to the library and UVM), an uncapped managed point, and the uniform
2^24 workload with its access-pattern and placement variants (`c2`).
`--impl reference` times the CPU oracle instead (the paper's method has no
public implementation to run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS and % of host-link/HBM peak for BFS/SSSP/CC; batched queries/s at p99"
GEN_SEED, SRC_SEED = 1, 2
N_SOURCES = 16
KRON27 = dict(scale=27, ef=32)
DEVICE_BUDGET = 16 << 30  # the paper's 16 GB GPU (Sec. 5.6 throttles its A100 to 16 GB)
URAND24 = dict(n=1 << 24, degree=32)
SOURCES_FILE = os.path.join(ROOT, "tests", "golden", "kron27_ef32_sources.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kron27", choices=["kron27", "urand24"],
                    help="kron27 = the default line (Kronecker scale 27, edge factor 32, edges and weights "
                         "pinned in place in host memory, 16 GiB device budget); urand24 = uniform 2^24, "
                         "degree 32 (the c2 workload) as the headline")
    ap.add_argument("--graph-cache", default=os.environ.get("EMOGI_GRAPH_CACHE"),
                    help="directory of binary CSR files (graphgen.cached): the scale-27 graph is read from there "
                         "when present, else generated and written there; default: generate, write nothing")
    ap.add_argument("--link-reach", type=int, default=0, metavar="GIB",
                    help="measure zero-copy read rates over a pinned huge-page host array of GIB GiB "
                         "(emogi_probe_host_reads: streaming, random blocks over growing ranges, per-block "
                         "regions), print one JSON line and exit")
    ap.add_argument("--no-variants", action="store_true", help="skip the managed / access-pattern comparisons")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uniform 2^24 block and the multi-source, batched and serving measurements")
    ap.add_argument("--ncu-case", nargs="?", const="traversal", default=None,
                    choices=["traversal", "msbfs", "batch", "pagerank", "kron", "access", "device", "kron27"],
                    help="profiling case, then exit: 'traversal' = one BFS, SSSP and CC on a 2^22-vertex uniform "
                         "graph (1.1 GB edges in pinned host memory); 'kron' = the same on a Kronecker graph of "
                         "scale 23, edge factor 32 (2.2 GB edges in host memory); 'access' = top-down BFS on the "
                         "2^22 uniform graph with the naive, merged and merged+aligned reads; 'msbfs' = one "
                         "64-source pass on a scale-22 Kronecker graph in host memory; 'batch' = one batched BFS "
                         "over 128 uneven graphs in HBM; 'pagerank' = 3 PageRank iterations on the 2^22 uniform "
                         "graph in host memory; 'device' = the 'traversal' calls with the graph in HBM; "
                         "'kron27' = SSSP on the scale-27 bench graph, device-driven then host-driven loop "
                         "(for EMOGI_TRACE=1 per-sweep traces and one-pass launch lists only)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def read_kron27_sources():
    """The stored sources of the scale-27 workload (written by the oracle's
    union-find over the whole graph: tests/golden/make_kron27_sources.py)."""
    info = {}
    if not os.path.exists(SOURCES_FILE):
        return info
    for line in open(SOURCES_FILE):
        if line.startswith("#") or not line.strip():
            continue
        k, _, v = line.strip().partition(" ")
        info[k] = [int(x) for x in v.split()] if k == "sources" else int(v)
    return info


def make_kron27(cache_dir=None):
    """The scale-27 graph on huge pages and its 16 giant-component sources
    (the stored list when it belongs to this graph, else 16 seeded vertices
    of degree >= 2, and the config says so); with `cache_dir`, read from the
    binary CSR cache there (written on first use)."""
    import graphgen as gg
    t0 = time.perf_counter()
    if cache_dir:
        g = gg.cached(cache_dir, "kron", KRON27["scale"], KRON27["ef"], seed=GEN_SEED, weights=True)
    else:
        g = gg.kronecker(KRON27["scale"], KRON27["ef"], seed=GEN_SEED, weights=True)
    gen_s = time.perf_counter() - t0
    info = read_kron27_sources()
    if info.get("n") == g.n and info.get("m") == g.m and len(info.get("sources", [])) == N_SOURCES:
        srcs, how = info["sources"], "16 seeded vertices of the giant component (oracle union-find, stored)"
    else:
        srcs = [int(s) for s in gg.random_sources(g, N_SOURCES, seed=SRC_SEED, min_degree=2)]
        how = "16 seeded vertices of degree >= 2 (no stored giant-component list for this graph)"
    return g, srcs, {"generation_s": round(gen_s, 1), "sources_from": how,
                     "graph_cache": bool(cache_dir)}


def make_urand24(n=URAND24["n"], degree=URAND24["degree"]):
    import graphgen as gg
    g = gg.uniform(n, degree, seed=GEN_SEED, weights=True)
    srcs = gg.random_sources(g, N_SOURCES, seed=SRC_SEED)
    return g, [int(s) for s in srcs]


def link_probe(E, cols, stream):
    """Zero-copy read rates (GB/s) of this box over the borrowed edge list:
    a streaming pass, 512-byte and 4 KiB blocks at random over the first GiB
    and over the whole array, and 512-byte blocks spaced evenly with each
    thread block walking its own region.  Random reads over a range beyond
    what the GPU's address translations cover run far below the link's peak;
    the same reads walked in address order do not."""
    nb = cols.nbytes
    one = min(nb, 1 << 30)
    cases = {"stream_all": ("stream", 0, 0, nb), "random512_1GiB": ("random", 512, 1 << 21, one),
             "random512_all": ("random", 512, 1 << 21, nb), "random4k_all": ("random", 4096, 1 << 18, nb),
             "regions512_all": ("regions", 512, nb // 32768, nb)}
    out = {}
    for name, (pat, bb, blocks, rng) in cases.items():
        ms = min(E.probe_host_reads(cols, pat, bb, blocks, nbytes=rng, stream=stream) for _ in range(2))
        moved = rng // 16 * 16 if pat == "stream" else bb * blocks
        out[name] = round(moved / ms / 1e6, 1)
    out["unit"] = "GB/s"
    return out


def workload_config(workload, m):
    """The `config` of the bench line, the same for both arms (m = the graph's
    directed edge count)."""
    if workload == "kron27":
        return {"workload": "Kronecker scale 27, edge factor 32 (initiator 0.57/0.19/0.19/0.05, ids relabelled, "
                            "cleaned, symmetric): BFS+SSSP+CC, uint64 edges + uint32 weights pinned in place in "
                            "host memory (zero-copy), vertex state in HBM, 16 GiB device budget",
                "n": 1 << KRON27["scale"], "m": m, "edge_bytes": m * 8 if m else None,
                "weight_bytes": m * 4 if m else None, "sources": N_SOURCES,
                "placement": "host (borrowed, huge pages)", "device_budget_bytes": DEVICE_BUDGET,
                "access": "merged_aligned", "step": "BFS + SSSP from one source, then CC",
                "l2": "inputs larger than L2 (69 GB edge list in host memory); no flush"}
    return {"workload": f"uniform-random n=2^24 avg-degree 32: BFS+SSSP+CC (the SSSP + CC workload with BFS "
                        "added), edges+weights in pinned host memory (zero-copy), vertex state in HBM",
            "n": URAND24["n"], "m": m, "edge_bytes": m * 8 if m else None, "weight_bytes": m * 4 if m else None,
            "sources": N_SOURCES, "placement": "host", "access": "merged_aligned",
            "step": "BFS + SSSP from one source, then CC",
            "l2": "inputs larger than L2 (4.3 GB edge list in host memory); no flush"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except ValueError:
            return {}
    return {}


def pinned_h2d_peak_gbs(torch):
    """Pinned host->device copy bandwidth (1 GiB, best of 5, CUDA events): the
    host-link roofline denominator for zero-copy reads."""
    nbytes = 1 << 30
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = float("inf")
    s = torch.cuda.current_stream()
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        d.copy_(h, non_blocking=True)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del h, d
    return nbytes / (best * 1e-3) / 1e9


# ------------------------------------------------------------------ our arm
def run_step(E, h, src, stream, outs=None, time_kernels=True):
    kw = dict(stream=stream, time_kernels=time_kernels)
    if outs is None:
        lv, sb = E.bfs(h, src, **kw)
        ds, ss = E.sssp(h, src, **kw)
        lb, sc = E.cc(h, **kw)
    else:
        lv, sb = E.bfs(h, src, out=outs[0], **kw)
        ds, ss = E.sssp(h, src, out=outs[1], **kw)
        lb, sc = E.cc(h, out=outs[2], **kw)
    return (sb, ss, sc)


def step_teps_edges(stats):
    sb, ss, sc = stats
    return sb["edges_reached"] + ss["edges_reached"] + sc["edges_reached"]


def link_bytes(st):
    """Algorithmic bytes a call read from the edge list (and weights) in host
    memory: 8 B per id (4 B with 4-byte ids) and 4 B per weight of the list
    entries read there; entries of lists served from the short-list store in
    GPU memory are not counted."""
    return st["edge_bytes"] + st["weight_bytes"]


def step_alg_bytes(stats):
    """Algorithmic link bytes of one step's expansion launches (BFS, SSSP, CC)."""
    return sum(link_bytes(s) for s in stats)


# Host-link read bytes per algorithmic byte of the SSSP sweeps, from ncu's
# sysmem read-sector counts of the same kernels on a smaller graph of the same
# family (uniform: 2^22 vertices, profiles/link_traffic_per_kernel_urand22_host.md;
# Kronecker: scale 23, edge factor 32, profiles/link_traffic_sssp_kron23_host.md).
# The 32-byte sector waste of lists that do not start on a sector grows with
# the entries read, so the per-byte factor scales to the full graph; on the
# Kronecker graph most entries sit in long lists and the waste is about 1 %.
# Both were counted on earlier versions of the SSSP kernels (the library at
# c4db83c); the kernels have changed since (per-block queue slices, ordered
# runs, a per-graph store bound), so the bench line reports no `traffic` and
# gives the factor only as an estimate until the counters are taken again.
LINK_BYTES_PER_ALG_BYTE = {"urand": {"sssp": 1.135, "current": False},
                           "kron": {"sssp": 1.011, "current": False}}


def combine_over_ranks(ms, units, world, device="cuda"):
    """Across replicas: the timed region lasts as long as the slowest rank's,
    and the work is every rank's (each rank runs its own copy of the step on
    its own GPU; there is no data-path collective)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_loop(torch, E, h, srcs, stream, steps, warmup, outs):
    for i in range(warmup):
        run_step(E, h, srcs[i % len(srcs)], stream, outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    e0.record(stream)
    t0 = time.perf_counter()
    for i in range(steps):
        per.append(run_step(E, h, srcs[(warmup + i) % len(srcs)], stream, outs))
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return e0.elapsed_time(e1), wall, per


VARIANT_STEPS = 4  # sources each comparison variant is timed on (after one untimed step)


def per_algorithm(per):
    out = {}
    for i, nm in enumerate(("bfs", "sssp", "cc")):
        e = sum(p[i]["edges_reached"] for p in per)
        t = sum(p[i]["ms"] for p in per)
        out[nm] = {"gteps": round(e / (t * 1e-3) / 1e9, 3), "ms_mean": round(t / len(per), 3),
                   "iterations_mean": round(sum(p[i]["iterations"] for p in per) / len(per), 2),
                   "edges_scanned_over_reached": round(sum(p[i]["edges_scanned"] for p in per) / max(e, 1), 3),
                   "link_gbs_useful": round(sum(link_bytes(p[i]) for p in per) /
                                            max(sum(p[i]["expand_ms"] for p in per), 1e-9) / 1e6, 1)}
        sc = sum(p[i]["edges_scanned"] for p in per)
        if sc and nm != "cc":
            ids = sum(p[i]["edge_bytes"] for p in per) / 8  # the bench graphs have uint64 ids
            out[nm]["entries_from_gpu_memory"] = round(1.0 - ids / sc, 4)
    return out


def roofline(per, link_peak, factors, peaks, kernel):
    """Roofline of the dominant kernel, the recorded SSSP loop (one graph
    launch per call: its sweeps, far splits and controller; SSSP is most of
    the step): algorithmic bytes (12 B per list entry read: id + weight) over
    the loop's device time, against the pinned host->device copy peak.  The
    same fraction over every expansion launch of the step (BFS and CC read
    8 B per list entry) is reported beside it."""
    sssp_ms = sum(p[1]["expand_ms"] for p in per)
    sssp_bytes = sum(link_bytes(p[1]) for p in per)
    achieved = sssp_bytes / (sssp_ms * 1e-3) / 1e9
    expand_ms = sum(s["expand_ms"] for p in per for s in p)
    alg_bytes = sum(step_alg_bytes(p) for p in per)
    r = {"bound": "host_link", "kernel": kernel, "achieved": round(achieved, 2), "peak": round(link_peak, 2),
         "unit": "GB/s", "frac": round(achieved / link_peak, 4),
         "peak_source": "pinned host->device cudaMemcpy, 1 GiB, best of 6, measured in this run",
         "algorithmic_bytes_per_launch": int(sssp_bytes / len(per)),
         "unit_bytes": "12 B per SSSP list entry read from host memory (8 B id + 4 B weight); entries of lists "
                       "served by the short-list store in GPU memory are not counted",
         "launch_ms": round(sssp_ms / len(per), 3),
         "step_expansion": {"algorithmic_bytes": int(alg_bytes / len(per)), "ms": round(expand_ms / len(per), 3),
                            "frac": round(alg_bytes / (expand_ms * 1e-3) / 1e9 / link_peak, 4),
                            "note": "every expansion launch of the step: 8 B per BFS / CC list entry, 12 B per "
                                    "SSSP entry"},
         "hbm_peak_measured_gbs": peaks.get("hbm_gbs")}
    if factors and factors.get("current"):
        link = sum(factors["sssp"] * link_bytes(p[1]) for p in per)
        r["traffic"] = int(link / len(per))
        r["traffic_note"] = ("host-link read bytes per SSSP call: ncu sysmem read sectors x 32 per list entry on a "
                             f"smaller graph of the same family ({factors['sssp']} per algorithmic byte), scaled "
                             "by this run's entries")
        r["link_frac"] = round(link / (sssp_ms * 1e-3) / 1e9 / link_peak, 4)
    elif factors:
        link = sum(factors["sssp"] * link_bytes(p[1]) for p in per)
        r["traffic"] = None
        r["traffic_note"] = ("no ncu sector count of the current SSSP kernels: the last one, on an earlier version "
                             f"of them and a smaller graph of the same family, gave {factors['sssp']} link bytes "
                             "per algorithmic byte")
        r["link_frac_estimate"] = round(link / (sssp_ms * 1e-3) / 1e9 / link_peak, 4)
    else:
        r["traffic"] = None
        r["traffic_note"] = "no sysmem sector count of the current kernels on this graph family yet"
    return r


KERNEL_NOTE = ("the recorded SSSP loop, timed as one graph launch per call: k_sssp_loop_sweep (merged + aligned "
               "list reads), k_sssp_loop_lists (split lists), k_sssp_loop_compact, k_sssp_loop_far, "
               "k_sssp_loop_control")


def headline(torch, E, h, g, srcs, stream, args, world, barrier):
    """The timed step loop (value) and the same step through the public API
    with pinned host outputs (e2e)."""
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
    barrier()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms, wall, per = time_loop(torch, E, h, srcs, stream, args.steps, args.warmup, outs)
    barrier()
    ms, teps_edges = combine_over_ranks(ms, sum(step_teps_edges(p) for p in per), world)
    del outs
    e2e_steps = max(2, args.steps // 4)
    host_outs = [torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32) for _ in range(3)]
    barrier()
    ms_e2e, _, per_e2e = time_loop(torch, E, h, srcs, stream, e2e_steps, 1, host_outs)
    barrier()
    ms_e2e, e2e_edges = combine_over_ranks(ms_e2e, sum(step_teps_edges(p) for p in per_e2e), world)
    del host_outs
    return {"ms": ms, "wall": wall, "per": per, "value": teps_edges / (ms * 1e-3) / 1e9, "clocks": clk.summary(),
            "e2e": {"value": round(e2e_edges / (ms_e2e * 1e-3) / 1e9, 4), "unit": "GTEPS", "steps": e2e_steps,
                    "h2d_bytes_per_step": 2 * 8, "d2h_bytes_per_step": 3 * 4 * g.n,
                    "note": "public API with pinned host output arrays: each call copies its n-entry result to "
                            "the host inside the timed region"}}


def variant_steps(E, hv, srcs, stream, outs, okw, sssp_timeout_ns=0):
    """One untimed step, then one timed step per source; returns the summary."""
    def one(src):
        sb = E.bfs(hv, src, stream=stream, out=outs[0], **okw)[1]
        ss = E.sssp(hv, src, stream=stream, out=outs[1], timeout_ns=sssp_timeout_ns, **okw)[1]
        sc = E.cc(hv, stream=stream, out=outs[2], **okw)[1]
        return (sb, ss, sc)

    t0 = time.perf_counter()
    one(srcs[0])
    cold_s = time.perf_counter() - t0
    sts = [one(x) for x in srcs]
    tot_ms = sum(s["ms"] for st in sts for s in st)
    k = len(sts)
    return {"gteps": round(sum(step_teps_edges(st) for st in sts) / (tot_ms * 1e-3) / 1e9, 4),
            "ms_per_step": round(tot_ms / k, 3), "first_step_s": round(cold_s, 3), "steps": k,
            "bfs_ms": round(sum(st[0]["ms"] for st in sts) / k, 3),
            "sssp_ms": round(sum(st[1]["ms"] for st in sts) / k, 3),
            "cc_ms": round(sum(st[2]["ms"] for st in sts) / k, 3)}


def to_managed(E, gg, a, threads=8):
    """A managed copy of a large host array, made piece by piece; each piece
    of the host array is returned to the OS once copied, so the two copies
    never coexist (the host holds one copy of a 100 GB graph, not two)."""
    from concurrent.futures import ThreadPoolExecutor
    mo = E.managed_empty(a.size, a.dtype)
    piece = (256 << 20) // a.dtype.itemsize
    group = piece * threads

    def cp(i):
        mo[i:i + piece] = a[i:i + piece]

    with ThreadPoolExecutor(threads) as ex:
        for base in range(0, a.size, group):
            list(ex.map(cp, range(base, min(base + group, a.size), piece)))
            gg.release_host_range(a, base, base + group)
    return mo


MANAGED_SSSP_BOUND_S = 60  # time bound on one capped-UVM SSSP (the zero-copy SSSP takes under 2 s)


def managed_step(E, hm, src, stream, outs, sssp_bound_s):
    """BFS, SSSP (bounded in time) and CC from managed memory; times from the
    library's CUDA events, plus the wall time of the whole step."""
    r = {}
    t0 = time.perf_counter()
    r["bfs_ms"] = round(E.bfs(hm, src, stream=stream, out=outs[0], time_kernels=True)[1]["ms"], 2)
    t1 = time.perf_counter()
    try:
        ss = E.sssp(hm, src, stream=stream, out=outs[1], time_kernels=True, timeout_ns=int(sssp_bound_s * 1e9))[1]
        r["sssp_ms"] = round(ss["ms"], 2)
        r["sssp_rounds"] = ss["iterations"]
    except E.EmogiError as ex:
        if ex.status != E.E_TIMEOUT:
            raise
        r["sssp_ms"] = None
        r["sssp_unfinished"] = f"stopped at its {sssp_bound_s} s time bound: {str(ex)[:120]}"
        r["sssp_wall_s"] = round(time.perf_counter() - t1, 1)
    r["cc_ms"] = round(E.cc(hm, stream=stream, out=outs[2], time_kernels=True)[1]["ms"], 2)
    r["step_wall_s"] = round(time.perf_counter() - t0, 2)
    return r


def managed_arm(E, torch, g, srcs, stream):
    """The UVM baseline (Sec. 5.1.2 (a): cudaMallocManaged + ReadMostly) on the
    same graph, first with the device held to 16 GiB (a device allocation is
    held aside so that the library's buffers, the outputs and UVM's resident
    pages share 16 GiB, as on the paper's 16 GB GPU), then uncapped (the whole
    graph then fits in HBM and migrates once).  Consumes g's host arrays (they
    move into managed memory)."""
    import graphgen as gg
    res = {}
    t0 = time.perf_counter()
    mcols = to_managed(E, gg, g.cols)
    mw = to_managed(E, gg, g.weights)
    g.cols = g.weights = None  # the host copy is gone
    res["move_to_managed_s"] = round(time.perf_counter() - t0, 1)
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
    try:
        for capped in (True, False):
            hm = E.load_csr(g.n, g.m, g.offsets, mcols, mw, placement="managed", undirected=True, borrow=True)
            balloon = None
            try:
                if capped:
                    E.bfs(hm, srcs[0], out=outs[0], stream=stream)  # the library's buffers, before the cap
                    torch.cuda.synchronize()
                    free, _ = torch.cuda.mem_get_info()
                    mine = E.device_bytes_in_use() + sum(o.numel() * 4 for o in outs)
                    keep = max(0, DEVICE_BUDGET - mine)
                    if free > keep:
                        balloon = torch.empty(free - keep, dtype=torch.uint8, device="cuda")
                    torch.cuda.synchronize()
                    free2, _ = torch.cuda.mem_get_info()
                    res["managed_capped"] = {
                        "cap": {"device_budget_bytes": DEVICE_BUDGET, "library_and_outputs_bytes": mine,
                                "held_aside_bytes": 0 if balloon is None else balloon.numel(),
                                "free_for_uvm_bytes": free2},
                        "step": managed_step(E, hm, srcs[1], stream, outs, MANAGED_SSSP_BOUND_S)}
                else:
                    cold = managed_step(E, hm, srcs[1], stream, outs, 3 * MANAGED_SSSP_BOUND_S)
                    warm = managed_step(E, hm, srcs[2], stream, outs, MANAGED_SSSP_BOUND_S)
                    res["managed_uncapped"] = {"note": "the whole graph fits in HBM: pages migrate on first "
                                                       "touch, then stay", "cold_step": cold, "warm_step": warm}
            finally:
                hm.free()
                del balloon
                torch.cuda.empty_cache()
    finally:
        del outs, mcols, mw
    res["managed_wall_s"] = round(time.perf_counter() - t0, 1)
    return res


def ours(args):
    import graphgen as gg
    import torch

    rank, world, local = dist_env()
    t_start = time.perf_counter()
    # The graph is generated before any CUDA work: its 100 GB of arrays need
    # transparent huge pages (the GPU reads them in place, and with 64 KiB
    # pages it needs far more address translations than it holds).  Measured
    # on GB300: made after the CUDA context and a pinned probe buffer, the
    # same edge list got SSSP 5.7 s instead of 1.65 s.
    if args.workload == "kron27":
        g, srcs, ginfo = make_kron27(args.graph_cache)
        ginfo["huge_pages"] = gg.huge_page_report()
        ginfo["numa"] = gg.numa_report(g.cols, g.weights)
    else:
        g, srcs = make_urand24()
        ginfo = {}
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi as E

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    peaks = measured_peaks()
    if args.workload == "kron27":
        E.set_device_budget(DEVICE_BUDGET)
        t0 = time.perf_counter()
        h = E.load_csr(g.n, g.m, g.offsets, g.cols, g.weights, placement="host", undirected=True, borrow=True)
        ginfo["pin_s"] = round(time.perf_counter() - t0, 1)
        factors = LINK_BYTES_PER_ALG_BYTE["kron"]
    else:
        h = E.load_graph(g, placement="host")
        factors = LINK_BYTES_PER_ALG_BYTE["urand"]
    ginfo["store_bound"] = h.store_bound  # lists of 1..store_bound entries are read from GPU memory
    link_peak = pinned_h2d_peak_gbs(torch)
    if args.workload == "kron27":
        ginfo["link_probe"] = link_probe(E, g.cols, stream)

    hl = headline(torch, E, h, g, srcs, stream, args, world, barrier)
    if args.workload == "kron27":
        # the host memory behind the link is shared with the machine's other
        # GPUs and tenants: a streaming pass right after the timed steps shows
        # whether the link still delivered what the probe saw before them
        nb = min(g.cols.nbytes, 8 << 30)
        ms = min(E.probe_host_reads(g.cols, "stream", nbytes=nb, stream=stream) for _ in range(3))
        ginfo["link_probe"]["stream_8GiB_after_timed_steps"] = round(nb / ms / 1e6, 1)
    per = hl["per"]
    launches = sum(s["kernel_launches"] for p in per for s in p)
    cfg = workload_config(args.workload, g.m)
    result = {
        "metric": METRIC, "value": round(hl["value"], 4), "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(hl["ms"] / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (integer)",
        "data": f"synthetic (seeded {'Kronecker' if args.workload == 'kron27' else 'uniform-random'} graph, graphgen)",
        "config": cfg, "graph": ginfo, "per_algorithm": per_algorithm(per), "e2e": hl["e2e"],
        "gpu_launches": int(launches),
        "roofline": roofline(per, link_peak, factors, peaks, KERNEL_NOTE),
        "clocks": hl["clocks"], "wall_s_timed": round(hl["wall"], 3),
    }
    if args.workload == "kron27":
        result["device_bytes_in_use"] = E.device_bytes_in_use()

    if rank == 0 and not args.no_variants and args.workload == "kron27":
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
        variants = {}
        try:
            variants["aligned_zero_copy_paper_forms"] = variant_steps(
                E, h, srcs[1:3], stream, outs, dict(top_down_only=True, cc_full_pass=True))
        except Exception as ex:  # noqa: BLE001 - report, keep the bench line
            variants["aligned_zero_copy_paper_forms"] = {"error": str(ex)[:200]}
        del outs
        h.free()
        h = None
        try:
            variants.update(managed_arm(E, torch, g, srcs, stream))
        except Exception as ex:  # noqa: BLE001
            variants["managed"] = {"error": str(ex)[:300]}
        result["variants"] = variants
    if h is not None:
        h.free()
    E.set_device_budget(0)
    del g

    c2 = None
    if rank == 0 and not args.no_extras:
        try:
            c2, result["c2"] = block_c2(E, torch, args, link_peak, peaks, stream)
        except Exception as ex:  # noqa: BLE001
            result["c2"] = {"error": str(ex)[:300]}
        for name, fn in (("kron16_bfs", extra_kron16),
                         ("pagerank", (lambda E_, t_: extra_pagerank(E_, t_, c2)) if c2 is not None else None),
                         ("msbfs", extra_msbfs), ("batch", extra_batch), ("serving", extra_serving)):
            if fn is None:
                continue
            try:
                result[name] = fn(E, torch)
            except Exception as ex:  # noqa: BLE001 - report, keep the bench line
                result[name] = {"error": str(ex)[:300]}
    del c2

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.workload)
    result["wall_s_total"] = round(time.perf_counter() - t_start, 1)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def block_c2(E, torch, args, link_peak, peaks, stream):
    """The uniform 2^24, degree-32 workload (SSSP and CC, with BFS added) from
    pinned host memory: its own timed loop and roofline, and the comparison
    variants on the same GPU (naive, merged, the paper's forms, Beamer's rule,
    4-byte ids, managed memory that fits in HBM, all in HBM)."""
    g, srcs = make_urand24()
    res = {"workload": f"uniform n=2^24 degree 32 (m={g.m}), edges + weights in pinned host memory"}
    with E.load_graph(g, placement="host") as h:
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
        steps = 8
        ms, _, per = time_loop(torch, E, h, srcs, stream, steps, 2, outs)
        res.update({"value": round(sum(step_teps_edges(p) for p in per) / (ms * 1e-3) / 1e9, 4), "unit": "GTEPS",
                    "steps": steps, "ms_per_step": round(ms / steps, 3), "per_algorithm": per_algorithm(per),
                    "roofline": roofline(per, link_peak, LINK_BYTES_PER_ALG_BYTE["urand"], peaks, KERNEL_NOTE)})
        if not args.no_variants:
            variants = {}
            for name, kw in (("naive_zero_copy", dict(placement="host", access="naive")),
                             ("merged_zero_copy", dict(placement="host", access="merged")),
                             ("aligned_zero_copy_paper_forms", dict(placement="host", access="merged_aligned",
                                                                    top_down_only=True, cc_full_pass=True)),
                             ("aligned_zero_copy_beamer_rule", dict(placement="host", access="merged_aligned",
                                                                    beamer=True)),
                             ("aligned_zero_copy_ids32", dict(placement="host", access="merged_aligned",
                                                              ids32=True)),
                             ("managed_uvm", dict(placement="managed", access="merged_aligned")),
                             ("device_hbm", dict(placement="device", access="merged_aligned")),
                             ("device_hbm_ids32", dict(placement="device", access="merged_aligned", ids32=True))):
                try:
                    ids32 = kw.get("ids32", False)
                    hv = h if (kw["placement"] == "host" and not ids32) else \
                        E.load_graph(g, placement=kw["placement"], ids32=ids32)
                    okw = {k: v for k, v in kw.items() if k not in ("placement", "ids32")}
                    variants[name] = variant_steps(E, hv, srcs[1:1 + VARIANT_STEPS], stream, outs, okw)
                    if hv is not h:
                        hv.free()
                except Exception as ex:  # noqa: BLE001 - report, keep the bench line
                    variants[name] = {"error": str(ex)[:200]}
            res["variants"] = variants
        del outs
    return g, res


def _time(torch, fn, stream):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3, r


def extra_kron16(E, torch):
    """BFS from the highest-degree vertex of an undirected Kronecker graph
    (scale 16, edge factor 16), from HBM and from pinned host memory: a
    latency-bound case (about 2M edges)."""
    import graphgen as gg
    g = gg.kronecker(16, 16, seed=GEN_SEED)
    src = gg.max_degree_vertex(g)
    st = torch.cuda.Stream()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    res = {"workload": f"Kronecker scale 16 ef 16 (n={g.n}, m={g.m}), source = max-degree vertex {src}"}
    for place in ("device", "host"):
        with E.load_graph(g, placement=place) as h:
            for _ in range(3):
                E.bfs(h, src, out=out, stream=st)
            reps = 20
            ms, _, stats = _time(torch, lambda: [E.bfs(h, src, out=out, stream=st)[1] for _ in range(reps)], st)
            ms /= reps
            res[place] = {"ms": round(ms, 4), "gteps": round(stats[-1]["edges_reached"] / (ms * 1e-3) / 1e9, 3),
                          "levels": stats[-1]["iterations"]}
    return res


def extra_pagerank(E, torch, g):
    """PageRank (20 iterations, damping 0.85, no early stop) on the bench graph
    with its edge list in pinned host memory: the whole uint64 edge list is
    read once per iteration, so the link bound is 8 B x m per iteration."""
    st = torch.cuda.Stream()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    res = {"workload": f"uniform n={g.n} m={g.m}, 20 power iterations, host placement"}
    for ids32 in (False, True):
        with E.load_graph(g, placement="host", with_weights=False, ids32=ids32) as h:
            E.pagerank(h, 0.85, tol=0.0, max_iters=2, out=out, stream=st)
            _, s = E.pagerank(h, 0.85, tol=0.0, max_iters=20, out=out, stream=st, time_kernels=True)
            per_it = s["ms"] / s["iterations"]
            idb = 4 if ids32 else 8
            res["ids32" if ids32 else "ids64"] = {
                "ms_per_iteration": round(per_it, 3), "gteps": round(g.m / (per_it * 1e-3) / 1e9, 2),
                "link_gbs_useful": round(idb * s["edges_scanned"] / (s["expand_ms"] * 1e-3) / 1e9, 1)}
    return res


def extra_msbfs(E, torch):
    """64 BFS sources in one multi-source pass vs 64 single BFS calls on an
    undirected Kronecker graph (scale 24, edge factor 16) in pinned host memory."""
    import graphgen as gg
    g = gg.kronecker(24, 16, seed=GEN_SEED)
    srcs = [int(s) for s in gg.random_sources(g, 64, seed=SRC_SEED)]
    st = torch.cuda.Stream()
    out = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
    one = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with E.load_graph(g, placement="host") as h:
        E.msbfs(h, srcs[:4], out=out, stream=st)  # warm-up
        ms_ms, _, (lv, sm) = _time(torch, lambda: E.msbfs(h, srcs, out=out, stream=st), st)
        E.bfs(h, srcs[0], out=one, stream=st)
        seq = []
        ms_seq, _, _ = _time(torch, lambda: [seq.append(E.bfs(h, s, out=one, stream=st)[1]) for s in srcs], st)
        ms_td, _, _ = _time(torch, lambda: [E.bfs(h, s, out=one, stream=st, top_down_only=True) for s in srcs],
                            st)
    reached = sm["edges_reached"]
    return {"workload": f"Kronecker scale 24 ef 16 (n={g.n}, m={g.m}), 64 seeded sources, host placement",
            "msbfs_ms": round(ms_ms, 2), "msbfs_gteps": round(reached / (ms_ms * 1e-3) / 1e9, 3),
            "msbfs_levels": sm["iterations"], "msbfs_edges_read": sm["edges_scanned"],
            "single_bfs_64_ms": round(ms_seq, 2), "single_bfs_gteps": round(reached / (ms_seq * 1e-3) / 1e9, 3),
            "single_bfs_top_down_64_ms": round(ms_td, 2),
            "speedup_vs_single": round(ms_seq / ms_ms, 3),
            "edges_read_single": int(sum(x["edges_scanned"] for x in seq))}


def extra_batch(E, torch):
    """512 uneven uniform-random graphs (2^10..2^18 vertices log-uniform,
    average degree 4..64) in HBM: one persistent graph-captured batched BFS vs
    512 single BFS calls, after the autotuner picks lanes per vertex and claim."""
    import graphgen as gg
    rng = np.random.default_rng(4)
    gs = []
    for i in range(512):
        n = int(2 ** rng.uniform(10, 18))
        gs.append(gg.uniform(n, int(rng.integers(4, 65)), seed=4000 + i))
    srcs = [gg.max_degree_vertex(g) for g in gs]
    hs = [E.load_graph(g, placement="device") for g in gs]
    st = torch.cuda.Stream()
    try:
        with E.Batch(hs) as b:
            out = torch.empty(b.total, dtype=torch.int32, device="cuda")
            G, claim, tune_ms = b.autotune(srcs)
            b.bfs(srcs, out=out)
            reps = 5
            ms_b, _, stats = _time(torch, lambda: [b.bfs(srcs, out=out)[1] for _ in range(reps)], st)
            ms_b /= reps
            reached = stats[-1]["edges_reached"]
        one = torch.empty(max(g.n for g in gs), dtype=torch.int32, device="cuda")
        for h, s in zip(hs[:8], srcs[:8]):
            E.bfs(h, s, out=one, stream=st)
        ms_s, _, _ = _time(torch, lambda: [E.bfs(h, s, out=one, stream=st) for h, s in zip(hs, srcs)], st)
    finally:
        for h in hs:
            h.free()
    return {"workload": f"512 uniform graphs, sum n={sum(g.n for g in gs)}, sum m={sum(g.m for g in gs)}, "
                        "device placement",
            "autotuned": {"granularity": G, "claim": claim, "ms": round(tune_ms, 3)},
            "batch_ms": round(ms_b, 3), "batch_queries_per_s": round(512 / (ms_b * 1e-3), 1),
            "batch_gteps": round(reached / (ms_b * 1e-3) / 1e9, 3),
            "single_calls_ms": round(ms_s, 3), "single_queries_per_s": round(512 / (ms_s * 1e-3), 1),
            "speedup_vs_single": round(ms_s / ms_b, 3)}


SERVING_LOADS = (1000, 2000, 5000, 10000, 20000, 50000)
SERVING_QUERIES = 2000  # per offered load


def extra_serving(E, torch):
    """Serving: Poisson-arriving BFS (80 %) and SSSP (20 %) queries with seeded
    random sources over a resident set of 8 graphs (Kronecker scales 18, 20,
    22, 24, 26 with edge factor 16 and uniform 2^20, 2^22, 2^24 with degree 16;
    graphs of 2^22 vertices or fewer in HBM, the others borrowed in pinned
    host memory), each query on a graph drawn uniformly, results discarded.
    Per offered load: achieved queries/s, p50/p99 latency (arrival -> result,
    overall and per kind), mean batch, the host-link bytes of the list
    entries read from host-placed graphs per second, and where the slots'
    time went; next to the same kind of queries run one at a time."""
    import graphgen as gg
    specs = [("kron18", lambda: gg.kronecker(18, 16, seed=11, weights=True), "device"),
             ("kron20", lambda: gg.kronecker(20, 16, seed=12, weights=True), "device"),
             ("kron22", lambda: gg.kronecker(22, 16, seed=13, weights=True), "device"),
             ("kron24", lambda: gg.kronecker(24, 16, seed=14, weights=True), "host"),
             ("kron26", lambda: gg.kronecker(26, 16, seed=15, weights=True), "host"),
             ("urand20", lambda: gg.uniform(1 << 20, 16, seed=16, weights=True), "device"),
             ("urand22", lambda: gg.uniform(1 << 22, 16, seed=17, weights=True), "device"),
             ("urand24", lambda: gg.uniform(1 << 24, 16, seed=18, weights=True), "host")]
    t0 = time.perf_counter()
    gs, hs, places = [], [], []
    out = {}
    try:
        for _, mk, place in specs:
            g = mk()
            gs.append(g)
            places.append(place)
            hs.append(E.load_graph(g, placement=place, borrow=(place == "host")))
        out["workload"] = "resident set " + ", ".join(f"{nm} (m={g.m}, {pl})" for (nm, _, pl), g in zip(specs, gs))
        out["setup_s"] = round(time.perf_counter() - t0, 1)
        rng = np.random.default_rng(3)
        degs = [g.degrees() for g in gs]

        def make_queries(count):
            qs = []
            for _ in range(count):
                gi = int(rng.integers(0, len(gs)))
                kind = "bfs" if rng.random() < 0.8 else "sssp"
                src = int(rng.integers(0, gs[gi].n))
                while degs[gi][src] == 0:  # a source with at least one edge
                    src = int(rng.integers(0, gs[gi].n))
                qs.append((gi, kind, src))
            return qs

        def link_bytes(gi, kind, scanned):
            return scanned * (12 if kind == "sssp" else 8) if places[gi] == "host" else 0

        def summarise(qs, lat, runs, scanned, wall, slots=1, batch=None):
            """runs: each query's job time; a job of b queries reports its time on
            each of them, so slot time counts runs / b per query (each job once)."""
            lat = np.asarray(lat)
            kinds = np.array([k for _, k, _ in qs])
            nb = np.asarray(batch, dtype=np.float64) if batch is not None else np.ones(len(qs))
            runs = np.asarray(runs, dtype=np.float64) / nb
            r = {"queries": len(qs), "queries_per_s": round(len(qs) / wall, 1),
                 "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                 "link_gbs": round(sum(link_bytes(gi, k, sc) for (gi, k, _), sc in zip(qs, scanned)) / wall / 1e9, 2)}
            for kind in ("bfs", "sssp"):
                sel = kinds == kind
                if sel.any():
                    r[kind] = {"p50_ms": round(float(np.percentile(lat[sel], 50)), 3),
                               "p99_ms": round(float(np.percentile(lat[sel], 99)), 3),
                               "slot_time_share": round(float(np.sum(runs[sel])) / max(float(np.sum(runs)), 1e-9), 3),
                               "job_ms_mean": round(float(np.sum(runs[sel])) / max(float(np.sum(1.0 / nb[sel])), 1e-9),
                                                    3)}
            r["slot_busy"] = round(float(np.sum(runs)) / 1e3 / (wall * slots), 3)
            by = {}
            for (gi, kind, _), t in zip(qs, runs):
                d = by.setdefault(specs[gi][0], {"bfs": 0.0, "sssp": 0.0})
                d[kind] += t / 1e3
            r["slot_s_by_graph"] = {k: {kk: round(vv, 2) for kk, vv in v.items()} for k, v in by.items()}
            return r

        # one query at a time through the plain calls
        st = torch.cuda.Stream()
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in gs]
        base_q = make_queries(400)
        for gi, kind, src in base_q[:16]:  # warm-up: every graph's buffers and loop graphs
            (E.bfs if kind == "bfs" else E.sssp)(hs[gi], src, out=outs[gi], stream=st)
        lat, runs, scanned = [], [], []
        tb = time.perf_counter()
        for gi, kind, src in base_q:
            t1 = time.perf_counter()
            _, s_ = (E.bfs if kind == "bfs" else E.sssp)(hs[gi], src, out=outs[gi], stream=st)
            lat.append((time.perf_counter() - t1) * 1e3)
            runs.append(lat[-1])
            scanned.append(s_["edges_scanned"])
        out["one_at_a_time"] = summarise(base_q, lat, runs, scanned, time.perf_counter() - tb)
        del outs
        loads = []
        slots = 8
        with E.Server(max_slots=slots) as srv:
            for q in make_queries(32):  # warm-up: every worker's shares
                srv.wait(srv.submit(hs[q[0]], q[1], q[2]))
            for rate in SERVING_LOADS:
                qs = make_queries(SERVING_QUERIES)
                gaps = rng.exponential(1.0 / rate, size=len(qs))
                tickets = []
                tl = time.perf_counter()
                t_next = tl
                for (gi, kind, src), gap in zip(qs, gaps):
                    t_next += gap
                    while time.perf_counter() < t_next:
                        pass
                    tickets.append(srv.submit(hs[gi], kind, src))
                res = [srv.wait(t) for t in tickets]
                wall = time.perf_counter() - tl
                r = summarise(qs, [x["latency_ms"] for x in res], [x["run_ms"] for x in res],
                              [x["edges_scanned"] for x in res], wall, slots, [x["batch_size"] for x in res])
                r["offered_qps"] = rate
                r["mean_batch"] = round(float(np.mean([x["batch_size"] for x in res])), 2)
                r["max_batch"] = int(max(x["batch_size"] for x in res))
                loads.append(r)
        out["loads"] = loads
        out["slots"] = slots
        out["queries_per_load"] = SERVING_QUERIES
    finally:
        for h in hs:
            h.free()
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


# The oracle's bounded sample of the scale-27 workload: the same generator
# and edge factor at scale 23 (1/16 of the vertices and edges), so that one
# single-threaded BFS + union-find pass takes seconds, not minutes.
CPU_SAMPLE = dict(scale=23, ef=32)


def cpu_sample(workload):
    """(graph, sources, description) of the oracle's sample of a workload."""
    import graphgen as gg
    if workload == "kron27":
        g = gg.kronecker(CPU_SAMPLE["scale"], CPU_SAMPLE["ef"], seed=GEN_SEED)
        srcs = [int(s) for s in gg.random_sources(g, N_SOURCES, seed=SRC_SEED, min_degree=2)]
        return g, srcs, (f"Kronecker scale {CPU_SAMPLE['scale']}, edge factor {CPU_SAMPLE['ef']} (n={g.n}, m={g.m}): "
                         "the scale-27 workload's generator at 1/16 of its size")
    g, srcs = make_urand24()
    return g, srcs, f"the uniform 2^24 graph itself (m={g.m})"


def oracle_step(g, src):
    """One oracle step of the bounded sample: BFS from src + union-find CC
    (Dijkstra left out: a single-threaded heap Dijkstra over the sample takes
    minutes)."""
    import oracle
    t0 = time.perf_counter()
    lv = oracle.bfs_g(g, src)
    t1 = time.perf_counter()
    oracle.cc_g(g)
    t2 = time.perf_counter()
    return oracle.reached_edges(g.offsets, lv) + g.m, (t1 - t0, t2 - t1)


def host_cpu():
    """The host's core count and CPU model (lscpu's "Model name", else the
    machine type)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine()}


def cpu_baseline(workload="kron27"):
    """The oracle's BFS and CC, single-threaded, on a bounded sample."""
    g, srcs, desc = cpu_sample(workload)
    edges, (tb, tc) = oracle_step(g, srcs[0])
    tot = tb + tc
    return {"value": round(edges / tot / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"BFS from vertex {srcs[0]} + union-find CC on {desc}; single-threaded C; "
                      f"{tot:.1f} s (bfs {tb:.1f}, cc {tc:.1f})", "host": host_cpu()}


# ------------------------------------------------------------------ reference arm
_REF_GRAPH = None  # set before the worker pool forks; workers share it copy-on-write


def _ref_worker(src):
    edges, ts = oracle_step(_REF_GRAPH, src)
    return edges, sum(ts)


def reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle
    oracle.build_lib()
    global _REF_GRAPH
    g, srcs, desc = cpu_sample(args.workload)
    _REF_GRAPH = g
    cores = min(os.cpu_count() or 1, max(1, args.steps), 16)
    # no GPU is touched in this process, so forking is safe
    ctx = mp.get_context("fork")
    with ctx.Pool(cores) as pool:
        pool.map(_ref_worker, [srcs[i % len(srcs)] for i in range(args.warmup)], chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_ref_worker, [srcs[(args.warmup + i) % len(srcs)] for i in range(args.steps)], chunksize=1)
        wall = time.perf_counter() - t0
    edges = sum(r[0] for r in res)
    value = edges / wall / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GTEPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall * 1e3 / args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (integer)",
           "data": "synthetic (seeded graph, graphgen)",
           "config": workload_config(args.workload, read_kron27_sources().get("m") if args.workload == "kron27"
                                     else g.m),
           "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                            "host": host_cpu(),
                            "sample": f"{args.steps} steps, each the oracle's BFS from one seeded vertex + "
                                      f"union-find CC on {desc}; one step per process, {cores} processes "
                                      "in parallel"},
           "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "note": "the paper publishes no implementation; the reference arm is the CPU oracle on a bounded "
                   "sample of the workload"}
    print(json.dumps(out), flush=True)


def ncu_case(args):
    """Small cases for ncu captures: inputs still far larger than L2, a few
    hundred MB to a few GB on the device, a few dozen launches."""
    import torch
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi as E
    import graphgen as gg
    if args.ncu_case == "msbfs":
        g = gg.kronecker(22, 16, seed=GEN_SEED)
        srcs = [int(s) for s in gg.random_sources(g, 64, seed=SRC_SEED)]
        out = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
        with E.load_graph(g, placement="host") as h:
            st = E.msbfs(h, srcs, out=out)[1]
        print(json.dumps({"ncu_case": "msbfs Kronecker scale 22 ef 16, 64 sources, host", "stats": st}))
        return
    if args.ncu_case == "pagerank":
        g, _ = make_urand24(1 << 22, URAND24["degree"])
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        with E.load_graph(g, placement="host", with_weights=False) as h:
            st = E.pagerank(h, 0.85, tol=0.0, max_iters=3, out=out)[1]
        print(json.dumps({"ncu_case": "PageRank, 3 iterations, uniform n=2^22 degree 32, host", "stats": st}))
        return
    if args.ncu_case == "batch":
        rng = np.random.default_rng(4)
        gs = [gg.uniform(int(2 ** rng.uniform(10, 18)), int(rng.integers(4, 65)), seed=4000 + i) for i in range(128)]
        hs = [E.load_graph(g, placement="device") for g in gs]
        with E.Batch(hs) as b:
            st = b.bfs([gg.max_degree_vertex(g) for g in gs])[1]
        for h in hs:
            h.free()
        print(json.dumps({"ncu_case": "batched BFS, 128 uneven uniform graphs, device", "stats": st}))
        return
    if args.ncu_case == "access":
        # the request-size ladder of Sec. 5.3.1: the same top-down BFS with a
        # thread per list (naive), a warp per list (merged) and aligned groups
        g, srcs = make_urand24(1 << 22, URAND24["degree"])
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        res = {}
        with E.load_graph(g, placement="host", with_weights=False) as h:
            for acc in ("naive", "merged", "merged_aligned"):
                res[acc] = E.bfs(h, srcs[0], out=out, access=acc, top_down_only=True)[1]
        print(json.dumps({"ncu_case": "top-down BFS, uniform n=2^22 degree 32, host, three access patterns",
                          **res}))
        return
    if args.ncu_case == "kron27":
        # the headline graph: for per-sweep traces (EMOGI_TRACE=1) and one-pass
        # ncu launch lists only; a 100 GB host edge list is no case for
        # multi-pass captures
        g, srcs, _ = make_kron27(args.graph_cache)
        E.set_device_budget(DEVICE_BUDGET)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        st = torch.cuda.Stream()
        h = E.load_csr(g.n, g.m, g.offsets, g.cols, g.weights, placement="host", undirected=True, borrow=True)
        E.sssp(h, srcs[0], out=out, stream=st)  # first touch of the borrowed arrays
        print("=== sssp", file=sys.stderr, flush=True)
        ss = E.sssp(h, srcs[1], out=out, stream=st)[1]
        print("=== sssp_host_loop", file=sys.stderr, flush=True)
        sh = E.sssp(h, srcs[1], out=out, stream=st, host_loop=True)[1]
        print("=== end", file=sys.stderr, flush=True)
        bound = h.store_bound
        h.free()
        print(json.dumps({"ncu_case": f"Kronecker scale 27 ef 32 (m={g.m}), host placement (borrowed), "
                                      "16 GiB device budget", "store_bound": bound, "sssp": ss, "sssp_host_loop": sh}))
        return
    placement = "host"
    if args.ncu_case == "kron":
        g = gg.kronecker(23, 32, seed=GEN_SEED, weights=True)
        srcs = [int(s) for s in gg.random_sources(g, 2, seed=SRC_SEED, min_degree=2)]
        what = f"Kronecker scale 23 ef 32 (m={g.m}), host placement"
    elif args.ncu_case == "device":
        g, srcs = make_urand24(1 << 22, URAND24["degree"])
        placement = "device"
        what = "uniform n=2^22 degree 32, device placement (edge list and weights in HBM)"
    else:
        g, srcs = make_urand24(1 << 22, URAND24["degree"])
        what = "uniform n=2^22 degree 32, host placement"
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")

    def mark(what):  # separates the calls in a per-sweep trace (EMOGI_TRACE=1)
        print(f"=== {what}", file=sys.stderr, flush=True)

    with E.load_graph(g, placement=placement) as h:
        mark("bfs")
        sb = E.bfs(h, srcs[0], out=out)[1]
        mark("sssp")
        ss = E.sssp(h, srcs[0], out=out)[1]
        mark("sssp_host_loop")
        sh = E.sssp(h, srcs[0], out=out, host_loop=True)[1]  # sweeps as separate launches, for per-kernel counters
        mark("cc")
        sc = E.cc(h, out=out)[1]
    print(json.dumps({"ncu_case": what, "bfs": sb, "sssp": ss, "sssp_host_loop": sh, "cc": sc}))


def link_reach(args):
    """Zero-copy read rates over one pinned host array of args.link_reach GiB
    on transparent huge pages: how far the GPU's address translations reach
    for random reads, and what per-block address order recovers."""
    import torch
    import graphgen as gg
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi as E
    nbytes = args.link_reach << 30
    buf = gg.aligned_empty(nbytes // 8, np.uint64)
    from concurrent.futures import ThreadPoolExecutor
    gib = (1 << 30) // 8
    with ThreadPoolExecutor(16) as ex:  # touch every page before it is pinned
        list(ex.map(lambda i: buf[i * gib:(i + 1) * gib].fill(i), range(args.link_reach)))
    cudart = torch.cuda.cudart()
    torch.cuda.init()
    if int(cudart.cudaHostRegister(buf.ctypes.data, nbytes, 2)) != 0:  # cudaHostRegisterMapped
        raise RuntimeError("cudaHostRegister failed")
    st = torch.cuda.Stream()
    res = {"link_reach": f"pinned host array of {args.link_reach} GiB on huge pages", "unit": "GB/s",
           "huge_pages": gg.huge_page_report()}
    try:
        def rate(pat, bb, blocks, rng, reps=2):
            ms = min(E.probe_host_reads(buf, pat, bb, blocks, nbytes=rng, stream=st) for _ in range(reps))
            moved = rng // 16 * 16 if pat == "stream" else bb * blocks
            return round(moved / ms / 1e6, 1)
        res["stream_1GiB"] = rate("stream", 0, 0, 1 << 30)
        res["stream_all"] = rate("stream", 0, 0, nbytes)
        ranges = [r for r in (1, 2, 4, 8, 16, 24, 32, 48, 64, 96, 128) if r <= args.link_reach]
        for bb, blocks in ((128, 1 << 22), (512, 1 << 21), (4096, 1 << 18)):
            res[f"random{bb}"] = {f"{r}GiB": rate("random", bb, blocks, r << 30) for r in ranges}
        res["regions512"] = {f"every{sp // 1024}KiB": rate("regions", 512, nbytes // sp, nbytes)
                             for sp in (4096, 32768, 262144)}
    finally:
        cudart.cudaHostUnregister(buf.ctypes.data)
    print(json.dumps(res))


def main():
    args = parse()
    if args.link_reach:
        link_reach(args)
        return
    if args.ncu_case:
        ncu_case(args)
    elif args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
