"""Benchmark: BFS + SSSP + CC over an undirected uniform-random graph whose edge
and weight arrays sit in pinned host memory and are read zero-copy.

Workload: 2^24 vertices, 2^28 uniform samples stored in both directions
(about 5.4e8 directed uint64 edges = 4.3 GB, plus 2.1 GB of uint32 weights in
[1, 255]); vertex state in GPU memory.  One step = BFS + SSSP from the same
seeded source (16 sources, used in turn) + CC.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is GTEPS over the whole step (edges out of
reached vertices for BFS and SSSP, all m edges for CC, divided by the
device-timed step), with the graph resident (edges in pinned host memory,
offsets in HBM).  `e2e` repeats the step through the public API with host
output buffers, so every step's D2H result copy (and the source ids sent to
the device) sit inside the timed region.  `--impl reference` times the CPU
oracle instead (the paper's method has no public implementation to run).
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
SCALE_N = 1 << 24
AVG_DEGREE = 32
GEN_SEED, SRC_SEED = 1, 2
N_SOURCES = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=SCALE_N, help="vertices (power of two)")
    ap.add_argument("--degree", type=int, default=AVG_DEGREE)
    ap.add_argument("--no-variants", action="store_true", help="skip the naive/managed/device comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="urand24", choices=["urand24", "kron27"],
                    help="urand24 = the default bench line; kron27 = BFS, SSSP and CC from 4 seeded sources on an "
                         "undirected Kronecker graph of scale 27, edge factor 32 (about 7e9 edges, 60+ GB edges "
                         "and 30 GB weights) pinned in place in host memory, with a 16 GB device budget")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the multi-source, batched and serving measurements")
    ap.add_argument("--ncu-case", nargs="?", const="traversal", default=None,
                    choices=["traversal", "msbfs", "batch", "pagerank"],
                    help="profiling case, then exit: 'traversal' = one BFS, SSSP and CC on a 2^22-vertex uniform "
                         "graph (1.1 GB edges in pinned host memory); 'msbfs' = one 64-source pass on a scale-22 "
                         "Kronecker graph in host memory; 'batch' = one batched BFS over 128 uneven graphs in HBM; "
                         "'pagerank' = 3 PageRank iterations on the 2^22-vertex uniform graph in host memory")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_graph(n, degree):
    import graphgen as gg
    g = gg.uniform(n, degree, seed=GEN_SEED, weights=True)
    srcs = gg.random_sources(g, N_SOURCES, seed=SRC_SEED)
    return g, [int(s) for s in srcs]


def workload_config(g, n, degree, extra=None):
    cfg = {"workload": f"uniform-random n=2^{n.bit_length() - 1} avg-degree {degree}: BFS+SSSP+CC, "
                       "edges+weights in pinned host memory (zero-copy), vertex state in HBM",
           "n": g.n, "m": g.m, "edge_bytes": g.m * 8, "weight_bytes": g.m * 4,
           "sources": N_SOURCES, "placement": "host", "access": "merged_aligned",
           "l2": "inputs larger than L2 (4.3 GB edge list in host memory); no flush"}
    if extra:
        cfg.update(extra)
    return cfg


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


def step_alg_bytes(stats):
    """Algorithmic link bytes of the expansion launches: 8 B per list entry read
    (BFS, CC) and 12 B per entry (SSSP: id + weight), over the entries the
    launches actually process (direction-optimising BFS and sampled CC read
    fewer entries than the reached edges; SSSP re-expands a few)."""
    sb, ss, sc = stats
    return 8 * sb["edges_scanned"] + 12 * ss["edges_scanned"] + 8 * sc["edges_scanned"]


# Host-link read bytes per algorithmic byte of the expansion kernels, from the
# ncu sysmem read-sector counts of the same kernels on the 2^22-vertex case
# (profiles/link_traffic_per_kernel_urand22_host.md); the 32-byte sector waste
# of lists that do not start on a sector grows with the entries read, so the
# per-entry factor scales to the 2^24 graph.
LINK_BYTES_PER_ALG_BYTE = {"bfs": 1.130, "sssp": 1.135, "cc": 1.0}


def step_link_bytes(stats):
    sb, ss, sc = stats
    return (LINK_BYTES_PER_ALG_BYTE["bfs"] * 8 * sb["edges_scanned"] +
            LINK_BYTES_PER_ALG_BYTE["sssp"] * 12 * ss["edges_scanned"] +
            LINK_BYTES_PER_ALG_BYTE["cc"] * 8 * sc["edges_scanned"])


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


def ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi as E

    g, srcs = make_graph(args.n, args.degree)
    stream = torch.cuda.Stream()
    peaks = measured_peaks()
    link_peak = pinned_h2d_peak_gbs(torch)

    h = E.load_graph(g, placement="host")
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing (value)
    barrier()
    with ClockSampler(local) as clk:
        ms, wall, per = time_loop(torch, E, h, srcs, stream, args.steps, args.warmup, outs)
    barrier()
    ms, teps_edges = combine_over_ranks(ms, sum(step_teps_edges(p) for p in per), world)
    value = teps_edges / (ms * 1e-3) / 1e9
    expand_ms = sum(s["expand_ms"] for p in per for s in p)
    alg_bytes = sum(step_alg_bytes(p) for p in per)
    launches = sum(s["kernel_launches"] for p in per for s in p)
    achieved = alg_bytes / (expand_ms * 1e-3) / 1e9
    per_alg = {}
    for i, nm in enumerate(("bfs", "sssp", "cc")):
        e = sum(p[i]["edges_reached"] for p in per)
        t = sum(p[i]["ms"] for p in per)
        per_alg[nm] = {"gteps": round(e / (t * 1e-3) / 1e9, 3), "ms_mean": round(t / len(per), 3),
                       "iterations_mean": round(sum(p[i]["iterations"] for p in per) / len(per), 2),
                       "edges_scanned_over_reached": round(sum(p[i]["edges_scanned"] for p in per) / max(e, 1), 3)}

    # ---- end to end through the public API with host output buffers: pinned
    # host arrays (as a serving caller keeps them), so each result crosses to
    # the host by DMA; pageable arrays are timed too
    e2e_steps = max(2, args.steps // 2)
    host_outs = [torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32) for _ in range(3)]
    barrier()
    ms_e2e, wall_e2e, per_e2e = time_loop(torch, E, h, srcs, stream, e2e_steps, 1, host_outs)
    barrier()
    ms_e2e, e2e_edges = combine_over_ranks(ms_e2e, sum(step_teps_edges(p) for p in per_e2e), world)
    e2e_value = e2e_edges / (ms_e2e * 1e-3) / 1e9
    barrier()
    ms_pg, _, per_pg = time_loop(torch, E, h, srcs, stream, e2e_steps, 1, None)
    barrier()
    ms_pg, pg_edges = combine_over_ranks(ms_pg, sum(step_teps_edges(p) for p in per_pg), world)
    e2e_pageable = pg_edges / (ms_pg * 1e-3) / 1e9
    del host_outs

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (integer)",
        "data": "synthetic (seeded uniform-random graph, graphgen)",
        "config": workload_config(g, args.n, args.degree, {"parallelism": "replicas" if world > 1 else "single"}),
        "per_algorithm": per_alg,
        "e2e": {"value": round(e2e_value, 4), "unit": "GTEPS", "steps": e2e_steps,
                "h2d_bytes_per_step": 2 * 8, "d2h_bytes_per_step": 3 * 4 * g.n,
                "note": "public API with pinned host output arrays: each call copies its n-entry result to the host",
                "pageable_outputs_value": round(e2e_pageable, 4)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "host_link",
                     "kernel": "expansion launches: k_expand_group / k_expand_split (BFS top-down, CC final), "
                               "k_bfs_bottom_up, k_cc_sample, and the recorded SSSP loop (k_sssp_loop_*)",
                     "achieved": round(achieved, 2), "peak": round(link_peak, 2), "unit": "GB/s",
                     "frac": round(achieved / link_peak, 4),
                     "traffic": int(sum(step_link_bytes(p) for p in per) / len(per)),
                     "traffic_note": "host-link read bytes per step of the expansion kernels: ncu sysmem read "
                                     "sectors x 32 per list entry on the 2^22 case (BFS 1.130, SSSP 1.135 per "
                                     "algorithmic byte), scaled by this run's entries",
                     "link_frac": round(sum(step_link_bytes(p) for p in per) / (expand_ms * 1e-3) / 1e9 / link_peak, 4),
                     "peak_source": "pinned host->device cudaMemcpy, 1 GiB, best of 6, measured in this run",
                     "algorithmic_bytes_per_step": int(alg_bytes / len(per)),
                     "unit_bytes": "8 B per list entry read (BFS, CC), 12 B (SSSP)",
                     "expand_ms_per_step": round(expand_ms / len(per), 3),
                     "hbm_peak_measured_gbs": peaks.get("hbm_gbs")},
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 3),
    }

    # ---- comparison points on the same GPU (one timed step each)
    if not args.no_variants and rank == 0:
        variants = {}
        for name, kw in (("naive_zero_copy", dict(placement="host", access="naive")),
                         ("merged_zero_copy", dict(placement="host", access="merged")),
                         ("aligned_zero_copy_paper_forms", dict(placement="host", access="merged_aligned",
                                                                top_down_only=True, cc_full_pass=True)),
                         ("aligned_zero_copy_beamer_rule", dict(placement="host", access="merged_aligned",
                                                                beamer=True)),
                         ("aligned_zero_copy_ids32", dict(placement="host", access="merged_aligned", ids32=True)),
                         ("managed_uvm", dict(placement="managed", access="merged_aligned")),
                         ("device_hbm", dict(placement="device", access="merged_aligned")),
                         ("device_hbm_ids32", dict(placement="device", access="merged_aligned", ids32=True))):
            try:
                ids32 = kw.get("ids32", False)
                hv = h if (kw["placement"] == "host" and not ids32) else \
                    E.load_graph(g, placement=kw["placement"], ids32=ids32)
                okw = {k: v for k, v in kw.items() if k not in ("placement", "ids32")}

                def one(src):
                    sb = E.bfs(hv, src, stream=stream, out=outs[0], **okw)[1]
                    ss = E.sssp(hv, src, stream=stream, out=outs[1], **okw)[1]
                    sc = E.cc(hv, stream=stream, out=outs[2], **okw)[1]
                    return (sb, ss, sc)

                t0 = time.perf_counter()
                first = one(srcs[0])  # cold for managed: pages migrate
                cold_s = time.perf_counter() - t0
                sts = [one(x) for x in srcs[1:1 + VARIANT_STEPS]]
                tot_ms = sum(s["ms"] for st in sts for s in st)
                edges = sum(step_teps_edges(st) for st in sts)
                k = len(sts)
                variants[name] = {"gteps": round(edges / (tot_ms * 1e-3) / 1e9, 4),
                                  "ms_per_step": round(tot_ms / k, 3), "first_step_s": round(cold_s, 3),
                                  "steps": k,
                                  "bfs_ms": round(sum(st[0]["ms"] for st in sts) / k, 3),
                                  "sssp_ms": round(sum(st[1]["ms"] for st in sts) / k, 3),
                                  "cc_ms": round(sum(st[2]["ms"] for st in sts) / k, 3)}
                del first
                if hv is not h:
                    hv.free()
            except Exception as ex:  # noqa: BLE001 - report, keep the bench line
                variants[name] = {"error": str(ex)[:200]}
        result["variants"] = variants

    # ---- multi-source BFS, batched many-graph BFS and serving (rank 0)
    if rank == 0 and not args.no_extras:
        for name, fn in (("kron16_bfs", extra_kron16), ("pagerank", lambda E_, t_: extra_pagerank(E_, t_, g)),
                         ("msbfs", extra_msbfs), ("batch", extra_batch), ("serving", extra_serving)):
            try:
                result[name] = fn(E, torch)
            except Exception as ex:  # noqa: BLE001 - report, keep the bench line
                result[name] = {"error": str(ex)[:300]}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(g, srcs[0])

    h.free()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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


def extra_serving(E, torch):
    """Poisson-arriving BFS (80 %) and SSSP (20 %) queries with seeded random
    sources over a resident set (Kronecker scales 16, 18, 20 and uniform 2^18,
    2^20, degree 16; the two smallest in HBM, the rest in pinned host memory),
    results discarded; p50/p99 latency and throughput per offered load, next
    to the same queries run one at a time."""
    import graphgen as gg
    specs = [("kron16", lambda: gg.kronecker(16, 16, seed=11, weights=True), "device"),
             ("urand18", lambda: gg.uniform(1 << 18, 16, seed=12, weights=True), "device"),
             ("kron18", lambda: gg.kronecker(18, 16, seed=13, weights=True), "host"),
             ("kron20", lambda: gg.kronecker(20, 16, seed=14, weights=True), "host"),
             ("urand20", lambda: gg.uniform(1 << 20, 16, seed=15, weights=True), "host")]
    gs, hs = [], []
    for _, mk, place in specs:
        g = mk()
        gs.append(g)
        hs.append(E.load_graph(g, placement=place))
    rng = np.random.default_rng(3)
    out = {"workload": "resident set " + ", ".join(f"{nm} ({pl})" for nm, _, pl in specs)}
    try:
        def make_queries(count):
            qs = []
            for _ in range(count):
                gi = int(rng.integers(0, len(gs)))
                qs.append((gi, "bfs" if rng.random() < 0.8 else "sssp", int(rng.integers(0, gs[gi].n))))
            return qs

        # one query at a time through the plain calls
        base_q = make_queries(300)
        st = torch.cuda.Stream()
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in gs]
        t0 = time.perf_counter()
        lat = []
        for gi, kind, src in base_q:
            t1 = time.perf_counter()
            (E.bfs if kind == "bfs" else E.sssp)(hs[gi], src, out=outs[gi], stream=st)
            lat.append((time.perf_counter() - t1) * 1e3)
        wall = time.perf_counter() - t0
        out["one_at_a_time"] = {"queries_per_s": round(len(base_q) / wall, 1),
                                "p50_ms": round(float(np.percentile(lat, 50)), 3),
                                "p99_ms": round(float(np.percentile(lat, 99)), 3)}
        loads = []
        with E.Server(max_slots=8) as srv:
            for rate in (1000, 5000, 20000):
                qs = make_queries(2000)
                gaps = rng.exponential(1.0 / rate, size=len(qs))
                tickets = []
                t0 = time.perf_counter()
                t_next = t0
                for (gi, kind, src), gap in zip(qs, gaps):
                    t_next += gap
                    while time.perf_counter() < t_next:
                        pass
                    tickets.append(srv.submit(hs[gi], kind, src))
                res = [srv.wait(t) for t in tickets]
                wall = time.perf_counter() - t0
                lat = np.array([r["latency_ms"] for r in res])
                loads.append({"offered_qps": rate, "achieved_qps": round(len(qs) / wall, 1),
                              "p50_ms": round(float(np.percentile(lat, 50)), 3),
                              "p99_ms": round(float(np.percentile(lat, 99)), 3),
                              "mean_batch": round(float(np.mean([r["batch_size"] for r in res])), 2),
                              "max_batch": int(max(r["batch_size"] for r in res))})
        out["loads"] = loads
    finally:
        for h in hs:
            h.free()
    return out


def oracle_step(g, src):
    import oracle
    t0 = time.perf_counter()
    lv = oracle.bfs_g(g, src)
    t1 = time.perf_counter()
    ds = oracle.sssp_g(g, src)
    t2 = time.perf_counter()
    oracle.cc_g(g)
    t3 = time.perf_counter()
    edges = oracle.reached_edges(g.offsets, lv) + oracle.reached_edges(g.offsets, ds) + g.m
    return edges, (t1 - t0, t2 - t1, t3 - t2)


def cpu_baseline(g, src):
    """The oracle's BFS and CC on the full graph (Dijkstra alone takes over a
    minute on one core, so it is left out of this bounded sample)."""
    import oracle
    t0 = time.perf_counter()
    lv = oracle.bfs_g(g, src)
    t1 = time.perf_counter()
    oracle.cc_g(g)
    t2 = time.perf_counter()
    edges = oracle.reached_edges(g.offsets, lv) + g.m
    tot = t2 - t0
    return {"value": round(edges / tot / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"BFS from vertex {src} + union-find CC on the full graph, single-threaded C; "
                      f"{tot:.1f} s (bfs {t1 - t0:.1f}, cc {t2 - t1:.1f})"}


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
    g, srcs = make_graph(args.n, args.degree)
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
           "data": "synthetic (seeded uniform-random graph, graphgen)",
           "config": workload_config(g, args.n, args.degree),
           "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} full steps (BFS + Dijkstra + union-find CC), one per "
                                      f"process, {cores} processes in parallel"},
           "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "note": "the paper publishes no implementation; the reference arm is the CPU oracle"}
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
        g, _ = make_graph(1 << 22, args.degree)
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        with E.load_graph(g, placement="host", with_weights=False) as h:
            st = E.pagerank(h, 0.85, tol=0.0, max_iters=3, out=out)[1]
        print(json.dumps({"ncu_case": f"PageRank, 3 iterations, uniform n=2^22 degree {args.degree}, host", "stats": st}))
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
    g, srcs = make_graph(1 << 22, args.degree)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with E.load_graph(g, placement="host") as h:
        sb = E.bfs(h, srcs[0], out=out)[1]
        ss = E.sssp(h, srcs[0], out=out)[1]
        sh = E.sssp(h, srcs[0], out=out, host_loop=True)[1]  # sweeps as separate launches, for per-kernel counters
        sc = E.cc(h, out=out)[1]
    print(json.dumps({"ncu_case": f"uniform n=2^22 degree {args.degree}, host placement",
                      "bfs": sb, "sssp": ss, "sssp_host_loop": sh, "cc": sc}))


def kron27(args):
    """The paper's scale: a graph whose edge list and weights do not fit a
    16 GB device (the budget the paper's A100 runs were held to).  Edges and
    weights are generated in place and pinned where they are (BORROW, no
    copy); vertex state and offsets stay within the 16 GB device budget."""
    import torch
    from paper_2006_06890_gb300 import _build
    _build.build()
    from paper_2006_06890_gb300 import emogi as E
    import graphgen as gg
    t0 = time.perf_counter()
    g = gg.kronecker(27, 32, seed=GEN_SEED, weights=True)
    gen_s = time.perf_counter() - t0
    E.set_device_budget(16 << 30)
    srcs = [int(s) for s in gg.random_sources(g, 4, seed=SRC_SEED, min_degree=2)]
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    res = {"workload": f"Kronecker scale 27 ef 32 (n={g.n}, m={g.m}), edges {g.m * 8 / 1e9:.1f} GB + weights "
                       f"{g.m * 4 / 1e9:.1f} GB pinned in place in host memory, 16 GB device budget",
           "generation_s": round(gen_s, 1)}
    t0 = time.perf_counter()
    h = E.load_csr(g.n, g.m, g.offsets, g.cols, g.weights, placement="host", undirected=True, borrow=True)
    res["load_s"] = round(time.perf_counter() - t0, 1)
    try:
        link_peak = pinned_h2d_peak_gbs(torch)
        runs = {"bfs": [], "sssp": [], "cc": []}
        E.bfs(h, srcs[0], out=out, stream=st)
        for s_ in srcs:
            runs["bfs"].append(E.bfs(h, s_, out=out, stream=st, time_kernels=True)[1])
            runs["sssp"].append(E.sssp(h, s_, out=out, stream=st, time_kernels=True)[1])
        runs["cc"].append(E.cc(h, out=out, stream=st, time_kernels=True)[1])
        runs["cc"].append(E.cc(h, out=out, stream=st, time_kernels=True)[1])
        for nm, lst in runs.items():
            ms = float(np.mean([x["ms"] for x in lst]))
            reached = float(np.mean([x["edges_reached"] for x in lst]))
            scanned = float(np.mean([x["edges_scanned"] for x in lst]))
            ub = 12 if nm == "sssp" else 8
            res[nm] = {"ms_mean": round(ms, 2), "gteps": round(reached / (ms * 1e-3) / 1e9, 3),
                       "edges_scanned_over_reached": round(scanned / max(reached, 1), 4),
                       "link_gbs_useful": round(ub * scanned / (float(np.mean([x["expand_ms"] for x in lst])) * 1e-3)
                                                / 1e9, 1)}
        res["link_peak_gbs"] = round(link_peak, 1)
        res["device_bytes_in_use"] = E.device_bytes_in_use()
        _, tdo = E.bfs(h, srcs[0], out=out, stream=st, top_down_only=True)
        res["bfs_top_down_only_ms"] = round(tdo["ms"], 2)
    finally:
        h.free()
        E.set_device_budget(0)
    print(json.dumps({"workload_extra": "kron27", **res}), flush=True)


def main():
    args = parse()
    if args.workload == "kron27":
        kron27(args)
    elif args.ncu_case:
        ncu_case(args)
    elif args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
