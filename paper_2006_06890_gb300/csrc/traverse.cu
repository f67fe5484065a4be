// Host drivers of BFS, SSSP and CC: the level loop of Sec. 4.2 ("the input
// graph is traversed by a single vertex depth on every kernel execution") run
// until no vertex is active (Algorithm "High-level Graph Traversal Flow").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "kernels.cuh"

namespace emogi {
namespace {

using dev::Sweep;

constexpr int kThreads = 256;

constexpr uint32_t kLargeLines = 32;  // lists above 32 lines (4 KiB) are split

// EMOGI_TRACE=1 in the environment prints one line per sweep to stderr
// (algorithm, sweep, frontier size, event-timed duration).  It forces the
// per-sweep events on, so it is for diagnosis, not for timed runs.
bool trace_enabled() {
    static const bool on = [] {
        const char* e = getenv("EMOGI_TRACE");
        return e && *e && *e != '0';
    }();
    return on;
}

struct Ctx {
    emogi_graph g;
    Opts o;
    cudaStream_t st;
    uint32_t G;
    uint32_t chunk;
    int sms;
    double expand_ms = 0.0;
    uint64_t expand_launches = 0;
    uint64_t kernel_launches = 0;
};

// Lanes per vertex when the caller leaves it open: enough for a mean list in
// about two 16-byte steps per lane.  Measured on GB300 with a uniform degree-32
// graph: with uint64 ids 8 lanes (16 ids per step) beat 16 and 32 for both
// placements, because more lists are in flight per warp, and beat 4 (SSSP
// 43.3 against 44.5 ms); with uint32 ids 4 lanes (16 ids per step) beat 8
// (SSSP 37.5 against 38.8 ms).
uint32_t auto_granularity(double avg_degree, uint32_t id_bytes) {
    uint32_t G = 4;
    if (avg_degree >= 96.0) G = 32;
    else if (avg_degree >= 48.0) G = 16;
    else if (avg_degree >= 12.0) G = 8;
    if (id_bytes == 4 && G > 4) G /= 2;  // a step carries twice the ids
    return G;
}

// SSSP window width: a few times the weight of a vertex's cheapest out-edge
// (about mean weight / mean degree), so a window holds about one hop of the
// shortest-path tree.  Measured on GB300 with weights in [1, 255] and degree
// 32: width 16 re-expands 3% of the edges in 100 rounds, width 8 0.7% in 155
// rounds, plain Bellman-Ford 360% in 35 rounds.
// A window's tail: once a sweep leaves fewer near vertices than this, the far
// pile is split at once and the tail joins the next window's first sweep
// instead of draining in a run of small, latency-bound sweeps (0 = off).
// Measured on GB300, uniform 2^24 degree 32: SSSP 43.6 -> 42.7 ms from host
// memory, 12.6 -> 11.7 ms from HBM, the same re-expansion.  On graphs with
// long lists (Kronecker scale 24) it let hubs be improved after their window
// moved on and doubled the re-expansion (46 -> 77 ms), so it is off there.
#ifndef EMOGI_SSSP_TAIL_SHIFT
#define EMOGI_SSSP_TAIL_SHIFT 12
#endif
uint64_t sssp_tail(emogi_graph g) {
    if (!EMOGI_SSSP_TAIL_SHIFT || g->max_degree > dev::kHeavyEntries) return 0;
    return std::max<uint64_t>(g->n >> EMOGI_SSSP_TAIL_SHIFT, 256);
}

uint64_t auto_delta(emogi_graph g) {
    const double d = g->avg_degree > 1.0 ? g->avg_degree : 1.0;
    const double x = g->avg_weight * 4.0 / d;
    return x < 1.0 ? 1 : (uint64_t)x;
}

emogi_status setup(emogi_graph g, const emogi_opts* opts, Ctx* c) {
    if (!g) return fail(EMOGI_E_ARG, "graph is NULL");
    EMOGI_TRY(parse_opts(opts, &c->o));
    c->g = g;
    EMOGI_CUDA_TRY(cudaSetDevice(g->device));
    EMOGI_TRY(ensure_workspace(g));
    c->st = c->o.stream ? c->o.stream : g->stream;
    c->G = c->o.granularity ? c->o.granularity : auto_granularity(g->avg_degree, g->id_bytes);
    c->chunk = c->o.chunk_lines ? c->o.chunk_lines : 32;
    c->sms = sm_count(g->device);
    if (trace_enabled()) c->o.flags |= EMOGI_OPT_TIME_KERNELS;
    return EMOGI_OK;
}

int grid_for(const Ctx& c, uint64_t threads_needed) {
    uint64_t b = (threads_needed + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)c.sms * 8;
    if (b < 1) b = 1;
    return (int)std::min(b, cap);
}

Sweep make_sweep(const Ctx& c, int side, bool all_vertices) {
    emogi_graph g = c.g;
    Workspace& ws = g->ws;
    Sweep s;
    s.off = g->d_off;
    s.cols = g->cols;
    s.w = g->w;
    s.shift = g->shift;
    s.in_q = all_vertices ? nullptr : ws.q[side];
    s.in_count = &ws.ctr->qcount[side];
    s.all_n = (uint32_t)g->n;
    s.out_q = ws.q[side ^ 1];
    s.out_count = &ws.ctr->qcount[side ^ 1];
    s.lq_v = ws.lq_v;
    s.lq_base = ws.lq_base;
    s.lq_state = ws.lq_state;
    s.large = &ws.ctr->large[0];
    s.large_lines = kLargeLines;
    s.chunk_lines = c.chunk;
    s.scanned = &ws.ctr->scanned;
    s.heads = g->d_heads;
    s.short_off = g->d_short_off;
    s.short_ids = g->d_short_ids;
    s.short_w = g->d_short_w;
    s.short_max = g->short_max;
    s.scanned_heads = &ws.ctr->scanned_heads;
    s.m = g->m;
    s.qcap = (uint32_t)g->n;
    return s;
}

// One sweep over k active vertices: the neighbour expansion of the chosen
// access variant (plus the split-list pass for MERGED_ALIGNED).
template <class Op, class Id>
emogi_status sweep_ids(Ctx& c, const Sweep& s, const Op& op, uint64_t k) {
    Workspace& ws = c.g->ws;
    const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
    switch (c.o.access) {
        case EMOGI_ACCESS_NAIVE:
            dev::k_expand_naive<Op, Id><<<grid_for(c, k), kThreads, 0, c.st>>>(s, op);
            c.kernel_launches += 1;
            break;
        case EMOGI_ACCESS_MERGED:
            dev::k_expand_merged<Op, Id><<<grid_for(c, k * 32), kThreads, 0, c.st>>>(s, op);
            c.kernel_launches += 1;
            break;
        default: {
            if (!s.in_q) {  // every vertex: one lane per vertex first, G lanes per kept list
                const int grid = grid_for(c, k);
                switch (c.G) {
                    case 4: dev::k_expand_all<Op, 4, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                    case 8: dev::k_expand_all<Op, 8, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                    case 16: dev::k_expand_all<Op, 16, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                    default: dev::k_expand_all<Op, 32, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                }
                dev::k_expand_split<Op, Id><<<c.sms * 4, kThreads, 0, c.st>>>(s, op);
                c.kernel_launches += 2;
                break;
            }
            const int grid = grid_for(c, k * c.G);
            switch (c.G) {
                case 4: dev::k_expand_group<Op, 4, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                case 8: dev::k_expand_group<Op, 8, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                case 16: dev::k_expand_group<Op, 16, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
                default: dev::k_expand_group<Op, 32, Id><<<grid, kThreads, 0, c.st>>>(s, op); break;
            }
            dev::k_expand_split<Op, Id><<<c.sms * 4, kThreads, 0, c.st>>>(s, op);
            c.kernel_launches += 2;
        }
    }
    EMOGI_CUDA_TRY(cudaGetLastError());
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
    c.expand_launches++;
    return EMOGI_OK;
}

template <class Op>
emogi_status sweep(Ctx& c, const Sweep& s, const Op& op, uint64_t k) {
    return c.g->id_bytes == 4 ? sweep_ids<Op, uint32_t>(c, s, op, k) : sweep_ids<Op, uint64_t>(c, s, op, k);
}

// One bottom-up BFS sweep over all vertices at level L.
template <class Id>
emogi_status sweep_bottom_up_ids(Ctx& c, const Sweep& s, uint32_t* level, uint32_t L) {
    Workspace& ws = c.g->ws;
    const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
    const uint32_t G = std::min<uint32_t>(c.G, 8);
    const int grid = grid_for(c, c.g->n);  // one vertex per lane, then G lanes per undecided list
    unsigned long long* fe = &ws.ctr->fedges;
    switch (G) {
        case 4: dev::k_bfs_bottom_up<4, Id><<<grid, kThreads, 0, c.st>>>(s, level, L, fe); break;
        default: dev::k_bfs_bottom_up<8, Id><<<grid, kThreads, 0, c.st>>>(s, level, L, fe); break;
    }
    EMOGI_CUDA_TRY(cudaGetLastError());
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
    c.kernel_launches++;
    c.expand_launches++;
    return EMOGI_OK;
}

emogi_status sweep_bottom_up(Ctx& c, const Sweep& s, uint32_t* level, uint32_t L) {
    return c.g->id_bytes == 4 ? sweep_bottom_up_ids<uint32_t>(c, s, level, L)
                              : sweep_bottom_up_ids<uint64_t>(c, s, level, L);
}

// Turns the next-frontier flags into queue `side` (in vertex order) and
// clears them.
emogi_status compact_next(Ctx& c, int side) {
    Workspace& ws = c.g->ws;
    const uint64_t chunks = c.g->n / 16 + 1;
    dev::k_compact_flags<<<grid_for(c, chunks), kThreads, 0, c.st>>>(ws.nflag, chunks, ws.q[side],
                                                                     &ws.ctr->qcount[side], (uint32_t)c.g->n);
    EMOGI_CUDA_TRY(cudaGetLastError());
    c.kernel_launches++;
    return EMOGI_OK;
}

// Clears what a call that ended early may have left set (far flags, the
// next-frontier flags), and marks them in use until the call completes.
emogi_status begin_flags(Ctx& c) {
    Workspace& ws = c.g->ws;
    if (ws.flags_dirty) {
        EMOGI_CUDA_TRY(cudaMemsetAsync(ws.fflag, 0, c.g->n * 4, c.st));
        EMOGI_CUDA_TRY(cudaMemsetAsync(ws.nflag, 0, (c.g->n / 16 + 1) * 16, c.st));
    }
    ws.flags_dirty = true;
    return EMOGI_OK;
}

// One bottom-up multi-source BFS level (k_ms_bottom_up).
template <class Id>
emogi_status ms_bottom_up_ids(Ctx& c, const Sweep& s, unsigned long long active) {
    Workspace& ws = c.g->ws;
    const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
    const int grid = grid_for(c, c.g->n);
    if (std::min<uint32_t>(c.G, 8) == 4)
        dev::k_ms_bottom_up<4, Id><<<grid, kThreads, 0, c.st>>>(s, ws.ms_front, ws.ms_visit, ws.ms_next, ws.nflag,
                                                                 active);
    else
        dev::k_ms_bottom_up<8, Id><<<grid, kThreads, 0, c.st>>>(s, ws.ms_front, ws.ms_visit, ws.ms_next, ws.nflag,
                                                                 active);
    EMOGI_CUDA_TRY(cudaGetLastError());
    if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
    c.kernel_launches++;
    c.expand_launches++;
    return EMOGI_OK;
}

// Multi-source BFS direction: bottom-up when the frontier's lists hold more
// than 1/EMOGI_MS_ALPHA of the edges each source has left to explore on
// average.  A pull for several sources stops only once every source it still
// needs is found, so it pays later than a single-source pull (Beamer's 1/14).
#ifndef EMOGI_MS_ALPHA
#define EMOGI_MS_ALPHA 4
#endif
bool ms_bottom_up_pays(uint64_t mf, uint64_t m, uint32_t k, uint64_t pairs_edges) {
    const double left = ((double)k * (double)m - (double)pairs_edges) / (double)k;
    return (double)mf * EMOGI_MS_ALPHA > left;
}

emogi_status read_counters(Ctx& c, bool after_sweep = true) {
    Workspace& ws = c.g->ws;
    EMOGI_CUDA_TRY(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(c.st));
    // a queue holds n entries and every append past them was dropped: a count
    // above n is a broken invariant, reported before the queue is read again
    for (int i = 0; i < 2; i++)
        if (ws.h_ctr->qcount[i] > c.g->n)
            return fail(EMOGI_E_CUDA, "internal error: frontier queue %d holds %u entries for n = %llu", i,
                        ws.h_ctr->qcount[i], (unsigned long long)c.g->n);
    if (after_sweep && (c.o.flags & EMOGI_OPT_TIME_KERNELS)) {
        float ms = 0.f;
        EMOGI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev[2], ws.ev[3]));
        c.expand_ms += ms;
        if (trace_enabled())
            fprintf(stderr, "[emogi] sweep %llu in=%u/%u out=%u/%u far=%u/%u scanned=%llu stored=%llu ms=%.4f\n",
                    (unsigned long long)c.expand_launches, ws.h_ctr->qcount[0], ws.h_ctr->qcount[1],
                    ws.h_ctr->qcount[1], ws.h_ctr->qcount[0], ws.h_ctr->fcount[0], ws.h_ctr->fcount[1],
                    (unsigned long long)ws.h_ctr->scanned, (unsigned long long)ws.h_ctr->scanned_heads, ms);
    }
    return EMOGI_OK;
}

// Clears the next-side queue counter and the split-list counter.
emogi_status reset_sweep_counters(Ctx& c, int side) {
    Workspace& ws = c.g->ws;
    EMOGI_CUDA_TRY(cudaMemsetAsync(&ws.ctr->qcount[side ^ 1], 0, sizeof(uint32_t), c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(&ws.ctr->large[0], 0, sizeof(unsigned long long), c.st));
    return EMOGI_OK;
}

emogi_status finish(Ctx& c, uint32_t* state, uint32_t* out, bool count_reached, uint32_t iterations,
                    emogi_stats* stats, bool weights) {
    emogi_graph g = c.g;
    Workspace& ws = g->ws;
    if (count_reached && stats && g->n) {
        dev::k_reached_edges<<<grid_for(c, g->n), kThreads, 0, c.st>>>(state, g->d_off, (uint32_t)g->n,
                                                                         &ws.ctr->reached);
        c.kernel_launches++;
    }
    EMOGI_CUDA_TRY(cudaGetLastError());
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[1], c.st));
    if (!c.o.out_on_device && g->n)
        EMOGI_CUDA_TRY(cudaMemcpyAsync(out, state, g->n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(c.st));
    if (stats) {
        float ms = 0.f;
        EMOGI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev[0], ws.ev[1]));
        memset(stats, 0, sizeof *stats);
        stats->iterations = iterations;
        stats->edges_scanned = ws.h_ctr->scanned;
        stats->edges_reached = count_reached ? ws.h_ctr->reached : g->m;
        stats->edge_bytes = (ws.h_ctr->scanned - ws.h_ctr->scanned_heads) * g->id_bytes;
        stats->weight_bytes = weights ? (ws.h_ctr->scanned - ws.h_ctr->scanned_heads) * 4ull : 0;
        stats->ms = ms;
        stats->expand_ms = c.expand_ms;
        stats->expand_launches = c.expand_launches;
        stats->kernel_launches = c.kernel_launches;
    }
    return EMOGI_OK;
}

// Level-synchronous loop shared by BFS and SSSP: sweep the active queue until
// the next queue comes back empty.  make_op(level) builds the sweep's policy.
template <class MakeOp>
emogi_status level_loop(Ctx& c, MakeOp make_op, uint32_t* iterations) {
    int side = 0;
    uint64_t k = 1;
    uint32_t it = 0;
    while (k > 0) {
        // BFS needs at most n sweeps and frontier Bellman-Ford at most n rounds
        if (it > c.g->n + 1) return fail(EMOGI_E_TIMEOUT, "traversal did not converge in %u sweeps", it);
        EMOGI_TRY(reset_sweep_counters(c, side));
        Sweep s = make_sweep(c, side, false);
        EMOGI_TRY(sweep(c, s, make_op(it + 1), k));
        EMOGI_TRY(read_counters(c));
        k = c.g->ws.h_ctr->qcount[side ^ 1];
        side ^= 1;
        it++;
    }
    *iterations = it;
    return EMOGI_OK;
}

// Direction of the next BFS level by the list entries each would read (over
// the host link every entry costs the same, whichever direction reads it).
// Top-down reads the frontier's lists: mf entries.  Bottom-up reads, for each
// of the nu unreached vertices, its list up to its first neighbour in the
// frontier.  A list entry points into the frontier with probability
// p = mf / m (the frontier's share of edge endpoints), so a vertex of the
// unreached vertices' mean degree d reads sum_{i<d} (1-p)^i entries, of which
// the first `heads` come from GPU memory when the list heads are mirrored
// there; the scan of all n levels adds a fixed cost of about n/32 entries.
bool bottom_up_reads_less(uint64_t n, uint64_t m, uint64_t mf, uint64_t nu, uint64_t mu, bool heads) {
    if (mf == 0 || m == 0) return false;
    if (nu == 0) return (double)n / 32.0 < (double)mf;  // nothing left to find: only the level scan
    const double p = std::min(1.0, (double)mf / (double)m), q = 1.0 - p;
    const double d = (double)mu / (double)nu;
    const double H = heads ? (double)dev::kHeads : 0.0;
    double per = 0.0;  // link entries per unreached vertex
    if (p < 1.0 && d > H) per = std::pow(q, H) * (1.0 - std::pow(q, d - H)) / p;
    return (double)nu * per + (double)n / 32.0 < (double)mf;
}

emogi_status check_output(emogi_graph g, const Opts& o, void* out) {
    if (!out && g->n) return fail(EMOGI_E_ARG, "output pointer is NULL");
    if (o.out_on_device && out) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(EMOGI_E_ARG, "out_on_device is set but the output is not device memory");
        }
    }
    return EMOGI_OK;
}

template <class Id, bool kFlags>
void record_sssp_sweeps(uint32_t G, int big, int lists, cudaStream_t cs, const dev::SsspFixed& f, dev::SsspLoop* L,
                        DevCounters* ctr) {
    switch (G) {
        case 4: dev::k_sssp_loop_sweep<DevCounters, 4, Id, kFlags><<<big, kThreads, 0, cs>>>(f, L, ctr); break;
        case 8: dev::k_sssp_loop_sweep<DevCounters, 8, Id, kFlags><<<big, kThreads, 0, cs>>>(f, L, ctr); break;
        case 16: dev::k_sssp_loop_sweep<DevCounters, 16, Id, kFlags><<<big, kThreads, 0, cs>>>(f, L, ctr); break;
        default: dev::k_sssp_loop_sweep<DevCounters, 32, Id, kFlags><<<big, kThreads, 0, cs>>>(f, L, ctr); break;
    }
    dev::k_sssp_loop_lists<DevCounters, Id, kFlags><<<lists, kThreads, 0, cs>>>(f, L, ctr);
    if (kFlags) dev::k_sssp_loop_compact<DevCounters><<<big, kThreads, 0, cs>>>(f, L, ctr);
}

// Whether SSSP rebuilds its near frontiers in vertex order: for edge lists
// (with weights) of 16 GiB or more, which a sweep in arrival order reads
// scattered over more address range than the GPU's translations cover
// (EMOGI_OPT_ORDERED_FRONTIER forces it).
bool ordered_frontier(const Ctx& c) {
    const emogi_graph g = c.g;
    const uint64_t bytes = g->m * (g->id_bytes + (g->w ? 4u : 0u));
    return (c.o.flags & EMOGI_OPT_ORDERED_FRONTIER) || bytes >= (16ull << 30);
}

// Records the device-driven SSSP loop of graph g as a CUDA graph (once per
// granularity / chunk choice): a conditional while-node whose body runs the
// sweep kernels, the far split and the controller.
emogi_status build_sssp_exec(Ctx& c) {
    emogi_graph g = c.g;
    Workspace& ws = g->ws;
    const uint32_t key = c.chunk * 2 + (ordered_frontier(c) ? 1u : 0u);
    if (ws.sssp_exec && ws.sssp_exec_G == c.G && ws.sssp_exec_chunk == key) return EMOGI_OK;
    if (ws.sssp_exec) {
        cudaGraphExecDestroy(ws.sssp_exec);
        ws.sssp_exec = nullptr;
    }
    dev::SsspFixed f;
    f.base = make_sweep(c, 0, false);
    f.base.block_slices = ordered_frontier(c) ? 1u : 0u;  // the queue holds vertex-ordered runs
    f.q[0] = ws.q[0];
    f.q[1] = ws.q[1];
    f.qround = ws.qround;
    f.fflag = ws.fflag;
    f.xd = ws.xd;
    f.nflag = ws.nflag;
    f.nchunks = g->n / 16 + 1;
    dev::SsspLoop* L = (dev::SsspLoop*)ws.sssp_loop;
    cudaGraph_t graph = nullptr;
    EMOGI_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(EMOGI_E_CUDA, "SSSP loop graph: %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cs = g->stream;  // record on the graph's own (non-default) stream
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const int big = c.sms * 8, lists = c.sms * 4;
        const bool ord = ordered_frontier(c);
        if (g->id_bytes == 4) {
            if (ord) record_sssp_sweeps<uint32_t, true>(c.G, big, lists, cs, f, L, ws.ctr);
            else record_sssp_sweeps<uint32_t, false>(c.G, big, lists, cs, f, L, ws.ctr);
        } else {
            if (ord) record_sssp_sweeps<uint64_t, true>(c.G, big, lists, cs, f, L, ws.ctr);
            else record_sssp_sweeps<uint64_t, false>(c.G, big, lists, cs, f, L, ws.ctr);
        }
        dev::k_sssp_loop_far<DevCounters><<<big, kThreads, 0, cs>>>(f, L, ws.ctr);
        dev::k_sssp_loop_control<DevCounters><<<1, 1, 0, cs>>>(L, ws.ctr, handle);
        cudaGraph_t captured = body;
        e = cudaStreamEndCapture(cs, &captured);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ws.sssp_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        ws.sssp_exec = nullptr;
        return fail(EMOGI_E_CUDA, "recording the SSSP loop: %s", cudaGetErrorString(e));
    }
    ws.sssp_exec_G = c.G;
    ws.sssp_exec_chunk = key;
    return EMOGI_OK;
}

}  // namespace
}  // namespace emogi

using namespace emogi;

extern "C" {

emogi_status emogi_bfs(emogi_graph g, uint64_t src, uint32_t* level, const emogi_opts* opts, emogi_stats* stats) {
    clear_error();
    Ctx c;
    EMOGI_TRY(setup(g, opts, &c));
    if (src >= g->n) return fail(EMOGI_E_ARG, "source %llu is not below n = %llu", (unsigned long long)src,
                                 (unsigned long long)g->n);
    EMOGI_TRY(check_output(g, c.o, level));
    Workspace& ws = g->ws;
    uint32_t* state = c.o.out_on_device ? level : ws.state;
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[0], c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ctr, 0, sizeof(DevCounters), c.st));
    dev::k_init_single<<<grid_for(c, g->n), kThreads, 0, c.st>>>(state, (uint32_t)g->n, (uint32_t)src, ws.q[0],
                                                                  nullptr, &ws.ctr->qcount[0]);
    EMOGI_CUDA_TRY(cudaGetLastError());
    c.kernel_launches++;
    EMOGI_TRY(begin_flags(c));
    const bool diropt = (g->flags & EMOGI_LOAD_UNDIRECTED) && !(c.o.flags & EMOGI_OPT_TOP_DOWN_ONLY) &&
                        c.o.access == EMOGI_ACCESS_MERGED_ALIGNED;
    const bool beamer = c.o.flags & EMOGI_OPT_BEAMER;
    int side = 0;
    uint64_t nf = 1, mf = 0, mu = g->m, reached = 1;
    bool top_down = true;
    uint32_t it = 0;
    while (nf > 0) {
        if (it > g->n + 1) return fail(EMOGI_E_TIMEOUT, "BFS did not converge in %u levels", it);
        if (diropt && it > 0) {
            if (beamer) {
                // the rule of Beamer et al.: bottom-up when the frontier's edges
                // exceed 1/14 of the unreached vertices' edges, back to top-down
                // when the frontier holds fewer than n/24 vertices
                if (top_down && mf > mu / 14) top_down = false;
                else if (!top_down && nf < g->n / 24) top_down = true;
            } else {
                top_down = !bottom_up_reads_less(g->n, g->m, mf, g->n - reached, mu, g->d_heads != nullptr);
            }
        }
        EMOGI_TRY(reset_sweep_counters(c, side));
        EMOGI_CUDA_TRY(cudaMemsetAsync(&ws.ctr->fedges, 0, sizeof(unsigned long long), c.st));
        Sweep s = make_sweep(c, side, !top_down);
        if (top_down) {
            dev::BfsBitsOp op{state, it + 1, diropt ? g->d_off : nullptr, diropt ? &ws.ctr->fedges : nullptr, 0,
                              ws.nflag};
            EMOGI_TRY(sweep(c, s, op, nf));
            EMOGI_TRY(compact_next(c, side ^ 1));
        } else {
            EMOGI_TRY(sweep_bottom_up(c, s, state, it));
        }
        EMOGI_TRY(read_counters(c));
        nf = ws.h_ctr->qcount[side ^ 1];
        mf = ws.h_ctr->fedges;
        mu -= std::min(mu, mf);
        reached += nf;
        side ^= 1;
        it++;
    }
    ws.flags_dirty = false;
    return finish(c, state, level, true, it, stats, false);
}

emogi_status emogi_sssp(emogi_graph g, uint64_t src, uint32_t* dist, const emogi_opts* opts, emogi_stats* stats) {
    clear_error();
    Ctx c;
    EMOGI_TRY(setup(g, opts, &c));
    if (src >= g->n) return fail(EMOGI_E_ARG, "source %llu is not below n = %llu", (unsigned long long)src,
                                 (unsigned long long)g->n);
    if (!g->w) return fail(EMOGI_E_UNSUPPORTED, "graph was loaded without weights");
    EMOGI_TRY(check_output(g, c.o, dist));
    Workspace& ws = g->ws;
    DevCounters* ctr = ws.ctr;
    uint32_t* state = c.o.out_on_device ? dist : ws.state;
    const uint64_t n = g->n;
    EMOGI_TRY(begin_flags(c));
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[0], c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->far_min, 0xFF, sizeof(uint32_t), c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.xd, 0xFF, n * 4, c.st));
    uint32_t* qround = ws.qround;  // sweep stamps; all 0 = "queued for sweep 0" only matters for the source
    EMOGI_CUDA_TRY(cudaMemsetAsync(qround, 0, n * 4, c.st));
    dev::k_init_single<<<grid_for(c, n), kThreads, 0, c.st>>>(state, (uint32_t)n, (uint32_t)src, ws.q[0],
                                                               nullptr, &ctr->qcount[0]);
    EMOGI_CUDA_TRY(cudaGetLastError());
    c.kernel_launches++;
    ws.flags_dirty = true;

    const uint64_t delta = c.o.delta ? c.o.delta : auto_delta(g);
    uint32_t it = 0, sweeps = 0;
    const bool device_loop = c.o.access == EMOGI_ACCESS_MERGED_ALIGNED && !(c.o.flags & EMOGI_OPT_HOST_LOOP);
    if (device_loop) {
        if (!ws.sssp_loop) {
            EMOGI_TRY(dev_alloc(&ws.sssp_loop, 256, "SSSP loop state"));
            EMOGI_CUDA_TRY(cudaHostAlloc(&ws.h_sssp_loop, 256, cudaHostAllocDefault));
        }
        EMOGI_TRY(build_sssp_exec(c));
        dev::SsspLoop* hl = (dev::SsspLoop*)ws.h_sssp_loop;
        memset(hl, 0, sizeof *hl);
        hl->T = (uint32_t)std::min<uint64_t>(delta, dev::INF);
        hl->delta = (uint32_t)std::min<uint64_t>(delta, dev::INF);
        hl->cap = 4 * n + 8;
        hl->dist = state;
        hl->delta_heavy = (uint32_t)std::max<uint64_t>(std::min<uint64_t>(delta, dev::INF) / 8, 1);
        hl->Th = dev::heavy_threshold(0, hl->delta_heavy, hl->T);
        hl->tail = sssp_tail(g);
        hl->qcap = (uint32_t)n;
        // the loop runs on the device: bound it in time as well (the caller's
        // timeout_ns when given, else one minute)
        hl->timeout_ns = (opts && opts->timeout_ns) ? opts->timeout_ns : 60000000000ull;
        EMOGI_CUDA_TRY(cudaMemcpyAsync(ws.sssp_loop, hl, sizeof *hl, cudaMemcpyHostToDevice, c.st));
        const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
        if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
        EMOGI_CUDA_TRY(cudaGraphLaunch(ws.sssp_exec, c.st));
        if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
        EMOGI_CUDA_TRY(cudaMemcpyAsync(hl, ws.sssp_loop, sizeof *hl, cudaMemcpyDeviceToHost, c.st));
        EMOGI_TRY(read_counters(c));
        if (hl->error == 1) return fail(EMOGI_E_TIMEOUT, "SSSP did not converge in %u rounds", hl->iters);
        if (hl->error == 3)
            return fail(EMOGI_E_CUDA, "internal error: an SSSP frontier queue passed n = %llu entries after %u rounds",
                        (unsigned long long)n, hl->iters);
        if (hl->error)
            return fail(EMOGI_E_TIMEOUT, "SSSP loop passed its time bound of %llu ns after %u rounds",
                        (unsigned long long)hl->timeout_ns, hl->iters);
        it = hl->iters;
        sweeps = hl->sweeps;
        c.expand_launches += sweeps;
        c.kernel_launches += (ordered_frontier(c) ? 5ull : 4ull) * it;
    }
    uint64_t T = std::min<uint64_t>(delta, dev::INF);
    int side = 0;
    uint64_t nk = device_loop ? 0 : 1, fk = 0;
    const bool ordered = ordered_frontier(c);
    const uint64_t tail = sssp_tail(g);
    const uint64_t delta_heavy = std::max<uint64_t>(std::min<uint64_t>(delta, dev::INF) / 8, 1);
    uint32_t Th = dev::heavy_threshold(0, delta_heavy, T);
    bool merge_tail = false;
    while (nk > 0 || fk > 0) {
        // every sweep or split either expands a vertex with a smaller distance
        // than before or raises T; both are bounded
        if (it > 4 * n + 8) return fail(EMOGI_E_TIMEOUT, "SSSP did not converge in %u rounds", it);
        if (nk > 0 && !merge_tail) {
            EMOGI_TRY(reset_sweep_counters(c, side));
            Sweep s = make_sweep(c, side, false);
            s.block_slices = ordered ? 1u : 0u;  // the queue holds vertex-ordered runs
            if (ordered) {
                dev::SsspFlagsOp op{state, qround, ws.fflag, ws.xd, &ctr->far_min, &ctr->overflow, (uint32_t)T,
                                    sweeps, dev::INF, g->d_off, Th, ws.nflag};
                EMOGI_TRY(sweep(c, s, op, nk));
                EMOGI_TRY(compact_next(c, side ^ 1));
            } else {
                dev::SsspOp op{state, qround, ws.fflag, ws.xd, &ctr->far_min, &ctr->overflow, (uint32_t)T, sweeps,
                               dev::INF, g->d_off, Th, nullptr};
                EMOGI_TRY(sweep(c, s, op, nk));
            }
            sweeps++;
            EMOGI_TRY(read_counters(c));
            nk = ws.h_ctr->qcount[side ^ 1];
            fk = (ws.h_ctr->fcount[0] > 0 || ws.h_ctr->far_min != dev::INF) ? 1 : 0;
            side ^= 1;
            merge_tail = nk > 0 && nk < tail && fk > 0;
        } else {
            // near frontier empty, or down to the window's tail: raise T past
            // the smallest pending far distance; a tail stays in the queue and
            // the split appends behind it
            const uint64_t fmin = ws.h_ctr->far_min;
            uint64_t Tn = fmin + delta;
            if (Tn <= T) Tn = T + 1;
            T = std::min<uint64_t>(Tn, dev::INF);
            Th = dev::heavy_threshold(fmin, delta_heavy, T);
            if (!merge_tail) EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->qcount[side], 0, sizeof(uint32_t), c.st));
            merge_tail = false;
            EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->fcount[0], 0, sizeof(uint32_t), c.st));
            EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->far_min, 0xFF, sizeof(uint32_t), c.st));
            dev::k_far_split<<<grid_for(c, n), kThreads, 0, c.st>>>((uint32_t)n, ws.fflag, state, ws.xd, qround,
                                                                     (uint32_t)T, sweeps, ws.q[side],
                                                                     &ctr->qcount[side], &ctr->fcount[0],
                                                                     &ctr->far_min);
            EMOGI_CUDA_TRY(cudaGetLastError());
            c.kernel_launches++;
            EMOGI_TRY(read_counters(c, false));
            nk = ws.h_ctr->qcount[side];
            fk = ws.h_ctr->fcount[0] > 0 ? 1 : 0;
        }
        it++;
    }
    ws.flags_dirty = false;
    if (ws.h_ctr->overflow) {
        // some relaxation overflowed: find out whether a reachable vertex was
        // left without a distance (its true distance is >= UINT32_MAX)
        EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->error, 0, sizeof(uint32_t), c.st));
        EMOGI_TRY(reset_sweep_counters(c, 0));
        Sweep s = make_sweep(c, 0, true);
        EMOGI_TRY(sweep(c, s, dev::OverflowCheckOp{state, &ctr->error}, n));
        EMOGI_TRY(read_counters(c));
        if (ws.h_ctr->error)
            return fail(EMOGI_E_OVERFLOW, "a shortest-path distance from %llu does not fit below UINT32_MAX",
                        (unsigned long long)src);
    }
    return finish(c, state, dist, true, it, stats, true);
}

emogi_status emogi_msbfs(emogi_graph g, const uint64_t* srcs, uint32_t k, uint32_t* levels, const emogi_opts* opts,
                         emogi_stats* stats) {
    clear_error();
    Ctx c;
    EMOGI_TRY(setup(g, opts, &c));
    if (k < 1 || k > EMOGI_MAX_SOURCES) return fail(EMOGI_E_ARG, "k = %u sources; 1 to 64 are supported", k);
    if (!srcs) return fail(EMOGI_E_ARG, "srcs is NULL");
    dev::MsSources ms;
    ms.k = k;
    for (uint32_t b = 0; b < k; b++) {
        if (srcs[b] >= g->n)
            return fail(EMOGI_E_ARG, "source %u = %llu is not below n = %llu", b, (unsigned long long)srcs[b],
                        (unsigned long long)g->n);
        ms.v[b] = (uint32_t)srcs[b];
    }
    EMOGI_TRY(check_output(g, c.o, levels));
    Workspace& ws = g->ws;
    const uint64_t n = g->n;
    if (!ws.ms_visit) {
        EMOGI_TRY(dev_alloc((void**)&ws.ms_visit, n * 8, "multi-source visit masks"));
        EMOGI_TRY(dev_alloc((void**)&ws.ms_front, n * 8, "multi-source frontier masks"));
        EMOGI_TRY(dev_alloc((void**)&ws.ms_next, n * 8, "multi-source next masks"));
    }
    uint32_t* out = levels;
    if (!c.o.out_on_device) {
        const size_t need = (size_t)k * n * 4;
        if (ws.ms_out_bytes < need) {
            dev_free(ws.ms_out, ws.ms_out_bytes);
            ws.ms_out = nullptr;
            ws.ms_out_bytes = 0;
            EMOGI_TRY(dev_alloc((void**)&ws.ms_out, need, "multi-source levels"));
            ws.ms_out_bytes = need;
        }
        out = ws.ms_out;
    }
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[0], c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ctr, 0, sizeof(DevCounters), c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ms_visit, 0, n * 8, c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ms_front, 0, n * 8, c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ms_next, 0, n * 8, c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(out, 0xFF, (size_t)k * n * 4, c.st));
    EMOGI_TRY(begin_flags(c));
    dev::k_ms_init<<<1, 64, 0, c.st>>>(ms, ws.ms_visit, ws.ms_front, out, n, ws.q[0], &ws.ctr->qcount[0]);
    EMOGI_CUDA_TRY(cudaGetLastError());
    c.kernel_launches++;
    EMOGI_TRY(read_counters(c, false));
    uint64_t kq = ws.h_ctr->qcount[0];
    // direction-optimising as emogi_bfs (undirected graphs, aligned access)
    const bool diropt = (g->flags & EMOGI_LOAD_UNDIRECTED) && !(c.o.flags & EMOGI_OPT_TOP_DOWN_ONLY) &&
                        c.o.access == EMOGI_ACCESS_MERGED_ALIGNED;
    unsigned long long active = k == 64 ? ~0ull : ((1ull << k) - 1ull);
    uint64_t mf = 0;
    const dev::MsLevelStats lst{&ws.ctr->fedges, &ws.ctr->ms_pairs_edges, &ws.ctr->ms_active};
    int side = 0;
    uint32_t it = 0;
    while (kq > 0) {
        if (it > n + 1) return fail(EMOGI_E_TIMEOUT, "multi-source BFS did not converge in %u levels", it);
        EMOGI_TRY(reset_sweep_counters(c, side));
        Sweep s = make_sweep(c, side, false);
        const bool bottom_up = diropt && it > 0 && ms_bottom_up_pays(mf, g->m, k, ws.h_ctr->ms_pairs_edges);
        if (bottom_up) {
            if (g->id_bytes == 4) EMOGI_TRY(ms_bottom_up_ids<uint32_t>(c, make_sweep(c, side, true), active));
            else EMOGI_TRY(ms_bottom_up_ids<uint64_t>(c, make_sweep(c, side, true), active));
            dev::k_ms_clear_front<<<grid_for(c, kq), kThreads, 0, c.st>>>(ws.q[side], &ws.ctr->qcount[side],
                                                                          ws.ms_front);
            EMOGI_CUDA_TRY(cudaGetLastError());
            c.kernel_launches++;
        } else {
            EMOGI_TRY(sweep(c, s, dev::MsBfsOp{ws.ms_front, ws.ms_visit, ws.ms_next, ws.nflag}, kq));
        }
        EMOGI_TRY(compact_next(c, side ^ 1));
        EMOGI_CUDA_TRY(cudaMemsetAsync(&ws.ctr->fedges, 0, sizeof(unsigned long long), c.st));
        EMOGI_CUDA_TRY(cudaMemsetAsync(&ws.ctr->ms_active, 0, sizeof(unsigned long long), c.st));
        dev::k_ms_finalize<<<grid_for(c, n), kThreads, 0, c.st>>>(ws.q[side ^ 1], &ws.ctr->qcount[side ^ 1],
                                                                   ws.ms_visit, ws.ms_front, ws.ms_next, out, n,
                                                                   it + 1, g->d_off, lst);
        EMOGI_CUDA_TRY(cudaGetLastError());
        c.kernel_launches++;
        EMOGI_TRY(read_counters(c));
        kq = ws.h_ctr->qcount[side ^ 1];
        mf = ws.h_ctr->fedges;
        active = ws.h_ctr->ms_active;
        side ^= 1;
        it++;
    }
    ws.flags_dirty = false;
    if (stats && n) {
        dev::k_ms_reached_edges<<<grid_for(c, n), kThreads, 0, c.st>>>(ws.ms_visit, g->d_off, (uint32_t)n,
                                                                         &ws.ctr->reached);
        EMOGI_CUDA_TRY(cudaGetLastError());
        c.kernel_launches++;
    }
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[1], c.st));
    if (!c.o.out_on_device)
        EMOGI_CUDA_TRY(cudaMemcpyAsync(levels, out, (size_t)k * n * 4, cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(c.st));
    if (stats) {
        float ms = 0.f;
        EMOGI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev[0], ws.ev[1]));
        memset(stats, 0, sizeof *stats);
        stats->iterations = it;
        stats->edges_scanned = ws.h_ctr->scanned;
        stats->edges_reached = ws.h_ctr->reached;
        stats->edge_bytes = (ws.h_ctr->scanned - ws.h_ctr->scanned_heads) * g->id_bytes;
        stats->ms = ms;
        stats->expand_ms = c.expand_ms;
        stats->expand_launches = c.expand_launches;
        stats->kernel_launches = c.kernel_launches;
    }
    return EMOGI_OK;
}

emogi_status emogi_pagerank(emogi_graph g, double damping, double tolerance, uint32_t max_iters, double* rank,
                            const emogi_opts* opts, emogi_stats* stats) {
    clear_error();
    Ctx c;
    EMOGI_TRY(setup(g, opts, &c));
    if (!(damping >= 0.0 && damping < 1.0)) return fail(EMOGI_E_ARG, "damping %g is not in [0, 1)", damping);
    if (!(tolerance >= 0.0)) return fail(EMOGI_E_ARG, "tolerance %g is negative", tolerance);
    if (max_iters < 1) return fail(EMOGI_E_ARG, "max_iters must be at least 1");
    EMOGI_TRY(check_output(g, c.o, rank));
    Workspace& ws = g->ws;
    const uint64_t n = g->n;
    if (!ws.pr_contrib) {
        EMOGI_TRY(dev_alloc((void**)&ws.pr_contrib, n * 8, "PageRank contributions"));
        EMOGI_TRY(dev_alloc((void**)&ws.pr_acc, n * 8, "PageRank sums"));
        EMOGI_TRY(dev_alloc(&ws.pr_ctr, 64, "PageRank counters"));
        EMOGI_CUDA_TRY(cudaHostAlloc(&ws.h_pr_ctr, 64, cudaHostAllocDefault));
        EMOGI_CUDA_TRY(cudaMemsetAsync(ws.pr_acc, 0, n * 8, c.st));  // on the call's stream, before its kernels
    }
    double* r = rank;
    if (!c.o.out_on_device) {
        if (!ws.pr_rank) EMOGI_TRY(dev_alloc((void**)&ws.pr_rank, n * 8, "PageRank ranks"));
        r = ws.pr_rank;
    }
    dev::PrCounters* pc = (dev::PrCounters*)ws.pr_ctr;
    dev::PrCounters* hpc = (dev::PrCounters*)ws.h_pr_ctr;
    const bool pull = g->flags & EMOGI_LOAD_UNDIRECTED;
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[0], c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ctr, 0, sizeof(DevCounters), c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(pc, 0, sizeof(dev::PrCounters), c.st));
    uint32_t it = 0;
    if (n) {
        dev::k_pr_init<<<grid_for(c, n), kThreads, 0, c.st>>>(n, g->d_off, r, ws.pr_contrib, pc);
        EMOGI_CUDA_TRY(cudaGetLastError());
        c.kernel_launches++;
        for (; it < max_iters; it++) {
            EMOGI_TRY(reset_sweep_counters(c, 0));
            Sweep s = make_sweep(c, 0, true);
            const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
            if (pull) {
                if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
                const int grid = grid_for(c, n * c.G);
                if (g->id_bytes == 4) {
                    switch (c.G) {
                        case 4: dev::k_pr_pull<4, uint32_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        case 8: dev::k_pr_pull<8, uint32_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        case 16: dev::k_pr_pull<16, uint32_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        default: dev::k_pr_pull<32, uint32_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                    }
                    dev::k_pr_pull_split<uint32_t><<<c.sms * 4, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc);
                } else {
                    switch (c.G) {
                        case 4: dev::k_pr_pull<4, uint64_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        case 8: dev::k_pr_pull<8, uint64_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        case 16: dev::k_pr_pull<16, uint64_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                        default: dev::k_pr_pull<32, uint64_t><<<grid, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc); break;
                    }
                    dev::k_pr_pull_split<uint64_t><<<c.sms * 4, kThreads, 0, c.st>>>(s, ws.pr_contrib, ws.pr_acc);
                }
                EMOGI_CUDA_TRY(cudaGetLastError());
                if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
                c.kernel_launches += 2;
                c.expand_launches++;
            } else {
                EMOGI_TRY(sweep(c, s, dev::PrPushOp{ws.pr_contrib, ws.pr_acc}, n));
            }
            EMOGI_CUDA_TRY(cudaMemsetAsync(&pc->change, 0, sizeof(double), c.st));
            EMOGI_CUDA_TRY(cudaMemsetAsync(&pc->dangling[(it + 1) & 1], 0, sizeof(double), c.st));
            dev::k_pr_finalize<<<grid_for(c, n), kThreads, 0, c.st>>>(n, g->d_off, r, ws.pr_contrib, ws.pr_acc, pc,
                                                                      damping, it);
            EMOGI_CUDA_TRY(cudaGetLastError());
            c.kernel_launches++;
            EMOGI_CUDA_TRY(cudaMemcpyAsync(hpc, pc, sizeof(dev::PrCounters), cudaMemcpyDeviceToHost, c.st));
            EMOGI_TRY(read_counters(c));
            if (hpc->change < tolerance) {
                it++;
                break;
            }
        }
    }
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[1], c.st));
    if (!c.o.out_on_device && n)
        EMOGI_CUDA_TRY(cudaMemcpyAsync(rank, r, n * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c.st));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(c.st));
    if (stats) {
        float ms = 0.f;
        EMOGI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev[0], ws.ev[1]));
        memset(stats, 0, sizeof *stats);
        stats->iterations = it;
        stats->edges_scanned = ws.h_ctr->scanned;
        stats->edges_reached = g->m * (uint64_t)it;
        stats->edge_bytes = (ws.h_ctr->scanned - ws.h_ctr->scanned_heads) * g->id_bytes;
        stats->ms = ms;
        stats->expand_ms = c.expand_ms;
        stats->expand_launches = c.expand_launches;
        stats->kernel_launches = c.kernel_launches;
    }
    return EMOGI_OK;
}

emogi_status emogi_cc(emogi_graph g, uint32_t* label, const emogi_opts* opts, emogi_stats* stats) {
    clear_error();
    Ctx c;
    EMOGI_TRY(setup(g, opts, &c));
    if (!(g->flags & EMOGI_LOAD_UNDIRECTED))
        return fail(EMOGI_E_UNSUPPORTED, "connected components needs a graph loaded with EMOGI_LOAD_UNDIRECTED");
    EMOGI_TRY(check_output(g, c.o, label));
    Workspace& ws = g->ws;
    uint32_t* parent = c.o.out_on_device ? label : ws.state;
    EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[0], c.st));
    EMOGI_CUDA_TRY(cudaMemsetAsync(ws.ctr, 0, sizeof(DevCounters), c.st));
    const bool sampled = !(c.o.flags & EMOGI_OPT_CC_FULL_PASS) && c.o.access == EMOGI_ACCESS_MERGED_ALIGNED;
    if (g->n) {
        const uint32_t n = (uint32_t)g->n;
        dev::k_init_identity<<<grid_for(c, n), kThreads, 0, c.st>>>(parent, n);
        EMOGI_CUDA_TRY(cudaGetLastError());
        c.kernel_launches++;
        Sweep s = make_sweep(c, 0, true);
        if (sampled) {
            const bool timed = c.o.flags & EMOGI_OPT_TIME_KERNELS;
            if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[2], c.st));
            if (g->id_bytes == 4)
                dev::k_cc_sample<uint32_t><<<grid_for(c, n), kThreads, 0, c.st>>>(g->d_off, g->cols, g->d_heads,
                                                                                   parent, n, 2, &ws.ctr->scanned);
            else
                dev::k_cc_sample<uint64_t><<<grid_for(c, n), kThreads, 0, c.st>>>(g->d_off, g->cols, g->d_heads,
                                                                                   parent, n, 2, &ws.ctr->scanned);
            EMOGI_CUDA_TRY(cudaGetLastError());
            if (timed) EMOGI_CUDA_TRY(cudaEventRecord(ws.ev[3], c.st));
            c.expand_launches++;
            if (timed) EMOGI_TRY(read_counters(c));
            dev::k_compress<<<grid_for(c, n), kThreads, 0, c.st>>>(parent, n);
            dev::k_cc_giant<<<1, 1024, 0, c.st>>>(parent, g->d_off, n, &ws.ctr->giant);
            EMOGI_CUDA_TRY(cudaGetLastError());
            EMOGI_TRY(read_counters(c, false));
            c.kernel_launches += 3;
            EMOGI_TRY(reset_sweep_counters(c, 0));
            EMOGI_TRY(sweep(c, s, dev::CcFinalOp{parent, ws.h_ctr->giant}, n));
        } else {
            EMOGI_TRY(sweep(c, s, dev::CcOp{parent}, n));
        }
        dev::k_compress<<<grid_for(c, n), kThreads, 0, c.st>>>(parent, n);
        EMOGI_CUDA_TRY(cudaGetLastError());
        c.kernel_launches++;
        if (c.o.flags & EMOGI_OPT_TIME_KERNELS) EMOGI_TRY(read_counters(c));
    }
    return finish(c, parent, label, false, sampled ? 2 : 1, stats, false);
}

}  // extern "C"
