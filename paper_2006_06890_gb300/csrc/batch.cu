// Batched BFS over many graphs in one persistent launch.
//
// The paper traverses one graph per run, launching one kernel per level
// (Sec. 4.2).  Serving many small or uneven graphs that way pays a launch and
// a host round trip per level per graph.  Here every graph of a batch advances
// one level per round of a single persistent, cooperatively launched kernel:
// the frontiers of all graphs form one combined queue of (graph, vertex)
// entries, warps claim chunks of it dynamically (graphs differ in degree, so
// static striding would leave warps idle), and a grid-wide barrier with a
// bounded wait separates levels.  The whole call (source upload, init, the
// persistent kernel) is one CUDA graph, instantiated once per batch and
// replayed.  The lanes per vertex (G) and the claim size are picked by
// measurement (emogi_batch_autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace emogi {
namespace {

struct BatchGraph {
    const uint64_t* off;
    const void* cols;
    uint64_t base;   // first entry of this graph in the combined level array
    uint64_t m;      // entries in the edge list
    uint32_t n;
    uint32_t shift;
    uint32_t ids32;  // 1: uint32 ids, 0: uint64 ids
    uint32_t pad;
};

struct BatchCtl {
    uint32_t qcount[3];     // rotating frontier counters
    uint32_t wclaim[3];     // rotating work-claim counters
    uint32_t bar_count;
    uint32_t bar_gen;
    uint32_t error;         // 1 = a barrier wait timed out
    uint32_t levels;        // rounds run
    unsigned long long scanned;
};

struct BatchParams {
    const BatchGraph* graphs;
    uint32_t* level;        // combined levels, graph g at graphs[g].base
    uint2* q[2];            // combined frontier queues of (graph, vertex)
    BatchCtl* ctl;
    uint64_t timeout_ns;
    uint32_t claim;         // frontier entries a warp claims at once, in units of its groups
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks are co-resident).
// The wait is bounded: after timeout_ns the block records an error and every
// block leaves the kernel at its next barrier.  Returns false on error.
__device__ bool grid_barrier(BatchCtl* ctl, uint64_t timeout_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile uint32_t* gen = &ctl->bar_gen;
        const uint32_t g = *gen;
        __threadfence();
        if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*gen == g) {
                if (*(volatile uint32_t*)&ctl->error) { ok = 0; break; }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(&ctl->error, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile uint32_t*)&ctl->error) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// Per-warp staging of (graph, vertex) appends in shared memory: one
// atomicAdd and one coalesced copy per buffer instead of one atomicAdd per
// warp and step on the round's single queue counter.
constexpr uint32_t kStage = 128;
struct Stage {
    uint2* buf;     // this warp's kStage entries
    uint32_t cnt;   // entries held (the same in every lane)
};

__device__ __forceinline__ void stage_flush(Stage& st, uint2* q, uint32_t* count) {
    if (st.cnt == 0) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(count, st.cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    for (uint32_t i = lane; i < st.cnt; i += 32) q[base + i] = st.buf[i];
    __syncwarp();
    st.cnt = 0;
}

// Stages up to two entries per lane (whole warp, converged).
__device__ __forceinline__ void stage_push2(Stage& st, uint2* q, uint32_t* count, bool p0, uint2 e0, bool p1,
                                            uint2 e1) {
    const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
    const uint32_t n0 = __popc(b0), total = n0 + __popc(b1);
    if (total == 0) return;
    if (st.cnt + total > kStage) stage_flush(st, q, count);
    const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
    if (p0) st.buf[st.cnt + __popc(b0 & below)] = e0;
    if (p1) st.buf[st.cnt + n0 + __popc(b1 & below)] = e1;
    st.cnt += total;
}

// level[*] = INF for every graph.
__global__ void k_batch_init(uint32_t* level, uint64_t total) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = tid; i < total; i += nt) level[i] = dev::INF;
}

// level[src_g] = 0 and queue = {(g, src_g)} for every graph g.
__global__ void k_batch_sources(BatchParams p, const uint32_t* srcs, uint32_t count) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    const BatchGraph d = p.graphs[g];
    p.level[d.base + srcs[g]] = 0;
    p.q[0][g] = make_uint2(g, srcs[g]);
    if (g == 0) p.ctl->qcount[0] = count;
}

// Level-synchronous BFS of every graph in the batch, one round per level.
template <int G>
__global__ void __launch_bounds__(256) k_batch_bfs(BatchParams p) {
    constexpr int GPW = 32 / G;
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    BatchCtl* ctl = p.ctl;
    __shared__ uint2 stage_bufs[8 * kStage];
    Stage stg{stage_bufs + (threadIdx.x >> 5) * kStage, 0u};
    unsigned long long scanned = 0;
    for (uint32_t L = 0;; L++) {
        const uint32_t* in_cnt = &ctl->qcount[L % 3];
        uint32_t* out_cnt = &ctl->qcount[(L + 1) % 3];
        uint32_t* claim = &ctl->wclaim[L % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->qcount[(L + 2) % 3] = 0;  // next round's output, unused this round
            ctl->wclaim[(L + 1) % 3] = 0;
        }
        const uint2* in_q = p.q[L & 1];
        uint2* out_q = p.q[(L + 1) & 1];
        const uint32_t k = *(volatile const uint32_t*)in_cnt;
        const uint32_t step = p.claim * GPW;
        for (;;) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(claim, step);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= k) break;
            for (uint32_t c0 = base; c0 < base + step && c0 < k; c0 += GPW) {
                const uint32_t idx = c0 + grp;
                uint64_t s = 0, e = 0, a = 0;
                BatchGraph d = {nullptr, nullptr, 0, 0, 0, 0, 0, 0};
                uint32_t v = 0, gi = 0;
                if (idx < k && idx < base + step) {
                    const uint2 en = in_q[idx];
                    gi = en.x;
                    v = en.y;
                    d = p.graphs[gi];
                    s = d.off[v];
                    e = d.off[v + 1];
                    a = d.ids32 ? dev::aligned_start<uint32_t>(s, d.shift) : dev::aligned_start<uint64_t>(s, d.shift);
                    if (glane == 0) scanned += e - s;
                }
                const uint32_t steps = e > s ? (uint32_t)((e - a + 2 * G - 1) / (2 * G)) : 0u;
                const uint32_t maxsteps = __reduce_max_sync(0xffffffffu, steps);
                uint32_t* lev = p.level + d.base;
                for (uint32_t t = 0; t < maxsteps; t++) {
                    const uint64_t j = a + (uint64_t)t * (2 * G) + 2 * glane;
                    // two ids per lane and step: 16 bytes of uint64 ids or 8 of uint32
                    uint32_t u[2] = {0, 0};
                    bool ok[2] = {false, false};
                    if (t < steps && j + 1 >= s) {
                        // a list's last ids too come in one whole load, unless it would pass
                        // the end of the edge list
                        if (j + 1 < e || (EMOGI_WHOLE_TAIL_LOADS && j < e && j + 2 <= d.m)) {
                            if (d.ids32) {
                                const uint2 pr = dev::ld_w2((const uint32_t*)d.cols + j);
                                u[0] = pr.x;
                                u[1] = pr.y;
                            } else {
                                const ulonglong2 pr = dev::ld_edge2((const uint64_t*)d.cols + j);
                                u[0] = (uint32_t)pr.x;
                                u[1] = (uint32_t)pr.y;
                            }
                            ok[0] = j >= s;
                            ok[1] = j + 1 < e;
                        } else if (j < e && j >= s) {
                            u[0] = d.ids32 ? dev::ld_id<uint32_t>(d.cols, j) : dev::ld_id<uint64_t>(d.cols, j);
                            ok[0] = true;
                        }
                    }
                    // read both neighbours' levels before either update
                    uint32_t cur[2] = {0, 0};
#pragma unroll
                    for (int x = 0; x < 2; x++)
                        if (ok[x]) cur[x] = lev[(uint32_t)u[x]];
                    bool pushed[2] = {false, false};
#pragma unroll
                    for (int x = 0; x < 2; x++)
                        if (ok[x] && cur[x] == dev::INF)
                            pushed[x] = atomicCAS(lev + (uint32_t)u[x], dev::INF, L + 1) == dev::INF;
                    stage_push2(stg, out_q, out_cnt, pushed[0], make_uint2(gi, u[0]), pushed[1],
                                make_uint2(gi, u[1]));
                }
            }
        }
        stage_flush(stg, out_q, out_cnt);
        if (!grid_barrier(ctl, p.timeout_ns)) break;
        const uint32_t next = *(volatile const uint32_t*)out_cnt;
        if (next == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->levels = L + 1;
            break;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) scanned += __shfl_xor_sync(0xffffffffu, scanned, o);
    if (lane == 0 && scanned) atomicAdd(&ctl->scanned, scanned);
}

template <int G>
const void* batch_kernel() {
    return (const void*)k_batch_bfs<G>;
}

const void* kernel_for(uint32_t G) {
    switch (G) {
        case 4: return batch_kernel<4>();
        case 8: return batch_kernel<8>();
        case 16: return batch_kernel<16>();
        default: return batch_kernel<32>();
    }
}

}  // namespace
}  // namespace emogi

struct emogi_batch_s {
    int device = 0;
    uint32_t count = 0;
    uint64_t total = 0;           // sum of n over the graphs
    std::vector<uint64_t> base;   // first entry of each graph in the combined levels
    std::vector<emogi_graph> graphs;
    emogi::BatchGraph* d_graphs = nullptr;
    uint32_t* d_level = nullptr;
    uint2* d_q[2] = {nullptr, nullptr};
    emogi::BatchCtl* d_ctl = nullptr;
    emogi::BatchCtl* h_ctl = nullptr;
    uint32_t* d_srcs = nullptr;
    uint32_t* h_srcs = nullptr;   // pinned staging for the sources
    size_t dev_bytes[5] = {0, 0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    uint32_t G = 8, claim = 4;    // current configuration
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    uint32_t exec_G = 0, exec_claim = 0;
    uint64_t exec_timeout = 0;
};

using namespace emogi;

namespace {

emogi_status batch_grid(emogi_batch b, uint32_t G, int* grid) {
    int per_sm = 0;
    EMOGI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(G), 256, 0));
    if (per_sm < 1) return fail(EMOGI_E_CUDA, "batched kernel cannot be resident");
    *grid = per_sm * sm_count(b->device);
    return EMOGI_OK;
}

emogi_status launch_batch_kernel(emogi_batch b, cudaStream_t st, uint32_t G, uint32_t claim, uint64_t timeout_ns) {
    int grid = 0;
    EMOGI_TRY(batch_grid(b, G, &grid));
    BatchParams p;
    p.graphs = b->d_graphs;
    p.level = b->d_level;
    p.q[0] = b->d_q[0];
    p.q[1] = b->d_q[1];
    p.ctl = b->d_ctl;
    p.timeout_ns = timeout_ns;
    p.claim = claim;
    void* args[] = {&p};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    EMOGI_CUDA_TRY(cudaLaunchKernelExC(&cfg, kernel_for(G), args));
    return EMOGI_OK;
}

// Records the whole call (source upload, init, persistent kernel) into
// b->exec for configuration (G, claim).
emogi_status build_exec(emogi_batch b, uint32_t G, uint32_t claim, uint64_t timeout_ns) {
    if (b->exec && b->exec_G == G && b->exec_claim == claim && b->exec_timeout == timeout_ns) return EMOGI_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t st = b->stream;
    EMOGI_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    BatchParams p;
    p.graphs = b->d_graphs;
    p.level = b->d_level;
    p.q[0] = b->d_q[0];
    p.q[1] = b->d_q[1];
    p.ctl = b->d_ctl;
    p.timeout_ns = timeout_ns;
    p.claim = claim;
    cudaMemcpyAsync(b->d_srcs, b->h_srcs, b->count * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), st);
    const int sms = sm_count(b->device);
    k_batch_init<<<sms * 8, 256, 0, st>>>(b->d_level, b->total);
    k_batch_sources<<<(b->count + 255) / 256, 256, 0, st>>>(p, b->d_srcs, b->count);
    emogi_status s = launch_batch_kernel(b, st, G, claim, timeout_ns);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != EMOGI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "capturing the batched BFS: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "instantiating the batched BFS: %s", cudaGetErrorString(e));
    b->exec_G = G;
    b->exec_claim = claim;
    b->exec_timeout = timeout_ns;
    return EMOGI_OK;
}

emogi_status run_batch(emogi_batch b, const uint64_t* srcs, uint32_t G, uint32_t claim, uint64_t timeout_ns,
                       float* ms) {
    for (uint32_t g = 0; g < b->count; g++) {
        if (srcs[g] >= b->graphs[g]->n)
            return fail(EMOGI_E_ARG, "source of graph %u (%llu) is not below its n = %llu", g,
                        (unsigned long long)srcs[g], (unsigned long long)b->graphs[g]->n);
        b->h_srcs[g] = (uint32_t)srcs[g];
    }
    EMOGI_TRY(build_exec(b, G, claim, timeout_ns));
    EMOGI_CUDA_TRY(cudaEventRecord(b->ev[0], b->stream));
    EMOGI_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    EMOGI_CUDA_TRY(cudaEventRecord(b->ev[1], b->stream));
    EMOGI_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(b->stream));
    EMOGI_CUDA_TRY(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
    if (b->h_ctl->error)
        return fail(EMOGI_E_TIMEOUT, "a level barrier of the batched BFS waited longer than %llu ns",
                    (unsigned long long)timeout_ns);
    return EMOGI_OK;
}

void free_batch(emogi_batch b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    dev_free(b->d_graphs, b->dev_bytes[0]);
    dev_free(b->d_level, b->dev_bytes[1]);
    dev_free(b->d_q[0], b->dev_bytes[2]);
    dev_free(b->d_q[1], b->dev_bytes[2]);
    dev_free(b->d_ctl, b->dev_bytes[3]);
    dev_free(b->d_srcs, b->dev_bytes[4]);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_srcs) cudaFreeHost(b->h_srcs);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

emogi_status emogi_batch_create(const emogi_graph* graphs, uint32_t count, emogi_batch* out) {
    clear_error();
    if (!out) return fail(EMOGI_E_ARG, "out is NULL");
    *out = nullptr;
    if (!graphs || count == 0) return fail(EMOGI_E_ARG, "a batch needs at least one graph");
    emogi_batch b = new (std::nothrow) emogi_batch_s();
    if (!b) return fail(EMOGI_E_NOMEM, "batch handle");
    b->count = count;
    b->base.resize(count);
    b->graphs.assign(graphs, graphs + count);
    std::vector<BatchGraph> table(count);
    for (uint32_t g = 0; g < count; g++) {
        emogi_graph gr = graphs[g];
        if (!gr || gr->n == 0) {
            free_batch(b);
            return fail(EMOGI_E_ARG, "graph %u of the batch is NULL or empty", g);
        }
        if (g && gr->device != graphs[0]->device) {
            free_batch(b);
            return fail(EMOGI_E_ARG, "all graphs of a batch must be on one device");
        }
        b->base[g] = b->total;
        table[g] = BatchGraph{gr->d_off, gr->cols, b->total, gr->m, (uint32_t)gr->n, gr->shift,
                              gr->id_bytes == 4 ? 1u : 0u, 0u};
        b->total += gr->n;
    }
    if (b->total >= 0xFFFFFFFFull) {
        free_batch(b);
        return fail(EMOGI_E_ARG, "a batch holds at most 2^32 - 2 vertices in total");
    }
    b->device = graphs[0]->device;
    auto bail = [&](emogi_status s) {
        free_batch(b);
        return s;
    };
    if (cudaSetDevice(b->device) != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "cudaSetDevice"));
    b->dev_bytes[0] = count * sizeof(BatchGraph);
    b->dev_bytes[1] = b->total * sizeof(uint32_t);
    b->dev_bytes[2] = b->total * sizeof(uint2);
    b->dev_bytes[3] = sizeof(BatchCtl);
    b->dev_bytes[4] = count * sizeof(uint32_t);
    emogi_status s;
    if ((s = dev_alloc((void**)&b->d_graphs, b->dev_bytes[0], "batch graph table")) != EMOGI_OK) return bail(s);
    if ((s = dev_alloc((void**)&b->d_level, b->dev_bytes[1], "batch levels")) != EMOGI_OK) return bail(s);
    if ((s = dev_alloc((void**)&b->d_q[0], b->dev_bytes[2], "batch queue 0")) != EMOGI_OK) return bail(s);
    if ((s = dev_alloc((void**)&b->d_q[1], b->dev_bytes[2], "batch queue 1")) != EMOGI_OK) return bail(s);
    if ((s = dev_alloc((void**)&b->d_ctl, b->dev_bytes[3], "batch control")) != EMOGI_OK) return bail(s);
    if ((s = dev_alloc((void**)&b->d_srcs, b->dev_bytes[4], "batch sources")) != EMOGI_OK) return bail(s);
    cudaError_t e = cudaHostAlloc((void**)&b->h_ctl, sizeof(BatchCtl), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_srcs, count * sizeof(uint32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_graphs, table.data(), count * sizeof(BatchGraph), cudaMemcpyHostToDevice);
    // the copy ran on the legacy default stream, which the batch's non-blocking
    // stream does not wait for: finish it before the batch is handed out
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "batch set-up: %s", cudaGetErrorString(e)));
    double deg = 0.0;
    for (auto* gr : b->graphs) deg += gr->avg_degree;
    deg /= count;
    b->G = deg >= 96 ? 32 : deg >= 48 ? 16 : deg >= 12 ? 8 : 4;
    *out = b;
    return EMOGI_OK;
}

emogi_status emogi_batch_free(emogi_batch b) {
    free_batch(b);
    return EMOGI_OK;
}

uint64_t emogi_batch_offset(emogi_batch b, uint32_t g) {
    return (b && g < b->count) ? b->base[g] : 0;
}

uint64_t emogi_batch_total_vertices(emogi_batch b) { return b ? b->total : 0; }

emogi_status emogi_bfs_batch(const emogi_graph* graphs, const uint64_t* srcs, uint32_t* levels, uint32_t count,
                             const emogi_opts* opts, emogi_stats* stats) {
    emogi_batch b = nullptr;
    EMOGI_TRY(emogi_batch_create(graphs, count, &b));
    emogi_status s = emogi_batch_bfs(b, srcs, levels, opts, stats);
    std::string err = s != EMOGI_OK ? std::string(emogi_last_error()) : std::string();
    free_batch(b);
    if (s != EMOGI_OK) set_error(err);
    return s;
}

emogi_status emogi_batch_bfs(emogi_batch b, const uint64_t* srcs, uint32_t* levels, const emogi_opts* opts,
                             emogi_stats* stats) {
    clear_error();
    if (!b) return fail(EMOGI_E_ARG, "batch is NULL");
    if (!srcs || !levels) return fail(EMOGI_E_ARG, "srcs and levels must be non-NULL");
    Opts o;
    EMOGI_TRY(parse_opts(opts, &o));
    if (o.access != EMOGI_ACCESS_MERGED_ALIGNED)
        return fail(EMOGI_E_UNSUPPORTED, "batched BFS reads lists merged and aligned only");
    EMOGI_CUDA_TRY(cudaSetDevice(b->device));
    const uint32_t G = o.granularity ? o.granularity : b->G;
    const uint32_t claim = o.chunk_lines ? o.chunk_lines : b->claim;
    float ms = 0.f;
    EMOGI_TRY(run_batch(b, srcs, G, claim, o.timeout_ns, &ms));
    const cudaMemcpyKind kind = o.out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    EMOGI_CUDA_TRY(cudaMemcpyAsync(levels, b->d_level, b->total * sizeof(uint32_t), kind, b->stream));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->iterations = b->h_ctl->levels;
        stats->edges_scanned = b->h_ctl->scanned;
        stats->edges_reached = b->h_ctl->scanned;  // BFS expands each reached vertex once
        stats->edge_bytes = b->h_ctl->scanned * 8ull;
        stats->ms = ms;
        stats->expand_ms = ms;
        stats->expand_launches = 1;
        stats->kernel_launches = 3;
    }
    return EMOGI_OK;
}

emogi_status emogi_batch_autotune(emogi_batch b, const uint64_t* srcs, uint32_t* best_granularity,
                                  uint32_t* best_claim, double* best_ms) {
    clear_error();
    if (!b || !srcs) return fail(EMOGI_E_ARG, "batch and srcs must be non-NULL");
    EMOGI_CUDA_TRY(cudaSetDevice(b->device));
    static const uint32_t Gs[] = {4, 8, 16, 32};
    static const uint32_t claims[] = {1, 4, 16, 64};
    float best = 1e30f;
    uint32_t bg = b->G, bc = b->claim;
    const uint64_t timeout = 2000000000ull;
    for (uint32_t G : Gs) {
        for (uint32_t claim : claims) {
            float ms = 0.f, t = 1e30f;
            for (int rep = 0; rep < 2; rep++) {  // first run warms the graph up
                EMOGI_TRY(run_batch(b, srcs, G, claim, timeout, &ms));
                t = std::min(t, ms);
            }
            if (t < best) {
                best = t;
                bg = G;
                bc = claim;
            }
        }
    }
    b->G = bg;
    b->claim = bc;
    if (best_granularity) *best_granularity = bg;
    if (best_claim) *best_claim = bc;
    if (best_ms) *best_ms = best;
    return EMOGI_OK;
}

}  // extern "C"
