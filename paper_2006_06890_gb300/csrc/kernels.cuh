// Device code of the traversal path.
//
// One level (BFS), relaxation round (SSSP) or edge pass (CC) is a
// vertex-centric sweep (paper Sec. 2.1, Algorithm "High-level Graph Traversal
// Flow"): every active vertex's neighbour list is read and an
// application-dependent update is applied to each neighbour; neighbours that
// satisfy the application's condition become active for the next sweep.
//
// The neighbour-list reads are the hot loop.  With the edge list in pinned
// host memory every read crosses the host link, so how a list is read decides
// the request sizes on the link (Sec. 3.3, Sec. 4.3):
//   * k_expand_group  - merged + aligned: a group of G lanes reads one list
//                       starting from the 128-byte line that holds its first
//                       element (16 ids per line), 16 bytes per lane, masking
//                       the lanes outside [start, end).  Lists longer than
//                       `large_lines` lines are not read here but appended
//                       to a split-list queue;
//   * k_expand_split  - the split lists, cut into work items of chunk_lines
//                       lines, one warp per item;
//   * k_expand_merged - the paper's "Merged" variant: a warp per vertex,
//                       8 bytes per lane from the list's own start;
//   * k_expand_naive  - the paper's "Naive" variant: a thread per vertex
//                       walking its list one element at a time.
// The per-neighbour work is a policy class (BfsOp, SsspOp, CcOp).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace emogi {
namespace dev {

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr unsigned long long SLOT_SHIFT = 34;  // items < 2^34, slots < 2^30
constexpr unsigned long long CHUNK_MASK = (1ull << SLOT_SHIFT) - 1;

// Everything a sweep needs besides the per-application state.
struct Sweep {
    const uint64_t* off;       // row offsets (GPU memory)
    const uint64_t* cols;      // edge list (GPU, pinned host or managed memory)
    const uint32_t* w;         // weights beside the edges, or null
    uint32_t shift;            // (edge-list base address mod 128) / 8
    const uint32_t* in_q;      // active vertices, or null for "all vertices"
    const uint32_t* in_count;  // number of active vertices (when in_q != null)
    uint32_t all_n;            // number of vertices (when in_q == null)
    uint32_t* out_q;           // next active vertices
    uint32_t* out_count;
    uint32_t* lq_v;            // split-list queue: vertex
    unsigned long long* lq_base;   // split-list queue: first work item
    unsigned long long* large;     // (slots << 34) | items
    uint32_t large_lines;      // lists with more lines than this are split
    uint32_t chunk_lines;      // lines per split work item
    unsigned long long* scanned;   // neighbour entries read (statistics)
};

// ------------------------------------------------------------------ loads
// Edge-list reads go through the non-coherent read-only path and do not
// allocate in L1: every line is used once per sweep.  The edge list and the
// weights never change during a traversal, so these loads are free of side
// effects and the compiler may schedule them early.
__device__ __forceinline__ ulonglong2 ld_edge2(const uint64_t* p) {
    ulonglong2 r;
    asm("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
                 : "=l"(r.x), "=l"(r.y)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint64_t ld_edge(const uint64_t* p) {
    uint64_t r;
    asm("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_w2(const uint32_t* p) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_w(const uint32_t* p) {
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// First index the aligned read starts from: the largest index <= s whose
// address is on a 128-byte boundary (the listing "Coalesced Memory Access
// (Merged + Aligned)" masks the low four index bits for 8-byte ids; `shift`
// accounts for an edge list whose base is not itself line aligned).  Never
// below 0; always even, so 16-byte vector loads stay aligned.
__device__ __forceinline__ uint64_t aligned_start(uint64_t s, uint32_t shift) {
    uint64_t r = (s + shift) & 15u;
    return s >= r ? s - r : 0;
}

// ------------------------------------------------------------------ queue push
// Warp-aggregated append: the lanes that push at the same time share one
// atomicAdd on the counter.
__device__ __forceinline__ void push(uint32_t* q, uint32_t* count, uint32_t v) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    q[base + rank] = v;
}

// Append a long list to the split-list queue: one 64-bit atomic hands out both
// the slot and the first work item, so bases increase with slot numbers.
__device__ __forceinline__ void defer(const Sweep& c, uint32_t v, unsigned long long items) {
    unsigned long long old = atomicAdd(c.large, (1ull << SLOT_SHIFT) | items);
    unsigned long long slot = old >> SLOT_SHIFT;
    c.lq_v[slot] = v;
    c.lq_base[slot] = old & CHUNK_MASK;
}

// ------------------------------------------------------------------ applications
// The per-neighbour work of a sweep is a policy object.  Each thread works on
// its own copy, so a policy may keep per-thread accumulators.
//   begin(v)       one lane per active vertex, before the list is read: returns
//                  the 32-bit value broadcast to the lanes reading v's list, or
//                  INF to skip the list entirely;
//   begin_chunk(v) the same for one work item of a split (long) list;
//   visit(st,v,u,w) the update for edge (v, u) with weight w; true = push u to
//                  the next frontier;
//   flush()        once per thread at kernel end, whole warp converged.

// BFS (Sec. 2.1): an unvisited neighbour gets the next level and becomes active.
// The compare-and-swap makes exactly one visitor push it.
struct BfsOp {
    uint32_t* level;
    uint32_t next;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = true;
    __device__ __forceinline__ uint32_t begin(uint32_t) { return 0; }
    __device__ __forceinline__ uint32_t begin_chunk(uint32_t) { return 0; }
    __device__ __forceinline__ bool visit(uint32_t, uint32_t, uint64_t u, uint32_t) {
        uint32_t* p = level + (uint32_t)u;
        if (*p != INF) return false;
        return atomicCAS(p, INF, next) == INF;
    }
    __device__ __forceinline__ void flush() {}
};

// Warp-reduced atomic minimum of a per-thread value (whole warp converged).
__device__ __forceinline__ void warp_atomic_min(uint32_t* out, uint32_t x) {
    x = __reduce_min_sync(0xffffffffu, x);
    if ((threadIdx.x & 31) == 0 && x != INF) atomicMin(out, x);
}

// SSSP (Sec. 5.1.2, Sec. 5.4: weights are read beside the edges).  Relaxation
// by atomic minimum with a near/far split of the active set (delta-stepping
// order): an improved neighbour whose new distance is below the threshold T
// joins the next near frontier, otherwise the far pile.  When the near
// frontier empties, the far pile is split again with T raised past its
// smallest distance.  Every vertex is expanded with its final distance, so
// the fixed point is the exact shortest distance whatever the order.
//   nflag / fflag: "queued in the near frontier / far pile" (one entry each);
//   xd: the distance v was last expanded with, so a vertex queued twice
//   (near and far) is not expanded twice with the same distance.
// A vertex clears its near flag before it reads its distance, so an
// improvement landing after the read queues it again.
struct SsspOp {
    uint32_t* dist;
    uint32_t* nflag;
    uint32_t* fflag;
    uint32_t* xd;
    uint32_t* far_q;
    uint32_t* far_count;
    uint32_t* far_min;
    uint32_t* overflow;
    uint32_t T;
    uint32_t lmin;  // per-thread smallest distance sent to the far pile
    static constexpr bool kWeights = true;
    static constexpr bool kPush = true;
    __device__ __forceinline__ uint32_t begin(uint32_t v) {
        atomicExch(nflag + v, 0u);
        __threadfence();
        const uint32_t d = __ldcg(dist + v);
        if (d >= __ldcg(xd + v)) return INF;  // already expanded with this distance
        __stcg(xd + v, d);
        return d;
    }
    __device__ __forceinline__ uint32_t begin_chunk(uint32_t v) { return __ldcg(dist + v); }
    // A relaxation whose sum does not fit below INF is dropped and noted; the
    // host then checks whether some reachable vertex was left at INF.
    __device__ __forceinline__ bool visit(uint32_t dv, uint32_t, uint64_t u64, uint32_t w) {
        const uint32_t u = (uint32_t)u64;
        const uint64_t nd64 = (uint64_t)dv + (uint64_t)w;
        if (nd64 >= (uint64_t)INF) {
            if (dv != INF) atomicExch(overflow, 1u);
            return false;
        }
        const uint32_t nd = (uint32_t)nd64;
        uint32_t* p = dist + u;
        if (nd >= *p) return false;
        const uint32_t old = atomicMin(p, nd);
        if (nd >= old) return false;
        __threadfence();
        if (nd < T) return atomicExch(nflag + u, 1u) == 0u;
        lmin = nd < lmin ? nd : lmin;
        if (atomicExch(fflag + u, 1u) == 0u) push(far_q, far_count, u);
        return false;
    }
    __device__ __forceinline__ void flush() { warp_atomic_min(far_min, lmin); }
};

// Union-find root with path halving.  Parents only ever point to smaller ids
// and a non-root never becomes a root again, so racing halving stores always
// write an ancestor.  Reads bypass L1 so that hooks made by other SMs are seen.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x) {
    for (;;) {
        const uint32_t px = __ldcg(parent + x);
        if (px == x) return x;
        const uint32_t gp = __ldcg(parent + px);
        if (gp != px) __stcg(parent + x, gp);
        x = gp;
    }
}

// CC hooking (Sec. 5.4, all vertices active, one pass over the edge list):
// each undirected edge (seen from its larger endpoint) joins the two trees by
// linking the larger root under the smaller with compare-and-swap, so the root
// of every component is its smallest vertex id.
struct CcOp {
    uint32_t* parent;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    __device__ __forceinline__ uint32_t begin(uint32_t) { return 0; }
    __device__ __forceinline__ uint32_t begin_chunk(uint32_t) { return 0; }
    __device__ __forceinline__ bool visit(uint32_t, uint32_t v, uint64_t u64, uint32_t) {
        uint32_t u = (uint32_t)u64;
        if (u >= v) return false;
        uint32_t a = v, b = u;
        for (;;) {
            a = uf_find(parent, a);
            b = uf_find(parent, b);
            if (a == b) return false;
            const uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
            if (atomicCAS(parent + hi, hi, lo) == hi) return false;
        }
    }
    __device__ __forceinline__ void flush() {}
};

// SSSP overflow check, run only when some relaxation overflowed: an edge from
// a vertex with a finite distance to one left at INF means that neighbour is
// reachable but its shortest distance does not fit below UINT32_MAX.
struct OverflowCheckOp {
    const uint32_t* dist;
    uint32_t* found;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    __device__ __forceinline__ uint32_t begin(uint32_t v) { return __ldcg(dist + v); }
    __device__ __forceinline__ uint32_t begin_chunk(uint32_t v) { return __ldcg(dist + v); }
    __device__ __forceinline__ bool visit(uint32_t dv, uint32_t, uint64_t u, uint32_t) {
        if (dv != INF && __ldcg(dist + (uint32_t)u) == INF) atomicExch(found, 1u);
        return false;
    }
    __device__ __forceinline__ void flush() {}
};

// ------------------------------------------------------------------ statistics
__device__ __forceinline__ void add_scanned(const Sweep& c, unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(c.scanned, x);
}

// One 16-byte step of a list read: lane covers ids j and j+1 of [s, e).
template <class Op>
__device__ __forceinline__ void read_pair(const Sweep& c, Op& op, uint32_t st, uint32_t v, uint64_t j,
                                          uint64_t s, uint64_t e, bool active) {
    uint64_t u0 = 0, u1 = 0;
    uint32_t w0 = 0, w1 = 0;
    bool v0 = false, v1 = false;
    if (active && j + 1 >= s) {
        if (j + 1 < e) {
            const ulonglong2 pr = ld_edge2(c.cols + j);
            u0 = pr.x;
            u1 = pr.y;
            if (Op::kWeights) {
                const uint2 wp = ld_w2(c.w + j);
                w0 = wp.x;
                w1 = wp.y;
            }
            v0 = j >= s;
            v1 = true;
        } else if (j < e && j >= s) {
            u0 = ld_edge(c.cols + j);
            if (Op::kWeights) w0 = ld_w(c.w + j);
            v0 = true;
        }
    }
    const bool p0 = v0 && op.visit(st, v, u0, w0);
    const bool p1 = v1 && op.visit(st, v, u1, w1);
    if (Op::kPush) {
        if (p0) push(c.out_q, c.out_count, (uint32_t)u0);
        if (p1) push(c.out_q, c.out_count, (uint32_t)u1);
    }
}

// ------------------------------------------------------------------ kernels
// Merged + aligned expansion with G lanes per vertex (G = 4, 8, 16, 32).
// Loops are warp-uniform: a warp runs as many steps as its longest group.
template <class Op, int G>
__global__ void __launch_bounds__(256) k_expand_group(Sweep c, Op op_in) {
    constexpr int GPW = 32 / G;
    Op op = op_in;
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0;
    for (uint64_t base = warp * GPW; base < k; base += nwarps * GPW) {
        const uint64_t idx = base + grp;
        uint32_t v = 0, st = INF;
        if (idx < k) {
            v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
            if (glane == 0) st = op.begin(v);
        }
        st = __shfl_sync(0xffffffffu, st, grp * G);
        uint64_t s = 0, e = 0;
        if (idx < k && st != INF) {
            s = c.off[v];
            e = c.off[v + 1];
        }
        uint64_t a = aligned_start(s, c.shift);
        const uint64_t lines = e > s ? (e - a + 15) >> 4 : 0;
        if (glane == 0) scanned += e - s;
        if (lines > c.large_lines) {
            if (glane == 0) defer(c, v, (lines + c.chunk_lines - 1) / c.chunk_lines);
            s = e = a = 0;
        }
        const uint32_t steps = e > s ? (uint32_t)((e - a + 2 * G - 1) / (2 * G)) : 0u;
        const uint32_t maxsteps = __reduce_max_sync(0xffffffffu, steps);
        for (uint32_t t = 0; t < maxsteps; t++)
            read_pair(c, op, st, v, a + (uint64_t)t * (2 * G) + 2 * glane, s, e, t < steps);
    }
    add_scanned(c, scanned);
    op.flush();
}

// Split lists: work item i of vertex lq_v[slot] covers lines
// [i * chunk_lines, (i + 1) * chunk_lines) of its aligned list; one warp per
// item, 16 bytes per lane (four 128-byte lines per step).
template <class Op>
__global__ void __launch_bounds__(256) k_expand_split(Sweep c, Op op_in) {
    Op op = op_in;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long tot = *c.large;
    const uint32_t nslots = (uint32_t)(tot >> SLOT_SHIFT);
    const unsigned long long nitems = tot & CHUNK_MASK;
    for (unsigned long long item = warp; item < nitems; item += nwarps) {
        uint32_t lo = 0, hi = nslots;  // last slot whose base <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (c.lq_base[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t v = c.lq_v[lo];
        const unsigned long long ci = item - c.lq_base[lo];
        const uint64_t s = c.off[v], e = c.off[v + 1];
        const uint64_t a = aligned_start(s, c.shift);
        const uint64_t cs = a + ci * 16ull * c.chunk_lines;
        uint64_t ce = cs + 16ull * c.chunk_lines;
        if (ce > e) ce = e;
        uint32_t st = 0;
        if (lane == 0) st = op.begin_chunk(v);
        st = __shfl_sync(0xffffffffu, st, 0);
        for (uint64_t j0 = cs; j0 < ce; j0 += 64) read_pair(c, op, st, v, j0 + 2 * lane, s, ce, true);
    }
    op.flush();
}

// The paper's "Merged" variant: one warp per vertex, lanes read consecutive
// 8-byte entries starting at the list's own first element.
template <class Op>
__global__ void __launch_bounds__(256) k_expand_merged(Sweep c, Op op_in) {
    Op op = op_in;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0;
    for (uint64_t idx = warp; idx < k; idx += nwarps) {
        const uint32_t v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
        uint32_t st = 0;
        if (lane == 0) st = op.begin(v);
        st = __shfl_sync(0xffffffffu, st, 0);
        if (st == INF) continue;
        const uint64_t s = c.off[v], e = c.off[v + 1];
        if (lane == 0) scanned += e - s;
        for (uint64_t i = s + lane; i < e; i += 32) {
            const uint64_t u = ld_edge(c.cols + i);
            const uint32_t w = Op::kWeights ? ld_w(c.w + i) : 0u;
            if (op.visit(st, v, u, w) && Op::kPush) push(c.out_q, c.out_count, (uint32_t)u);
        }
    }
    __syncwarp();
    add_scanned(c, scanned);
    op.flush();
}

// The paper's "Naive" variant: one thread per vertex, element by element.
template <class Op>
__global__ void __launch_bounds__(256) k_expand_naive(Sweep c, Op op_in) {
    Op op = op_in;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0;
    for (uint64_t idx = tid; idx < k; idx += nt) {
        const uint32_t v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
        const uint32_t st = op.begin(v);
        if (st == INF) continue;
        const uint64_t s = c.off[v], e = c.off[v + 1];
        scanned += e - s;
        for (uint64_t i = s; i < e; i++) {
            const uint64_t u = ld_edge(c.cols + i);
            const uint32_t w = Op::kWeights ? ld_w(c.w + i) : 0u;
            if (op.visit(st, v, u, w) && Op::kPush) push(c.out_q, c.out_count, (uint32_t)u);
        }
    }
    __syncwarp();
    add_scanned(c, scanned);
    op.flush();
}

// SSSP far-pile split (the near frontier is empty): every pending far vertex
// whose distance is below the new threshold T moves to the near frontier, the
// others stay in the far pile; vertices already expanded with their current
// distance are dropped.  Each vertex is in the pile once, and nothing else
// runs meanwhile, so plain flag updates suffice.
static __global__ void k_far_split(const uint32_t* fq_in, const uint32_t* fcount_in, uint32_t* fq_out,
                            uint32_t* fcount_out, uint32_t* nq_out, uint32_t* ncount_out, const uint32_t* dist,
                            uint32_t* nflag, uint32_t* fflag, const uint32_t* xd, uint32_t T,
                            uint32_t* far_min) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t k = *fcount_in;
    uint32_t lmin = INF;
    for (uint64_t base = tid - (threadIdx.x & 31); base < k; base += nt) {
        const uint64_t i = base + (threadIdx.x & 31);
        if (i < k) {
            const uint32_t v = fq_in[i];
            const uint32_t d = dist[v];
            if (d >= xd[v]) {
                fflag[v] = 0u;
            } else if (d < T) {
                fflag[v] = 0u;
                nflag[v] = 1u;
                push(nq_out, ncount_out, v);
            } else {
                lmin = d < lmin ? d : lmin;
                push(fq_out, fcount_out, v);
            }
        }
    }
    warp_atomic_min(far_min, lmin);
}

// ------------------------------------------------------------------ small kernels
// state[v] = INF for all v, except state[src] = 0; queue = {src}.
static __global__ void k_init_single(uint32_t* state, uint32_t n, uint32_t src, uint32_t* q, uint32_t* flag,
                              uint32_t* count) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = tid; v < n; v += nt) state[v] = (v == src) ? 0u : INF;
    if (tid == 0) {
        q[0] = src;
        *count = 1u;
        if (flag) flag[src] = 1u;
    }
}

// parent[v] = v.
static __global__ void k_init_identity(uint32_t* parent, uint32_t n) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = tid; v < n; v += nt) parent[v] = (uint32_t)v;
}

// Root of x without writes.
__device__ __forceinline__ uint32_t uf_root(const uint32_t* parent, uint32_t x) {
    for (;;) {
        const uint32_t px = __ldcg(parent + x);
        if (px == x) return x;
        x = px;
    }
}

// label[v] = root of v.  Only roots are written here: a path-halving store
// (which writes an ancestor that need not be the root) could land after the
// owner of that entry stored its root and leave a non-root label behind.
static __global__ void k_compress(uint32_t* parent, uint32_t n) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = tid; v < n; v += nt) {
        const uint32_t r = uf_root(parent, (uint32_t)v);
        __stcg(parent + v, r);
    }
}

// Sum of out-degrees of vertices with a finite value (the TEPS numerator).
static __global__ void k_reached_edges(const uint32_t* state, const uint64_t* off, uint32_t n,
                                unsigned long long* out) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (uint64_t v = tid; v < n; v += nt)
        if (state[v] != INF) acc += off[v + 1] - off[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

}  // namespace dev
}  // namespace emogi
