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
    const uint64_t* off = nullptr;       // row offsets (GPU memory)
    const void* cols = nullptr;          // edge list of uint64 or uint32 ids (GPU, pinned host or managed)
    const uint32_t* w = nullptr;         // weights beside the edges, or null
    uint32_t shift = 0;                  // (edge-list base address mod 128) / bytes per id
    const uint32_t* in_q = nullptr;      // active vertices, or null for "all vertices"
    const uint32_t* in_count = nullptr;  // number of active vertices (when in_q != null)
    uint32_t all_n = 0;                  // number of vertices (when in_q == null)
    uint32_t* out_q = nullptr;           // next active vertices
    uint32_t* out_count = nullptr;
    uint32_t* lq_v = nullptr;                      // split-list queue: vertex
    unsigned long long* lq_base = nullptr;         // split-list queue: first work item
    unsigned long long* lq_state = nullptr;        // split-list queue: the vertex's begin() value
    unsigned long long* large = nullptr;           // (slots << 34) | items
    uint32_t large_lines = 0xFFFFFFFFu;  // lists with more lines than this are split
    uint32_t chunk_lines = 1;            // lines per split work item
    unsigned long long* scanned = nullptr;         // neighbour entries read (statistics)
    const uint32_t* heads = nullptr;     // first kHeads ids of every list in GPU memory, or null
    const uint32_t* short_off = nullptr; // short-list store: start of v's list / 4, or null
    const uint32_t* short_ids = nullptr;
    const uint32_t* short_w = nullptr;   // its weights (weighted graphs), or null
    uint32_t short_max = 0;              // longest list the store holds
    uint32_t block_slices = 0;           // 1: each block walks its own contiguous slice of in_q
    unsigned long long* scanned_heads = nullptr;  // entries read from the store instead of the edge list
    uint64_t m = 0;                      // entries in the edge list (and weights): a lane's 16-byte
                                         // load at index j is whole when j + ids per load <= m
    uint32_t qcap = 0xFFFFFFFFu;         // entries out_q holds: an append at or past it is dropped
                                         // while the count still grows, so the host sees count > qcap
};

// Entries of each list mirrored in GPU memory ("list heads", INF-padded).
constexpr int kHeads = 4;


// ------------------------------------------------------------------ loads
// Edge-list reads go through the non-coherent read-only path and do not
// allocate in L1: every line is used once per sweep.  They are volatile so
// that they issue where they are written, all of a lane's loads of a batch
// before its first neighbour read: left free, the compiler sinks a weight
// load to its use after the neighbour reads (fewer live registers), which
// adds a second host-link round trip to every step (measured on GB300: the
// largest SSSP sweep from host memory 11.8 -> 18.2 ms).
//
// Ids are uint64 (the paper's main format) or uint32 (the 4-byte edge list
// of Sec. 5.4, 32 ids per 128-byte line as Sec. 4.1 counts them, which halves
// the link bytes of an id); either way a
// lane reads 16 bytes per step: two 8-byte or four 4-byte ids, plus the same
// number of 4-byte weights.  Vertex ids are below 2^32 in both formats, so
// the loaded ids are narrowed to uint32 at once.
template <class Id> struct IdWidth;
template <> struct IdWidth<uint64_t> {
    static constexpr int kPerStep = 2;   // ids per 16-byte lane load
    static constexpr int kPerLine = 16;  // ids per 128-byte line
};
template <> struct IdWidth<uint32_t> {
    static constexpr int kPerStep = 4;
    static constexpr int kPerLine = 32;
};

__device__ __forceinline__ ulonglong2 ld_edge2(const uint64_t* p) {
    ulonglong2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
                 : "=l"(r.x), "=l"(r.y)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint64_t ld_edge(const uint64_t* p) {
    uint64_t r;
    asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_w2(const uint32_t* p) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint4 ld_u32x4(const uint32_t* p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_w(const uint32_t* p) {
    uint32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// One id at index i of an edge list of Id.
template <class Id>
__device__ __forceinline__ uint32_t ld_id(const void* cols, uint64_t i) {
    if constexpr (sizeof(Id) == 8) return (uint32_t)ld_edge((const uint64_t*)cols + i);
    else return ld_w((const uint32_t*)cols + i);
}

// The ids at [j, j + kPerStep), j a multiple of kPerStep: one 16-byte vector
// load.
template <class Id>
__device__ __forceinline__ void ld_ids(const void* cols, uint64_t j, uint32_t* id) {
    if constexpr (sizeof(Id) == 8) {
        const ulonglong2 r = ld_edge2((const uint64_t*)cols + j);
        id[0] = (uint32_t)r.x;
        id[1] = (uint32_t)r.y;
    } else {
        const uint4 r = ld_u32x4((const uint32_t*)cols + j);
        id[0] = r.x;
        id[1] = r.y;
        id[2] = r.z;
        id[3] = r.w;
    }
}
// First index the aligned read starts from: the largest index <= s whose
// address is on a 128-byte boundary (the listing "Coalesced Memory Access
// (Merged + Aligned)" masks the low index bits: four for 8-byte ids, five
// for 4-byte ids; `shift` accounts for an edge list whose base is not itself
// line aligned).  Never below 0; always a multiple of kPerStep, so 16-byte
// vector loads stay aligned.
template <class Id = uint64_t>
__device__ __forceinline__ uint64_t aligned_start(uint64_t s, uint32_t shift) {
    const uint64_t r = (s + shift) & (uint64_t)(IdWidth<Id>::kPerLine - 1);
    return s >= r ? s - r : 0;
}

// ------------------------------------------------------------------ queue push
// Warp-aggregated append: the lanes that push at the same time share one
// atomicAdd on the counter.  A slot at or past `cap` is not written (the
// count still records it, which the host reports).
__device__ __forceinline__ void push(uint32_t* q, uint32_t* count, uint32_t cap, uint32_t v) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    if ((uint64_t)base + rank < cap) q[base + rank] = v;
}

// Append a long list to the split-list queue: one 64-bit atomic hands out both
// the slot and the first work item, so bases increase with slot numbers.
__device__ __forceinline__ void defer(const Sweep& c, uint32_t v, unsigned long long items,
                                     unsigned long long st) {
    unsigned long long old = atomicAdd(c.large, (1ull << SLOT_SHIFT) | items);
    unsigned long long slot = old >> SLOT_SHIFT;
    c.lq_v[slot] = v;
    c.lq_base[slot] = old & CHUNK_MASK;
    c.lq_state[slot] = st;
}

// ------------------------------------------------------------------ applications
// The per-neighbour work of a sweep is a policy object.  Each thread works on
// its own copy, so a policy may keep per-thread accumulators.
//   S, kSkip       the per-vertex value type broadcast to the lanes reading a
//                  list, and the value meaning "do not read this list";
//   begin(v)       one lane per active vertex, before the list is read: returns
//                  that value (a split list's items reuse it);
//   visit(st,v,u,w) the update for edge (v, u) with weight w; true = push u to
//                  the next frontier;
//   flush()        once per thread at kernel end, whole warp converged.

// Warp-reduced atomic add of a per-thread count (whole warp converged).
__device__ __forceinline__ void warp_atomic_add(unsigned long long* out, unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(out, x);
}

// BFS (Sec. 2.1): an unvisited neighbour gets the next level and becomes active.
// The compare-and-swap makes exactly one visitor push it.  When `off` is set,
// the out-degrees of the vertices pushed are summed into `fedges` (the edge
// count of the next frontier, which picks the direction of the next level).
// kBits: the next frontier is a flag byte per vertex (`nflag`) that a
// compaction turns into the next queue in vertex order (k_compact_flags);
// otherwise visitors append to the queue directly.
template <bool kBits>
struct BfsOpT {
    uint32_t* level;
    uint32_t next;
    const uint64_t* off = nullptr;
    unsigned long long* fedges = nullptr;
    unsigned long long lf = 0;
    uint8_t* nflag = nullptr;
    using S = uint32_t;
    static constexpr S kSkip = INF;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = !kBits;
    static constexpr int kSteps = 4;
    static constexpr bool kPeek = true;
    __device__ __forceinline__ S begin(uint32_t) { return 0; }
    __device__ __forceinline__ uint32_t peek(uint64_t u) const { return level[(uint32_t)u]; }
    __device__ __forceinline__ bool visit(S, uint32_t, uint64_t u, uint32_t, uint32_t cur) {
        uint32_t* p = level + (uint32_t)u;
        if (cur != INF) return false;
        if (atomicCAS(p, INF, next) != INF) return false;
        if (off) lf += off[(uint32_t)u + 1] - off[(uint32_t)u];
        if (kBits) {
            nflag[(uint32_t)u] = 1;  // the CAS made this visitor the only one
            return false;
        }
        return true;
    }
    __device__ __forceinline__ void flush() {
        if (fedges) warp_atomic_add(fedges, lf);
    }
};
using BfsOp = BfsOpT<false>;
using BfsBitsOp = BfsOpT<true>;

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
//   qround: the sweep a vertex is queued for.  An improvement in sweep r
//     queues its vertex for sweep r + 1 unless an earlier improvement in the
//     same sweep already did (atomicMax returns the previous stamp).  A vertex
//     that is being expanded in sweep r and improved meanwhile is therefore
//     always queued again, whichever distance its expansion read, and no
//     ordering between the distance and the stamp is needed.
//   fflag: "in the far pile".  The pile is a flag per vertex, set with a
//     plain store; the split kernel scans all flags.  (A queue needed an
//     atomic exchange plus an append on one shared counter per vertex sent
//     to the pile.)
//   nflag: the next near frontier as a flag byte per vertex (a plain store:
//     the stamp already picked one improver per sweep); after the sweep a
//     compaction kernel turns it into the next queue in vertex order, so that
//     the next sweep reads its lists in address order (see k_compact_flags).
//   xd: the distance v was last expanded with, so a vertex queued twice
//     (near and far) is not expanded twice with the same distance.
//   Th: long lists (more than kHeavyEntries entries) are expanded only when
//     their distance is below Th, the start of the window plus a fraction of
//     its width; a long-listed vertex of the near frontier at or above Th
//     goes back to the far pile.  A vertex that many short paths reach
//     (the hubs of a skewed graph) is improved several times inside a wide
//     window, and each improvement re-reads its whole list; a narrow window
//     for long lists only keeps those re-reads rare while short lists keep
//     the wide window's few rounds.  Measured on GB300, Kronecker scale 24
//     (hubs of 400 k entries) from host memory: re-expansion 2.49x -> 1.19x,
//     84 -> 46 ms; no effect on graphs without long lists.
//   kFlags: the next near frontier goes to `nflag` (compacted in vertex order)
//     instead of the sweep's queue; for edge lists larger than the GPU's
//     address translations cover (the compaction costs a scan of n bytes per
//     sweep, 1.5 % of SSSP on a 6.4 GB graph that does not need it).
constexpr uint32_t kHeavyEntries = 512;
template <bool kFlags>
struct SsspOpT {
    uint32_t* dist;
    uint32_t* qround;
    uint32_t* fflag;
    uint32_t* xd;
    uint32_t* far_min;
    uint32_t* overflow;
    uint32_t T;
    uint32_t round;
    uint32_t lmin;  // per-thread smallest distance sent to the far pile
    const uint64_t* off = nullptr;  // row offsets (for the list length of a vertex at or above Th)
    uint32_t Th = INF;
    uint8_t* nflag = nullptr;       // next near frontier
    using S = uint32_t;
    static constexpr S kSkip = INF;
    static constexpr bool kWeights = true;
    static constexpr bool kPush = !kFlags;
    static constexpr int kSteps = 1;
    __device__ __forceinline__ S begin(uint32_t v) {
        const uint32_t d = __ldcg(dist + v);
        if (d >= __ldcg(xd + v)) return INF;  // already expanded with this distance
        if (d >= Th && off[v + 1] - off[v] > kHeavyEntries) {  // a long list waits for a narrower window
            lmin = d < lmin ? d : lmin;
            fflag[v] = 1u;
            return INF;
        }
        __stcg(xd + v, d);
        return d;
    }
    // A relaxation whose sum does not fit below INF is dropped and noted; the
    // host then checks whether some reachable vertex was left at INF.
    static constexpr bool kPeek = true;
    __device__ __forceinline__ uint32_t peek(uint64_t u) const { return dist[(uint32_t)u]; }
    __device__ __forceinline__ bool visit(uint32_t dv, uint32_t, uint64_t u64, uint32_t w, uint32_t cur) {
        const uint32_t u = (uint32_t)u64;
        const uint64_t nd64 = (uint64_t)dv + (uint64_t)w;
        if (nd64 >= (uint64_t)INF) {
            if (dv != INF) atomicExch(overflow, 1u);
            return false;
        }
        const uint32_t nd = (uint32_t)nd64;
        uint32_t* p = dist + u;
        if (nd >= cur) return false;  // cur may be stale, but only ever larger than the true value
        const uint32_t old = atomicMin(p, nd);
        if (nd >= old) return false;
        if (nd < T) {
            const bool fresh = atomicMax(qround + u, round + 1) < round + 1;
            if (!kFlags) return fresh;
            if (fresh) nflag[u] = 1;
            return false;
        }
        lmin = nd < lmin ? nd : lmin;
        fflag[u] = 1u;  // idempotent: the split scans the flags, no queue to append to
        return false;
    }
    // The relaxations of one load step (N entries of a lane) taken together:
    // every improving entry's atomicMin is issued before any result is used,
    // then the round stamps of those that improved, so a lane waits for two
    // L2 round trips per step rather than two per entry.  Same outcome as N
    // calls of visit() in entry order: atomics on one address stay in program
    // order, and min / max commute across addresses.
#ifndef EMOGI_SSSP_BATCHED_RELAX
#define EMOGI_SSSP_BATCHED_RELAX 1
#endif
    static constexpr bool kVisitN = EMOGI_SSSP_BATCHED_RELAX != 0;
    template <int N>
    __device__ __forceinline__ void visit_n(uint32_t dv, const uint32_t (&u)[N], const uint32_t (&w)[N],
                                            const uint32_t (&cur)[N], uint32_t valid, bool (&push)[N]) {
        uint32_t nd[N];
        bool go[N];
#pragma unroll
        for (int i = 0; i < N; i++) {
            const uint64_t nd64 = (uint64_t)dv + (uint64_t)w[i];
            const bool in = (valid >> i) & 1u;
            if (in && nd64 >= (uint64_t)INF && dv != INF) atomicExch(overflow, 1u);
            nd[i] = (uint32_t)nd64;
            go[i] = in && nd64 < (uint64_t)INF && nd[i] < cur[i];
        }
        uint32_t old[N];
#pragma unroll
        for (int i = 0; i < N; i++) old[i] = go[i] ? atomicMin(dist + u[i], nd[i]) : 0u;
        bool near[N];
#pragma unroll
        for (int i = 0; i < N; i++) {
            const bool better = go[i] && nd[i] < old[i];
            near[i] = better && nd[i] < T;
            if (better && !near[i]) {
                lmin = nd[i] < lmin ? nd[i] : lmin;
                fflag[u[i]] = 1u;
            }
        }
        uint32_t stamp[N];
#pragma unroll
        for (int i = 0; i < N; i++) stamp[i] = near[i] ? atomicMax(qround + u[i], round + 1) : round + 1;
#pragma unroll
        for (int i = 0; i < N; i++) {
            const bool fresh = near[i] && stamp[i] < round + 1;
            if (kFlags && fresh) nflag[u[i]] = 1;
            push[i] = !kFlags && fresh;
        }
    }
    __device__ __forceinline__ void flush() { warp_atomic_min(far_min, lmin); }
};
using SsspOp = SsspOpT<false>;
using SsspFlagsOp = SsspOpT<true>;

// Multi-source BFS over up to 64 sources at once: bit b of a vertex's masks
// belongs to source b.  One read of a list serves every source whose frontier
// holds the vertex: the neighbour gains the frontier bits it has not been
// visited by (visit is fixed during a sweep), collected with an atomic OR; the
// first OR that lands on an empty mask queues the neighbour (through the
// next-frontier flags, compacted in vertex order).
struct MsBfsOp {
    unsigned long long* front;
    const unsigned long long* seen;  // visit masks
    unsigned long long* next;
    uint8_t* nflag;                  // newly reached vertices (compacted into the queue in vertex order)
    using S = unsigned long long;
    static constexpr S kSkip = 0ull;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    static constexpr int kSteps = 4;
    __device__ __forceinline__ S begin(uint32_t v) {
        const S f = front[v];
        if (f) front[v] = 0ull;  // each vertex is queued once per sweep
        return f;
    }
    __device__ __forceinline__ bool visit_edge(S f, uint64_t u64) {
        const uint32_t u = (uint32_t)u64;
        const S nb = f & ~seen[u];
        if (!nb) return false;
        if ((next[u] & nb) == nb) return false;  // a stale read only shows fewer bits
        if (atomicOr(next + u, nb) == 0ull) nflag[u] = 1;
        return false;
    }
    static constexpr bool kPeek = false;
    __device__ __forceinline__ uint32_t peek(uint64_t) const { return 0; }
    __device__ __forceinline__ bool visit(S f, uint32_t, uint64_t u, uint32_t, uint32_t) { return visit_edge(f, u); }
    __device__ __forceinline__ void flush() {}
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
    using S = uint32_t;
    static constexpr S kSkip = INF;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    static constexpr int kSteps = 1;
    static constexpr bool kPeek = false;
    __device__ __forceinline__ S begin(uint32_t) { return 0; }
    __device__ __forceinline__ uint32_t peek(uint64_t) const { return 0; }
    __device__ __forceinline__ bool visit(S, uint32_t v, uint64_t u64, uint32_t, uint32_t) {
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

// Sampled CC (Afforest, Sutton, Ben-Nun and Barak, IPDPS 2018), final pass:
// vertices already joined to the sampled largest tree (parent == giant) are
// skipped; every other vertex links itself with each of its neighbours, in
// either id order, because its neighbour may have been skipped.  Skipping is
// safe: a skipped vertex's parent pointer already ties it to the giant tree,
// and each edge to a vertex outside that tree is linked from the other end.
struct CcFinalOp {
    uint32_t* parent;
    uint32_t giant;
    using S = uint32_t;
    static constexpr S kSkip = INF;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    static constexpr int kSteps = 1;
    static constexpr bool kPeek = false;
    __device__ __forceinline__ S begin(uint32_t v) { return __ldcg(parent + v) == giant ? kSkip : 0u; }
    __device__ __forceinline__ uint32_t peek(uint64_t) const { return 0; }
    __device__ __forceinline__ bool visit(S, uint32_t v, uint64_t u64, uint32_t, uint32_t) {
        uint32_t a = v, b = (uint32_t)u64;
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

// Union of a and b (larger root under the smaller).
__device__ __forceinline__ void uf_union(uint32_t* parent, uint32_t a, uint32_t b) {
    for (;;) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        const uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
        if (atomicCAS(parent + hi, hi, lo) == hi) return;
    }
}

// SSSP overflow check, run only when some relaxation overflowed: an edge from
// a vertex with a finite distance to one left at INF means that neighbour is
// reachable but its shortest distance does not fit below UINT32_MAX.
struct OverflowCheckOp {
    const uint32_t* dist;
    uint32_t* found;
    using S = uint32_t;
    static constexpr S kSkip = INF;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    static constexpr int kSteps = 1;
    static constexpr bool kPeek = false;
    __device__ __forceinline__ S begin(uint32_t v) { return __ldcg(dist + v); }
    __device__ __forceinline__ uint32_t peek(uint64_t) const { return 0; }
    __device__ __forceinline__ bool visit(S dv, uint32_t, uint64_t u, uint32_t, uint32_t) {
        if (dv != INF && __ldcg(dist + (uint32_t)u) == INF) atomicExch(found, 1u);
        return false;
    }
    __device__ __forceinline__ void flush() {}
};

// ------------------------------------------------------------------ statistics
__device__ __forceinline__ void add_scanned(const Sweep& c, unsigned long long x, unsigned long long xh = 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        xh += __shfl_xor_sync(0xffffffffu, xh, o);
    }
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(c.scanned, x);
    if ((threadIdx.x & 31) == 0 && xh && c.scanned_heads) atomicAdd(c.scanned_heads, xh);
}

// One 16-byte step of a list read: the lane covers ids [j, j + E) of [s, e),
// E = kPerStep.  Loading and visiting are split so that a lane can issue
// several steps' loads before it waits on the first (more 16-byte requests in
// flight).  The two widths are written out separately (a pair of uint64 ids,
// a quad of uint32 ids) rather than as loops over E: the loop form compiled
// to code that was 50 % slower from host memory on GB300 (the largest SSSP
// sweep 11.8 -> 18.2 ms) with the same loads and updates.
struct PairLoad {
    ulonglong2 id;
    uint2 w;
    uint32_t valid;  // bit 0: id j, bit 1: id j + 1
};
struct QuadLoad {
    uint4 id;
    uint4 w;
    uint32_t valid;  // bit i: id j + i
};
template <class Id> struct StepOf { using T = PairLoad; };
template <> struct StepOf<uint32_t> { using T = QuadLoad; };

// A list's last load, which may hold ids of the next list, is a whole
// 16-byte load (its extra ids masked off) unless it would pass the end of the
// edge list.  Element loads there cost up to three more requests per lane,
// and some fetched a host sector a second time (measured on GB300, uniform
// degree 32 from host memory: SSSP link bytes per algorithmic byte 1.188 ->
// 1.135; SSSP 42.65 -> 40.6 ms with uint64 ids, 37.1 -> 30.1 ms with uint32).
#ifndef EMOGI_WHOLE_TAIL_LOADS
#define EMOGI_WHOLE_TAIL_LOADS 1
#endif
template <class Op>
__device__ __forceinline__ PairLoad load_pair(const Sweep& c, uint64_t j, uint64_t s, uint64_t e, bool active) {
    const uint64_t* cols = (const uint64_t*)c.cols;
    PairLoad p;
    p.id = make_ulonglong2(0, 0);
    p.w = make_uint2(0, 0);
    p.valid = 0;
    if (active && j + 1 >= s) {
        if (j + 1 < e || (EMOGI_WHOLE_TAIL_LOADS && j < e && j + 2 <= c.m)) {
            p.id = ld_edge2(cols + j);
            if (Op::kWeights) p.w = ld_w2(c.w + j);
            p.valid = (j >= s ? 1u : 0u) | (j + 1 < e ? 2u : 0u);
        } else if (j < e && j >= s) {
            p.id.x = ld_edge(cols + j);
            if (Op::kWeights) p.w.x = ld_w(c.w + j);
            p.valid = 1u;
        }
    }
    return p;
}

template <class Op>
__device__ __forceinline__ QuadLoad load_quad(const Sweep& c, uint64_t j, uint64_t s, uint64_t e, bool active) {
    const uint32_t* cols = (const uint32_t*)c.cols;
    QuadLoad p;
    p.id = make_uint4(0, 0, 0, 0);
    p.w = make_uint4(0, 0, 0, 0);
    p.valid = 0;
    if (active && j + 3 >= s && j < e) {
        if (j + 3 < e || (EMOGI_WHOLE_TAIL_LOADS && j + 4 <= c.m)) {
            p.id = ld_u32x4(cols + j);
            if (Op::kWeights) p.w = ld_u32x4(c.w + j);
            p.valid = (j >= s ? 1u : 0u) | (j + 1 >= s && j + 1 < e ? 2u : 0u) | (j + 2 >= s && j + 2 < e ? 4u : 0u) |
                      (j + 3 < e ? 8u : 0u);
        } else {  // the last load of the whole edge list: element loads, nothing read at or past m
            if (j >= s) {
                p.id.x = ld_w(cols + j);
                if (Op::kWeights) p.w.x = ld_w(c.w + j);
                p.valid |= 1u;
            }
            if (j + 1 >= s && j + 1 < e) {
                p.id.y = ld_w(cols + j + 1);
                if (Op::kWeights) p.w.y = ld_w(c.w + j + 1);
                p.valid |= 2u;
            }
            if (j + 2 >= s && j + 2 < e) {
                p.id.z = ld_w(cols + j + 2);
                if (Op::kWeights) p.w.z = ld_w(c.w + j + 2);
                p.valid |= 4u;
            }
        }
    }
    return p;
}

template <class Op, class Id>
__device__ __forceinline__ typename StepOf<Id>::T load_step(const Sweep& c, uint64_t j, uint64_t s, uint64_t e,
                                                             bool active) {
    if constexpr (sizeof(Id) == 8) return load_pair<Op>(c, j, s, e, active);
    else return load_quad<Op>(c, j, s, e, active);
}

// Whole lists of at most short_max entries are read from the short-list store
// in GPU memory (ids, and weights when the op reads them) instead of the edge
// list, in the same steps a list read makes, so peek and visit are unchanged.
// Where an edge list sits in host memory, a sweep over a sparse frontier (a
// few of every hundred vertices, most of them of low degree, spread over the
// whole array) lands each list read on a different part of the array, and the
// GPU's address translations of a 100 GB array then bound it, not the link:
// measured on GB300, Kronecker scale 27 (67 GB of ids + 33 GB of weights),
// such SSSP sweeps read 7.5 GB/s while dense ones read 164 GB/s.  Short lists
// are most of those reads.  A store list starts on a 4-entry boundary, so a
// lane's two or four entries are one 8- or 16-byte load.
template <class Op>
__device__ __forceinline__ bool reads_store(const Sweep& c, uint64_t s, uint64_t e) {
    return c.short_off && (!Op::kWeights || c.short_w) && e > s && e - s <= (uint64_t)c.short_max;
}
template <class Op, class Id>
__device__ __forceinline__ typename StepOf<Id>::T store_step(const Sweep& c, uint32_t v, uint32_t j, uint32_t len,
                                                              bool active) {
    typename StepOf<Id>::T p;
    p.valid = 0;
    const uint64_t b = (uint64_t)c.short_off[v] * 4 + j;  // j: the lane's first entry, a multiple of E
    if constexpr (sizeof(Id) == 8) {
        p.id = make_ulonglong2(0, 0);
        p.w = make_uint2(0, 0);
        if (active && j < len) {
            const uint2 id = *reinterpret_cast<const uint2*>(c.short_ids + b);
            p.id = make_ulonglong2(id.x, id.y);
            if (Op::kWeights) p.w = *reinterpret_cast<const uint2*>(c.short_w + b);
            p.valid = 1u | (j + 1 < len ? 2u : 0u);
        }
    } else {
        p.id = make_uint4(0, 0, 0, 0);
        p.w = make_uint4(0, 0, 0, 0);
        if (active && j < len) {
            p.id = *reinterpret_cast<const uint4*>(c.short_ids + b);
            if (Op::kWeights) p.w = *reinterpret_cast<const uint4*>(c.short_w + b);
            const uint32_t k = len - j < 4 ? len - j : 4;
            p.valid = (1u << k) - 1u;
        }
    }
    return p;
}

// The neighbours' current values (level, distance) a step's updates compare
// against, read before any update so that all of a lane's reads are in
// flight together rather than one after another.
template <class Op>
__device__ __forceinline__ uint2 peek_step(const Op& op, const PairLoad& p) {
    uint2 cur = make_uint2(0, 0);
    if (Op::kPeek) {
        if (p.valid & 1u) cur.x = op.peek(p.id.x);
        if (p.valid & 2u) cur.y = op.peek(p.id.y);
    }
    return cur;
}
template <class Op>
__device__ __forceinline__ uint4 peek_step(const Op& op, const QuadLoad& p) {
    uint4 cur = make_uint4(0, 0, 0, 0);
    if (Op::kPeek) {
        if (p.valid & 1u) cur.x = op.peek(p.id.x);
        if (p.valid & 2u) cur.y = op.peek(p.id.y);
        if (p.valid & 4u) cur.z = op.peek(p.id.z);
        if (p.valid & 8u) cur.w = op.peek(p.id.w);
    }
    return cur;
}
template <class Id> struct CurOf { using T = uint2; };
template <> struct CurOf<uint32_t> { using T = uint4; };

// Per-warp staging of queue appends in shared memory: a warp collects the ids
// it pushes and appends them to the global queue with one atomicAdd (and one
// coalesced copy) per buffer, instead of one atomicAdd per warp and step on
// the single queue counter, which every warp of a dense level contends for.
constexpr int kWarpBuf = 256;
struct WarpQ {
    uint32_t* buf;  // this warp's kWarpBuf entries of shared memory
    uint32_t cnt;   // entries held (the same in every lane)
};

// Appends the held entries (whole warp, converged).  Slots at or past `cap`
// are not written; the count still records them, which the host reports.
__device__ __forceinline__ void warpq_flush(WarpQ& wq, uint32_t* q, uint32_t* count, uint32_t cap) {
    if (wq.cnt == 0) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(count, wq.cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    for (uint32_t i = lane; i < wq.cnt; i += 32)
        if ((uint64_t)base + i < cap) q[base + i] = wq.buf[i];
    __syncwarp();
    wq.cnt = 0;
}

// Stages up to four ids per lane (whole warp, converged); the slots come from
// ballot prefix counts.
__device__ __forceinline__ void warpq_push4(WarpQ& wq, uint32_t* q, uint32_t* count, uint32_t cap, bool p0, bool p1,
                                            bool p2, bool p3, uint4 id) {
    const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
    const unsigned b2 = __ballot_sync(0xffffffffu, p2), b3 = __ballot_sync(0xffffffffu, p3);
    const uint32_t n0 = __popc(b0), n1 = __popc(b1), n2 = __popc(b2);
    const uint32_t total = n0 + n1 + n2 + __popc(b3);
    if (total == 0) return;
    if (wq.cnt + total > (uint32_t)kWarpBuf) warpq_flush(wq, q, count, cap);
    const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
    uint32_t* b = wq.buf + wq.cnt;
    if (p0) b[__popc(b0 & below)] = id.x;
    if (p1) b[n0 + __popc(b1 & below)] = id.y;
    if (p2) b[n0 + n1 + __popc(b2 & below)] = id.z;
    if (p3) b[n0 + n1 + n2 + __popc(b3 & below)] = id.w;
    wq.cnt += total;
}

// Ops with a batched visit (visit_n) declare kVisitN.
template <class Op, class = void> struct HasVisitN { static constexpr bool value = false; };
template <class Op> struct HasVisitN<Op, decltype((void)Op::kVisitN)> { static constexpr bool value = Op::kVisitN; };

template <class Op>
__device__ __forceinline__ void visit_step(const Sweep& c, Op& op, typename Op::S st, uint32_t v, const PairLoad& p,
                                           uint2 cur, WarpQ& wq) {
    bool p0, p1;
    if constexpr (HasVisitN<Op>::value) {
        const uint32_t u[2] = {(uint32_t)p.id.x, (uint32_t)p.id.y}, w[2] = {p.w.x, p.w.y}, cu[2] = {cur.x, cur.y};
        bool pu[2];
        op.template visit_n<2>(st, u, w, cu, p.valid, pu);
        p0 = pu[0];
        p1 = pu[1];
    } else {
        p0 = (p.valid & 1u) && op.visit(st, v, p.id.x, p.w.x, cur.x);
        p1 = (p.valid & 2u) && op.visit(st, v, p.id.y, p.w.y, cur.y);
    }
    if (Op::kPush)
        warpq_push4(wq, c.out_q, c.out_count, c.qcap, p0, p1, false, false,
                    make_uint4((uint32_t)p.id.x, (uint32_t)p.id.y, 0u, 0u));
}
template <class Op>
__device__ __forceinline__ void visit_step(const Sweep& c, Op& op, typename Op::S st, uint32_t v, const QuadLoad& p,
                                           uint4 cur, WarpQ& wq) {
    bool p0, p1, p2, p3;
    if constexpr (HasVisitN<Op>::value) {
        const uint32_t u[4] = {p.id.x, p.id.y, p.id.z, p.id.w}, w[4] = {p.w.x, p.w.y, p.w.z, p.w.w},
                       cu[4] = {cur.x, cur.y, cur.z, cur.w};
        bool pu[4];
        op.template visit_n<4>(st, u, w, cu, p.valid, pu);
        p0 = pu[0];
        p1 = pu[1];
        p2 = pu[2];
        p3 = pu[3];
    } else {
        p0 = (p.valid & 1u) && op.visit(st, v, p.id.x, p.w.x, cur.x);
        p1 = (p.valid & 2u) && op.visit(st, v, p.id.y, p.w.y, cur.y);
        p2 = (p.valid & 4u) && op.visit(st, v, p.id.z, p.w.z, cur.z);
        p3 = (p.valid & 8u) && op.visit(st, v, p.id.w, p.w.w, cur.w);
    }
    if (Op::kPush) warpq_push4(wq, c.out_q, c.out_count, c.qcap, p0, p1, p2, p3, p.id);
}

// Shared-memory staging buffers of the (at most 8) warps of a 256-thread block.
template <class Op>
__device__ __forceinline__ WarpQ warpq_begin() {
    __shared__ uint32_t bufs[Op::kPush ? 8 * kWarpBuf : 1];
    WarpQ wq;
    wq.buf = bufs + (Op::kPush ? (threadIdx.x >> 5) * kWarpBuf : 0);
    wq.cnt = 0;
    return wq;
}

// Steps whose loads (and neighbour reads) a lane issues back to back before
// it updates any neighbour: Op::kSteps.  Measured on GB300: 4 helps top-down
// BFS from HBM (uniform degree 32: 8.5 -> 7.6 ms) and the 64-source BFS from
// host memory (Kronecker scale 24: 199 -> 88 ms); for SSSP and CC more steps
// only cost registers (SSSP: 46 -> 91 registers, 5 -> 2 blocks per SM).

// With 4-byte ids a step carries twice the ids, so the same ids in flight
// take half the steps: batches of Op::kSteps / EMOGI_IDS32_STEP_DIV steps
// (measured on GB300, uniform degree 32 from host memory: BFS 3.7 -> 3.4 ms
// with 2 instead of 4 steps of four ids).
#ifndef EMOGI_IDS32_STEP_DIV
#define EMOGI_IDS32_STEP_DIV 2
#endif
template <class Op, class Id>
constexpr int batch_steps() {
    return (IdWidth<Id>::kPerStep == 4 && Op::kSteps >= EMOGI_IDS32_STEP_DIV) ? Op::kSteps / EMOGI_IDS32_STEP_DIV
                                                                               : Op::kSteps;
}

// ------------------------------------------------------------------ kernels
// Merged + aligned expansion with G lanes per vertex (G = 4, 8, 16, 32).
// Loops are warp-uniform: a warp runs as many steps as its longest group.
template <class Op, int G, class Id = uint64_t>
__device__ __forceinline__ void expand_group_body(const Sweep& c, Op& op) {
    constexpr int GPW = 32 / G, E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
    constexpr int KS = batch_steps<Op, Id>();
    WarpQ wq = warpq_begin<Op>();
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    // Which queue entries a group takes: by default the whole grid strides
    // over the queue, so a group's successive lists lie nwarps * GPW entries
    // apart.  With block_slices each block takes one contiguous slice of the
    // queue and its warps stride within it, so that where the queue is in
    // vertex order (runs of it, at least) a block's successive list reads stay
    // close in the address space.  Measured on GB300 over a 96 GiB pinned host
    // array: random 512-byte reads ran at 19.7 GB/s, the same reads at 4 KiB
    // or 32 KiB spacing walked per block at 203-211 GB/s (the link's peak);
    // beyond 16 GiB of such an array, random reads are bound by the GPU's
    // address translations.
    uint64_t hi = k, first = warp * GPW, stride = nwarps * GPW;
    if (c.block_slices && c.in_q) {
        const uint64_t lo = k * blockIdx.x / gridDim.x;
        hi = k * (blockIdx.x + 1) / gridDim.x;
        first = lo + (threadIdx.x >> 5) * GPW;
        stride = (blockDim.x >> 5) * GPW;
    }
    for (uint64_t base = first; base < hi; base += stride) {
        const uint64_t idx = base + grp;
        uint32_t v = 0;
        typename Op::S st = Op::kSkip;
        if (idx < hi) {
            v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
            if (glane == 0) st = op.begin(v);
        }
        st = __shfl_sync(0xffffffffu, st, grp * G);
        uint64_t s = 0, e = 0;
        if (idx < hi && st != Op::kSkip) {
            s = c.off[v];
            e = c.off[v + 1];
        }
        uint64_t a = aligned_start<Id>(s, c.shift);
        const uint64_t lines = e > s ? (e - a + LINE - 1) / LINE : 0;
        const bool hd = reads_store<Op>(c, s, e);
        if (glane == 0) {
            scanned += e - s;
            if (hd) scanned_h += e - s;
        }
        if (lines > c.large_lines) {
            if (glane == 0) defer(c, v, (lines + c.chunk_lines - 1) / c.chunk_lines, (unsigned long long)st);
            s = e = a = 0;
        }
        const uint64_t from = hd ? s : a;  // a store list starts at its first entry
        const uint32_t steps = e > s ? (uint32_t)((e - from + E * G - 1) / (E * G)) : 0u;
        const uint32_t maxsteps = __reduce_max_sync(0xffffffffu, steps);
        for (uint32_t t0 = 0; t0 < maxsteps; t0 += KS) {
            typename StepOf<Id>::T p[KS];
            typename CurOf<Id>::T cur[KS];
#pragma unroll
            for (int u = 0; u < KS; u++)
                p[u] = hd ? store_step<Op, Id>(c, v, (t0 + u) * (E * G) + E * glane, (uint32_t)(e - s), t0 + u < steps)
                          : load_step<Op, Id>(c, a + (uint64_t)(t0 + u) * (E * G) + E * glane, s, e, t0 + u < steps);
#pragma unroll
            for (int u = 0; u < KS; u++) cur[u] = peek_step(op, p[u]);
#pragma unroll
            for (int u = 0; u < KS; u++) visit_step(c, op, st, v, p[u], cur[u], wq);
        }
    }
    if (Op::kPush) warpq_flush(wq, c.out_q, c.out_count, c.qcap);
    add_scanned(c, scanned, scanned_h);
    op.flush();
}

template <class Op, int G, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_expand_group(Sweep c, Op op_in) {
    Op op = op_in;
    expand_group_body<Op, G, Id>(c, op);
}

// Merged + aligned expansion over all vertices (CC's passes, the SSSP
// overflow check), where begin() skips most vertices: a lane first takes one
// vertex and calls begin() (32 vertices per warp and pass instead of 32/G),
// then the vertices it keeps are read G lanes per list as above.
template <class Op, int G, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_expand_all(Sweep c, Op op_in) {
    Op op = op_in;
    constexpr int GPW = 32 / G, E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
    constexpr int KS = batch_steps<Op, Id>();
    WarpQ wq = warpq_begin<Op>();
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n = c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
        const uint64_t v = base + lane;
        typename Op::S st = Op::kSkip;
        uint64_t s = 0, e = 0;
        if (v < n) st = op.begin((uint32_t)v);
        bool pending = false;
        if (st != Op::kSkip) {
            s = c.off[v];
            e = c.off[v + 1];
            scanned += e - s;
            if (reads_store<Op>(c, s, e)) scanned_h += e - s;
            const uint64_t a = aligned_start<Id>(s, c.shift);
            const uint64_t lines = e > s ? (e - a + LINE - 1) / LINE : 0;
            if (lines > c.large_lines) defer(c, (uint32_t)v, (lines + c.chunk_lines - 1) / c.chunk_lines,
                                             (unsigned long long)st);
            else pending = e > s;
        }
        unsigned pend = __ballot_sync(0xffffffffu, pending);
        while (pend) {
            unsigned rest = pend;
            for (uint32_t i = 0; i < grp && rest; i++) rest &= rest - 1u;  // this group's pending lane
            const int src = rest ? __ffs((int)rest) - 1 : 0;
            const bool mine = rest != 0;
            for (uint32_t i = 0; i < (uint32_t)GPW && pend; i++) pend &= pend - 1u;
            const uint32_t vv = (uint32_t)__shfl_sync(0xffffffffu, v, src);
            const typename Op::S sv = __shfl_sync(0xffffffffu, st, src);
            uint64_t ss = __shfl_sync(0xffffffffu, s, src);
            uint64_t ee = __shfl_sync(0xffffffffu, e, src);
            if (!mine) ss = ee = 0;
            const uint64_t a = aligned_start<Id>(ss, c.shift);
            const bool hd = reads_store<Op>(c, ss, ee);
            const uint32_t steps = ee > ss ? (uint32_t)((ee - (hd ? ss : a) + E * G - 1) / (E * G)) : 0u;
            const uint32_t maxsteps = __reduce_max_sync(0xffffffffu, steps);
            for (uint32_t t0 = 0; t0 < maxsteps; t0 += KS) {
                typename StepOf<Id>::T p[KS];
                typename CurOf<Id>::T cur[KS];
#pragma unroll
                for (int u = 0; u < KS; u++)
                    p[u] = hd ? store_step<Op, Id>(c, vv, (t0 + u) * (E * G) + E * glane, (uint32_t)(ee - ss),
                                                   t0 + u < steps)
                              : load_step<Op, Id>(c, a + (uint64_t)(t0 + u) * (E * G) + E * glane, ss, ee,
                                                  t0 + u < steps);
#pragma unroll
                for (int u = 0; u < KS; u++) cur[u] = peek_step(op, p[u]);
#pragma unroll
                for (int u = 0; u < KS; u++) visit_step(c, op, sv, vv, p[u], cur[u], wq);
            }
        }
    }
    if (Op::kPush) warpq_flush(wq, c.out_q, c.out_count, c.qcap);
    add_scanned(c, scanned, scanned_h);
    op.flush();
}

// Split lists: work item i of vertex lq_v[slot] covers lines
// [i * chunk_lines, (i + 1) * chunk_lines) of its aligned list.  The items of
// all split lists (in slot order) are cut into one contiguous run per warp: a
// warp finds the slot of its first item once (binary search over the slots'
// first items) and then walks on item by item and list by list, 16 bytes per
// lane and step (32 lanes: four 128-byte lines), with kSplitSteps steps of
// loads in flight before their neighbours are read and updated.  Lists above
// 32 lines hold most of the edges of a skewed graph (Kronecker scale 22,
// edge factor 32: 72 %), so this path carries most of its link traffic; a
// warp per item with a search of its own and one step in flight left it
// latency-bound.
#ifndef EMOGI_SPLIT_STEPS
#define EMOGI_SPLIT_STEPS 4
#endif
constexpr int kSplitSteps = EMOGI_SPLIT_STEPS;
#ifndef EMOGI_SPLIT_RUNS
#define EMOGI_SPLIT_RUNS 1
#endif

#if !EMOGI_SPLIT_RUNS
template <class Op, class Id = uint64_t>
__device__ __forceinline__ void expand_split_body(const Sweep& c, Op& op) {
    constexpr int E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
    constexpr int KS = batch_steps<Op, Id>();
    WarpQ wq = warpq_begin<Op>();
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
        const uint64_t a = aligned_start<Id>(s, c.shift);
        const uint64_t cs = a + ci * (uint64_t)LINE * c.chunk_lines;
        uint64_t ce = cs + (uint64_t)LINE * c.chunk_lines;
        if (ce > e) ce = e;
        const typename Op::S st = (typename Op::S)c.lq_state[lo];
        for (uint64_t j0 = cs; j0 < ce; j0 += 32 * E * KS) {
            typename StepOf<Id>::T p[KS];
            typename CurOf<Id>::T cur[KS];
#pragma unroll
            for (int u = 0; u < KS; u++) p[u] = load_step<Op, Id>(c, j0 + 32 * E * u + E * lane, s, ce, true);
#pragma unroll
            for (int u = 0; u < KS; u++) cur[u] = peek_step(op, p[u]);
#pragma unroll
            for (int u = 0; u < KS; u++) visit_step(c, op, st, v, p[u], cur[u], wq);
        }
    }
    if (Op::kPush) warpq_flush(wq, c.out_q, c.out_count, c.qcap);
    op.flush();
}
#else
template <class Op, class Id = uint64_t>
__device__ __forceinline__ void expand_split_body(const Sweep& c, Op& op) {
    constexpr int E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
    // a step of 4-byte ids carries twice the ids: half the steps in flight
    constexpr int KS = E == 4 && kSplitSteps >= EMOGI_IDS32_STEP_DIV ? kSplitSteps / EMOGI_IDS32_STEP_DIV
                                                                      : kSplitSteps;
    constexpr uint64_t STEP = 32 * E;  // ids per warp step
    WarpQ wq = warpq_begin<Op>();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long tot = *c.large;
    const uint32_t nslots = (uint32_t)(tot >> SLOT_SHIFT);
    const unsigned long long nitems = tot & CHUNK_MASK;
    const unsigned long long per = (nitems + nwarps - 1) / nwarps;
    unsigned long long item = warp * per;
    const unsigned long long iend = item + per < nitems ? item + per : nitems;
    const uint64_t item_ids = (uint64_t)LINE * c.chunk_lines;
    if (item < iend) {  // warp-uniform
        uint32_t lo = 0, hi = nslots;  // last slot whose first item <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (c.lq_base[mid] <= item) lo = mid; else hi = mid;
        }
        uint32_t slot = lo, v = 0;
        typename Op::S st = Op::kSkip;
        uint64_t s = 0, e = 0, a = 0, pos = 0, ce = 0;
        unsigned long long first = 0, slot_end = 0;
        auto open_slot = [&]() {
            v = c.lq_v[slot];
            st = (typename Op::S)c.lq_state[slot];
            s = c.off[v];
            e = c.off[v + 1];
            a = aligned_start<Id>(s, c.shift);
            first = c.lq_base[slot];
            slot_end = slot + 1 < nslots ? c.lq_base[slot + 1] : nitems;
        };
        auto open_item = [&]() {
            pos = a + (item - first) * item_ids;
            ce = pos + item_ids < e ? pos + item_ids : e;
        };
        open_slot();
        open_item();
        bool more = true;
        while (more) {
            typename StepOf<Id>::T p[KS];
            typename CurOf<Id>::T cur[KS];
            uint32_t vs[KS];
            typename Op::S sts[KS];
#pragma unroll
            for (int u = 0; u < KS; u++) {
                vs[u] = v;
                sts[u] = st;
                p[u] = load_step<Op, Id>(c, pos + E * lane, s, ce, more);
                if (more) {
                    pos += STEP;
                    if (pos >= ce) {  // next item, and next list when the item was its last
                        if (++item >= iend) {
                            more = false;
                        } else {
                            if (item >= slot_end) {
                                slot++;
                                open_slot();
                            }
                            open_item();
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < KS; u++) cur[u] = peek_step(op, p[u]);
#pragma unroll
            for (int u = 0; u < KS; u++) visit_step(c, op, sts[u], vs[u], p[u], cur[u], wq);
        }
    }
    if (Op::kPush) warpq_flush(wq, c.out_q, c.out_count, c.qcap);
    op.flush();
}
#endif

template <class Op, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_expand_split(Sweep c, Op op_in) {
    Op op = op_in;
    expand_split_body<Op, Id>(c, op);
}

// Bottom-up BFS sweep (the pull direction of direction-optimising BFS, Beamer,
// Asanovic and Patterson, SC 2012), for undirected graphs: every vertex not yet
// reached looks for a neighbour on level L; it then takes level L + 1 and
// joins the next frontier.  A lane first checks one vertex (coalesced level
// reads) and its list heads in GPU memory, one at a time until a hit; only
// the lists that this leaves undecided are read from the edge list, G lanes
// per list in aligned 16-byte steps, stopping at the first hit.  When most
// vertices are already reached, or most have a parent among their first
// neighbours, this reads little of the edge list.
// Only the owner writes level[v], and a vertex set to L + 1 during this sweep
// never reads as L, so plain accesses suffice.
template <int G, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_bfs_bottom_up(Sweep c, uint32_t* level, uint32_t L,
                                                       unsigned long long* fedges) {
    constexpr int GPW = 32 / G, E = IdWidth<Id>::kPerStep;
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (grp * G);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n = c.all_n;
    unsigned long long scanned = 0, lf = 0;
    // one pass: 32 vertices per warp, one per lane
    for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
        const uint64_t v = base + lane;
        uint64_t s = 0, e = 0;
        bool found = false, pending = false;
        if (v < n && level[v] == INF) {
            s = c.off[v];
            e = c.off[v + 1];
            if (c.heads) {
                // the first kHeads neighbours are mirrored in GPU memory: check
                // them there one by one (the first hit ends it), and leave the
                // rest of the list, read from host memory, to the groups below
                const uint4 h = *reinterpret_cast<const uint4*>(c.heads + v * kHeads);
                const uint64_t k = e - s;
                found = (k > 0 && level[h.x] == L) || (k > 1 && level[h.y] == L) || (k > 2 && level[h.z] == L) ||
                        (k > 3 && level[h.w] == L);
                pending = !found && k > (uint64_t)kHeads;
                s += kHeads;
            } else {
                pending = e > s;
            }
        }
        if (found) {
            level[v] = L + 1;
            lf += e - (c.heads ? s - kHeads : s);
        }
        const unsigned fb = __ballot_sync(0xffffffffu, found);
        if (fb) {  // append the warp's finds in vertex order, one atomic per warp
            uint32_t pos = 0;
            if (lane == 0) pos = atomicAdd(c.out_count, (uint32_t)__popc(fb));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            const uint64_t slot = (uint64_t)pos + __popc(fb & ((1u << lane) - 1u));
            if (found && slot < c.qcap) c.out_q[slot] = (uint32_t)v;
        }
        // lists still undecided: GPW of them at a time, G lanes each, read in
        // aligned 16-byte steps until the first neighbour on level L
        unsigned pend = __ballot_sync(0xffffffffu, pending);
        while (pend) {
            unsigned rest = pend;
            for (uint32_t i = 0; i < grp && rest; i++) rest &= rest - 1u;  // this group's pending lane
            const int src = rest ? __ffs((int)rest) - 1 : 0;
            const bool mine = rest != 0;
            for (uint32_t i = 0; i < (uint32_t)GPW && pend; i++) pend &= pend - 1u;
            const uint64_t vv = __shfl_sync(0xffffffffu, v, src);
            uint64_t ss = __shfl_sync(0xffffffffu, s, src);
            uint64_t ee = __shfl_sync(0xffffffffu, e, src);
            if (!mine) ss = ee = 0;
            const uint64_t s0 = c.heads ? ss - kHeads : ss;
            const uint64_t a = aligned_start<Id>(ss, c.shift);
            const uint32_t steps = ee > ss ? (uint32_t)((ee - a + E * G - 1) / (E * G)) : 0u;
            bool gfound = false;
            for (uint32_t t = 0; __any_sync(0xffffffffu, t < steps && !gfound); t++) {
                bool hit = false;
                if (t < steps && !gfound) {
                    const uint64_t j = a + (uint64_t)t * (E * G) + E * glane;
                    if (j + E - 1 >= ss && j < ee) {
                        uint32_t id[E];
                        if (j + E - 1 < ee || (EMOGI_WHOLE_TAIL_LOADS && j + E <= c.m)) {
                            ld_ids<Id>(c.cols, j, id);
                        } else {
#pragma unroll
                            for (int x = 0; x < E; x++) id[x] = (j + x < ee) ? ld_id<Id>(c.cols, j + x) : 0u;
                        }
#pragma unroll
                        for (int x = 0; x < E; x++) {
                            if (j + x >= ss && j + x < ee) {
                                hit = hit || level[id[x]] == L;
                                scanned += 1;
                            }
                        }
                    }
                }
                // every lane must reach the ballot: evaluate it before combining
                const unsigned hits = __ballot_sync(0xffffffffu, hit);
                gfound = gfound || (hits & gmask) != 0;
            }
            if (mine && gfound && glane == 0) {
                level[vv] = L + 1;
                lf += ee - s0;
                push(c.out_q, c.out_count, c.qcap, (uint32_t)vv);
            }
        }
    }
    add_scanned(c, scanned);
    warp_atomic_add(fedges, lf);
}

// The paper's "Merged" variant: one warp per vertex, lanes read consecutive
// 8-byte entries starting at the list's own first element.
template <class Op, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_expand_merged(Sweep c, Op op_in) {
    Op op = op_in;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    for (uint64_t idx = warp; idx < k; idx += nwarps) {
        const uint32_t v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
        typename Op::S st = Op::kSkip;
        if (lane == 0) st = op.begin(v);
        st = __shfl_sync(0xffffffffu, st, 0);
        if (st == Op::kSkip) continue;
        const uint64_t s = c.off[v], e = c.off[v + 1];
        if (lane == 0) scanned += e - s;
        for (uint64_t i = s + lane; i < e; i += 32) {
            const uint32_t u = ld_id<Id>(c.cols, i);
            const uint32_t w = Op::kWeights ? ld_w(c.w + i) : 0u;
            if (op.visit(st, v, u, w, Op::kPeek ? op.peek(u) : 0u) && Op::kPush)
                push(c.out_q, c.out_count, c.qcap, (uint32_t)u);
        }
    }
    __syncwarp();
    add_scanned(c, scanned, scanned_h);
    op.flush();
}

// The paper's "Naive" variant: one thread per vertex, element by element.
template <class Op, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_expand_naive(Sweep c, Op op_in) {
    Op op = op_in;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t k = c.in_q ? (uint64_t)*c.in_count : (uint64_t)c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    for (uint64_t idx = tid; idx < k; idx += nt) {
        const uint32_t v = c.in_q ? c.in_q[idx] : (uint32_t)idx;
        const typename Op::S st = op.begin(v);
        if (st == Op::kSkip) continue;
        const uint64_t s = c.off[v], e = c.off[v + 1];
        scanned += e - s;
        for (uint64_t i = s; i < e; i++) {
            const uint32_t u = ld_id<Id>(c.cols, i);
            const uint32_t w = Op::kWeights ? ld_w(c.w + i) : 0u;
            if (op.visit(st, v, u, w, Op::kPeek ? op.peek(u) : 0u) && Op::kPush)
                push(c.out_q, c.out_count, c.qcap, (uint32_t)u);
        }
    }
    __syncwarp();
    add_scanned(c, scanned, scanned_h);
    op.flush();
}

// Block-aggregated queue append for kernels whose blocks step through the
// vertex range together: a block collects the ids its threads push in shared
// memory and appends them with one atomicAdd per kBlockBuf/2 ids or so,
// instead of one per warp and pass (every warp of a dense scan pushes, so
// per-warp appends meet on the one queue counter).
constexpr int kBlockBuf = 2048;
struct BlockQueue {
    uint32_t ids[kBlockBuf];
    uint32_t count;
    uint32_t base;
};

// Appends the buffered ids (whole block, converged).  Slots at or past `cap`
// are not written; the count still records them, which the host reports.
__device__ __forceinline__ void block_queue_flush(BlockQueue& bq, uint32_t* q, uint32_t* qcount, uint32_t cap) {
    __syncthreads();
    const uint32_t k = bq.count;
    if (threadIdx.x == 0 && k) bq.base = atomicAdd(qcount, k);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
        if ((uint64_t)bq.base + i < cap) q[bq.base + i] = bq.ids[i];
    __syncthreads();
    if (threadIdx.x == 0) bq.count = 0;
    __syncthreads();
}

// Adds this thread's id if `p` (whole block, converged); flushes first when
// one more pass of the block might not fit.
__device__ __forceinline__ void block_queue_push(BlockQueue& bq, uint32_t* q, uint32_t* qcount, uint32_t cap,
                                                 bool p, uint32_t id) {
    const unsigned b = __ballot_sync(0xffffffffu, p);
    const int lane = threadIdx.x & 31;
    uint32_t slot = 0;
    if (lane == 0 && b) slot = atomicAdd(&bq.count, (uint32_t)__popc(b));  // shared-memory atomic
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (p) bq.ids[slot + __popc(b & ((1u << lane) - 1u))] = id;
    __syncthreads();
    const uint32_t cnt = bq.count;
    __syncthreads();  // every thread has read the count before the next pass adds to it
    if (cnt + blockDim.x > (uint32_t)kBlockBuf) block_queue_flush(bq, q, qcount, cap);
}

// Frontier compaction: appends the vertices whose flag byte is set to q and
// clears the flags.  Each thread takes 16 flags (one 16-byte load); each block
// takes one contiguous range of the flags and stages its ids in shared memory,
// so that the queue is made of runs of up to kBlockBuf ids in vertex order
// (one atomicAdd per run), and a sweep whose blocks each take a slice of the
// queue walks the edge list in address order within each slice.  A sweep
// whose queue came from pushes in arrival order reads its lists at random
// across the whole edge list; once that list exceeds what the GPU's address
// translations cover (tens of GB of host memory), those reads ran 8x slower
// (measured on GB300, uniform 2^26 vertices with 25.8 GB of ids + weights:
// 21 GB/s in arrival order against 160 GB/s in vertex order).  Flags are
// bytes set with plain stores: a bitmap needs an atomic OR per vertex, and on
// a dense BFS level (14 M new vertices into a 2 MB bitmap) those contended.
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t x) {
    const uint32_t m = __vcmpne4(x, 0u);  // 0xff in every non-zero byte
    return ((m >> 7) & 1u) | ((m >> 14) & 2u) | ((m >> 21) & 4u) | ((m >> 28) & 8u);
}

__device__ __forceinline__ void compact_flags_body(uint8_t* flags, uint64_t nchunks, uint32_t* q, uint32_t* count,
                                                   uint32_t cap) {
    __shared__ uint32_t warp_off[32];
    __shared__ uint32_t pass_total, block_base;
    __shared__ BlockQueue bq;
    if (threadIdx.x == 0) bq.count = 0;
    __syncthreads();
    uint4* chunks = reinterpret_cast<uint4*>(flags);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // block b takes one contiguous range of chunks; every thread of a block
    // runs the same number of passes (the bounds are per block)
    const uint64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * per;
    const uint64_t lo = b0 < nchunks ? b0 : nchunks, hi = lo + per < nchunks ? lo + per : nchunks;
    for (uint64_t base = lo; base < hi; base += blockDim.x) {
        const uint64_t ci = base + threadIdx.x;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (ci < hi) w = chunks[ci];
        uint32_t mask = nonzero_bytes(w.x) | (nonzero_bytes(w.y) << 4) | (nonzero_bytes(w.z) << 8) |
                        (nonzero_bytes(w.w) << 12);
        if (mask) chunks[ci] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t c = __popc(mask);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        if (lane == 31) warp_off[wid] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (uint32_t i = 0; i < nw; i++) {
                const uint32_t x = warp_off[i];
                warp_off[i] = tot;
                tot += x;
            }
            pass_total = tot;
        }
        __syncthreads();
        const uint32_t tot = pass_total;
        if (bq.count + tot > (uint32_t)kBlockBuf) block_queue_flush(bq, q, count, cap);  // block-uniform
        const bool direct = tot > (uint32_t)kBlockBuf;  // more than the buffer holds: straight to the queue
        if (direct) {
            if (threadIdx.x == 0) block_base = atomicAdd(count, tot);
            __syncthreads();
        }
        uint32_t pos = (direct ? block_base : bq.count) + warp_off[wid] + incl - c;
        while (mask) {
            const uint32_t b = (uint32_t)__ffs((int)mask) - 1u;
            mask &= mask - 1u;
            const uint32_t id = (uint32_t)(ci * 16u + b);
            if (direct) {
                if (pos < cap) q[pos] = id;
            } else {
                bq.ids[pos] = id;
            }
            pos++;
        }
        __syncthreads();  // warp_off, pass_total and the buffer count are rewritten below / next pass
        if (threadIdx.x == 0 && !direct) bq.count += tot;
        __syncthreads();
    }
    block_queue_flush(bq, q, count, cap);
}

static __global__ void __launch_bounds__(256) k_compact_flags(uint8_t* flags, uint64_t nchunks, uint32_t* q,
                                                              uint32_t* count, uint32_t cap) {
    compact_flags_body(flags, nchunks, q, count, cap);
}

__device__ __forceinline__ void far_split_body(uint32_t n, uint32_t* fflag, const uint32_t* dist, const uint32_t* xd,
                                               uint32_t* qround, uint32_t T, uint32_t round, uint32_t* nq_out,
                                               uint32_t* ncount_out, uint32_t* kept, uint32_t* far_min) {
    __shared__ BlockQueue bq;
    if (threadIdx.x == 0) bq.count = 0;
    __syncthreads();
    uint32_t lmin = INF, lkept = 0;
    // block b takes one contiguous range of vertices, so the near vertices it
    // appends form runs in vertex order (see compact_flags_body); every thread
    // of a block runs the same number of passes (the bounds are per block)
    const uint64_t per = ((uint64_t)n + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * per;
    const uint64_t lo = b0 < n ? b0 : n, hi = lo + per < n ? lo + per : n;
    for (uint64_t base = lo; base < hi; base += blockDim.x) {
        const uint64_t v = base + threadIdx.x;
        bool near = false;
        if (v < hi && fflag[v]) {
            const uint32_t d = dist[v];
            if (d >= xd[v] || qround[v] == round) {
                // already expanded with this distance, or already in the queue:
                // a vertex improved first to a far and then to a near distance
                // in the last sweep is flagged and queued for sweep `round`
                // (the window's tail, which this split appends behind)
                fflag[v] = 0u;
            } else if (d < T) {
                fflag[v] = 0u;
                qround[v] = round;  // queued for the next sweep
                near = true;
            } else {
                lmin = d < lmin ? d : lmin;
                lkept++;
            }
        }
        block_queue_push(bq, nq_out, ncount_out, n, near, (uint32_t)v);
    }
    block_queue_flush(bq, nq_out, ncount_out, n);
    warp_atomic_min(far_min, lmin);
    const uint32_t wk = __reduce_add_sync(0xffffffffu, lkept);
    if ((threadIdx.x & 31) == 0 && wk) atomicAdd(kept, wk);
}

// SSSP far split over all vertices (the near frontier is empty): every
// vertex flagged "far" whose distance is below the new threshold T moves to
// the near frontier of sweep `round`, the others stay flagged (counted in
// *kept); vertices already expanded with their current distance are dropped.
// Nothing else runs meanwhile, so plain updates suffice.
static __global__ void k_far_split(uint32_t n, uint32_t* fflag, const uint32_t* dist, const uint32_t* xd,
                                   uint32_t* qround, uint32_t T, uint32_t round, uint32_t* nq_out,
                                   uint32_t* ncount_out, uint32_t* kept, uint32_t* far_min) {
    far_split_body(n, fflag, dist, xd, qround, T, round, nq_out, ncount_out, kept, far_min);
}

// ------------------------------------------------------------------ device-driven SSSP loop
// The near/far SSSP loop with its decisions on the device: one iteration of a
// CUDA graph's conditional while-node runs the sweep kernels, the far split
// and a one-thread controller; the kernel that is not due this iteration
// returns at once.  No host round trip separates iterations.
struct SsspLoop {
    uint32_t side;        // near frontier parity
    uint32_t mode;        // 0 = sweep next, 1 = far split next, 2 = done
    uint32_t T;           // current threshold
    uint32_t sweeps;      // sweeps run (sweep stamp of the next sweep)
    uint32_t iters;       // sweeps + splits run
    uint32_t delta;       // window width
    uint32_t error;       // 1 = the iteration cap was reached, 2 = the time bound, 3 = a queue count above n
    unsigned long long cap;
    unsigned long long t0, timeout_ns;  // %globaltimer at the first iteration; bound on the loop
    uint32_t* dist;       // this call's distance array
    uint32_t Th;          // long lists wait while their distance is at or above this
    uint32_t delta_heavy; // width of the long lists' part of a window
    unsigned long long tail;  // a sweep leaving fewer near vertices than this splits the far pile at once
    uint32_t qcap;        // entries each frontier queue holds (n)
};

// The long lists' threshold of a window that starts at `lo`.
__host__ __device__ __forceinline__ uint32_t heavy_threshold(uint64_t lo, uint64_t delta_heavy, uint64_t T) {
    const uint64_t th = lo + delta_heavy;
    return (uint32_t)(th < T ? th : T);
}

// Fixed pointers of one graph's SSSP loop (recorded once in the CUDA graph).
struct SsspFixed {
    Sweep base;           // off, cols, w, shift, split-list queue, scanned
    uint32_t* q[2];
    uint32_t* qround;
    uint32_t* fflag;
    uint32_t* xd;
    uint8_t* nflag;       // next near frontier flags
    uint64_t nchunks;     // 16-byte chunks of nflag
};

template <class Ctr, class OpT>
__device__ __forceinline__ void sssp_loop_views(const SsspFixed& f, const SsspLoop& L, Ctr* ctr, Sweep* s,
                                                OpT* op) {
    *s = f.base;
    s->in_q = f.q[L.side];
    s->in_count = &ctr->qcount[L.side];
    s->out_q = f.q[L.side ^ 1];
    s->out_count = &ctr->qcount[L.side ^ 1];
    s->large = &ctr->large[0];
    *op = OpT{L.dist, f.qround, f.fflag, f.xd, &ctr->far_min, &ctr->overflow, L.T, L.sweeps, INF, f.base.off,
                 L.Th, f.nflag};
}

template <class Ctr, int G, class Id, bool kFlags>
__global__ void __launch_bounds__(256) k_sssp_loop_sweep(SsspFixed f, const SsspLoop* Lp, Ctr* ctr) {
    const SsspLoop L = *Lp;
    if (L.mode != 0) return;
    Sweep s;
    SsspOpT<kFlags> op;
    sssp_loop_views(f, L, ctr, &s, &op);
    expand_group_body<SsspOpT<kFlags>, G, Id>(s, op);
}

template <class Ctr, class Id, bool kFlags>
__global__ void __launch_bounds__(256) k_sssp_loop_lists(SsspFixed f, const SsspLoop* Lp, Ctr* ctr) {
    const SsspLoop L = *Lp;
    if (L.mode != 0) return;
    Sweep s;
    SsspOpT<kFlags> op;
    sssp_loop_views(f, L, ctr, &s, &op);
    expand_split_body<SsspOpT<kFlags>, Id>(s, op);
}

template <class Ctr>
__global__ void __launch_bounds__(256) k_sssp_loop_compact(SsspFixed f, const SsspLoop* Lp, Ctr* ctr) {
    const SsspLoop L = *Lp;
    if (L.mode != 0) return;
    compact_flags_body(f.nflag, f.nchunks, f.q[L.side ^ 1], &ctr->qcount[L.side ^ 1], f.base.qcap);
}

template <class Ctr>
__global__ void __launch_bounds__(256) k_sssp_loop_far(SsspFixed f, const SsspLoop* Lp, Ctr* ctr) {
    const SsspLoop L = *Lp;
    if (L.mode != 1) return;
    far_split_body(f.base.all_n, f.fflag, L.dist, f.xd, f.qround, L.T, L.sweeps, f.q[L.side], &ctr->qcount[L.side],
                   &ctr->fcount[0], &ctr->far_min);
}

// One thread: account for the iteration that just ran, pick the next one
// (sweep while the near frontier is non-empty, else split the far pile with
// a raised threshold, else stop), clear the counters it will fill, and set
// the loop condition.
template <class Ctr>
__global__ void k_sssp_loop_control(SsspLoop* Lp, Ctr* ctr, cudaGraphConditionalHandle handle) {
    SsspLoop L = *Lp;
    uint64_t nk = 0;
    // far vertices are pending if the last split kept some or a sweep since
    // sent some (it then lowered far_min below INF)
    const bool far_pending = ctr->fcount[0] > 0 || ctr->far_min != INF;
    const bool after_sweep = L.mode == 0;
    if (L.mode == 0) {
        nk = ctr->qcount[L.side ^ 1];
        L.side ^= 1;
        L.sweeps++;
    } else {
        nk = ctr->qcount[L.side];
    }
    const uint64_t fk = far_pending ? 1 : 0;
    L.iters++;
    unsigned long long now;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(now));
    if (L.t0 == 0) L.t0 = now;
    if (ctr->qcount[0] > L.qcap || ctr->qcount[1] > L.qcap) {
        // appends past a queue's n entries were dropped: stop before a sweep
        // reads the queue (this cannot happen while every vertex is queued at
        // most once per sweep; the check makes a broken invariant an error)
        L.error = 3;
        L.mode = 2;
    } else if (L.iters > L.cap) {
        L.error = 1;
        L.mode = 2;
    } else if (now - L.t0 > L.timeout_ns) {
        L.error = 2;
        L.mode = 2;
    } else if (nk > 0 && !(after_sweep && fk > 0 && nk < L.tail)) {
        L.mode = 0;
        ctr->qcount[L.side ^ 1] = 0;
        ctr->large[0] = 0;
    } else if (fk > 0) {
        // near frontier empty, or down to the window's tail (which stays in
        // the queue; the split appends behind it)
        L.mode = 1;
        uint64_t Tn = (uint64_t)ctr->far_min + (uint64_t)L.delta;
        if (Tn <= L.T) Tn = (uint64_t)L.T + 1;
        L.T = Tn < (uint64_t)INF ? (uint32_t)Tn : INF;
        L.Th = heavy_threshold(ctr->far_min, L.delta_heavy, L.T);
        if (nk == 0) ctr->qcount[L.side] = 0;
        ctr->fcount[0] = 0;
        ctr->far_min = INF;
    } else {
        L.mode = 2;
    }
    *Lp = L;
    __threadfence();
    cudaGraphSetConditional(handle, L.mode != 2 ? 1u : 0u);
}

// ------------------------------------------------------------------ PageRank
// The fourth application of Sec. 5.4: every vertex is active in every
// iteration and the whole edge list is read.  Power iteration in double
// precision: rank'(v) = (1 - d)/n + d * dangling/n + d * sum of contrib(u)
// over the edges u -> v, with contrib(u) = rank(u) / outdeg(u) and dangling
// the rank held by vertices without out-edges.
struct PrCounters {
    double change;        // L1 change of the iteration (sum of |rank' - rank|)
    double dangling[2];   // rank on vertices without out-edges, by iteration parity
    double pad;
};

// List loads without weights, for the PageRank kernels.
struct PrLoads {
    static constexpr bool kWeights = false;
};

template <int E>
__device__ __forceinline__ double pr_sum_step(const double* contrib, const PairLoad& p) {
    double x = 0.0;
    if (p.valid & 1u) x += contrib[(uint32_t)p.id.x];
    if (p.valid & 2u) x += contrib[(uint32_t)p.id.y];
    return x;
}
template <int E>
__device__ __forceinline__ double pr_sum_step(const double* contrib, const QuadLoad& p) {
    double x = 0.0;
    if (p.valid & 1u) x += contrib[p.id.x];
    if (p.valid & 2u) x += contrib[p.id.y];
    if (p.valid & 4u) x += contrib[p.id.z];
    if (p.valid & 8u) x += contrib[p.id.w];
    return x;
}

// Pull form for undirected graphs (a vertex's list is also its in-list):
// acc[v] = sum of contrib over v's list, G lanes per list in aligned 16-byte
// steps, the group's partial sums added by a shuffle tree and stored by its
// first lane; lists longer than large_lines go to the split queue (their
// items add into acc[v], which the previous finalize left at 0).  No atomics
// on the common path.
template <int G, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_pr_pull(Sweep c, const double* contrib, double* acc) {
    constexpr int GPW = 32 / G, E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n = c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    for (uint64_t base = warp * GPW; base < n; base += nwarps * GPW) {
        const uint64_t v = base + grp;
        uint64_t s = 0, e = 0;
        if (v < n) {
            s = c.off[v];
            e = c.off[v + 1];
        }
        uint64_t a = aligned_start<Id>(s, c.shift);
        const uint64_t lines = e > s ? (e - a + LINE - 1) / LINE : 0;
        if (glane == 0) scanned += e - s;
        const bool split = lines > c.large_lines;
        if (split) {
            if (glane == 0) defer(c, (uint32_t)v, (lines + c.chunk_lines - 1) / c.chunk_lines, 0ull);
            s = e = a = 0;
        }
        const uint32_t steps = e > s ? (uint32_t)((e - a + E * G - 1) / (E * G)) : 0u;
        const uint32_t maxsteps = __reduce_max_sync(0xffffffffu, steps);
        double sum = 0.0;
        // the loads of KS steps go out before their contributions are gathered
        constexpr int KS = E == 2 ? 4 : 2;
        for (uint32_t t0 = 0; t0 < maxsteps; t0 += KS) {
            typename StepOf<Id>::T p[KS];
#pragma unroll
            for (int u = 0; u < KS; u++)
                p[u] = load_step<PrLoads, Id>(c, a + (uint64_t)(t0 + u) * (E * G) + E * glane, s, e, t0 + u < steps);
#pragma unroll
            for (int u = 0; u < KS; u++) sum += pr_sum_step<E>(contrib, p[u]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (glane == 0 && v < n && !split) acc[v] = sum;
    }
    add_scanned(c, scanned, scanned_h);
}

// The split lists of k_pr_pull: one warp per item, its sum added into acc[v].
template <class Id = uint64_t>
__global__ void __launch_bounds__(256) k_pr_pull_split(Sweep c, const double* contrib, double* acc) {
    constexpr int E = IdWidth<Id>::kPerStep, LINE = IdWidth<Id>::kPerLine;
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
        const uint64_t a = aligned_start<Id>(s, c.shift);
        const uint64_t cs = a + ci * (uint64_t)LINE * c.chunk_lines;
        uint64_t ce = cs + (uint64_t)LINE * c.chunk_lines;
        if (ce > e) ce = e;
        double sum = 0.0;
        constexpr int KS = E == 2 ? 4 : 2;
        for (uint64_t j0 = cs; j0 < ce; j0 += 32 * E * KS) {
            typename StepOf<Id>::T p[KS];
#pragma unroll
            for (int u = 0; u < KS; u++) p[u] = load_step<PrLoads, Id>(c, j0 + 32 * E * u + E * lane, s, ce, true);
#pragma unroll
            for (int u = 0; u < KS; u++) sum += pr_sum_step<E>(contrib, p[u]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) atomicAdd(acc + v, sum);
    }
}

// Push form for directed graphs (only out-lists are stored): every edge
// v -> u adds contrib(v) into acc[u].  The per-vertex value is the bit
// pattern of contrib(v) (vertices without out-edges are skipped).
struct PrPushOp {
    const double* contrib;
    double* acc;
    using S = unsigned long long;
    static constexpr S kSkip = ~0ull;
    static constexpr bool kWeights = false;
    static constexpr bool kPush = false;
    static constexpr int kSteps = 1;
    static constexpr bool kPeek = false;
    __device__ __forceinline__ S begin(uint32_t v) {
        const double x = contrib[v];
        return x > 0.0 ? (S)__double_as_longlong(x) : kSkip;
    }
    __device__ __forceinline__ uint32_t peek(uint64_t) const { return 0; }
    __device__ __forceinline__ bool visit(S st, uint32_t, uint64_t u, uint32_t, uint32_t) {
        atomicAdd(acc + (uint32_t)u, __longlong_as_double((long long)st));
        return false;
    }
    __device__ __forceinline__ void flush() {}
};

__device__ __forceinline__ double block_sum(double x) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (uint32_t i = 0; i < (blockDim.x >> 5); i++) t += part[i];
    __syncthreads();
    return t;  // valid in thread 0
}

// Iteration 0: rank = 1/n, contrib = rank / outdeg, and the dangling rank.
static __global__ void k_pr_init(uint64_t n, const uint64_t* off, double* rank, double* contrib, PrCounters* pc) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const double r0 = 1.0 / (double)n;
    double dang = 0.0;
    for (uint64_t base = tid - threadIdx.x; base < n; base += nt) {  // same trip count in a block
        const uint64_t v = base + threadIdx.x;
        if (v < n) {
            const uint64_t deg = off[v + 1] - off[v];
            rank[v] = r0;
            contrib[v] = deg ? r0 / (double)deg : 0.0;
            if (!deg) dang += r0;
        }
    }
    const double t = block_sum(dang);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(&pc->dangling[0], t);
}

// End of iteration `it`: rank' = base + d * acc, with base from the dangling
// rank of this iteration; the L1 change and the next dangling rank are summed
// per block; contrib is refreshed and acc cleared for the next iteration.
static __global__ void k_pr_finalize(uint64_t n, const uint64_t* off, double* rank, double* contrib, double* acc,
                                     PrCounters* pc, double damping, uint32_t it) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const double base = (1.0 - damping) / (double)n + damping * pc->dangling[it & 1] / (double)n;
    double chg = 0.0, dang = 0.0;
    for (uint64_t b = tid - threadIdx.x; b < n; b += nt) {  // same trip count in a block
        const uint64_t v = b + threadIdx.x;
        if (v < n) {
            const double r = base + damping * acc[v];
            chg += fabs(r - rank[v]);
            rank[v] = r;
            acc[v] = 0.0;
            const uint64_t deg = off[v + 1] - off[v];
            contrib[v] = deg ? r / (double)deg : 0.0;
            if (!deg) dang += r;
        }
    }
    const double tc = block_sum(chg);
    const double td = block_sum(dang);
    if (threadIdx.x == 0) {
        if (tc != 0.0) atomicAdd(&pc->change, tc);
        if (td != 0.0) atomicAdd(&pc->dangling[(it + 1) & 1], td);
    }
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

// Multi-source BFS, end of a sweep: each newly reached vertex takes its new
// bits into visit and into its frontier mask, and level L is written for each
// new (source, vertex) pair; levels is k rows of n entries.  For the choice
// of the next level's direction it also sums the new frontier's out-degrees
// (fedges), the out-degrees weighted by new sources (pairs_edges), and ORs
// the sources whose frontier is non-empty (active).
struct MsLevelStats {
    unsigned long long* fedges;
    unsigned long long* pairs_edges;
    unsigned long long* active;
};

static __global__ void k_ms_finalize(const uint32_t* q, const uint32_t* count, unsigned long long* visit,
                                     unsigned long long* front, unsigned long long* next, uint32_t* levels,
                                     uint64_t n, uint32_t level, const uint64_t* off, MsLevelStats st) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t k = *count;
    unsigned long long fe = 0, pe = 0, act = 0;
    for (uint64_t base = tid - (threadIdx.x & 31); base < k; base += nt) {
        const uint64_t i = base + (threadIdx.x & 31);
        if (i < k) {
            const uint32_t u = q[i];
            unsigned long long nb = next[u];
            next[u] = 0ull;
            visit[u] |= nb;
            front[u] = nb;
            const unsigned long long deg = off[u + 1] - off[u];
            fe += deg;
            pe += deg * (unsigned long long)__popcll(nb);
            act |= nb;
            while (nb) {
                const int b = __ffsll((long long)nb) - 1;
                nb &= nb - 1;
                levels[(uint64_t)b * n + u] = level;
            }
        }
    }
    warp_atomic_add(st.fedges, fe);
    warp_atomic_add(st.pairs_edges, pe);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) act |= __shfl_xor_sync(0xffffffffu, act, o);
    if ((threadIdx.x & 31) == 0 && act) atomicOr(st.active, act);
}

// Multi-source BFS: clears the frontier masks of the level a bottom-up sweep
// just finished with (a top-down sweep clears each one as it expands it).
static __global__ void k_ms_clear_front(const uint32_t* q, const uint32_t* count, unsigned long long* front) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t k = *count;
    for (uint64_t i = tid; i < k; i += nt) front[q[i]] = 0ull;
}

// Multi-source BFS, bottom-up level (the pull direction applied to all
// sources at once, as Then et al., VLDB 2014, do for multi-source BFS over
// bit sets): every vertex that some source with a non-empty frontier has not
// reached (need = active & ~visit) ORs the frontier masks of its neighbours
// into `got`, stopping once got == need.  A lane first takes one vertex and
// its list heads in GPU memory; the lists this leaves undecided are read from
// the edge list, G lanes per list, with the group's OR combined after every
// step.  A vertex with new bits stores them in next (it is their only writer)
// and flags itself for the ordered compaction.
template <int G, class Id = uint64_t>
__global__ void __launch_bounds__(256) k_ms_bottom_up(Sweep c, const unsigned long long* front,
                                                      const unsigned long long* visit, unsigned long long* next,
                                                      uint8_t* nflag, unsigned long long active) {
    constexpr int GPW = 32 / G, E = IdWidth<Id>::kPerStep;
    const uint32_t lane = threadIdx.x & 31u, glane = lane % G, grp = lane / G;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n = c.all_n;
    unsigned long long scanned = 0, scanned_h = 0;
    for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
        const uint64_t v = base + lane;
        uint64_t s = 0, e = 0;
        unsigned long long need = 0, got = 0;
        bool pending = false;
        if (v < n) need = active & ~visit[v];
        if (need) {
            s = c.off[v];
            e = c.off[v + 1];
            if (c.heads) {
                const uint4 h = *reinterpret_cast<const uint4*>(c.heads + v * kHeads);
                const uint64_t k = e - s;
                if (k > 0) got |= front[h.x] & need;
                if (k > 1 && got != need) got |= front[h.y] & need;
                if (k > 2 && got != need) got |= front[h.z] & need;
                if (k > 3 && got != need) got |= front[h.w] & need;
                pending = got != need && k > (uint64_t)kHeads;
                s += kHeads;
            } else {
                pending = e > s;
            }
        }
        if (!pending && got) {
            next[v] = got;
            nflag[v] = 1;
        }
        unsigned pend = __ballot_sync(0xffffffffu, pending);
        while (pend) {
            unsigned rest = pend;
            for (uint32_t i = 0; i < grp && rest; i++) rest &= rest - 1u;  // this group's pending lane
            const int src = rest ? __ffs((int)rest) - 1 : 0;
            const bool mine = rest != 0;
            for (uint32_t i = 0; i < (uint32_t)GPW && pend; i++) pend &= pend - 1u;
            const uint64_t vv = __shfl_sync(0xffffffffu, v, src);
            uint64_t ss = __shfl_sync(0xffffffffu, s, src);
            uint64_t ee = __shfl_sync(0xffffffffu, e, src);
            unsigned long long nd = __shfl_sync(0xffffffffu, need, src);
            unsigned long long gg = __shfl_sync(0xffffffffu, got, src);
            if (!mine) {
                ss = ee = 0;
                nd = 0ull;
            }
            const uint64_t a = aligned_start<Id>(ss, c.shift);
            const uint32_t steps = ee > ss ? (uint32_t)((ee - a + E * G - 1) / (E * G)) : 0u;
            bool done = !mine;
            for (uint32_t t = 0; __any_sync(0xffffffffu, t < steps && !done); t++) {
                unsigned long long part = 0;
                if (t < steps && !done) {
                    const uint64_t j = a + (uint64_t)t * (E * G) + E * glane;
                    if (j + E - 1 >= ss && j < ee) {
                        uint32_t id[E];
                        if (j + E - 1 < ee || (EMOGI_WHOLE_TAIL_LOADS && j + E <= c.m)) {
                            ld_ids<Id>(c.cols, j, id);
                        } else {
#pragma unroll
                            for (int x = 0; x < E; x++) id[x] = (j + x < ee) ? ld_id<Id>(c.cols, j + x) : 0u;
                        }
#pragma unroll
                        for (int x = 0; x < E; x++) {
                            if (j + x >= ss && j + x < ee) {
                                part |= front[id[x]] & nd;
                                scanned += 1;
                            }
                        }
                    }
                }
                // every lane reaches the shuffles: the group's OR, then its test
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) part |= __shfl_xor_sync(0xffffffffu, part, o);
                gg |= part;
                done = done || gg == nd;
            }
            if (mine && glane == 0 && gg) {
                next[vv] = gg;
                nflag[vv] = 1;
            }
        }
    }
    add_scanned(c, scanned, scanned_h);
}

struct MsSources {
    uint32_t v[64];
    uint32_t k;
};

// Multi-source BFS start: source b sets bit b of its vertex and level 0 in
// row b; each distinct source vertex is queued once.
static __global__ void k_ms_init(MsSources src, unsigned long long* visit, unsigned long long* front,
                                 uint32_t* levels, uint64_t n, uint32_t* q, uint32_t* count) {
    const uint32_t b = threadIdx.x;
    if (b >= src.k) return;
    const uint32_t s = src.v[b];
    const unsigned long long bit = 1ull << b;
    atomicOr(visit + s, bit);
    const unsigned long long old = atomicOr(front + s, bit);
    levels[(uint64_t)b * n + s] = 0;
    if (old == 0ull) q[atomicAdd(count, 1u)] = s;
}

// Sum over vertices of out-degree x number of sources that reached it.
static __global__ void k_ms_reached_edges(const unsigned long long* visit, const uint64_t* off, uint32_t n,
                                          unsigned long long* out) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (uint64_t v = tid; v < n; v += nt) acc += (off[v + 1] - off[v]) * (unsigned long long)__popcll(visit[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// Sampled CC, first phase: every vertex is linked with its first `rounds`
// neighbours (one or two ids, usually one 32-byte sector of the edge list).
template <class Id>
__global__ void k_cc_sample(const uint64_t* off, const void* cols, const uint32_t* heads, uint32_t* parent,
                            uint32_t n, uint32_t rounds, unsigned long long* scanned) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (uint64_t v = tid; v < n; v += nt) {
        const uint64_t s = off[v], e = off[v + 1];
        const uint64_t k = e - s < rounds ? e - s : rounds;
        if (heads) {  // the ids are mirrored in GPU memory: no edge-list read
            for (uint64_t r = 0; r < k; r++) uf_union(parent, (uint32_t)v, heads[v * kHeads + r]);
            continue;
        }
        for (uint64_t r = 0; r < k; r++) uf_union(parent, (uint32_t)v, ld_id<Id>(cols, s + r));
        cnt += k;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(scanned, cnt);
}

// Sampled CC: the most frequent root among up to 1024 sample vertices of
// non-zero degree (one block of 1024 threads), written to *giant.
static __global__ void k_cc_giant(const uint32_t* parent, const uint64_t* off, uint32_t n, uint32_t* giant) {
    __shared__ uint32_t root[1024];
    __shared__ unsigned long long best;
    const uint32_t t = threadIdx.x;
    if (t == 0) best = 0;
    uint32_t r = INF;
    // sample vertex t * stride, stepping forward to the first vertex with edges
    const uint64_t stride = n > 1024 ? n / 1024 : 1;
    uint64_t v = (uint64_t)t * stride;
    for (uint32_t tries = 0; v < n && tries < 64; tries++, v++) {
        if (off[v + 1] > off[v]) {
            r = __ldcg(parent + v);
            break;
        }
    }
    root[t] = r;
    __syncthreads();
    uint32_t cnt = 0;
    if (r != INF)
        for (uint32_t i = 0; i < 1024; i++) cnt += root[i] == r;
    // the largest count wins; ties go to the smaller root id
    if (r != INF) atomicMax(&best, ((unsigned long long)cnt << 32) | (unsigned long long)(0xFFFFFFFFu - r));
    __syncthreads();
    if (t == 0) *giant = best ? 0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFu) : INF;
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
