// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "emogi.h"

namespace emogi {

// The short-list store (whole lists mirrored in GPU memory when the edge list
// is not there) holds every list of 1..kStoreBase entries, and of
// 1..kStoreWide entries when those hold at most 1/kStoreShare of the graph's
// entries: on degree-skewed graphs they are most of the vertices but few of
// the edges (Kronecker graphs of edge factor 32: 4-8 %), while on a uniform
// graph of mean degree 32 they are half of the edge list, which then stays
// where the caller placed it.  Measured on GB300, Kronecker scale 27 SSSP from host memory:
// 845 ms with a bound of 16 entries, 731 ms with 32 (1.0 GB more of GPU
// memory); 64 and 128 read 5 % fewer link bytes for 3.4 GB more and ran
// 666-1195 ms.  A bound whose store does not fit the device budget, with
// room left for the work buffers, is not taken.
constexpr uint32_t kStoreBase = 16, kStoreWide = 32, kStoreShare = 8;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
void clear_error();

// Records a failure with its message and returns the status.
emogi_status fail(emogi_status s, const char* fmt, ...);

#define EMOGI_CUDA_TRY(expr)                                                             \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::emogi::fail(EMOGI_E_CUDA, "%s failed: %s (%s:%d)", #expr,           \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

#define EMOGI_TRY(expr)                                                                  \
    do {                                                                                 \
        emogi_status s_ = (expr);                                                        \
        if (s_ != EMOGI_OK) return s_;                                                   \
    } while (0)

// ---------------------------------------------------------------- device memory
// Every device allocation of the library goes through these so that the
// budget of emogi_set_device_budget applies and tests can inject failures.
emogi_status dev_alloc(void** p, size_t bytes, const char* what);
emogi_status dev_free(void* p, size_t bytes);

// ---------------------------------------------------------------- options
struct Opts {
    uint32_t access = EMOGI_ACCESS_MERGED_ALIGNED;
    uint32_t granularity = 0;
    uint32_t chunk_lines = 0;
    uint32_t delta = 0;
    uint64_t timeout_ns = 2000000000ull;
    cudaStream_t stream = nullptr;
    bool out_on_device = false;
    uint32_t flags = 0;
};
emogi_status parse_opts(const emogi_opts* in, Opts* out);

// ---------------------------------------------------------------- work buffers
// Device counters of one traversal, kept in one small struct so that a single
// memset clears them.
struct DevCounters {
    uint32_t qcount[2];              // frontier sizes (ping-pong)
    uint32_t fcount[2];              // SSSP: [0] = far vertices kept by the last split
    uint32_t far_min;                // SSSP: smallest distance sent to the far pile
    uint32_t overflow;               // SSSP: a distance reached UINT32_MAX
    uint32_t error;                  // device-side error code (bounded waits)
    uint32_t pad;
    unsigned long long large[2];     // split-list work: (slots << 34) | items
    unsigned long long scanned;      // neighbour entries read
    unsigned long long reached;      // sum of out-degrees of reached vertices
    unsigned long long fedges;       // BFS / MS-BFS: sum of out-degrees of the next frontier
    unsigned long long ms_pairs_edges; // MS-BFS: sum over new (source, vertex) pairs of the out-degree
    unsigned long long ms_active;    // MS-BFS: sources whose frontier is non-empty
    uint32_t giant;                  // sampled CC: root of the largest sampled tree
    uint32_t pad2;
    unsigned long long scanned_heads; // of `scanned`: entries of whole lists read from the list heads in GPU memory
};

struct Workspace {
    uint64_t n = 0;
    uint32_t* q[2] = {nullptr, nullptr};   // frontier queues, n entries each
    uint32_t* state = nullptr;             // level / dist / parent when output is on the host
    uint32_t* qround = nullptr;            // SSSP sweep stamps: the sweep a vertex is queued for
    uint32_t* fflag = nullptr;             // SSSP "in the far pile" flags, all zero between calls
    uint32_t* xd = nullptr;                // SSSP distance of the last expansion
    uint8_t* nflag = nullptr;              // next frontier as one byte per vertex (n rounded up to 16), zero between calls
    bool flags_dirty = false;              // a call ended early and left flags set
    uint32_t* lq_v = nullptr;              // split-list vertices
    unsigned long long* lq_base = nullptr; // first chunk index of each split-list vertex
    unsigned long long* lq_state = nullptr;// the split-list vertex's per-sweep value
    uint64_t lq_cap = 0;
    DevCounters* ctr = nullptr;
    DevCounters* h_ctr = nullptr;          // pinned mirror for readback
    size_t dev_bytes = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // multi-source BFS state, allocated on first use
    unsigned long long* ms_visit = nullptr;  // sources that reached v
    unsigned long long* ms_front = nullptr;  // sources for which v is in the frontier
    unsigned long long* ms_next = nullptr;   // sources reaching v in the sweep under way
    uint32_t* ms_out = nullptr;              // k x n levels when the output is on the host
    size_t ms_out_bytes = 0;
    // PageRank state, allocated on first use
    double* pr_rank = nullptr;               // ranks when the output is on the host
    double* pr_contrib = nullptr;            // rank / out-degree
    double* pr_acc = nullptr;                // sums of the incoming contributions
    void* pr_ctr = nullptr;                  // dev::PrCounters
    void* h_pr_ctr = nullptr;                // pinned mirror
    // device-driven SSSP loop: its state block and its recorded CUDA graph
    void* sssp_loop = nullptr;               // dev::SsspLoop in device memory
    void* h_sssp_loop = nullptr;             // pinned staging copy
    cudaGraphExec_t sssp_exec = nullptr;
    uint32_t sssp_exec_G = 0;
    uint32_t sssp_exec_chunk = 0;
};

}  // namespace emogi

struct emogi_graph_s {
    int device = 0;
    uint64_t n = 0, m = 0;
    uint32_t flags = 0;
    int place = EMOGI_PLACE_DEVICE;
    uint64_t* d_off = nullptr;         // device row offsets (n + 1)
    uint32_t* d_heads = nullptr;       // first 4 ids of every list in GPU memory (edge lists off the GPU)
    // short-list store: every list of 1..short_max entries copied whole to GPU
    // memory (ids as uint32, and weights), each starting on a 4-entry boundary;
    // d_short_off[v] = start of v's list in units of 4 entries (edge lists off the GPU)
    uint32_t* d_short_off = nullptr;
    uint32_t* d_short_ids = nullptr;
    uint32_t* d_short_w = nullptr;
    uint32_t short_max = 0;            // longest list the store holds (0 = no store)
    uint64_t short_slots = 0;          // entries the store holds (padding included)
    uint64_t short_entries = 0;        // list entries it holds
    const void* cols = nullptr;        // kernel-visible edge list (uint64 or uint32 ids)
    uint32_t id_bytes = 8;             // bytes per id: 8, or 4 for a graph loaded by emogi_load_csr32
    const uint32_t* w = nullptr;       // kernel-visible weights or null
    void* cols_owned = nullptr;        // what to free (device / pinned / managed)
    void* w_owned = nullptr;
    const void* cols_borrowed = nullptr;  // what to unregister
    const void* w_borrowed = nullptr;
    uint32_t shift = 0;                // (edge-list base address mod 128) / id_bytes
    size_t dev_bytes = 0;              // budgeted device bytes of the graph arrays
    cudaStream_t stream = nullptr;
    emogi::Workspace ws;
    double avg_degree = 0.0;
    uint64_t max_degree = 0;
    double avg_weight = 0.0;           // mean of a sample of the weights
    bool shared = false;               // a view made by emogi_graph_share: the arrays belong to another handle
};

namespace emogi {
emogi_status ensure_workspace(emogi_graph g);
uint64_t workspace_need(uint64_t n, uint64_t m);  // device bytes ensure_workspace allocates
void release_workspace(emogi_graph g);
int sm_count(int device);
}  // namespace emogi
