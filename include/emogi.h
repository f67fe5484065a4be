/*
 * emogi.h - C ABI of the GB300 zero-copy graph-traversal library.
 *
 * The library runs level-synchronous BFS, SSSP and connected components over
 * a CSR graph whose edge (and weight) arrays may stay in pinned host memory
 * and are read by the GPU in place ("zero-copy", paper Sec. 3) with merged,
 * 128-byte-aligned warp accesses (Sec. 4.3), while the vertex list and all
 * vertex state live in GPU memory (Sec. 4.2).  Everything on the traversal
 * path runs in the library's own CUDA kernels (sm_103a); there is no CPU
 * fallback.
 *
 * Conventions shared by every entry point
 *  - Vertex ids at the API are uint64_t; the library requires
 *    n < 2^32 - 1 so that per-vertex state fits in uint32_t.
 *  - "Unreachable" / "no value" is UINT32_MAX (EMOGI_INF).
 *  - Calls are synchronous: when a call returns EMOGI_OK its outputs are
 *    complete (device outputs included).  A graph handle may be used by one
 *    thread at a time; distinct handles may be used concurrently.
 *  - No C++ exception crosses this boundary.  Every entry point returns an
 *    emogi_status; on failure emogi_last_error() returns a thread-local,
 *    human-readable description that stays valid until the next call on the
 *    same thread.  CUDA runtime failures map to EMOGI_E_CUDA.
 *  - Host arrays are read during the call only and never retained, except
 *    with EMOGI_LOAD_BORROW (see emogi_load_csr).
 */
#ifndef EMOGI_H
#define EMOGI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMOGI_INF 0xFFFFFFFFu
#define EMOGI_MAX_SOURCES 64u

typedef struct emogi_graph_s* emogi_graph;

typedef enum {
    EMOGI_OK = 0,
    EMOGI_E_ARG = 1,         /* invalid argument (bad CSR, source out of range, NULL pointer, ...) */
    EMOGI_E_NOMEM = 2,       /* a host or device allocation failed */
    EMOGI_E_BUDGET = 3,      /* the device-memory budget (emogi_set_device_budget) would be exceeded */
    EMOGI_E_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    EMOGI_E_TIMEOUT = 5,     /* a bounded device-side wait gave up (persistent kernels) */
    EMOGI_E_OVERFLOW = 6,    /* a shortest-path distance does not fit below UINT32_MAX */
    EMOGI_E_UNSUPPORTED = 7  /* operation not defined for this graph (e.g. CC on a directed graph) */
} emogi_status;

/* Where the edge list (col_idx) and the weights live.  The row offsets and all
 * vertex state are always in GPU memory (Sec. 4.2). */
typedef enum {
    EMOGI_PLACE_DEVICE = 0,  /* copied into GPU memory (all-in-HBM reference point) */
    EMOGI_PLACE_HOST = 1,    /* pinned, mapped host memory read zero-copy (Sec. 3.1, the EMOGI case) */
    EMOGI_PLACE_MANAGED = 2  /* cudaMallocManaged + ReadMostly advice: the UVM baseline (Sec. 5.1.2 (a)) */
} emogi_placement;

/* emogi_load_csr flags */
enum {
    EMOGI_LOAD_UNDIRECTED = 1u << 0, /* caller asserts the CSR is symmetric; required by emogi_cc */
    EMOGI_LOAD_BORROW = 1u << 1,     /* HOST: pin and map the caller's arrays in place, no copy;
                                        MANAGED: use the caller's managed arrays in place */
    EMOGI_LOAD_NO_HEADS = 1u << 2    /* HOST / MANAGED: mirror nothing of the edge list in GPU memory:
                                        neither the first 4 ids of every list (16 bytes per vertex, read
                                        by sampled CC and bottom-up BFS) nor the short-list store (every
                                        list of at most 16 or 32 entries, ids and weights, see
                                        emogi_graph_store_bound); every list entry is then read over
                                        the host link */
};

/* How a worker reads one neighbour list (Sec. 4.2, Sec. 4.3, Listings
 * "Uncoalesced Memory Access" and "Coalesced Memory Access (Merged + Aligned)"). */
typedef enum {
    EMOGI_ACCESS_MERGED_ALIGNED = 0, /* groups of lanes read the list from the 128-byte line that
                                        contains its first element, 16 bytes per lane; lists longer
                                        than a threshold are split across warps */
    EMOGI_ACCESS_MERGED = 1,         /* one warp per vertex, 8 bytes per lane, from the list's own
                                        (unaligned) start: the paper's "Merged" variant */
    EMOGI_ACCESS_NAIVE = 2           /* one thread per vertex walking its list element by element:
                                        the paper's "Naive" variant */
} emogi_access;

/* emogi_opts.flags */
enum {
    EMOGI_OPT_TIME_KERNELS = 1u << 0, /* bracket every neighbour-expansion launch with CUDA events and
                                         report their summed duration in emogi_stats.expand_ms */
    EMOGI_OPT_TOP_DOWN_ONLY = 1u << 1, /* BFS: expand every level from the frontier (push) as the paper
                                          does, never switch an undirected graph's dense levels to the
                                          bottom-up (pull) direction */
    EMOGI_OPT_CC_FULL_PASS = 1u << 2,  /* CC: stream the whole edge list as the paper does instead of
                                          linking sampled neighbours first and skipping the vertices
                                          already in the largest sampled component */
    EMOGI_OPT_HOST_LOOP = 1u << 3,     /* SSSP: drive the sweep loop from the host (one counter
                                          readback per sweep, as the paper's level loop) instead of a
                                          recorded CUDA graph whose conditional loop decides on the
                                          device */
    EMOGI_OPT_BEAMER = 1u << 4,        /* BFS: choose each level's direction by the fixed thresholds
                                          of Beamer et al. (alpha = 14, beta = 24) instead of the
                                          estimate of list entries each direction would read */
    EMOGI_OPT_ORDERED_FRONTIER = 1u << 5 /* SSSP: rebuild every near frontier in vertex order (flag
                                          per vertex, compacted after each sweep), as the library
                                          does by itself for edge lists (with weights) of 16 GiB or
                                          more, whose lists read in arrival order span more address
                                          range than the GPU's translations cover */
};

/* Per-call options.  Pass NULL for defaults.  struct_size must be
 * sizeof(emogi_opts) so that the struct can grow. */
typedef struct {
    uint32_t struct_size;
    uint32_t access;       /* emogi_access; default EMOGI_ACCESS_MERGED_ALIGNED */
    uint32_t granularity;  /* lanes per vertex for MERGED_ALIGNED: 4, 8, 16 or 32; 0 = automatic */
    uint32_t chunk_lines;  /* 128-byte lines per work item for split (long) lists; 0 = automatic */
    uint64_t timeout_ns;   /* bound on device-side waits of persistent kernels (0 = 2 s) and on
                              the device-driven SSSP loop (0 = 60 s); EMOGI_E_TIMEOUT when passed */
    void* cuda_stream;     /* cudaStream_t to run on; NULL = the graph's own stream */
    int32_t out_on_device; /* 1: output pointers are device pointers of the current device */
    uint32_t flags;        /* EMOGI_OPT_* */
    uint32_t delta;        /* SSSP bucket width: vertices are expanded in order of distance
                              windows [T - delta, T); 0 = automatic, UINT32_MAX = plain
                              frontier Bellman-Ford (one window) */
    uint32_t reserved0;
} emogi_opts;

/* Per-call statistics (optional output). */
typedef struct {
    uint32_t iterations;    /* levels (BFS), relaxation rounds (SSSP), edge passes (CC) */
    uint32_t reserved;
    uint64_t edges_scanned; /* neighbour-list entries read by the expansion kernels */
    uint64_t edges_reached; /* sum of out-degrees of reached vertices (the TEPS numerator; m for CC) */
    uint64_t edge_bytes;    /* bytes of ids read from the edge list: the entries of edges_scanned not
                               served by the short-list store in GPU memory (emogi_graph_store_bound),
                               * bytes per id (8, or 4 for emogi_load_csr32) */
    uint64_t weight_bytes;  /* weights read from the weight array (SSSP): those entries * 4 */
    double ms;              /* device time of the traversal, CUDA events on the launch stream */
    double expand_ms;       /* with EMOGI_OPT_TIME_KERNELS: summed duration of expansion launches */
    uint64_t expand_launches; /* neighbour-expansion sweeps */
    uint64_t kernel_launches; /* every kernel the call launched */
} emogi_stats;

/* Load a CSR graph (Sec. 2.1, Figure "Sample undirected graph and its CSR
 * representation"; placement as in Sec. 3.1 and Sec. 4.2).
 *   n            number of vertices, 0 <= n < 2^32 - 1
 *   m            number of stored (directed) edges
 *   row_offsets  host uint64_t[n+1], non-decreasing, row_offsets[0] == 0,
 *                row_offsets[n] == m; copied to GPU memory
 *   col_idx      host uint64_t[m], every entry < n; duplicates and self-loops
 *                are allowed
 *   weights      host uint32_t[m] or NULL (SSSP needs weights)
 *   place        emogi_placement of col_idx and weights
 *   flags        EMOGI_LOAD_* bits
 *   out          receives the handle; release it with emogi_free_graph
 * With EMOGI_LOAD_BORROW and EMOGI_PLACE_HOST the library registers col_idx
 * and weights with cudaHostRegister instead of copying; they must be 16-byte
 * aligned and the caller must keep them alive and unchanged until
 * emogi_free_graph.  With EMOGI_LOAD_BORROW and EMOGI_PLACE_MANAGED, col_idx
 * and weights must be managed memory (cudaMallocManaged, e.g. from
 * emogi_managed_alloc), 16-byte aligned; the library advises them read-mostly
 * and reads them in place (a graph larger than the host can hold twice then
 * needs no second copy); the caller frees them after emogi_free_graph.  A
 * borrowed DEVICE placement is rejected (EMOGI_E_ARG).
 * The GPU reads a borrowed list wherever it lies, so large borrowed arrays
 * should sit on huge pages (e.g. an anonymous mapping advised with
 * MADV_HUGEPAGE before it is filled): with 64 KiB pages a 50 GB edge list
 * needs far more address translations than the GPU holds, and random list
 * reads then run two orders of magnitude slower.  The library's own HOST
 * copies of arrays of 1 GiB or more are placed that way.
 * Errors: EMOGI_E_ARG (invalid CSR or flags), EMOGI_E_BUDGET, EMOGI_E_NOMEM,
 * EMOGI_E_CUDA.  On error *out is set to NULL and nothing is retained. */
emogi_status emogi_load_csr(uint64_t n, uint64_t m, const uint64_t* row_offsets,
                            const uint64_t* col_idx, const uint32_t* weights,
                            emogi_placement place, uint32_t flags, emogi_graph* out);

/* Load a CSR graph whose edge list holds 4-byte ids (Sec. 5.4 compares the
 * 4-byte edge list with the 8-byte one: it halves the link bytes of every id
 * read; Sec. 4.1: a 128-byte line then holds 32 ids instead of 16).  The
 * arguments, placement, flags, ownership and errors are those of
 * emogi_load_csr, except:
 *   col_idx      host uint32_t[m], every entry < n (with EMOGI_LOAD_BORROW,
 *                16-byte aligned, kept alive and unchanged until
 *                emogi_free_graph)
 * Every traversal, emogi_msbfs, the batch and the server accept the handle
 * and return exactly the results of the same graph loaded with 8-byte ids;
 * the kernels read four ids per 16-byte lane load and align list reads to
 * 32-id lines.  emogi_bfs_noalloc takes uint64 ids only. */
emogi_status emogi_load_csr32(uint64_t n, uint64_t m, const uint64_t* row_offsets,
                              const uint32_t* col_idx, const uint32_t* weights,
                              emogi_placement place, uint32_t flags, emogi_graph* out);

/* Breadth-first search from src (Sec. 2.1, Algorithm "High-level Graph
 * Traversal Flow" with the BFS condition: an unvisited neighbour of an active
 * vertex becomes active at the next depth; one kernel round per level, Sec. 4.2).
 * On graphs loaded with EMOGI_LOAD_UNDIRECTED and MERGED_ALIGNED access, a
 * level is expanded bottom-up instead (every unreached vertex reads its own
 * list up to its first neighbour on the current level; direction-optimising
 * BFS, Beamer et al. 2012) when that is estimated to read fewer list entries
 * than the frontier's own lists hold: with p the frontier's share of edge
 * endpoints, an unreached vertex of mean degree d reads about
 * sum_{i<d} (1-p)^i entries, the first four of them from GPU memory when the
 * list heads are mirrored there.  EMOGI_OPT_BEAMER uses Beamer's fixed
 * thresholds instead; EMOGI_OPT_TOP_DOWN_ONLY keeps the paper's push-only
 * form.  The levels are the same either way.
 *   level  uint32_t[n] output (host, or device if opts->out_on_device):
 *          level[src] = 0, hop distance for reached vertices, EMOGI_INF otherwise.
 * Errors: EMOGI_E_ARG (src >= n, NULL pointer), EMOGI_E_BUDGET, EMOGI_E_NOMEM,
 * EMOGI_E_CUDA.  The output is unspecified on error. */
emogi_status emogi_bfs(emogi_graph g, uint64_t src, uint32_t* level, const emogi_opts* opts,
                       emogi_stats* stats);

/* Single-source shortest paths with the graph's uint32 weights (Sec. 5.1.2,
 * Sec. 5.4: SSSP reads each weight beside its edge).  Active vertices relax
 * their out-edges with an atomic minimum and improved vertices become active,
 * until no distance changes; active vertices are expanded in distance windows
 * of width opts->delta (a near frontier below the threshold, a far pile above
 * it), which bounds re-expansions without changing the exact result.
 *   dist   uint32_t[n] output: exact shortest distance, EMOGI_INF if unreachable.
 * Errors: as emogi_bfs, plus EMOGI_E_UNSUPPORTED (graph loaded without
 * weights) and EMOGI_E_OVERFLOW (a finite distance >= UINT32_MAX). */
emogi_status emogi_sssp(emogi_graph g, uint64_t src, uint32_t* dist, const emogi_opts* opts,
                        emogi_stats* stats);

/* Connected components of an undirected graph (Sec. 5.4: every vertex starts
 * active and the entire edge list is streamed).  Edges hook the larger
 * union-find root under the smaller with compare-and-swap, then every vertex
 * is resolved to its root.  By default the edge stream is sampled first
 * (Afforest, Sutton et al. 2018): each vertex is linked with its first two
 * neighbours, the largest resulting tree is found from 1024 samples, and only
 * vertices outside it read their lists; EMOGI_OPT_CC_FULL_PASS streams every
 * list as the paper does.  The labels are the same either way.
 *   label  uint32_t[n] output: the smallest vertex id of the vertex's component.
 * Errors: EMOGI_E_UNSUPPORTED if the graph was not loaded with
 * EMOGI_LOAD_UNDIRECTED (the paper runs CC on undirected graphs only), and
 * the errors of emogi_bfs. */
emogi_status emogi_cc(emogi_graph g, uint32_t* label, const emogi_opts* opts, emogi_stats* stats);

/* PageRank (the fourth application of Sec. 5.4; every vertex is active in
 * every iteration and the whole edge list is read), by power iteration in
 * double precision: starting from 1/n, each iteration gives every vertex
 *   (1 - damping)/n + damping * D/n + damping * sum over edges u -> v of rank(u)/outdeg(u),
 * where D is the rank held by vertices without out-edges, and stops after
 * max_iters iterations or once the L1 change of an iteration is below
 * tolerance.  Parallel edges and self-loops count as edges.  Undirected graphs
 * are pulled (a vertex sums its own list, no atomics); directed graphs are
 * pushed along out-edges with atomic adds.  The result equals the definition
 * up to the order of floating-point additions.
 *   damping    in [0, 1)
 *   tolerance  >= 0 (0: run exactly max_iters iterations)
 *   max_iters  >= 1
 *   rank       double[n] output (host, or device if opts->out_on_device)
 *   stats->iterations = iterations run; edges_reached = m * iterations.
 * Errors: EMOGI_E_ARG (damping, tolerance, max_iters, NULL output), and the
 * errors of emogi_bfs. */
emogi_status emogi_pagerank(emogi_graph g, double damping, double tolerance, uint32_t max_iters, double* rank,
                            const emogi_opts* opts, emogi_stats* stats);

/* Multi-source BFS: k independent BFS traversals (1 <= k <= 64) in one
 * level-synchronous pass.  Each vertex carries 64-bit masks (visited, in the
 * frontier, reached this level), bit b for source b, so one read of a
 * neighbour list serves every source whose frontier holds the vertex.  The
 * paper runs its BFS from 64 sources one at a time (Sec. 5.2); the result
 * here is identical to k separate emogi_bfs calls.
 *   srcs    host uint64_t[k], each < n (repeats allowed)
 *   levels  uint32_t[k * n] output, row b = the levels from srcs[b] (host, or
 *           device if opts->out_on_device)
 * Errors: EMOGI_E_ARG (k out of range, a source >= n, NULL pointer) and the
 * errors of emogi_bfs. */
emogi_status emogi_msbfs(emogi_graph g, const uint64_t* srcs, uint32_t k, uint32_t* levels,
                         const emogi_opts* opts, emogi_stats* stats);

/* ---- Batched BFS over many graphs in one persistent launch ----------------
 * The paper traverses one graph per run with one kernel launch per level
 * (Sec. 4.2).  A batch advances every graph of a set by one level per round
 * of a single cooperatively launched, persistent kernel: the frontiers of all
 * graphs form one queue of (graph, vertex) entries that warps claim in
 * chunks, and rounds are separated by a grid-wide barrier whose wait is
 * bounded by opts->timeout_ns (EMOGI_E_TIMEOUT when exceeded).  Source upload,
 * initialisation and the persistent kernel are recorded once as a CUDA graph
 * and replayed on every call.  Results equal one emogi_bfs per graph.
 *
 * emogi_batch_create: graphs[0..count) are loaded graphs on one device (any
 *   placement); the batch keeps the handles (free it before them) and
 *   allocates its combined queues and levels (about 20 bytes per vertex).
 * emogi_batch_bfs: srcs host uint64_t[count], srcs[g] < n of graph g;
 *   levels uint32_t[emogi_batch_total_vertices(b)] output (host, or device if
 *   opts->out_on_device): graph g's levels start at emogi_batch_offset(b, g).
 *   opts->granularity = lanes per vertex (0 = the batch's current choice),
 *   opts->chunk_lines = frontier entries a warp claims at once, in units of
 *   its lane groups (0 = current choice).  Only MERGED_ALIGNED access.
 * emogi_batch_autotune: runs the batch from srcs with every lanes-per-vertex
 *   choice {4, 8, 16, 32} and claim size {1, 4, 16, 64}, keeps the fastest as
 *   the batch's choice and reports it (any output pointer may be NULL).
 * emogi_bfs_batch: one-shot create + bfs + free.
 * Errors: EMOGI_E_ARG (NULL, empty graph, mixed devices, a source out of
 * range), EMOGI_E_UNSUPPORTED (access other than MERGED_ALIGNED),
 * EMOGI_E_TIMEOUT, EMOGI_E_BUDGET, EMOGI_E_NOMEM, EMOGI_E_CUDA. */
typedef struct emogi_batch_s* emogi_batch;
emogi_status emogi_batch_create(const emogi_graph* graphs, uint32_t count, emogi_batch* out);
emogi_status emogi_batch_bfs(emogi_batch b, const uint64_t* srcs, uint32_t* levels, const emogi_opts* opts,
                             emogi_stats* stats);
emogi_status emogi_batch_autotune(emogi_batch b, const uint64_t* srcs, uint32_t* best_granularity,
                                  uint32_t* best_claim, double* best_ms);
uint64_t emogi_batch_offset(emogi_batch b, uint32_t g);
uint64_t emogi_batch_total_vertices(emogi_batch b);
emogi_status emogi_batch_free(emogi_batch b);
emogi_status emogi_bfs_batch(const emogi_graph* graphs, const uint64_t* srcs, uint32_t* levels, uint32_t count,
                             const emogi_opts* opts, emogi_stats* stats);

/* ---- Query server with continuous batching --------------------------------
 * The paper runs one traversal at a time.  A server accepts BFS and SSSP
 * queries over already loaded graphs from any thread and runs them on
 * max_slots worker slots, each with its own CUDA stream and its own share
 * (emogi_graph_share) of every graph it serves, so jobs overlap on the GPU.
 * When a slot is idle the oldest pending query forms the next job; a BFS job
 * also takes the other pending BFS queries of the same graph (up to
 * max_batch) and runs them as one multi-source pass (emogi_msbfs), so queries
 * that arrive while others run join the next pass.  A job is admitted only
 * when the device bytes the slots hold (their traversal buffers, kept
 * resident between jobs, and the batch's level rows, k * n * 4 bytes) fit
 * device_budget; idle slots release their buffers first, a job that does not
 * fit waits for running ones, and one that cannot fit on an idle server
 * fails with EMOGI_E_BUDGET.  Results equal the single-query calls.
 *   emogi_server_submit: out is a host uint32_t[n] for the result, or NULL to
 *     discard it; it must stay valid until the query is waited for.  The
 *     graph must outlive the server.
 *   emogi_server_wait: blocks until the query is done (timeout_ns = 0: no
 *     limit; otherwise EMOGI_E_TIMEOUT when it is not done in time, and the
 *     ticket stays valid), fills *res and releases the ticket; returns the
 *     query's own status.
 *   emogi_server_drain: waits until every submitted query is done.
 *   emogi_server_destroy: drains, stops the workers and frees their buffers. */
typedef struct emogi_server_s* emogi_server;
typedef enum { EMOGI_QUERY_BFS = 0, EMOGI_QUERY_SSSP = 1 } emogi_query_kind;
typedef struct {
    uint32_t struct_size;
    uint32_t max_slots;      /* worker slots; 0 = 4, at most 64 */
    uint64_t device_budget;  /* bytes the slots' buffers may hold; 0 = unlimited */
    uint32_t max_batch;      /* BFS queries per multi-source pass, 1..64; 0 = 64 */
    uint32_t reserved;
} emogi_server_config;
typedef struct {
    emogi_status status;
    uint32_t batch_size;     /* queries that ran in the same job */
    double queue_ms;         /* submit -> job start */
    double run_ms;           /* job start -> result ready */
    double latency_ms;       /* submit -> result ready */
    uint64_t edges_reached;  /* TEPS numerator (a batch reports its mean per query) */
    uint64_t edges_scanned;  /* list entries the job read (a batch reports its total divided by its
                                queries, so the sum over a batch's queries is what the pass read) */
} emogi_query_result;
emogi_status emogi_server_create(const emogi_server_config* cfg, emogi_server* out);
emogi_status emogi_server_submit(emogi_server s, emogi_graph g, uint32_t kind, uint64_t src, uint32_t* out,
                                 uint64_t* ticket);
emogi_status emogi_server_wait(emogi_server s, uint64_t ticket, uint64_t timeout_ns, emogi_query_result* res);
emogi_status emogi_server_drain(emogi_server s);
uint64_t emogi_server_device_bytes(emogi_server s);
emogi_status emogi_server_destroy(emogi_server s);

/* Set the device-memory budget in bytes for all graphs and work buffers the
 * library allocates from now on (0 = unlimited).  Allocations that would
 * exceed it fail with EMOGI_E_BUDGET.  Mirrors the paper's GPU memory cap of
 * its A100 runs (Sec. 5.6).  Returns EMOGI_OK. */
emogi_status emogi_set_device_budget(uint64_t bytes);

/* Bytes of device memory the library currently holds (graphs + work buffers). */
uint64_t emogi_device_bytes_in_use(void);

/* Managed (UVM) memory for arrays that a caller fills on the host and then
 * loads with EMOGI_PLACE_MANAGED | EMOGI_LOAD_BORROW (the UVM baseline of
 * Sec. 5.1.2 (a) without a second copy of the edge list).  The pages live in
 * host memory until the GPU touches them; they are not counted against the
 * device budget.  emogi_managed_alloc returns a 256-byte aligned pointer, or
 * EMOGI_E_ARG (out NULL or bytes 0) / EMOGI_E_NOMEM; emogi_managed_free(NULL)
 * is a no-op, and the memory must not be freed while a graph borrows it. */
emogi_status emogi_managed_alloc(uint64_t bytes, void** out);
emogi_status emogi_managed_free(void* p);

/* Release a graph and every buffer the library holds for it.  NULL is a no-op.
 * Returns EMOGI_E_CUDA if a CUDA free failed (the handle is released anyway). */
emogi_status emogi_free_graph(emogi_graph g);

/* A second handle onto a loaded graph: it reads the same row offsets, edge
 * list and weights (nothing is copied) but has its own stream and work
 * buffers, so that traversals through different handles of one graph can run
 * concurrently from different threads.  Free every share before the original
 * handle.  Errors: EMOGI_E_ARG, EMOGI_E_NOMEM, EMOGI_E_CUDA. */
emogi_status emogi_graph_share(emogi_graph g, emogi_graph* out);

/* Device bytes of the work buffers this handle holds (0 before its first traversal). */
uint64_t emogi_graph_workspace_bytes(emogi_graph g);

/* Properties of a loaded graph. */
uint64_t emogi_graph_num_vertices(emogi_graph g);
uint64_t emogi_graph_num_edges(emogi_graph g);
int emogi_graph_placement(emogi_graph g);

/* The longest list held by the graph's short-list store in GPU memory: the
 * traversals read every list of 1..this many entries there (ids, and weights
 * when loaded), not from the edge list, and leave those entries out of
 * emogi_stats.edge_bytes / weight_bytes.  32 when the lists of up to 32
 * entries hold at most 1/8 of the graph's entries (degree-skewed graphs),
 * else 16; 0 when there is no store: DEVICE placement, EMOGI_LOAD_NO_HEADS,
 * or no room for it in the device budget next to one handle's work buffers
 * (a store that does not fit is left out rather than failing the load).
 * This is a GB300-side cache with no counterpart in the paper, whose edge
 * list is read only over the link. */
uint32_t emogi_graph_store_bound(emogi_graph g);

/* Zero-copy read probe (a measurement aid with no counterpart among the
 * paper's operations; Sec. 5.3 measures how zero-copy request patterns set
 * the link's delivered bandwidth).  Times one kernel that reads the pinned,
 * mapped host range [host, host + bytes) over the link:
 *   EMOGI_PROBE_STREAM   the whole range, coalesced 16-byte loads
 *   EMOGI_PROBE_RANDOM   `blocks` reads of block_bytes each, a warp per read,
 *                        at pseudo-random block-aligned positions in the range
 *   EMOGI_PROBE_REGIONS  `blocks` reads of block_bytes each, spaced evenly over
 *                        the range (bytes / blocks apart); each thread block
 *                        of the grid reads one contiguous share of them
 *   host        16-byte aligned, pinned with cudaHostAlloc or cudaHostRegister
 *               (e.g. a borrowed edge list while its graph is loaded); only read
 *   cuda_stream stream to run on, or NULL for one the call creates
 *   ms          receives the kernel's duration (CUDA events)
 * The bytes read are `bytes` (rounded down to 16) for STREAM and
 * block_bytes * blocks otherwise.  Errors: EMOGI_E_ARG (NULL pointers, a
 * range under 16 bytes or not 16-byte aligned, memory that is not pinned and
 * mapped, block_bytes not a multiple of 16 in [16, bytes], blocks == 0, or
 * REGIONS blocks that do not fit apart), EMOGI_E_CUDA. */
enum { EMOGI_PROBE_STREAM = 0, EMOGI_PROBE_RANDOM = 1, EMOGI_PROBE_REGIONS = 2 };
emogi_status emogi_probe_host_reads(const void* host, uint64_t bytes, uint32_t pattern, uint32_t block_bytes,
                                    uint64_t blocks, void* cuda_stream, double* ms);

/* Static description of a status code. */
const char* emogi_status_string(emogi_status s);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* emogi_last_error(void);

/* Library version string. */
const char* emogi_version(void);

/* ---- Breadth-first search without any allocation --------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code running while another component owns the
 * whole device heap (a fixed arena reserved at start-up), code inside a
 * latency-critical loop that must not block or fail on allocation, or code
 * sharing a CUDA context whose allocator it may not touch.
 *
 * It computes exactly what emogi_bfs computes, but allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call) and needs no graph handle.
 * Its frontier queues and counters live in one fixed array inside the library
 * of 2 * EMOGI_NOALLOC_MAX_VERTICES * 4 + 256 bytes (16 MiB + 256 bytes), which
 * every GPU that loads the library holds until the process exits.
 *   n            number of vertices, 1 <= n <= EMOGI_NOALLOC_MAX_VERTICES;
 *                larger graphs are rejected with EMOGI_E_ARG
 *   row_offsets  device uint64_t[n+1] (CSR vertex list, as emogi_load_csr);
 *                the call reads row_offsets[n] (the edge count) once into a
 *                host variable
 *   col_idx      uint64_t[row_offsets[n]] readable by the current device:
 *                device memory or mapped pinned host memory; 16-byte aligned
 *                (not necessarily 128-byte aligned)
 *   src          source vertex, < n
 *   level        device uint32_t[n] output, as emogi_bfs
 *   cuda_stream  cudaStream_t to run on (NULL = the legacy default stream)
 * The call returns when the result is complete.  The first call on a device
 * looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture.  Every call on a
 * device shares the one array and the array keeps the previous call's
 * contents (the call clears what must start at zero), so calls whose work
 * overlaps on the GPU race: serialise them.
 * Errors: EMOGI_E_ARG (size or pointer rejected), EMOGI_E_CUDA, EMOGI_E_TIMEOUT. */
#define EMOGI_NOALLOC_MAX_VERTICES (1u << 21)
emogi_status emogi_bfs_noalloc(uint64_t n, const uint64_t* row_offsets, const uint64_t* col_idx,
                               uint64_t src, uint32_t* level, void* cuda_stream);

/* Testing hook: make the k-th device allocation from now on (k >= 1) fail as
 * if cudaMalloc had returned out-of-memory; 0 disarms.  Lets tests exercise
 * EMOGI_E_NOMEM handling without exhausting a real GPU. */
void emogi_test_fail_device_alloc_after(int k);

#ifdef __cplusplus
}
#endif

#endif /* EMOGI_H */
