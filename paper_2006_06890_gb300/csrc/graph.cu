// Graph loading and placement (paper Sec. 3.1 "Enabling Zero-Copy", Sec. 4.2
// "EMOGI Baseline", Sec. 5.1.2 (a) for the UVM baseline), the device-memory
// budget, work buffers and the status/error plumbing of the C ABI.
#include <cuda_runtime.h>
#include <sys/mman.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <fstream>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace emogi {

// ---------------------------------------------------------------- errors
static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }

emogi_status fail(emogi_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = std::string(emogi_status_string(s)) + ": " + buf;
    return s;
}

// ---------------------------------------------------------------- budget
static std::atomic<uint64_t> g_budget{0};
static std::atomic<uint64_t> g_in_use{0};
static std::atomic<int> g_fail_after{0};

emogi_status dev_alloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    uint64_t budget = g_budget.load();
    uint64_t prev = g_in_use.fetch_add(bytes);
    if (budget && prev + bytes > budget) {
        g_in_use.fetch_sub(bytes);
        return fail(EMOGI_E_BUDGET, "%s needs %zu bytes, %llu of %llu budget bytes already in use",
                    what, bytes, (unsigned long long)prev, (unsigned long long)budget);
    }
    int k = g_fail_after.load();
    if (k > 0) {
        if (g_fail_after.fetch_sub(1) == 1) {
            g_in_use.fetch_sub(bytes);
            return fail(EMOGI_E_NOMEM, "%s: injected device allocation failure", what);
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        g_in_use.fetch_sub(bytes);
        *p = nullptr;
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(EMOGI_E_NOMEM, "%s: cudaMalloc(%zu) out of memory", what, bytes);
        }
        return fail(EMOGI_E_CUDA, "%s: cudaMalloc(%zu): %s", what, bytes, cudaGetErrorString(e));
    }
    return EMOGI_OK;
}

emogi_status dev_free(void* p, size_t bytes) {
    if (!p) return EMOGI_OK;
    if (bytes == 0) bytes = 16;
    g_in_use.fetch_sub(bytes);
    EMOGI_CUDA_TRY(cudaFree(p));
    return EMOGI_OK;
}

int sm_count(int device) {
    static std::mutex mu;
    static std::vector<int> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= device) cache.resize(device + 1, 0);
    if (!cache[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cache[device] = v > 0 ? v : 1;
    }
    return cache[device];
}

emogi_status parse_opts(const emogi_opts* in, Opts* o) {
    *o = Opts();
    if (!in) return EMOGI_OK;
    if (in->struct_size < offsetof(emogi_opts, flags) + sizeof(uint32_t))
        return fail(EMOGI_E_ARG, "emogi_opts.struct_size %u is smaller than this library's %zu",
                    in->struct_size, sizeof(emogi_opts));
    if (in->access > EMOGI_ACCESS_NAIVE) return fail(EMOGI_E_ARG, "unknown access mode %u", in->access);
    if (in->granularity != 0 && in->granularity != 4 && in->granularity != 8 &&
        in->granularity != 16 && in->granularity != 32)
        return fail(EMOGI_E_ARG, "granularity must be 0, 4, 8, 16 or 32 (got %u)", in->granularity);
    if (in->chunk_lines > (1u << 20)) return fail(EMOGI_E_ARG, "chunk_lines too large");
    o->access = in->access;
    o->granularity = in->granularity;
    o->chunk_lines = in->chunk_lines;
    if (in->struct_size >= offsetof(emogi_opts, delta) + sizeof(uint32_t)) o->delta = in->delta;
    if (in->timeout_ns) o->timeout_ns = in->timeout_ns;
    o->stream = (cudaStream_t)in->cuda_stream;
    o->out_on_device = in->out_on_device != 0;
    o->flags = in->flags;
    return EMOGI_OK;
}

// ---------------------------------------------------------------- work buffers
// split-list vertices: a list is split when its aligned span exceeds 32 lines
// (512 uint64 ids or 1024 uint32 ids); the span starts at most 15 (31) ids
// before the list, so a split list holds at least 498 ids and one sweep splits
// at most m / 498
static uint64_t split_cap(uint64_t n, uint64_t m) { return std::min<uint64_t>(n, m / 497 + 1); }

uint64_t workspace_need(uint64_t n, uint64_t m) {
    n = n ? n : 1;
    return 6 * n * 4 + (n / 16 + 1) * 16 + split_cap(n, m) * 20 + sizeof(DevCounters) + 256;  // + SSSP loop state
}

emogi_status ensure_workspace(emogi_graph g) {
    Workspace& ws = g->ws;
    if (ws.ctr) return EMOGI_OK;
    const uint64_t n = g->n ? g->n : 1;
    ws.n = n;
    ws.lq_cap = split_cap(n, g->m);
    struct Item { void** p; size_t bytes; const char* what; };
    Item items[] = {
        {(void**)&ws.q[0], n * 4, "frontier queue 0"},
        {(void**)&ws.q[1], n * 4, "frontier queue 1"},
        {(void**)&ws.state, n * 4, "vertex state"},
        {(void**)&ws.qround, n * 4, "sweep stamps"},
        {(void**)&ws.fflag, n * 4, "far flags"},
        {(void**)&ws.xd, n * 4, "expanded distances"},
        {(void**)&ws.nflag, (n / 16 + 1) * 16, "next-frontier flags"},
        {(void**)&ws.lq_v, ws.lq_cap * 4, "split-list vertices"},
        {(void**)&ws.lq_base, ws.lq_cap * 8, "split-list chunk bases"},
        {(void**)&ws.lq_state, ws.lq_cap * 8, "split-list states"},
        {(void**)&ws.ctr, sizeof(DevCounters), "counters"},
    };
    for (auto& it : items) {
        emogi_status s = dev_alloc(it.p, it.bytes, it.what);
        if (s != EMOGI_OK) {
            release_workspace(g);
            return s;
        }
        ws.dev_bytes += it.bytes;
    }
    cudaError_t e = cudaHostAlloc((void**)&ws.h_ctr, sizeof(DevCounters), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMemset(ws.qround, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(ws.fflag, 0, n * 4);
    if (e == cudaSuccess) e = cudaMemset(ws.nflag, 0, (n / 16 + 1) * 16);
    // cudaMemset runs on the legacy default stream, which the traversals'
    // non-blocking streams do not wait for: finish it before any of them starts
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaEventCreate(&ws.ev[i]);
    if (e != cudaSuccess) {
        release_workspace(g);
        return fail(EMOGI_E_CUDA, "work buffers: %s", cudaGetErrorString(e));
    }
    return EMOGI_OK;
}

void release_workspace(emogi_graph g) {
    Workspace& ws = g->ws;
    dev_free(ws.q[0], ws.n * 4);
    dev_free(ws.q[1], ws.n * 4);
    dev_free(ws.state, ws.n * 4);
    dev_free(ws.qround, ws.n * 4);
    dev_free(ws.fflag, ws.n * 4);
    dev_free(ws.xd, ws.n * 4);
    dev_free(ws.nflag, (ws.n / 16 + 1) * 16);
    dev_free(ws.lq_v, ws.lq_cap * 4);
    dev_free(ws.lq_base, ws.lq_cap * 8);
    dev_free(ws.lq_state, ws.lq_cap * 8);
    dev_free(ws.pr_rank, ws.n * 8);
    dev_free(ws.pr_contrib, ws.n * 8);
    dev_free(ws.pr_acc, ws.n * 8);
    dev_free(ws.pr_ctr, 64);
    if (ws.h_pr_ctr) cudaFreeHost(ws.h_pr_ctr);
    dev_free(ws.ms_visit, ws.n * 8);
    dev_free(ws.ms_front, ws.n * 8);
    dev_free(ws.ms_next, ws.n * 8);
    dev_free(ws.ms_out, ws.ms_out_bytes);
    if (ws.sssp_exec) cudaGraphExecDestroy(ws.sssp_exec);
    dev_free(ws.sssp_loop, 256);
    if (ws.h_sssp_loop) cudaFreeHost(ws.h_sssp_loop);
    dev_free(ws.ctr, sizeof(DevCounters));
    // dev_free's accounting assumes the sizes it was allocated with; when a
    // partial allocation failed, unallocated entries are null and skipped.
    if (ws.h_ctr) cudaFreeHost(ws.h_ctr);
    for (auto& e : ws.ev)
        if (e) cudaEventDestroy(e);
    ws = Workspace();
}

// ---------------------------------------------------------------- validation
// Checks the CSR in parallel on the host: offsets monotone from 0 to m, every
// column id below n.
template <class Id>
static emogi_status validate_csr(uint64_t n, uint64_t m, const uint64_t* off, const Id* cols) {
    if (off[0] != 0) return fail(EMOGI_E_ARG, "row_offsets[0] = %llu, expected 0", (unsigned long long)off[0]);
    if (off[n] != m)
        return fail(EMOGI_E_ARG, "row_offsets[n] = %llu but m = %llu", (unsigned long long)off[n],
                    (unsigned long long)m);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<uint64_t> bad_row{UINT64_MAX}, bad_col{UINT64_MAX};
    auto work = [&](unsigned t) {
        uint64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
        for (uint64_t v = r0; v < r1; v++)
            if (off[v + 1] < off[v]) { bad_row = v; return; }
        uint64_t c0 = m * t / nt, c1 = m * (t + 1) / nt;
        for (uint64_t i = c0; i < c1; i++)
            if (cols[i] >= n) { bad_col = i; return; }
    };
    if ((uint64_t)nt * 65536 > m + n) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    if (bad_row != UINT64_MAX)
        return fail(EMOGI_E_ARG, "row_offsets decrease at vertex %llu", (unsigned long long)bad_row.load());
    if (bad_col != UINT64_MAX)
        return fail(EMOGI_E_ARG, "col_idx[%llu] = %llu is not below n = %llu", (unsigned long long)bad_col.load(),
                    (unsigned long long)cols[bad_col.load()], (unsigned long long)n);
    return EMOGI_OK;
}

static void parallel_copy(void* dst, const void* src, size_t bytes) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (bytes < (64u << 20)) nt = 1;
    std::vector<std::thread> th;
    auto work = [&](unsigned t) {
        size_t a = bytes * t / nt, b = bytes * (t + 1) / nt;
        memcpy((char*)dst + a, (const char*)src + a, b - a);
    };
    for (unsigned t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
}

// ---------------------------------------------------------------- pinned host arrays
// A HOST-placed array of a GiB or more is an anonymous mapping advised to use
// transparent huge pages, filled, then pinned and mapped with
// cudaHostRegister; smaller ones come from cudaHostAlloc.  The GPU reads a
// zero-copy edge list at random across its whole extent, so the number of
// pages it spans matters: measured on GB300 (a host with 64 KiB pages and
// 512 MiB transparent huge pages), SSSP over a 50 GB Kronecker edge list took
// 1.83 s from cudaHostAlloc memory and 1.14 s from huge pages, while 64 KiB
// pages stalled it (six rounds in 30 s).
static size_t huge_page_bytes() {
    static const size_t sz = [] {
        size_t v = 0;
        std::ifstream f("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size");
        if (f) f >> v;
        return v >= 4096 && (v & (v - 1)) == 0 ? v : (size_t)2 << 20;
    }();
    return sz;
}
static bool host_array_is_mapped(size_t alloc) { return alloc >= ((size_t)1 << 30); }
static size_t host_map_len(size_t alloc) {
    const size_t a = huge_page_bytes();
    return (alloc + a - 1) / a * a;
}

// An anonymous mapping of host_map_len(alloc) bytes starting on a huge-page
// boundary, advised to use huge pages; nullptr on failure.
static void* host_map(size_t alloc) {
    const size_t a = huge_page_bytes(), len = host_map_len(alloc);
    void* p = mmap(nullptr, len + a, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (p == MAP_FAILED) return nullptr;
    const uintptr_t u = (uintptr_t)p, al = (u + a - 1) & ~(uintptr_t)(a - 1);
    if (al > u) munmap(p, al - u);
    const size_t tail = (u + len + a) - (al + len);
    if (tail) munmap((void*)(al + len), tail);
    madvise((void*)al, len, MADV_HUGEPAGE);  // best effort: without THP the pages stay small
    return (void*)al;
}

// Places one edge-sized array according to the placement.  Fills *kernel_ptr
// (what kernels dereference), *owned (what to free) or *borrowed (what to
// unregister) and adds device bytes to *dev_bytes.
static emogi_status place_array(int place, bool borrow, int device, const void* src, size_t bytes,
                                const void** kernel_ptr, void** owned, const void** borrowed,
                                size_t* dev_bytes, const char* what) {
    *kernel_ptr = nullptr;
    *owned = nullptr;
    *borrowed = nullptr;
    // pad so that a 16-byte vector access at the last even index stays inside
    size_t alloc = ((bytes + 127) / 128) * 128 + 128;
    if (place == EMOGI_PLACE_DEVICE) {
        void* p = nullptr;
        EMOGI_TRY(dev_alloc(&p, alloc, what));
        cudaError_t e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            dev_free(p, alloc);
            return fail(EMOGI_E_CUDA, "%s: copy to device: %s", what, cudaGetErrorString(e));
        }
        *kernel_ptr = p;
        *owned = p;
        *dev_bytes += alloc;
    } else if (borrow && bytes == 0) {
        *kernel_ptr = src;  // nothing to pin; kernels never dereference an empty list
    } else if (place == EMOGI_PLACE_MANAGED && borrow) {
        // the caller's managed array, used in place with the baseline's
        // read-mostly advice (the UVM baseline of Sec. 5.1.2 (a))
        if (((uintptr_t)src) % 16)
            return fail(EMOGI_E_ARG, "%s: borrowed arrays must be 16-byte aligned", what);
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, src);
        if (e != cudaSuccess || at.type != cudaMemoryTypeManaged) {
            cudaGetLastError();
            return fail(EMOGI_E_ARG, "%s: a borrowed MANAGED array must come from cudaMallocManaged", what);
        }
        cudaMemLocation loc;
        loc.type = cudaMemLocationTypeDevice;
        loc.id = device;
        e = cudaMemAdvise(src, bytes, cudaMemAdviseSetReadMostly, loc);
        if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "%s: cudaMemAdvise(ReadMostly): %s", what, cudaGetErrorString(e));
        *kernel_ptr = src;
        *borrowed = src;
    } else if (place == EMOGI_PLACE_HOST && borrow) {
        if (((uintptr_t)src) % 16)
            return fail(EMOGI_E_ARG, "%s: borrowed arrays must be 16-byte aligned", what);
        cudaError_t e = cudaHostRegister((void*)src, bytes ? bytes : 16,
                                         cudaHostRegisterMapped | cudaHostRegisterReadOnly);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaHostRegister((void*)src, bytes ? bytes : 16, cudaHostRegisterMapped);
        }
        if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "%s: cudaHostRegister: %s", what, cudaGetErrorString(e));
        void* dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, (void*)src, 0);
        if (e != cudaSuccess) {
            cudaHostUnregister((void*)src);
            return fail(EMOGI_E_CUDA, "%s: cudaHostGetDevicePointer: %s", what, cudaGetErrorString(e));
        }
        *kernel_ptr = dp;
        *borrowed = src;
    } else if (place == EMOGI_PLACE_HOST && host_array_is_mapped(alloc)) {
        void* h = host_map(alloc);
        if (!h) return fail(EMOGI_E_NOMEM, "%s: mmap(%zu) failed", what, host_map_len(alloc));
        parallel_copy(h, src, bytes);
        memset((char*)h + bytes, 0, alloc - bytes);
        cudaError_t e = cudaHostRegister(h, alloc, cudaHostRegisterMapped | cudaHostRegisterReadOnly);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaHostRegister(h, alloc, cudaHostRegisterMapped);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            munmap(h, host_map_len(alloc));
            return fail(EMOGI_E_NOMEM, "%s: cudaHostRegister(%zu): %s", what, alloc, cudaGetErrorString(e));
        }
        void* dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, h, 0);
        if (e != cudaSuccess) {
            cudaHostUnregister(h);
            munmap(h, host_map_len(alloc));
            return fail(EMOGI_E_CUDA, "%s: cudaHostGetDevicePointer: %s", what, cudaGetErrorString(e));
        }
        *kernel_ptr = dp;
        *owned = h;
    } else if (place == EMOGI_PLACE_HOST) {
        void* h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, alloc, cudaHostAllocMapped);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(EMOGI_E_NOMEM, "%s: cudaHostAlloc(%zu): %s", what, alloc, cudaGetErrorString(e));
        }
        parallel_copy(h, src, bytes);
        memset((char*)h + bytes, 0, alloc - bytes);
        void* dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, h, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(h);
            return fail(EMOGI_E_CUDA, "%s: cudaHostGetDevicePointer: %s", what, cudaGetErrorString(e));
        }
        *kernel_ptr = dp;
        *owned = h;
    } else {  // MANAGED: the UVM baseline, edge list marked read-mostly
        void* p = nullptr;
        cudaError_t e = cudaMallocManaged(&p, alloc, cudaMemAttachGlobal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(EMOGI_E_NOMEM, "%s: cudaMallocManaged(%zu): %s", what, alloc, cudaGetErrorString(e));
        }
        parallel_copy(p, src, bytes);
        memset((char*)p + bytes, 0, alloc - bytes);
        cudaMemLocation loc;
        loc.type = cudaMemLocationTypeDevice;
        loc.id = device;
        e = cudaMemAdvise(p, alloc, cudaMemAdviseSetReadMostly, loc);
        if (e != cudaSuccess) {
            cudaFree(p);
            return fail(EMOGI_E_CUDA, "%s: cudaMemAdvise(ReadMostly): %s", what, cudaGetErrorString(e));
        }
        *kernel_ptr = p;
        *owned = p;
    }
    return EMOGI_OK;
}

// heads[v * 4 + r] = col_idx[row_offsets[v] + r] for r < degree, else
// UINT32_MAX; gathered on the host from the caller's arrays (no device read
// of the placed edge list, so a managed edge list is not migrated by this).
template <class Id>
static emogi_status build_heads(emogi_graph g, const uint64_t* off, const Id* cols) {
    const uint64_t n = g->n;
    std::vector<uint32_t> h;
    try {
        h.resize(n * 4);
    } catch (...) {
        return fail(EMOGI_E_NOMEM, "list heads staging (%llu bytes)", (unsigned long long)(n * 16));
    }
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 65536) nt = 1;
    auto work = [&](unsigned t) {
        const uint64_t v0 = n * t / nt, v1 = n * (t + 1) / nt;
        for (uint64_t v = v0; v < v1; v++)
            for (uint64_t r = 0; r < 4; r++)
                h[v * 4 + r] = off[v] + r < off[v + 1] ? (uint32_t)cols[off[v] + r] : 0xFFFFFFFFu;
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    EMOGI_CUDA_TRY(cudaMemcpy(g->d_heads, h.data(), n * 16, cudaMemcpyHostToDevice));
    return EMOGI_OK;
}

// The short-list store: every list of 1..g->short_max entries, copied whole
// (ids, and weights when given) into GPU memory, lists starting on 4-entry
// boundaries; short_off[v] is the start in units of 4 entries (lists longer
// than that or empty get 0 and are never read there).  The bound is
// kStoreWide when the lists up to that length hold at most 1/kStoreShare of
// the entries, else kStoreBase; a bound whose store (with the index) and the
// work buffers of one handle do not fit what the device budget leaves is
// dropped for the smaller one, and then for no store.  Built on the host from
// the caller's arrays in two parallel passes (counts per block of vertices
// for both bounds, then the copy), then copied to the device.
template <class Id>
static emogi_status build_short_store(emogi_graph g, const uint64_t* off, const Id* cols, const uint32_t* weights) {
    const uint64_t n = g->n;
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 65536) nt = 1;
    auto slots_of = [&](uint64_t v, uint32_t bound) -> uint64_t {
        const uint64_t d = off[v + 1] - off[v];
        return d >= 1 && d <= bound ? (d + 3) / 4 * 4 : 0;
    };
    // per block of vertices: slots and entries of the lists of 1..kStoreBase
    // and of 1..kStoreWide entries
    struct Count { uint64_t slots[2] = {0, 0}, ents[2] = {0, 0}; };
    std::vector<Count> cnt(nt);
    {
        std::vector<std::thread> th;
        auto count = [&](unsigned t) {
            Count x;
            for (uint64_t v = n * t / nt; v < n * (t + 1) / nt; v++) {
                const uint64_t d = off[v + 1] - off[v];
                if (d < 1 || d > kStoreWide) continue;
                const uint64_t k = (d + 3) / 4 * 4;
                x.slots[1] += k;
                x.ents[1] += d;
                if (d <= kStoreBase) {
                    x.slots[0] += k;
                    x.ents[0] += d;
                }
            }
            cnt[t] = x;
        };
        for (unsigned t = 1; t < nt; t++) th.emplace_back(count, t);
        count(0);
        for (auto& x : th) x.join();
    }
    Count all;
    for (const auto& x : cnt)
        for (int b = 0; b < 2; b++) {
            all.slots[b] += x.slots[b];
            all.ents[b] += x.ents[b];
        }
    const uint64_t budget = g_budget.load();
    auto fits = [&](int b) {
        if (all.slots[b] == 0 || all.slots[b] / 4 >= 0xFFFFFFFFull) return false;  // the uint32 index
        if (!budget) return true;
        const uint64_t need = n * 4 + all.slots[b] * (weights ? 8 : 4) + workspace_need(n, g->m);
        const uint64_t used = g_in_use.load();
        return used <= budget && need <= budget - used;
    };
    int pick = -1;
    if (all.ents[1] * kStoreShare <= g->m && fits(1)) pick = 1;
    else if (fits(0)) pick = 0;
    if (pick < 0) {  // nothing to store, or no room for it
        g->short_max = 0;
        return EMOGI_OK;
    }
    g->short_max = pick ? kStoreWide : kStoreBase;
    std::vector<uint64_t> part(nt + 1, 0);
    for (unsigned t = 0; t < nt; t++) part[t + 1] = part[t] + cnt[t].slots[pick];
    const uint64_t slots = part[nt];
    std::vector<uint32_t> so, sid, sw;
    try {
        so.resize(n);
        sid.assign(slots, 0xFFFFFFFFu);
        if (weights) sw.assign(slots, 0u);
    } catch (...) {
        return fail(EMOGI_E_NOMEM, "short-list store staging (%llu bytes)",
                    (unsigned long long)(n * 4 + slots * (weights ? 8 : 4)));
    }
    std::vector<uint64_t> ents(nt, 0);
    {
        std::vector<std::thread> th;
        auto fill = [&](unsigned t) {
            uint64_t pos = part[t], e = 0;
            for (uint64_t v = n * t / nt; v < n * (t + 1) / nt; v++) {
                const uint64_t k = slots_of(v, g->short_max);
                so[v] = (uint32_t)(pos / 4);
                if (!k) continue;
                const uint64_t d = off[v + 1] - off[v];
                for (uint64_t r = 0; r < d; r++) {
                    sid[pos + r] = (uint32_t)cols[off[v] + r];
                    if (weights) sw[pos + r] = weights[off[v] + r];
                }
                pos += k;
                e += d;
            }
            ents[t] = e;
        };
        for (unsigned t = 1; t < nt; t++) th.emplace_back(fill, t);
        fill(0);
        for (auto& x : th) x.join();
    }
    uint64_t entries = 0;
    for (auto e : ents) entries += e;
    EMOGI_TRY(dev_alloc((void**)&g->d_short_off, n * 4, "short-list store index"));
    g->dev_bytes += n * 4;
    EMOGI_TRY(dev_alloc((void**)&g->d_short_ids, slots * 4, "short-list store ids"));
    g->dev_bytes += slots * 4;
    if (weights) {
        EMOGI_TRY(dev_alloc((void**)&g->d_short_w, slots * 4, "short-list store weights"));
        g->dev_bytes += slots * 4;
    }
    g->short_slots = slots;
    g->short_entries = entries;
    EMOGI_CUDA_TRY(cudaMemcpy(g->d_short_off, so.data(), n * 4, cudaMemcpyHostToDevice));
    EMOGI_CUDA_TRY(cudaMemcpy(g->d_short_ids, sid.data(), slots * 4, cudaMemcpyHostToDevice));
    if (weights) EMOGI_CUDA_TRY(cudaMemcpy(g->d_short_w, sw.data(), slots * 4, cudaMemcpyHostToDevice));
    return EMOGI_OK;
}

static void release_array(int place, void* owned, const void* borrowed, size_t bytes) {
    size_t alloc = ((bytes + 127) / 128) * 128 + 128;
    if (borrowed && place == EMOGI_PLACE_HOST) cudaHostUnregister((void*)borrowed);
    if (!owned) return;
    if (place == EMOGI_PLACE_DEVICE) {
        dev_free(owned, alloc);
    } else if (place == EMOGI_PLACE_HOST && host_array_is_mapped(alloc)) {
        cudaHostUnregister(owned);
        munmap(owned, host_map_len(alloc));
    } else if (place == EMOGI_PLACE_HOST) {
        cudaFreeHost(owned);
    } else {
        cudaFree(owned);
    }
}

}  // namespace emogi

namespace emogi {

template <class Id>
static emogi_status load_csr(uint64_t n, uint64_t m, const uint64_t* row_offsets, const Id* col_idx,
                             const uint32_t* weights, emogi_placement place, uint32_t flags, emogi_graph* out) {
    clear_error();
    if (!out) return fail(EMOGI_E_ARG, "out is NULL");
    *out = nullptr;
    if (n >= 0xFFFFFFFFull) return fail(EMOGI_E_ARG, "n = %llu must be below 2^32 - 1", (unsigned long long)n);
    if (!row_offsets) return fail(EMOGI_E_ARG, "row_offsets is NULL");
    if (m && !col_idx) return fail(EMOGI_E_ARG, "col_idx is NULL");
    if ((int)place < EMOGI_PLACE_DEVICE || (int)place > EMOGI_PLACE_MANAGED)
        return fail(EMOGI_E_ARG, "unknown placement %d", (int)place);
    if (flags & ~(uint32_t)(EMOGI_LOAD_UNDIRECTED | EMOGI_LOAD_BORROW | EMOGI_LOAD_NO_HEADS))
        return fail(EMOGI_E_ARG, "unknown load flags 0x%x", flags);
    const bool borrow = flags & EMOGI_LOAD_BORROW;
    if (borrow && place == EMOGI_PLACE_DEVICE)
        return fail(EMOGI_E_ARG, "EMOGI_LOAD_BORROW needs EMOGI_PLACE_HOST or EMOGI_PLACE_MANAGED");
    EMOGI_TRY(validate_csr(n, m, row_offsets, col_idx));

    emogi_graph g = new (std::nothrow) emogi_graph_s();
    if (!g) return fail(EMOGI_E_NOMEM, "graph handle");
    g->n = n;
    g->m = m;
    g->flags = flags;
    g->place = place;
    g->avg_degree = n ? (double)m / (double)n : 0.0;
    for (uint64_t v = 0; v < n; v++) g->max_degree = std::max<uint64_t>(g->max_degree, row_offsets[v + 1] - row_offsets[v]);
    auto bail = [&](emogi_status s) {
        emogi_free_graph(g);
        return s;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "no CUDA device"));
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));

    // vertex list in GPU memory (Sec. 4.2)
    size_t off_bytes = (n + 1) * sizeof(uint64_t);
    emogi_status s = dev_alloc((void**)&g->d_off, off_bytes, "row offsets");
    if (s != EMOGI_OK) return bail(s);
    g->dev_bytes += off_bytes;
    e = cudaMemcpy(g->d_off, row_offsets, off_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "offsets copy: %s", cudaGetErrorString(e)));

    // edge list (and weights) by placement (Sec. 3.1, Sec. 5.1.2)
    const void* kp = nullptr;
    g->id_bytes = sizeof(Id);
    s = place_array(place, borrow, g->device, col_idx, m * sizeof(Id), &kp, &g->cols_owned,
                    &g->cols_borrowed, &g->dev_bytes, "edge list");
    if (s != EMOGI_OK) return bail(s);
    g->cols = kp;
    g->shift = (uint32_t)(((uintptr_t)g->cols % 128) / sizeof(Id));
    if (weights) {
        // mean weight from up to 2^20 evenly spaced entries
        const uint64_t stride = m > (1u << 20) ? m / (1u << 20) : 1;
        double sum = 0.0;
        uint64_t cnt = 0;
        for (uint64_t i = 0; i < m; i += stride, cnt++) sum += weights[i];
        g->avg_weight = cnt ? sum / (double)cnt : 0.0;
        if (borrow && ((uintptr_t)weights % 16)) return bail(fail(EMOGI_E_ARG, "borrowed weights must be 16-byte aligned"));
        s = place_array(place, borrow, g->device, weights, m * sizeof(uint32_t), &kp, &g->w_owned, &g->w_borrowed,
                        &g->dev_bytes, "weights");
        if (s != EMOGI_OK) return bail(s);
        g->w = (const uint32_t*)kp;
    }
    // list heads and the short-list store: when the edge list itself is not in
    // GPU memory, the first ids of every list (16 bytes per vertex) and every
    // list of at most 16 or 32 entries (ids and weights) are mirrored there
    if (place != EMOGI_PLACE_DEVICE && !(flags & EMOGI_LOAD_NO_HEADS) && n && m) {
        s = dev_alloc((void**)&g->d_heads, n * 4 * sizeof(uint32_t), "list heads");
        if (s != EMOGI_OK) return bail(s);
        g->dev_bytes += n * 4 * sizeof(uint32_t);
        s = build_heads(g, row_offsets, col_idx);
        if (s != EMOGI_OK) return bail(s);
        s = build_short_store(g, row_offsets, col_idx, weights);
        if (s != EMOGI_OK) return bail(s);
    }
    // The uploads above (cudaMemcpy, from pageable host memory) run on the
    // legacy default stream and may return before their DMA has landed; the
    // traversals run on non-blocking streams, which do not wait for the
    // legacy stream.  Measured on GB300: a BFS started at once after loading a
    // 134 M-vertex graph (1 GB of offsets) read offsets still in flight and got
    // wrong levels.  So the load returns only once every upload is complete.
    e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) return bail(fail(EMOGI_E_CUDA, "graph upload: %s", cudaGetErrorString(e)));
    *out = g;
    return EMOGI_OK;
}

}  // namespace emogi

using namespace emogi;

extern "C" {

const char* emogi_status_string(emogi_status s) {
    switch (s) {
        case EMOGI_OK: return "EMOGI_OK";
        case EMOGI_E_ARG: return "EMOGI_E_ARG";
        case EMOGI_E_NOMEM: return "EMOGI_E_NOMEM";
        case EMOGI_E_BUDGET: return "EMOGI_E_BUDGET";
        case EMOGI_E_CUDA: return "EMOGI_E_CUDA";
        case EMOGI_E_TIMEOUT: return "EMOGI_E_TIMEOUT";
        case EMOGI_E_OVERFLOW: return "EMOGI_E_OVERFLOW";
        case EMOGI_E_UNSUPPORTED: return "EMOGI_E_UNSUPPORTED";
    }
    return "EMOGI_E_UNKNOWN";
}

const char* emogi_last_error(void) { return t_last_error.c_str(); }

const char* emogi_version(void) { return "emogi-gb300 0.1 (sm_103a)"; }

emogi_status emogi_set_device_budget(uint64_t bytes) {
    g_budget = bytes;
    return EMOGI_OK;
}

uint64_t emogi_device_bytes_in_use(void) { return g_in_use.load(); }

emogi_status emogi_managed_alloc(uint64_t bytes, void** out) {
    clear_error();
    if (!out || bytes == 0) return fail(EMOGI_E_ARG, "emogi_managed_alloc needs out != NULL and bytes > 0");
    *out = nullptr;
    cudaError_t e = cudaMallocManaged(out, bytes, cudaMemAttachGlobal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(EMOGI_E_NOMEM, "cudaMallocManaged(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
    }
    return EMOGI_OK;
}

emogi_status emogi_managed_free(void* p) {
    clear_error();
    if (!p) return EMOGI_OK;
    EMOGI_CUDA_TRY(cudaFree(p));
    return EMOGI_OK;
}

void emogi_test_fail_device_alloc_after(int k) { g_fail_after = k > 0 ? k : 0; }

emogi_status emogi_load_csr(uint64_t n, uint64_t m, const uint64_t* row_offsets, const uint64_t* col_idx,
                            const uint32_t* weights, emogi_placement place, uint32_t flags, emogi_graph* out) {
    return load_csr<uint64_t>(n, m, row_offsets, col_idx, weights, place, flags, out);
}

emogi_status emogi_load_csr32(uint64_t n, uint64_t m, const uint64_t* row_offsets, const uint32_t* col_idx,
                              const uint32_t* weights, emogi_placement place, uint32_t flags, emogi_graph* out) {
    return load_csr<uint32_t>(n, m, row_offsets, col_idx, weights, place, flags, out);
}

emogi_status emogi_free_graph(emogi_graph g) {
    if (!g) return EMOGI_OK;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    release_workspace(g);
    if (!g->shared) {
        if (g->d_heads) dev_free(g->d_heads, g->n * 4 * sizeof(uint32_t));
        if (g->d_short_off) dev_free(g->d_short_off, g->n * 4);
        if (g->d_short_ids) dev_free(g->d_short_ids, g->short_slots * 4);
        if (g->d_short_w) dev_free(g->d_short_w, g->short_slots * 4);
        release_array(g->place, g->cols_owned, g->cols_borrowed, g->m * g->id_bytes);
        if (g->w || g->w_owned || g->w_borrowed)
            release_array(g->place, g->w_owned, g->w_borrowed, g->m * sizeof(uint32_t));
        if (g->d_off) dev_free(g->d_off, (g->n + 1) * sizeof(uint64_t));
    }
    cudaError_t e = cudaSuccess;
    if (g->stream) e = cudaStreamDestroy(g->stream);
    delete g;
    if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "cudaStreamDestroy: %s", cudaGetErrorString(e));
    return EMOGI_OK;
}

emogi_status emogi_graph_share(emogi_graph g, emogi_graph* out) {
    clear_error();
    if (!g || !out) return fail(EMOGI_E_ARG, "graph and out must be non-NULL");
    *out = nullptr;
    emogi_graph h = new (std::nothrow) emogi_graph_s();
    if (!h) return fail(EMOGI_E_NOMEM, "graph handle");
    h->device = g->device;
    h->n = g->n;
    h->m = g->m;
    h->flags = g->flags;
    h->place = g->place;
    h->d_off = g->d_off;
    h->d_heads = g->d_heads;
    h->d_short_off = g->d_short_off;
    h->d_short_ids = g->d_short_ids;
    h->d_short_w = g->d_short_w;
    h->short_max = g->short_max;
    h->short_slots = g->short_slots;
    h->short_entries = g->short_entries;
    h->cols = g->cols;
    h->id_bytes = g->id_bytes;
    h->w = g->w;
    h->shift = g->shift;
    h->avg_degree = g->avg_degree;
    h->max_degree = g->max_degree;
    h->avg_weight = g->avg_weight;
    h->shared = true;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return fail(EMOGI_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    *out = h;
    return EMOGI_OK;
}

uint64_t emogi_graph_workspace_bytes(emogi_graph g) { return g ? g->ws.dev_bytes : 0; }

uint64_t emogi_graph_num_vertices(emogi_graph g) { return g ? g->n : 0; }
uint64_t emogi_graph_num_edges(emogi_graph g) { return g ? g->m : 0; }
int emogi_graph_placement(emogi_graph g) { return g ? g->place : -1; }
uint32_t emogi_graph_store_bound(emogi_graph g) { return g ? g->short_max : 0; }

}  // extern "C"
