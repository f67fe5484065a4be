// emogi_bfs_noalloc: breadth-first search for callers that cannot allocate
// GPU memory.
//
// Some callers must not call cudaMalloc at all: code that runs while another
// component owns every byte of the device heap (a fixed arena carved out at
// start-up), code that must not block or fault on allocation inside a
// latency-critical loop, or hosts whose CUDA context is shared and whose
// allocator is off limits.  This entry point serves them: it allocates
// nothing.  The caller passes the graph (row offsets in device memory, the
// edge list in device memory or mapped pinned host memory) and the output
// array; the frontier queues and counters the traversal needs live in one
// fixed array in this file that every GPU holding the library keeps until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace emogi {
namespace {

// Scratch layout: two frontier queues of EMOGI_NOALLOC_MAX_VERTICES entries,
// then the counters.  16 MiB + 256 bytes per device.
constexpr uint64_t kMaxN = EMOGI_NOALLOC_MAX_VERTICES;
constexpr uint64_t kQueueWords = kMaxN;
constexpr uint64_t kCounterBytes = 256;
constexpr uint64_t kScratchBytes = 2 * kQueueWords * sizeof(uint32_t) + kCounterBytes;
static_assert(sizeof(DevCounters) <= kCounterBytes, "counters must fit the scratch tail");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (in host code the symbol itself is only a host-side
// stand-in and must never be passed to a kernel).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

emogi_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    EMOGI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(EMOGI_E_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(EMOGI_E_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_addr[dev];
    return EMOGI_OK;
}

}  // namespace
}  // namespace emogi

using namespace emogi;

extern "C" emogi_status emogi_bfs_noalloc(uint64_t n, const uint64_t* row_offsets, const uint64_t* col_idx,
                                          uint64_t src, uint32_t* level, void* cuda_stream) {
    clear_error();
    if (n == 0 || n > kMaxN)
        return fail(EMOGI_E_ARG, "emogi_bfs_noalloc handles 1 to %llu vertices (got %llu); use emogi_bfs",
                    (unsigned long long)kMaxN, (unsigned long long)n);
    if (src >= n) return fail(EMOGI_E_ARG, "source %llu is not below n = %llu", (unsigned long long)src,
                              (unsigned long long)n);
    if (!row_offsets || !level) return fail(EMOGI_E_ARG, "row_offsets and level must be non-NULL");
    if (((uintptr_t)col_idx) % 16) return fail(EMOGI_E_ARG, "col_idx must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* scratch = nullptr;
    EMOGI_TRY(scratch_for_current_device(&scratch));
    uint32_t* q0 = (uint32_t*)scratch;
    uint32_t* q1 = q0 + kQueueWords;
    DevCounters* ctr = (DevCounters*)(scratch + 2 * kQueueWords * sizeof(uint32_t));
    int dev = 0, sms = 1;
    EMOGI_CUDA_TRY(cudaGetDevice(&dev));
    EMOGI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, cap = sms * 8;
    auto grid = [&](uint64_t t) {
        uint64_t b = (t + threads - 1) / threads;
        return (int)(b < 1 ? 1 : (b > (uint64_t)cap ? (uint64_t)cap : b));
    };

    // The edge count (row_offsets[n]) lets a list's last ids come in one
    // whole 16-byte load wherever that load ends inside the edge list, as in
    // emogi_bfs; read into a host variable, which allocates nothing.
    uint64_t m = 0;
    EMOGI_CUDA_TRY(cudaMemcpyAsync(&m, row_offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    EMOGI_CUDA_TRY(cudaStreamSynchronize(st));

    // the array keeps the previous call's contents: clear the counters
    EMOGI_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st));
    dev::k_init_single<<<grid(n), threads, 0, st>>>(level, (uint32_t)n, (uint32_t)src, q0, nullptr,
                                                    &ctr->qcount[0]);
    EMOGI_CUDA_TRY(cudaGetLastError());

    uint32_t* q[2] = {q0, q1};
    uint64_t k = 1;
    int side = 0;
    for (uint32_t it = 0; k > 0; it++) {
        if (it > n + 1) return fail(EMOGI_E_TIMEOUT, "BFS did not converge in %u levels", it);
        EMOGI_CUDA_TRY(cudaMemsetAsync(&ctr->qcount[side ^ 1], 0, sizeof(uint32_t), st));
        dev::Sweep s;
        s.off = row_offsets;
        s.cols = col_idx;
        s.w = nullptr;
        s.shift = (uint32_t)(((uintptr_t)col_idx % 128) / 8);
        s.in_q = q[side];
        s.in_count = &ctr->qcount[side];
        s.all_n = (uint32_t)n;
        s.out_q = q[side ^ 1];
        s.out_count = &ctr->qcount[side ^ 1];
        s.lq_v = nullptr;  // long lists are read by their group here, never split
        s.lq_base = nullptr;
        s.large = &ctr->large[0];
        s.large_lines = 0xFFFFFFFFu;
        s.chunk_lines = 1;
        s.scanned = &ctr->scanned;
        s.m = m;
        s.qcap = (uint32_t)n;
        dev::k_expand_group<dev::BfsOp, 8><<<grid(k * 8), threads, 0, st>>>(s, dev::BfsOp{level, it + 1});
        EMOGI_CUDA_TRY(cudaGetLastError());
        uint32_t next = 0;
        EMOGI_CUDA_TRY(cudaMemcpyAsync(&next, &ctr->qcount[side ^ 1], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        EMOGI_CUDA_TRY(cudaStreamSynchronize(st));
        if (next > n) return fail(EMOGI_E_CUDA, "internal error: a BFS frontier of %u entries exceeds n = %llu",
                                  next, (unsigned long long)n);
        k = next;
        side ^= 1;
    }
    return EMOGI_OK;
}
