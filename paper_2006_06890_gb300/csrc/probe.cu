// emogi_probe_host_reads: times zero-copy reads of a pinned host range in
// three patterns (a measurement aid; it computes nothing of the traversals).
//
// Sec. 5.3 of the paper measures how the request pattern of zero-copy reads
// decides the bandwidth the link delivers.  On GB300 the link's rate also
// depends on how far apart in the address space successive reads of a warp or
// block fall: random 512-byte reads over a 96 GiB pinned array ran at
// 19.7 GB/s, over 16 GiB at 210 GB/s, and the same reads at a fixed spacing
// walked by each block in its own region at 203-211 GB/s.  The traversals are
// laid out around that (vertex-ordered frontiers, per-block queue slices, the
// short-list store); this entry point makes the measurement repeatable on the
// graph's own arrays.
#include <cuda_runtime.h>

#include "internal.h"

namespace emogi {
namespace dev {

__device__ unsigned long long g_probe_sink;

// SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014): a
// bijective mix of the read's index, so the random pattern needs no table.
__device__ __forceinline__ uint64_t probe_mix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Reads `w16` uint4 words at q[lane], q[lane + 32], ... and folds them into acc.
__device__ __forceinline__ uint32_t probe_block(const uint4* q, uint64_t w16, uint32_t lane, uint32_t acc) {
    for (uint64_t j = lane; j < w16; j += 32) {
        const uint4 v = q[j];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    return acc;
}

// pattern 0: the grid streams [0, n16) words; 1: warps read `blocks` blocks of
// blk16 words at mixed block-aligned positions; 2: `blocks` blocks spaced
// stride16 words apart, block b of the grid reading its own contiguous share
// of them with its warps interleaved.
__global__ void __launch_bounds__(256) k_probe_reads(const uint4* __restrict__ p, uint64_t n16, uint32_t pattern,
                                                     uint64_t blk16, uint64_t blocks, uint64_t stride16) {
    uint32_t acc = 0;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    if (pattern == EMOGI_PROBE_STREAM) {
        for (uint64_t i = tid; i < n16; i += nth) {
            const uint4 v = p[i];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    } else if (pattern == EMOGI_PROBE_RANDOM) {
        const uint64_t nslots = n16 / blk16;  // >= 1, checked by the host
        for (uint64_t r = tid >> 5; r < blocks; r += nth >> 5)
            acc = probe_block(p + (probe_mix(r) % nslots) * blk16, blk16, lane, acc);
    } else {
        const uint64_t per = blocks / gridDim.x, extra = blocks % gridDim.x;
        const uint64_t first = blockIdx.x * per + (blockIdx.x < extra ? blockIdx.x : extra);
        const uint64_t count = per + (blockIdx.x < extra ? 1 : 0);
        const uint32_t wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        for (uint64_t i = wid; i < count; i += wpb) acc = probe_block(p + (first + i) * stride16, blk16, lane, acc);
    }
    if (acc == 0x9E3779B9u) atomicAdd(&g_probe_sink, 1ull);  // keeps the loads
}

}  // namespace dev
}  // namespace emogi

using namespace emogi;

extern "C" emogi_status emogi_probe_host_reads(const void* host, uint64_t bytes, uint32_t pattern,
                                               uint32_t block_bytes, uint64_t blocks, void* cuda_stream,
                                               double* ms) {
    if (!host || !ms) return fail(EMOGI_E_ARG, "probe: host and ms must not be NULL");
    *ms = 0.0;
    if (bytes < 16) return fail(EMOGI_E_ARG, "probe: the range must hold at least 16 bytes");
    if ((uintptr_t)host % 16) return fail(EMOGI_E_ARG, "probe: the range must start on a 16-byte boundary");
    if (pattern > EMOGI_PROBE_REGIONS) return fail(EMOGI_E_ARG, "probe: unknown pattern %u", pattern);
    const uint64_t n16 = bytes / 16;
    uint64_t blk16 = 0, stride16 = 0;
    if (pattern != EMOGI_PROBE_STREAM) {
        if (block_bytes < 16 || block_bytes % 16 || block_bytes > bytes)
            return fail(EMOGI_E_ARG, "probe: block_bytes %u must be a multiple of 16 in [16, bytes]", block_bytes);
        if (blocks == 0) return fail(EMOGI_E_ARG, "probe: blocks must be at least 1");
        blk16 = block_bytes / 16;
        if (pattern == EMOGI_PROBE_REGIONS) {
            stride16 = n16 / blocks;
            if (stride16 < blk16)
                return fail(EMOGI_E_ARG, "probe: %llu blocks of %u bytes do not fit %llu bytes apart",
                            (unsigned long long)blocks, block_bytes, (unsigned long long)(stride16 * 16));
        }
    }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return fail(EMOGI_E_ARG, "probe: the range is not pinned host memory (cudaHostAlloc / cudaHostRegister)");
    }
    void* dptr = nullptr;
    if (cudaHostGetDevicePointer(&dptr, const_cast<void*>(host), 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(EMOGI_E_ARG, "probe: the pinned range is not mapped for the device");
    }
    int device = 0;
    EMOGI_CUDA_TRY(cudaGetDevice(&device));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    bool own = false;
    if (!st) {
        EMOGI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
        dev::k_probe_reads<<<sm_count(device) * 8, 256, 0, st>>>((const uint4*)dptr, n16, pattern, blk16, blocks,
                                                                 stride16);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (own) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(EMOGI_E_CUDA, "probe: %s", cudaGetErrorString(e));
    *ms = t;
    return EMOGI_OK;
}
