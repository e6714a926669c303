// Random-gather rate probe: the memory ceilings of the traversal kernels.
//
// The beam traversal (Sec. 2.2.1) reads one map cell (or one distance byte)
// at a data-dependent address per visit, and the lanes of a warp follow
// unrelated rays, so their addresses are effectively random.  Its ceiling is
// therefore not a streaming bandwidth but the rate at which the SMs can
// serve random single-byte gathers: from shared memory (bank conflicts set
// the rate) when the map is staged there, from L2 when it is read through
// the read-only path.  This kernel measures those rates with the same access
// shape: every lane keeps 8 independent linear congruential generators
// (s <- 1664525 s + 1013904223, Numerical Recipes' constants), takes the top
// log2(bytes) bits of each state as a byte offset into a table of `bytes`
// bytes and folds the byte into a per-block checksum.
//
// Address generation costs four or five instructions per read, below the
// shared-memory pipe's cost of a random 32-lane gather (several wavefronts),
// so the shared variant is bound by the gathers, not by issue.
#include <cuda_runtime.h>

#include <cstdint>

#include "nav_internal.h"

namespace flashnav {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kMaxProbeSmem = 192 * 1024;

// Byte j of the shared-memory table: the top byte of Knuth's multiplicative
// hash of j.
__device__ __forceinline__ uint32_t table_byte(uint32_t j) { return (j * 2654435761u) >> 24; }

__device__ __forceinline__ uint32_t chain_seed(uint32_t g) {
    return g * 2654435761u + 0x9E3779B9u;
}

template <bool kShared>
__global__ void __launch_bounds__(kProbeThreads)
    gather_probe(const uint8_t *__restrict__ table, int log2_bytes, int iters,
                 uint32_t *__restrict__ sums) {
    extern __shared__ __align__(16) uint8_t probe_smem[];
    __shared__ uint32_t red[kProbeThreads / 32];
    if constexpr (kShared) {
        uint32_t *w = reinterpret_cast<uint32_t *>(probe_smem);
        const uint32_t n_words = 1u << (log2_bytes - 2);
        for (uint32_t k = threadIdx.x; k < n_words; k += kProbeThreads) {
            const uint32_t j = 4u * k;
            w[k] = table_byte(j) | (table_byte(j + 1) << 8) | (table_byte(j + 2) << 16) |
                   (table_byte(j + 3) << 24);
        }
        __syncthreads();
    }
    const uint32_t g = (uint32_t)blockIdx.x * kProbeThreads + threadIdx.x;
    uint32_t s[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) s[c] = chain_seed(g * kChains + c);
    const int sh = 32 - log2_bytes; // offsets are the top log2_bytes bits: < bytes
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            s[c] = s[c] * 1664525u + 1013904223u;
            const uint32_t off = s[c] >> sh;
            if constexpr (kShared)
                acc += probe_smem[off];
            else
                acc += __ldg(table + off);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kProbeThreads / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

} // namespace
} // namespace flashnav

// C ABI: see include/flashnav.h (nav_gather_probe).
extern "C" int nav_gather_probe(int where, const void *table_dev, int64_t bytes, int n_blocks,
                                int iters, uint32_t *sums_dev, void *stream) {
    using namespace flashnav;
    if (where != 0 && where != 1) return NAV_E_INVAL;
    if (bytes < 1024 || (bytes & (bytes - 1)) || bytes > ((int64_t)1 << 31)) return NAV_E_INVAL;
    if (n_blocks < 1 || iters < 0 || !sums_dev) return NAV_E_INVAL;
    if (where == 0 && bytes > kMaxProbeSmem) return NAV_E_INVAL;
    if (where == 1 && !table_dev) return NAV_E_INVAL;
    int log2_bytes = 0;
    while (((int64_t)1 << log2_bytes) < bytes) ++log2_bytes;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (where == 0) {
        const size_t smem = (size_t)bytes;
        if (cudaFuncSetAttribute(gather_probe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return NAV_E_CUDA;
        gather_probe<true><<<n_blocks, kProbeThreads, smem, st>>>(nullptr, log2_bytes, iters,
                                                                 sums_dev);
    } else {
        gather_probe<false><<<n_blocks, kProbeThreads, 0, st>>>(
            static_cast<const uint8_t *>(table_dev), log2_bytes, iters, sums_dev);
    }
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}
