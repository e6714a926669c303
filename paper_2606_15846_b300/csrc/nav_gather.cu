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
#include "tc_util.cuh"

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

// ---------------------------------------------------------------------------
// Tensor-pipe rate probe: the costs behind the weight staging of the fused
// actor.  One thread of each CTA issues n_mma back-to-back tcgen05.mma
// (kind::f16, M 128, N n, K 16; A and B are zero BF16 tiles in shared
// memory with the 128-byte swizzle, 16 KiB of A and 32 KiB of B, the four
// K steps of one 64-wide chunk in turn) into a TMEM accumulator of 256
// columns, with a tcgen05.commit after every commit_every MMAs (0: none
// before the last) that it waits on when `wait` is set, then a final commit
// and wait; it records the %globaltimer nanoseconds from the first issue to
// the last completion.  The CTA's ~100 KiB of shared memory keeps at most
// two CTAs on an SM, so their TMEM allocations (256 columns each) never wait
// on each other.
// ---------------------------------------------------------------------------
constexpr int kMmaProbeThreads = 128;
constexpr unsigned kMmaProbeSmem = 100u * 1024u;

__device__ __forceinline__ unsigned long long probe_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kMmaProbeThreads)
    mma_probe(int n, int n_mma, int commit_every, int wait, unsigned long long *ns,
              int *status) {
    extern __shared__ __align__(1024) unsigned char mp_smem[];
    __shared__ unsigned tslot;
    __shared__ __align__(8) unsigned long long bar;    // the commits waited on
    __shared__ __align__(8) unsigned long long bar_nw; // the others (never completes a phase)
    const unsigned raw = smem_addr(mp_smem);
    const unsigned base = (raw + 1023u) & ~1023u; // A at base, B at base + 16 KiB
    unsigned char *tiles = mp_smem + (base - raw);
    for (unsigned o = threadIdx.x * 16u; o < 48u * 1024u; o += kMmaProbeThreads * 16u)
        *reinterpret_cast<uint4 *>(tiles + o) = make_uint4(0u, 0u, 0u, 0u);
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tslot)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar_nw)),
                     "r"((1u << 20) - 1u)
                     : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tslot;
    if (threadIdx.x == 0) {
        const unsigned idesc = instr_desc(128, n);
        const unsigned b = smem_addr(&bar);
        unsigned phase = 0;
        bool ok = true;
        const unsigned long long t0 = probe_clock_ns();
        for (int i = 0; i < n_mma; ++i) {
            mma_f16(tmem, smem_desc(base + 32u * (unsigned)(i & 3)),
                    smem_desc(base + 16384u + 32u * (unsigned)(i & 3)), idesc, i > 0 ? 1u : 0u);
            if (commit_every > 0 && (i + 1) % commit_every == 0 && i + 1 < n_mma) {
                if (wait) {
                    mma_commit(b);
                    ok = ok && mbar_wait(b, phase);
                    phase ^= 1u;
                } else {
                    // not waited on: its arrival goes to a barrier whose
                    // count is never reached, so `bar` holds one pending
                    // phase at a time and the waits on it are unambiguous
                    mma_commit(smem_addr(&bar_nw));
                }
            }
        }
        mma_commit(b);
        // commits complete in order: this one completes after every MMA
        ok = ok && mbar_wait(b, phase);
        const unsigned long long t1 = probe_clock_ns();
        ns[blockIdx.x] = t1 - t0;
        if (!ok) {
            atomicOr(status, 1);
            mbar_wait(b, phase); // once more (bounded) before the TMEM is freed
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
}

} // namespace
} // namespace flashnav

// C ABI: see include/flashnav.h (nav_mma_probe).
extern "C" int nav_mma_probe(int n, int n_mma, int commit_every, int wait, int n_blocks,
                             unsigned long long *ns_dev, int *status_dev, void *stream) {
    using namespace flashnav;
    if (n < 16 || n > 256 || (n % 16) != 0) return NAV_E_INVAL;
    if (n_mma < 1 || n_mma > (1 << 20) || commit_every < 0 || (wait != 0 && wait != 1))
        return NAV_E_INVAL;
    if (n_blocks < 1 || n_blocks > 1024 || !ns_dev || !status_dev) return NAV_E_INVAL;
    if (cudaFuncSetAttribute(mma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMmaProbeSmem) != cudaSuccess)
        return NAV_E_CUDA;
    mma_probe<<<n_blocks, kMmaProbeThreads, kMmaProbeSmem, static_cast<cudaStream_t>(stream)>>>(
        n, n_mma, commit_every, wait, ns_dev, status_dev);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

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
