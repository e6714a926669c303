// Tensor-core GEMM for the policy and critic MLPs (Sec. 2.1 MLPs; the
// FastDSAC learner of Sec. 2.3): C = A B^T with A [M][K] and B [N][K] BF16,
// both K-major, FP32 accumulation in tensor memory (tcgen05, sm_100-family).
//
// One CTA (4 warps) owns a 128 x BN output tile (BN <= 256, a multiple of 16).
// For each 64-wide K chunk the CTA copies A and B rows into shared memory in
// the 128-byte-swizzled K-major layout (8-row atoms of 1024 bytes, 16-byte
// piece c of row r stored at piece c ^ (r mod 8)), zero-filling rows past M/N
// and columns past K; one thread issues four tcgen05.mma (K = 16 each) into
// the TMEM accumulator and commits them to the chunk's stage mbarrier.  Four
// stages keep the copies of the next three chunks in flight behind the MMAs.  The epilogue reads
// the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
// rows), adds the bias, applies LeakyReLU if asked, and stores FP32 and/or
// BF16 and/or the BF16 transpose.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "nav_internal.h"
#include "tc_util.cuh"

namespace flashnav {
namespace {

constexpr int kTileM = 128;
constexpr int kChunkK = 64; // BF16 elements per 128-byte swizzle row
constexpr int kStages = 4;  // K chunks in flight
constexpr int kThreads = 128;
constexpr float kLeakySlope = 0.01f;

__global__ void __launch_bounds__(kThreads)
    gemm_bf16_tc(const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
                 int ldb, int M, int N, int K, int BN, const float *__restrict__ bias, int act,
                 float *C32, int ldc32, __nv_bfloat16 *C16, int ldc16, __nv_bfloat16 *C16T,
                 int ldct, int *status, int k_split) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[kStages];
    __shared__ unsigned tmem_base;
    // stage s: A tile at sA + s * stage_bytes, B tile after it (1024-aligned)
    const unsigned raw = smem_addr(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    const unsigned stage_bytes = (unsigned)(kTileM * 128 + BN * 128);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * BN;
    int ncols = 32;
    while (ncols < BN) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned idesc = instr_desc(kTileM, BN);
    bool ok = true;
    // split-K: CTA z covers chunks [z * k_split, (z + 1) * k_split) and adds
    // its partial product into C32 (zeroed by the caller)
    const int n_chunks_all = (K + kChunkK - 1) / kChunkK;
    const int kc0 = k_split > 0 ? blockIdx.z * k_split : 0;
    const int kc1 = k_split > 0 ? min(n_chunks_all, kc0 + k_split) : n_chunks_all;
    const int nk = kc1 - kc0;
    auto load_chunk = [&](int j) {
        const unsigned sa = base + (unsigned)(j % kStages) * stage_bytes;
        load_tile<kThreads>(sa, A, lda, m0, kTileM, M, (kc0 + j) * kChunkK, K);
        load_tile<kThreads>(sa + kTileM * 128, B, ldb, n0, BN, N, (kc0 + j) * kChunkK, K);
    };
    // pipeline: chunk j's copies form cp.async group j; chunk j + kStages - 1
    // is fetched into the stage of chunk j - 1 once that chunk's MMAs are done
    for (int j = 0; j < kStages - 1; ++j) {
        if (j < nk) load_chunk(j);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < nk; ++i) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const unsigned sa = base + (unsigned)(i % kStages) * stage_bytes;
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k16 = 0; k16 < kChunkK / 16; ++k16) {
                const unsigned long long da = smem_desc(sa + 32u * k16);
                const unsigned long long db = smem_desc(sa + kTileM * 128 + 32u * k16);
                const unsigned accum = (i > 0 || k16 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bar[i % kStages]))
                : "memory");
        }
        const int j = i + kStages - 1;
        if (j < nk) {
            if (i >= 1) ok = mbar_wait(smem_addr(&bar[(i - 1) % kStages]), ((i - 1) / kStages) & 1) && ok;
            load_chunk(j);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // the last commit covers every MMA issued before it
    if (nk > 0) ok = mbar_wait(smem_addr(&bar[(nk - 1) % kStages]), ((nk - 1) / kStages) & 1) && ok;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok && status && threadIdx.x == 0) atomicOr(status, 1);
    // epilogue: warp w holds rows m0 + 32 w + lane; 16 columns per TMEM load
    const int row = m0 + warp * 32 + lane;
    const bool vec16 = C16 && (ldc16 % 8) == 0;
    for (int cb = 0; cb < BN; cb += 16) {
        unsigned r[16];
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)cb;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row >= M) continue;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = n0 + cb + j;
            float x = __uint_as_float(r[j]);
            if (k_split == 0 && col < N) {
                if (bias) x += bias[col];
                if (act == 1) x = x > 0.0f ? x : kLeakySlope * x;
            }
            v[j] = x;
        }
        const int c0 = n0 + cb;
        if (k_split > 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < N) atomicAdd(&C32[(size_t)row * ldc32 + c0 + j], v[j]);
            continue;
        }
        if (C32) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < N) C32[(size_t)row * ldc32 + c0 + j] = v[j];
        }
        if (C16) {
            if (vec16 && c0 + 16 <= N) {
                uint4 pk[2];
                unsigned *w = reinterpret_cast<unsigned *>(pk);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    w[j] = *reinterpret_cast<const unsigned *>(&h2);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(C16 + (size_t)row * ldc16 + c0);
                dst[0] = pk[0];
                dst[1] = pk[1];
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < N) C16[(size_t)row * ldc16 + c0 + j] = __float2bfloat16_rn(v[j]);
            }
        }
        if (C16T) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < N) C16T[(size_t)(c0 + j) * ldct + row] = __float2bfloat16_rn(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

} // namespace

int launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                     const float *bias, int act, float *C32, int ldc32, void *C16, int ldc16,
                     void *C16T, int ldct, int *status, void *stream) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    const int BN = N >= 256 ? 256 : (N + 15) / 16 * 16;
    const size_t smem = 1024 + (size_t)kStages * ((size_t)kTileM * 128 + (size_t)BN * 128);
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    dim3 grid((M + kTileM - 1) / kTileM, (N + BN - 1) / BN);
    gemm_bf16_tc<<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(A), lda, static_cast<const __nv_bfloat16 *>(B), ldb, M,
        N, K, BN, bias, act, C32, ldc32, static_cast<__nv_bfloat16 *>(C16), ldc16,
        static_cast<__nv_bfloat16 *>(C16T), ldct, status, 0);
    return (int)cudaGetLastError();
}

int launch_gemm_bf16_splitk(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                            float *C32, int ldc32, int *status, void *stream) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    const int BN = N >= 256 ? 256 : (N + 15) / 16 * 16;
    const size_t smem = 1024 + (size_t)kStages * ((size_t)kTileM * 128 + (size_t)BN * 128);
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemset2DAsync(C32, (size_t)ldc32 * 4, 0, (size_t)N * 4, (size_t)M, s);
    if (e != cudaSuccess) return (int)e;
    const int n_chunks = (K + kChunkK - 1) / kChunkK;
    const int tiles = ((M + kTileM - 1) / kTileM) * ((N + BN - 1) / BN);
    // aim for >= 148 CTAs, at least 2 chunks each
    int splits = (148 + tiles - 1) / tiles;
    splits = std::max(1, std::min(splits, n_chunks / 2));
    const int per = (n_chunks + splits - 1) / splits;
    splits = (n_chunks + per - 1) / per;
    dim3 grid((M + kTileM - 1) / kTileM, (N + BN - 1) / BN, splits);
    gemm_bf16_tc<<<grid, kThreads, smem, s>>>(
        static_cast<const __nv_bfloat16 *>(A), lda, static_cast<const __nv_bfloat16 *>(B), ldb, M,
        N, K, BN, nullptr, 0, C32, ldc32, nullptr, 0, nullptr, 0, status, per);
    return (int)cudaGetLastError();
}

} // namespace flashnav

// C ABI: see include/flashnav.h (nav_gemm_bf16).
extern "C" int nav_gemm_bf16(const void *a_dev, int lda, const void *b_dev, int ldb, int m, int n,
                             int k, const float *bias_dev, int act, float *c32_dev, int ldc32,
                             void *c16_dev, int ldc16, void *c16t_dev, int ldct, int *status_dev,
                             void *stream) {
    if (!a_dev || !b_dev || m < 0 || n < 0 || k < 0 || (act != 0 && act != 1)) return NAV_E_INVAL;
    if ((lda % 8) || (ldb % 8) || lda < k || ldb < k) return NAV_E_INVAL;
    if ((reinterpret_cast<uintptr_t>(a_dev) & 15u) || (reinterpret_cast<uintptr_t>(b_dev) & 15u))
        return NAV_E_INVAL;
    if ((c32_dev && ldc32 < n) || (c16_dev && ldc16 < n) || (c16t_dev && ldct < m))
        return NAV_E_INVAL;
    const int rc = flashnav::launch_gemm_bf16(a_dev, lda, b_dev, ldb, m, n, k, bias_dev, act,
                                              c32_dev, ldc32, c16_dev, ldc16, c16t_dev, ldct,
                                              status_dev, stream);
    return rc == 0 ? NAV_OK : NAV_E_CUDA;
}
