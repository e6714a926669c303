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
//
// Large products run on a persistent, warp-specialised variant instead:
// warp 0 streams A and B chunks into a ring of shared-memory stages with
// tensor-map bulk copies (cp.async.bulk.tensor, 128-byte swizzle, zero fill
// past M, N and K), warp 1 issues the MMAs into one of two TMEM
// accumulators, and warps 2-9 drain the other accumulator (the epilogue of
// one tile overlaps the main loop of the next).  Stage and accumulator
// hand-offs are mbarriers; every wait is bounded and reports through the
// status word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "nav_internal.h"
#include "pdl.cuh"
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
    const bool vec16 = C16 && (ldc16 % 8) == 0 && (reinterpret_cast<uintptr_t>(C16) & 15u) == 0;
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


// ---------------------------------------------------------------------------
// Persistent warp-specialised GEMM (tensor-map loads, two TMEM accumulators)
// ---------------------------------------------------------------------------
constexpr int kWsThreads = 320; // warp 0 loads, warp 1 MMA, warps 2-9 epilogue
constexpr int kWsMaxStages = 8;
constexpr int kWaitLimit = 1 << 22; // polls of one mbarrier before giving up

struct WsArgs {
    int M, N, K, BN, n_mt, n_nt, n_tiles, per_split, stages;
    const float *bias;
    int bias_vec; // bias 16-byte aligned: read four columns per load
    int c16_v8;   // C16 rows 32-byte aligned: one 256-bit store per 16 columns
    int c32_v8;   // C32 rows 32-byte aligned: two 256-bit stores per 16 columns
    int act;
    float *C32;
    int ldc32;
    __nv_bfloat16 *C16;
    int ldc16;
    __nv_bfloat16 *C16T;
    int ldct;
    int *status;
};

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool ws_wait(unsigned bar, unsigned parity, volatile int *abort_flag) {
    for (int it = 0; it < kWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The k-th tile of this CTA: (m tile, n tile, chunk range) of tile
// blockIdx.x + k gridDim.x in (m, n, split) order; false past the last.
__device__ __forceinline__ bool ws_tile(const WsArgs &g, int k, int &mt, int &nt, int &c0,
                                        int &c1) {
    const int nkc = (g.K + kChunkK - 1) / kChunkK;
    const int t = blockIdx.x + k * gridDim.x;
    if (t >= g.n_tiles) return false;
    mt = t % g.n_mt;
    const int r = t / g.n_mt;
    nt = r % g.n_nt;
    const int z = r / g.n_nt;
    c0 = g.per_split > 0 ? z * g.per_split : 0;
    c1 = g.per_split > 0 ? min(nkc, c0 + g.per_split) : nkc;
    return true;
}

__global__ void __launch_bounds__(kWsThreads, 2)
    gemm_ws(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const WsArgs g) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kWsMaxStages], empty[kWsMaxStages];
    __shared__ __align__(8) unsigned long long accf[2], acce[2], fin;
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag;
    const unsigned base = (smem_addr(smem_raw) + 1023u) & ~1023u;
    const unsigned a_bytes = kTileM * 128;
    const unsigned stage_bytes = a_bytes + (unsigned)g.BN * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = g.stages;
    int ncols = 32;
    while (ncols < 2 * g.BN) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&accf[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_addr(&acce[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&fin)) : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    volatile int *abort_v = &abort_flag;
    auto give_up = [&]() {
        *abort_v = 1;
        if (g.status) atomicOr(g.status, 1);
    };

    if (warp == 0) {
        // producer: one elected lane streams every chunk of every tile
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmA))
                         : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmB))
                         : "memory");
            int mt, nt, c0, c1;
            int it = 0;
            bool ok = true;
            for (int k = 0; ok && ws_tile(g, k, mt, nt, c0, c1); ++k) {
                for (int c = c0; c < c1; ++c, ++it) {
                    const int s = it % S;
                    const unsigned u = (unsigned)(it / S);
                    if (it >= S && !ws_wait(smem_addr(&empty[s]), (u & 1u) ^ 1u, abort_v)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    const unsigned fb = smem_addr(&full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"(stage_bytes)
                                 : "memory");
                    const unsigned dst = base + (unsigned)s * stage_bytes;
                    tma_load_2d(dst, &tmA, c * kChunkK, mt * kTileM, fb);
                    tma_load_2d(dst + a_bytes, &tmB, c * kChunkK, nt * g.BN, fb);
                }
            }
            // every copy issued lands before the CTA exits (a no-op when the
            // MMA warp consumed them all)
            for (int q = max(0, it - S); q < it; ++q)
                ws_wait(smem_addr(&full[q % S]), (unsigned)(q / S) & 1u, abort_v) || (give_up(), true);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned idesc = instr_desc(kTileM, g.BN);
            int it = 0, tl = 0, mt, nt, c0, c1;
            bool ok = true, issued = false;
            for (int k = 0; ok && ws_tile(g, k, mt, nt, c0, c1); ++k, ++tl) {
                const int buf = tl & 1;
                const unsigned ub = (unsigned)(tl >> 1);
                if (tl >= 2 && !ws_wait(smem_addr(&acce[buf]), (ub & 1u) ^ 1u, abort_v)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned d = tmem + (unsigned)(buf * g.BN);
                for (int c = c0; c < c1; ++c, ++it) {
                    const int s = it % S;
                    if (!ws_wait(smem_addr(&full[s]), (unsigned)(it / S) & 1u, abort_v)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned sa = base + (unsigned)s * stage_bytes;
                    const unsigned sb = sa + a_bytes;
#pragma unroll
                    for (int k16 = 0; k16 < kChunkK / 16; ++k16)
                        mma_f16(d, smem_desc(sa + 32u * k16), smem_desc(sb + 32u * k16), idesc,
                                (c > c0 || k16 > 0) ? 1u : 0u);
                    mma_commit(smem_addr(&empty[s]));
                    issued = true;
                }
                if (ok) mma_commit(smem_addr(&accf[buf]));
            }
            // every MMA issued completes before the accumulators are freed
            if (issued) {
                mma_commit(smem_addr(&fin));
                ws_wait(smem_addr(&fin), 0u, abort_v) || (give_up(), true);
            }
        }
    } else {
        // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (its rows),
        // columns of its half of the tile (warps 2-5 the first 16-column
        // groups, warps 6-9 the rest)
        const int q = warp & 3;
        const int groups = g.BN / 16;
        const int g0 = warp < 6 ? 0 : (groups + 1) / 2, g1 = warp < 6 ? (groups + 1) / 2 : groups;
        int tl = 0, mt, nt, c0, c1;
        for (int k = 0; ws_tile(g, k, mt, nt, c0, c1); ++k, ++tl) {
            const int buf = tl & 1;
            // warp-uniform outcome: the TMEM loads below are warp-collective
            const bool got = __all_sync(0xffffffffu,
                                        ws_wait(smem_addr(&accf[buf]), (unsigned)(tl >> 1) & 1u, abort_v));
            if (!got) {
                if (lane == 0) give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = mt * kTileM + q * 32 + lane;
            const int n0 = nt * g.BN;
            const bool split = g.per_split > 0;
            const bool vec16 =
                g.C16 && (g.ldc16 % 8) == 0 && (reinterpret_cast<uintptr_t>(g.C16) & 15u) == 0;
            for (int gi = g0; gi < g1; ++gi) {
                const int cb = gi * 16;
                float v[16];
                tmem_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(buf * g.BN + cb), v);
                if (row >= g.M) continue;
                const int c0c = n0 + cb;
                if (!split && c0c + 16 <= g.N && (g.bias_vec || !g.bias)) {
                    // whole group inside N: bias as four 16-byte loads
                    if (g.bias) {
                        const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + c0c);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 bb = __ldg(b4 + j);
                            v[4 * j] += bb.x;
                            v[4 * j + 1] += bb.y;
                            v[4 * j + 2] += bb.z;
                            v[4 * j + 3] += bb.w;
                        }
                    }
                    if (g.act == 1) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = v[j] > 0.0f ? v[j] : kLeakySlope * v[j];
                    }
                } else if (!split) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = c0c + j;
                        float x = v[j];
                        if (col < g.N) {
                            if (g.bias) x += g.bias[col];
                            if (g.act == 1) x = x > 0.0f ? x : kLeakySlope * x;
                        }
                        v[j] = x;
                    }
                }
                if (split) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0c + j < g.N) atomicAdd(&g.C32[(size_t)row * g.ldc32 + c0c + j], v[j]);
                    continue;
                }
                if (g.C32) {
                    if (g.c32_v8 && c0c + 16 <= g.N) {
                        float *dst = g.C32 + (size_t)row * g.ldc32 + c0c;
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            asm volatile(
                                "st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst + 8 * h),
                                "r"(__float_as_uint(v[8 * h])), "r"(__float_as_uint(v[8 * h + 1])),
                                "r"(__float_as_uint(v[8 * h + 2])), "r"(__float_as_uint(v[8 * h + 3])),
                                "r"(__float_as_uint(v[8 * h + 4])), "r"(__float_as_uint(v[8 * h + 5])),
                                "r"(__float_as_uint(v[8 * h + 6])), "r"(__float_as_uint(v[8 * h + 7]))
                                : "memory");
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0c + j < g.N) g.C32[(size_t)row * g.ldc32 + c0c + j] = v[j];
                    }
                }
                if (g.C16) {
                    if (g.c16_v8 && c0c + 16 <= g.N) {
                        unsigned w[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            w[j] = *reinterpret_cast<const unsigned *>(&h2);
                        }
                        asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(
                                         g.C16 + (size_t)row * g.ldc16 + c0c),
                                     "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]),
                                     "r"(w[6]), "r"(w[7])
                                     : "memory");
                    } else if (vec16 && c0c + 16 <= g.N) {
                        uint4 pk[2];
                        unsigned *w = reinterpret_cast<unsigned *>(pk);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            w[j] = *reinterpret_cast<const unsigned *>(&h2);
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(g.C16 + (size_t)row * g.ldc16 + c0c);
                        dst[0] = pk[0];
                        dst[1] = pk[1];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0c + j < g.N)
                                g.C16[(size_t)row * g.ldc16 + c0c + j] = __float2bfloat16_rn(v[j]);
                    }
                }
                if (g.C16T) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0c + j < g.N)
                            g.C16T[(size_t)(c0c + j) * g.ldct + row] = __float2bfloat16_rn(v[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acce[buf]))
                             : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// K-major BF16 matrix [rows][ld] viewed as a 2-D tensor {K, rows}, boxes of
// 64 x box_rows elements with the 128-byte swizzle.  Encoded maps are kept
// in a small cache keyed by their arguments (the learner and the policy
// call the same products every step).
bool encode_map(CUtensorMap *map, const void *ptr, int ld, int rows, int K, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15u) || (ld % 8) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct MapKey {
    const void *ptr;
    int ld, rows, K, box;
    bool operator==(const MapKey &o) const {
        return ptr == o.ptr && ld == o.ld && rows == o.rows && K == o.K && box == o.box;
    }
};

bool make_map(CUtensorMap *map, const void *ptr, int ld, int rows, int K, int box_rows) {
    constexpr int kCache = 64;
    static MapKey keys[kCache];
    static CUtensorMap maps[kCache];
    static int n = 0, next = 0;
    static std::mutex mu;
    const MapKey key{ptr, ld, rows, K, box_rows};
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < n; ++i)
        if (keys[i] == key) {
            *map = maps[i];
            return true;
        }
    if (!encode_map(map, ptr, ld, rows, K, box_rows)) return false;
    keys[next] = key;
    maps[next] = *map;
    next = (next + 1) % kCache;
    n = std::min(n + 1, kCache);
    return true;
}

int sm_count() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    });
    return n;
}

// Launches the persistent GEMM (two CTAs per SM: n tiles of at most 128
// columns, stages within 96 KiB); returns false (nothing launched) when the
// operands cannot be described by tensor maps.
bool launch_ws(const void *A, int lda, const void *B, int ldb, int M, int N, int K, int BN,
               int per_split, int n_splits, const float *bias, int act, float *C32, int ldc32,
               void *C16, int ldc16, void *C16T, int ldct, int *status, cudaStream_t s, int &rc) {
    BN = std::min(BN, 128);
    const int n_mt = (M + kTileM - 1) / kTileM;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, lda, M, K, kTileM) || !make_map(&mb, B, ldb, N, K, BN)) return false;
    const int stage_bytes = kTileM * 128 + BN * 128;
    const int stages = std::min(kWsMaxStages, (96 * 1024) / stage_bytes);
    const size_t smem = 1024 + (size_t)stages * stage_bytes;
    {
        // the attribute only ever rises (a lower value would refuse later
        // launches still queued with a larger request)
        static int smem_set = 0;
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        if ((int)smem > smem_set) {
            cudaError_t e = cudaFuncSetAttribute(
                gemm_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) { rc = (int)e; return true; }
            smem_set = (int)smem;
        }
    }
    WsArgs g;
    g.M = M; g.N = N; g.K = K; g.BN = BN;
    g.n_mt = n_mt;
    g.n_nt = (N + BN - 1) / BN;
    g.n_tiles = g.n_mt * g.n_nt * n_splits;
    g.per_split = per_split;
    g.stages = stages;
    g.bias = bias; g.act = act;
    g.bias_vec = (reinterpret_cast<uintptr_t>(bias) & 15u) == 0;
    g.c16_v8 = C16 && (reinterpret_cast<uintptr_t>(C16) & 31u) == 0 && (ldc16 % 16) == 0;
    g.c32_v8 = C32 && (reinterpret_cast<uintptr_t>(C32) & 31u) == 0 && (ldc32 % 8) == 0;
    g.C32 = C32; g.ldc32 = ldc32;
    g.C16 = static_cast<__nv_bfloat16 *>(C16); g.ldc16 = ldc16;
    g.C16T = static_cast<__nv_bfloat16 *>(C16T); g.ldct = ldct;
    g.status = status;
    const int grid = std::min(g.n_tiles, 2 * sm_count());
    launch_pdl(gemm_ws, grid, kWsThreads, smem, s, ma, mb, g);
    rc = (int)cudaGetLastError();
    return true;
}

} // namespace

int launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                     const float *bias, int act, float *C32, int ldc32, void *C16, int ldc16,
                     void *C16T, int ldct, int *status, void *stream) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    const int BN = N >= 256 ? 256 : (N + 15) / 16 * 16;
    int rc = 0;
    if (launch_ws(A, lda, B, ldb, M, N, K, BN, 0, 1, bias, act, C32, ldc32, C16, ldc16, C16T, ldct,
                  status, static_cast<cudaStream_t>(stream), rc))
        return rc;
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
    int rc = 0;
    if (launch_ws(A, lda, B, ldb, M, N, K, BN, per, splits, nullptr, 0, C32, ldc32, nullptr, 0,
                  nullptr, 0, status, s, rc))
        return rc;
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
