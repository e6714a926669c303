// Fused passes of small MLPs on the tensor cores (Sec. 2.1 networks, (100) x 4
// in Table 3; the FastDSAC learner of Sec. 2.3).  The general GEMM path runs
// a network as one launch per layer and per gradient; at batch 1024 and width
// 100 each launch is a few microseconds of latency around almost no work, and
// an update of the twin critics and the actor is ~180 of them.  Here one CTA
// (16 warps) owns 128 batch rows of a network and walks all its layers:
//
// forward: per layer, the weight tile [out][in] is copied (cp.async) into a
//   swizzled K-major shared tile, one thread issues tcgen05.mma (M 128,
//   N = out rounded to 16, K = in in 64-wide chunks) into TMEM, and the
//   epilogue (tcgen05.ld, bias, LeakyReLU) writes the BF16 activation straight
//   into the next layer's A tile (ping-pong), plus optional saves for the
//   backward pass (row-major and transposed).
// backward: the upstream gradient G lives in shared memory twice, row-major
//   [128 rows][out] (A of dH = G W) and transposed [out][128 rows] (A of the
//   weight gradient dW = G^T H); per layer both MMAs run from shared tiles
//   into two TMEM regions; the dW epilogue writes this CTA's partial
//   [out][in]; the dH epilogue gates by LeakyReLU' (sign of the saved
//   activation), forms the next G in both layouts and its column sums (the
//   bias gradient partial).
// Partials are summed by the optimiser kernel (no atomics, deterministic).
// Rounding points equal the general path's: G rounded to BF16 for the
// GEMMs, FP32 for the bias sums, FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "nav_internal.h"
#include "pdl.cuh"
#include "nav_policy.h"
#include "tc_util.cuh"

namespace flashnav {
namespace {

typedef __nv_bfloat16 bf16;
constexpr int kTF = 512; // threads per CTA of the passes: warps w, w + 4, w + 8, ... share
                         // TMEM lanes 32 (w % 4) .. and split the columns (1024 threads,
                         // 16 columns a warp, measured slower)
constexpr int kGroups = kTF / 128;   // warps per TMEM lane quarter
constexpr int kSpan = 128 / kGroups; // columns per warp (16 or 32)
static_assert(kSpan == 16 || kSpan == 32, "a warp's columns must lie in one mask word");
constexpr unsigned kChunk = 128 * 128; // one 64-wide K chunk of 128 rows (bytes)
constexpr float kSlope = 0.01f;

__device__ __forceinline__ int round16(int n) { return (n + 15) & ~15; }

// zero `bytes` (multiple of 16 * NT) of shared memory at s with NT threads
template <int NT> __device__ __forceinline__ void zero_smem(unsigned char *s, unsigned bytes) {
    uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (unsigned o = threadIdx.x * 16u; o < bytes; o += 16u * NT)
        *reinterpret_cast<uint4 *>(s + o) = z;
}

__device__ __forceinline__ void wait_or_flag(unsigned bar, unsigned parity, int *status) {
    if (!mbar_wait(bar, parity) && status) atomicOr(status, 1);
}

// MMAs over n_chunks 64-wide K chunks: D [+]= A B^T, A and B chunk-tiled
__device__ __forceinline__ void mma_chunks(unsigned tmem_d, unsigned a, unsigned b, int n_chunks,
                                           unsigned idesc) {
    for (int c = 0; c < n_chunks; ++c)
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16)
            mma_f16(tmem_d, smem_desc(a + c * kChunk + 32u * k16),
                    smem_desc(b + c * kChunk + 32u * k16), idesc, (c > 0 || k16 > 0) ? 1u : 0u);
}

__device__ __forceinline__ unsigned tmem_alloc(unsigned *slot, unsigned ncols) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *slot;
}

__device__ __forceinline__ void tmem_free(unsigned tmem, unsigned ncols) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ncols)
                     : "memory");
}

// 8 BF16 of a row as one 16-byte word
__device__ __forceinline__ uint4 pack8(const float *v) {
    uint4 u;
    unsigned *w = reinterpret_cast<unsigned *>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<const unsigned *>(&h);
    }
    return u;
}

// Zero the 16-byte pieces of `row` in columns [c0, c1) of a 2-chunk tile.
__device__ __forceinline__ void zero_cols(unsigned char *tile, int row, int c0, int c1) {
    for (int c = c0; c < c1; c += 8)
        *reinterpret_cast<uint4 *>(tile + swz(row, c, kChunk)) = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------- forward ---
// smem: A (the layer input, 2 chunks; rewritten in place with the layer's
// output once its MMAs have completed) | W0 | W1 (weights, double-buffered:
// layer l + 1's tile is copied while layer l computes).  Warp w reads TMEM
// lanes 32 (w % 4) .. (batch rows) and columns [32 q, 32 q + 32), q = w / 4.
__global__ void __launch_bounds__(kTF) mlp_fwd_fused(const FGroup g) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_slot;
    __shared__ float sbias[2][kFusedMaxWidth];
    const FNet &N = g.net[blockIdx.y];
    const int tid = threadIdx.x, warp = tid >> 5, quad = warp & 3, qtr = warp >> 2;
    const int row = quad * 32 + (tid & 31), r0 = blockIdx.x * 128, grow = r0 + row;
    const unsigned raw = smem_addr(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *ap = smem_raw + (base - raw);
    const unsigned a = base, wb[2] = {base + 2 * kChunk, base + 4 * kChunk};
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    zero_smem<kTF>(ap, 2 * kChunk);
    const unsigned tmem = tmem_alloc(&tmem_slot, 128); // synchronises: A is zero
    const unsigned tlane = (unsigned)(quad * 32) << 16;
    auto fetch = [&](int l) { // weights and bias of layer l (and the input for l = 0)
        const FLayer &L = N.L[l];
        const int np = round16(L.out), nkc = (L.in + 63) >> 6;
        for (int c = 0; c < nkc; ++c)
            load_tile<kTF>(wb[l & 1] + c * kChunk, static_cast<const bf16 *>(L.W16), L.ld_in, 0,
                          np, L.out, 64 * c, L.in);
        if (l == 0)
            for (int c = 0; c < nkc; ++c)
                load_tile<kTF>(a + c * kChunk, static_cast<const bf16 *>(N.X), N.ldx, r0, 128, g.B,
                              64 * c, L.in);
        for (int t = tid; t < np; t += kTF) sbias[l & 1][t] = t < L.out ? L.b[t] : 0.0f;
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(0);
    for (int l = 0; l < N.n_layers; ++l) {
        const FLayer &L = N.L[l];
        const bool last = l == N.n_layers - 1;
        const int out = L.out, np = round16(out), nkc = (L.in + 63) >> 6;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mma_chunks(tmem, a, wb[l & 1], nkc, instr_desc(128, np));
            mma_commit(smem_addr(&bar));
        }
        if (!last) fetch(l + 1);
        wait_or_flag(smem_addr(&bar), (unsigned)(l & 1), g.status);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned mask = 0u;
        const int j0 = kSpan * qtr, j1 = min(np, j0 + kSpan);
        for (int j = j0; j < j1; j += 16) {
            float v[16];
            tmem_ld16(tmem + tlane + (unsigned)j, v);
            unsigned bits = 0u;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float x = v[i] + sbias[l & 1][j + i];
                if (!last) x = x > 0.0f ? x : kSlope * x;
                v[i] = j + i < out ? x : 0.0f;
                bits |= (v[i] > 0.0f ? 1u : 0u) << i;
            }
            mask |= bits << (j & 16);
            if (last) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (j + i < out) N.out32[(long long)grow * out + j + i] = v[i];
                continue;
            }
            *reinterpret_cast<uint4 *>(ap + swz(row, j, kChunk)) = pack8(v);
            *reinterpret_cast<uint4 *>(ap + swz(row, j + 8, kChunk)) = pack8(v + 8);
            if (N.H16[l]) {
                uint4 *d = reinterpret_cast<uint4 *>(static_cast<bf16 *>(N.H16[l]) +
                                                     (long long)grow * N.ldh + j);
                d[0] = pack8(v);
                d[1] = pack8(v + 8);
            }
            if (N.HT16[l]) {
                bf16 *d = static_cast<bf16 *>(N.HT16[l]);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (j + i < out) d[(long long)(j + i) * g.B + grow] = __float2bfloat16_rn(v[i]);
            }
        }
        if (!last) {
            zero_cols(ap, row, max(np, j0), j0 + kSpan); // the next layer reads whole chunks
            if (N.M[l] && j0 < np) {
                if (kSpan == 32)
                    N.M[l][(long long)grow * 4 + qtr] = mask;
                else // this warp's 16 columns: one half of a mask word
                    reinterpret_cast<unsigned short *>(N.M[l] + (long long)grow * 4)[qtr] =
                        (unsigned short)(mask >> (j0 & 16));
            }
        }
        // activations visible to the async proxy (next layer's MMA)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    tmem_free(tmem, 128);
}

// ------------------------------------------------------------ backward ---
// smem: Gn (row-major G, 2 chunks) | Gt (transposed G, 2 chunks of 64 batch
// rows) | HT0 | HT1 | WT0 | WT1 (layer operands, double-buffered).  G is
// rewritten in place once the layer's MMAs have completed.  As in the
// forward, warps w, w + 4, w + 8 and w + 12 share TMEM lanes and split the
// columns in quarters.
__global__ void __launch_bounds__(kTF) mlp_bwd_fused(const FGroup g) {
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_slot;
    __shared__ float sdb[kFusedMaxWidth];
    const FNet &N = g.net[blockIdx.y];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = warp & 3,
              qtr = warp >> 2;
    const int row = quad * 32 + lane, cta = blockIdx.x, r0 = cta * 128, grow = r0 + row;
    const unsigned raw = smem_addr(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    unsigned char *gnp = smem_raw + (base - raw), *gtp = gnp + 2 * kChunk;
    const unsigned gn = base, gt = base + 2 * kChunk;
    const unsigned htb[2] = {base + 4 * kChunk, base + 6 * kChunk};
    const unsigned wtb[2] = {base + 8 * kChunk, base + 10 * kChunk};
    const unsigned tlane = (unsigned)(quad * 32) << 16;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    zero_smem<kTF>(gnp, 4 * kChunk);
    for (int t = tid; t < kFusedMaxWidth; t += kTF) sdb[t] = 0.0f;
    const int top = N.n_layers - 1, nout = N.L[top].out;
    auto fetch = [&](int l, int buf) { // operands of layer l's MMAs
        const FLayer &L = N.L[l];
        const int inp = round16(L.in), koc = (L.out + 63) >> 6;
        if (N.gWp[l]) {
            const bf16 *src = static_cast<const bf16 *>(l > 0 ? N.HT16[l - 1] : N.XT);
            for (int c = 0; c < 2; ++c)
                load_tile<kTF>(htb[buf] + c * kChunk, src, g.B, 0, inp, L.in, r0 + 64 * c, g.B);
        }
        if (l > 0 || N.dX)
            for (int c = 0; c < koc; ++c)
                load_tile<kTF>(wtb[buf] + c * kChunk, static_cast<const bf16 *>(L.WT16), L.ld_out,
                              0, inp, L.in, 64 * c, L.out);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(top, 0);
    const unsigned tmem = tmem_alloc(&tmem_slot, 256); // synchronises: G is zero
    // top layer: G = dout (FP32 for the bias sums, BF16 in both layouts);
    // the quarters split its columns as in the epilogues
    {
        const int j0 = kSpan * qtr, j1 = min(round16(nout), j0 + kSpan);
        for (int j = j0; j < j1; j += 16) {
            float v[16];
            const float *src = N.dout + (long long)grow * nout + j;
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = j + i < nout ? src[i] : 0.0f;
            *reinterpret_cast<uint4 *>(gnp + swz(row, j, kChunk)) = pack8(v);
            *reinterpret_cast<uint4 *>(gnp + swz(row, j + 8, kChunk)) = pack8(v + 8);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                *reinterpret_cast<bf16 *>(gtp + swz(j + i, row, kChunk)) = __float2bfloat16_rn(v[i]);
            const float cs = colsum16(v, lane);
            if ((lane & 1) == 0) atomicAdd(&sdb[j + colsum16_col(lane)], cs);
        }
    }
    __syncthreads();
    if (N.gbp[top])
        for (int t = tid; t < nout; t += kTF) N.gbp[top][(long long)cta * N.cta_stride + t] = sdb[t];
    unsigned phase = 0;
    for (int l = top; l >= 0; --l) {
        const FLayer &L = N.L[l];
        const int in = L.in, out = L.out, inp = round16(in), onp = round16(out),
                  koc = (out + 63) >> 6, buf = (top - l) & 1;
        const bool wg = N.gWp[l] != nullptr;
        const bool dh = l > 0 || N.dX != nullptr;
        const bool next = l > 0;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads(); // operands and G ready; sdb read by the previous layer
        const bool any = wg || dh;
        if (tid == 0 && any) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // dW^T = H^T G: TMEM lanes are input features, columns outputs, so
            // that the partial's rows [out][in] are written coalesced
            if (wg) mma_chunks(tmem, htb[buf], gt, 2, instr_desc(128, onp));
            if (dh) mma_chunks(tmem + 128, gn, wtb[buf], koc, instr_desc(128, inp));
            mma_commit(smem_addr(&bar));
        }
        unsigned msk = 0u;
        if (next) {
            fetch(l - 1, buf ^ 1);
            if (dh) msk = N.M[l - 1][(long long)grow * 4 + (kSpan * qtr >> 5)];
            for (int t = tid; t < kFusedMaxWidth; t += kTF) sdb[t] = 0.0f;
        }
        if (any) wait_or_flag(smem_addr(&bar), phase & 1u, g.status);
        phase += any ? 1u : 0u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads(); // sdb cleared before the column sums
        if (wg) {
            // lane k holds dW[n][k] for 16 outputs n per load; quarters split n
            const int k = quad * 32 + lane;
            float *dst = N.gWp[l] + (long long)cta * N.cta_stride + k;
            for (int j = 16 * qtr; j < onp; j += 16 * kGroups) {
                float v[16];
                tmem_ld16(tmem + tlane + (unsigned)j, v);
                if (k < in) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (j + i < out) dst[(long long)(j + i) * in] = v[i];
                }
            }
        }
        if (dh) {
            const int j0 = kSpan * qtr, j1 = min(inp, j0 + kSpan);
            for (int j = j0; j < j1; j += 16) {
                float v[16];
                tmem_ld16(tmem + tlane + 128u + (unsigned)j, v);
                if (!next) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (j + i < in) N.dX[(long long)grow * N.lddx + j + i] = v[i];
                    continue;
                }
                // LeakyReLU' from the sign bits of layer l-1's activation
                const unsigned bits = msk >> (j & 16);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float z = v[i] * (((bits >> i) & 1u) ? 1.0f : kSlope);
                    v[i] = j + i < in ? z : 0.0f;
                }
                *reinterpret_cast<uint4 *>(gnp + swz(row, j, kChunk)) = pack8(v);
                *reinterpret_cast<uint4 *>(gnp + swz(row, j + 8, kChunk)) = pack8(v + 8);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    *reinterpret_cast<bf16 *>(gtp + swz(j + i, row, kChunk)) =
                        __float2bfloat16_rn(v[i]);
                const float cs = colsum16(v, lane);
                if ((lane & 1) == 0) atomicAdd(&sdb[j + colsum16_col(lane)], cs);
            }
            // the next layer's dH MMA reads whole 64-wide chunks of Gn
            if (next) zero_cols(gnp, row, max(inp, j0), j0 + kSpan);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (next && N.gbp[l - 1])
            for (int t = tid; t < in; t += kTF) N.gbp[l - 1][(long long)cta * N.cta_stride + t] = sdb[t];
    }
    tmem_free(tmem, 256);
}

// ----------------------------------------------------------- optimiser ---
struct OptNet {
    float *p[2 * kMaxLayers], *m[2 * kMaxLayers], *v[2 * kMaxLayers], *g[2 * kMaxLayers];
    const float *src[2 * kMaxLayers]; // Polyak sources
    bf16 *W16[kMaxLayers], *WT16[kMaxLayers];
    int n[2 * kMaxLayers]; // parameter tensors: W0, b0, W1, b1, ...
    int in[kMaxLayers], out[kMaxLayers], ld_in[kMaxLayers], ld_out[kMaxLayers];
    int n_tensors;
    long long total;
    const float *part; // [n_cta][total] partial gradients (Adam)
};
struct OptGroup {
    OptNet net[2];
};

// flat index -> (tensor, index)
__device__ __forceinline__ int locate(const OptNet &o, long long &i) {
    int t = 0;
    while (t < o.n_tensors - 1 && i >= o.n[t]) {
        i -= o.n[t];
        ++t;
    }
    return t;
}

__device__ __forceinline__ void refresh_w(const OptNet &o, int t, long long i, float w) {
    if (t & 1) return; // biases have no BF16 copy
    const int l = t >> 1, in = o.in[l];
    const int r = (int)(i / in), k = (int)(i - (long long)r * in);
    const bf16 h = __float2bfloat16_rn(w);
    o.W16[l][(long long)r * o.ld_in[l] + k] = h;
    o.WT16[l][(long long)k * o.ld_out[l] + r] = h;
}

// With tau > 0, Tg holds target networks of the same shapes: each target
// parameter then takes its Polyak step from the new value in the same pass
// (what polyak_fused would do after this kernel, element by element).
__global__ void adam_fused(const OptGroup G, int n_cta, float lr, float b1, float b2,
                           const float *__restrict__ corr, float wd, const OptGroup Tg,
                           float tau) {
    pdl_enter();
    const OptNet &o = G.net[blockIdx.y];
    const long long fi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= o.total) return;
    long long i = fi;
    const int t = locate(o, i);
    float gi = 0.0f;
    if (o.part) { // per-CTA partials of the fused backward: their sum
        for (int c = 0; c < n_cta; ++c) gi += o.part[(long long)c * o.total + fi];
        o.g[t][i] = gi;
    } else {      // the per-layer path's gradient tensors
        gi = o.g[t][i];
    }
    const float c1 = corr[0], c2 = corr[1];
    const float mi = b1 * o.m[t][i] + (1.0f - b1) * gi;
    const float vi = b2 * o.v[t][i] + (1.0f - b2) * gi * gi;
    o.m[t][i] = mi;
    o.v[t][i] = vi;
    const float p0 = o.p[t][i];
    const float pd = wd != 0.0f ? p0 * (1.0f - lr * wd) : p0;
    const float pn = pd - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    o.p[t][i] = pn;
    refresh_w(o, t, i, pn);
    if (tau > 0.0f) {
        const OptNet &tn = Tg.net[blockIdx.y];
        const float tv = (1.0f - tau) * tn.p[t][i] + tau * pn;
        tn.p[t][i] = tv;
        refresh_w(tn, t, i, tv);
    }
}

__global__ void polyak_fused(const OptGroup G, float tau) {
    pdl_enter();
    const OptNet &o = G.net[blockIdx.y];
    const long long fi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= o.total) return;
    long long i = fi;
    const int t = locate(o, i);
    const float pn = (1.0f - tau) * o.p[t][i] + tau * o.src[t][i];
    o.p[t][i] = pn;
    refresh_w(o, t, i, pn);
}

void fill_opt(const Mlp &m, OptNet &o) {
    o.n_tensors = 2 * m.n_layers;
    o.total = 0;
    for (int l = 0; l < m.n_layers; ++l) {
        const Layer &L = m.layer[l];
        o.p[2 * l] = L.W;
        o.p[2 * l + 1] = L.b;
        o.m[2 * l] = L.mW;
        o.m[2 * l + 1] = L.mb;
        o.v[2 * l] = L.vW;
        o.v[2 * l + 1] = L.vb;
        o.g[2 * l] = L.gW;
        o.g[2 * l + 1] = L.gb;
        o.n[2 * l] = L.in * L.out;
        o.n[2 * l + 1] = L.out;
        o.W16[l] = static_cast<bf16 *>(L.W16);
        o.WT16[l] = static_cast<bf16 *>(L.WT16);
        o.in[l] = L.in;
        o.out[l] = L.out;
        o.ld_in[l] = L.ld_in;
        o.ld_out[l] = L.ld_out;
        o.total += (long long)L.in * L.out + L.out;
    }
}

constexpr size_t kFwdSmem = 1024 + 6 * (size_t)kChunk;
constexpr size_t kBwdSmem = 1024 + 12 * (size_t)kChunk;
static_assert(kBwdSmem + 2048 <= 227 * 1024, "shared memory");

} // namespace

bool fused_ok(const Mlp &m, int B) {
    if (B <= 0 || B % 128 || m.n_layers < 2) return false;
    for (int l = 0; l < m.n_layers; ++l) {
        if (m.layer[l].in > kFusedMaxWidth || m.layer[l].out > kFusedMaxWidth) return false;
        // one saved-activation row stride: every hidden layer has one width
        if (l < m.n_layers - 1 && m.layer[l].out != m.layer[0].out) return false;
    }
    return true;
}

void fused_layers(const Mlp &m, FNet &f) {
    f.n_layers = m.n_layers;
    for (int l = 0; l < m.n_layers; ++l) {
        const Layer &L = m.layer[l];
        f.L[l] = FLayer{L.W16, L.WT16, L.b, L.ld_in, L.ld_out, L.in, L.out};
    }
}

int launch_mlp_fwd_fused(const FGroup &g, void *stream) {
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return (int)e;
    launch_pdl(mlp_fwd_fused, dim3(g.B / 128, g.n_nets), kTF, kFwdSmem, static_cast<cudaStream_t>(stream), g);
    return (int)cudaGetLastError();
}

int launch_mlp_bwd_fused(const FGroup &g, void *stream) {
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBwdSmem);
    if (e != cudaSuccess) return (int)e;
    launch_pdl(mlp_bwd_fused, dim3(g.B / 128, g.n_nets), kTF, kBwdSmem, static_cast<cudaStream_t>(stream), g);
    return (int)cudaGetLastError();
}

int launch_adam_fused(Mlp *const *nets, float *const *part, int n_nets, int n_cta, float lr,
                      float b1, float b2, const float *corr, float wd, void *stream,
                      Mlp *const *targets, float tau) {
    OptGroup G{}, Tg{};
    long long mx = 0;
    for (int k = 0; k < n_nets; ++k) {
        fill_opt(*nets[k], G.net[k]);
        G.net[k].part = part ? part[k] : nullptr;
        mx = mx > G.net[k].total ? mx : G.net[k].total;
        if (targets) {
            fill_opt(*targets[k], Tg.net[k]);
            if (Tg.net[k].total != G.net[k].total) return (int)cudaErrorInvalidValue;
        }
    }
    launch_pdl(adam_fused, dim3((unsigned)((mx + 255) / 256), n_nets), 256, 0,
               static_cast<cudaStream_t>(stream), G, n_cta, lr, b1, b2, corr, wd, Tg,
               targets ? tau : 0.0f);
    return (int)cudaGetLastError();
}

int launch_polyak_fused(Mlp *const *tgt, Mlp *const *src, int n_nets, float tau, void *stream) {
    OptGroup G{};
    long long mx = 0;
    for (int k = 0; k < n_nets; ++k) {
        fill_opt(*tgt[k], G.net[k]);
        for (int l = 0; l < src[k]->n_layers; ++l) {
            G.net[k].src[2 * l] = src[k]->layer[l].W;
            G.net[k].src[2 * l + 1] = src[k]->layer[l].b;
        }
        mx = mx > G.net[k].total ? mx : G.net[k].total;
    }
    launch_pdl(polyak_fused, dim3((unsigned)((mx + 255) / 256), n_nets), 256, 0,
                   static_cast<cudaStream_t>(stream), G, tau);
    return (int)cudaGetLastError();
}

} // namespace flashnav
