// tcgen05 / mbarrier / cp.async helpers shared by the tensor-core kernels
// (nav_mlp.cu: general GEMM; nav_fused.cu: fused small-MLP passes).
// Operand tiles are K-major with the 128-byte swizzle: rows of 64 BF16
// (128 bytes), 8-row atoms of 1024 bytes, the 16-byte piece c of row r
// stored at piece c ^ (r mod 8).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace flashnav {
namespace {

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), start address in 16-byte units.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)1 << 16;                 // leading byte offset (unused here)
    d |= (unsigned long long)(1024u >> 4) << 32;      // stride byte offset
    d |= (unsigned long long)1 << 46;                 // descriptor version
    d |= (unsigned long long)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ unsigned instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) |
           ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Copies rows [r0, r0 + rows) x K-chunk [k0, k0 + 64) of a K-major matrix
// into a swizzled tile; out-of-range rows and columns are zero.
template <int NT>
__device__ __forceinline__ void load_tile(unsigned dst, const __nv_bfloat16 *src, int ld,
                                          int r0, int rows, int nrows_total, int k0, int K) {
    for (int p = threadIdx.x; p < rows * 8; p += NT) {
        const int r = p >> 3, c = p & 7;
        const int gr = r0 + r, k = k0 + c * 8;
        int bytes = 0;
        const __nv_bfloat16 *g = src;
        if (gr < nrows_total && k < K) {
            bytes = K - k >= 8 ? 16 : 2 * (K - k);
            g = src + (size_t)gr * ld + k;
        }
        const unsigned d = dst + (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(bytes)
                     : "memory");
    }
}

// D (TMEM) [+]= A B^T for one K = 16 step, issued by one thread.
__device__ __forceinline__ void mma_f16(unsigned tmem_d, unsigned long long da,
                                        unsigned long long db, unsigned idesc, unsigned accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp
// w reads lanes 32 w .. 32 w + 31).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Byte offset of element (r, k) in a swizzled operand of 128-row tiles
// stored one 64-wide K chunk after another (chunk_bytes apart).
__device__ __forceinline__ unsigned swz(int r, int k, unsigned chunk_bytes) {
    return (unsigned)(k >> 6) * chunk_bytes +
           (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) +
                      (k & 7) * 2);
}

// Column sums of a 32-row x 16-column block held one row per lane: after
// 16 shuffles lane l (even) holds the sum of column ((l >> 1) & 15) in the
// butterfly order below; returns it (odd lanes return their pair's sum too).
__device__ __forceinline__ float colsum16(const float *v, int lane) {
    float a[8];
    const bool up16 = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float send = up16 ? v[i] : v[i + 8];
        const float keep = up16 ? v[i + 8] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    const bool up8 = lane & 8;
    float b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = up8 ? a[i] : a[i + 4];
        const float keep = up8 ? a[i + 4] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const bool up4 = lane & 4;
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = up4 ? b[i] : b[i + 2];
        const float keep = up4 ? b[i + 2] : b[i];
        c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const bool up2 = lane & 2;
    const float send = up2 ? c[0] : c[1];
    const float keep = up2 ? c[1] : c[0];
    float d = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}
// the column whose sum colsum16 leaves in lane l
__device__ __forceinline__ int colsum16_col(int lane) {
    return ((lane & 16) ? 8 : 0) + ((lane & 8) ? 4 : 0) + ((lane & 4) ? 2 : 0) + ((lane & 2) ? 1 : 0);
}

} // namespace
} // namespace flashnav
