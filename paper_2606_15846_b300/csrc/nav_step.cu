// Fused simulator step for sm_103a (FlashNav Sec. 2.2, Eq. 7).
//
// One CTA owns a tile of envs that share a map and a beam count.  It stages
// the tile's packed bitmap into shared memory with one bulk TMA copy
// (cp.async.bulk + mbarrier) when it fits, otherwise reads it through L1/L2.
// Phase 1 (one thread per env): action decode, exact-arc integration, moving
// discs, footprint collision, reward and flags, sparse reset.  Phase 2 (all
// warps): every beam of every env in the tile is cast by Amanatides-Woo grid
// traversal over the bitmap; warps fetch 32-ray chunks from a shared counter
// and a warp retires a chunk when its last ray stops.
//
// Geometry is compiled with FMA contraction off (-fmad=false) and IEEE
// division and square root, so every binary32 operation rounds once and the
// results (hit cells, flags, resets) are a fixed function of the inputs.
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "nav_geom.cuh"
#include "nav_internal.h"
#include "tc_util.cuh"

namespace flashnav {
namespace {

// ---------------------------------------------------------------------------
// Ray phase
// ---------------------------------------------------------------------------
template <bool DYN, bool MARCH, class B>
__device__ void ray_phase(const StepArgs &A, const B &bits, const MapDev &M, const TileDev &T,
                          int K, const float2 *beams, const EnvSlot *slots, const int *fin_slot,
                          int n_fin, const DynEnv *dyn, int *next_chunk) {
    const int lane = threadIdx.x & 31;
    const int n_main = T.env_count * K;
    const int total = n_main + n_fin * K;
    const float rmax_c = A.max_range * M.inv_res;
    const float step_c = A.p.march_step * M.inv_res;
    const float inv_k = 1.0f / (float)K; // rr / K by a multiply and one correction
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(next_chunk, 1);
        chunk = __shfl_sync(kFull, chunk, 0);
        const int base = chunk * 32;
        if (base >= total) break;
        const int rid = base + lane;
        unsigned vis = 0;
        float *row = nullptr;
        float range = 0.0f;
        int k = 0;
        if (rid < total) {
            const bool fin = rid >= n_main;
            const int rr = fin ? rid - n_main : rid; // < 2^24: exact as a float
            int q = (int)((float)rr * inv_k);
            q -= q * K > rr ? 1 : 0;
            q += (q + 1) * K <= rr ? 1 : 0;
            k = rr - q * K;
            const int s = fin ? fin_slot[q] : q;
            const EnvSlot &es = slots[s];
            const float sx = fin ? es.fst : es.st, cx = fin ? es.fct : es.ct;
            const float ox = fin ? es.fxc : es.xc, oy = fin ? es.fyc : es.yc;
            const float2 ab = beams[k];
            // Eq. 4: direction of theta + alpha_k by angle addition
            const float dx = cx * ab.x - sx * ab.y;
            const float dy = sx * ab.x + cx * ab.y;
            const DynEnv *de = DYN ? &dyn[2 * s + (fin ? 1 : 0)] : nullptr;
            int hit;
            range = MARCH ? march_ray<DYN>(bits, M, ox, oy, dx, dy, step_c, rmax_c, A.max_range,
                                           de, hit, vis)
                          : cast_ray<DYN>(bits, M, ox, oy, dx, dy, rmax_c, A.max_range, de,
                                          hit, vis);
            row = (fin ? A.final_obs : A.obs) + es.obs_off;
            if (!fin && A.dbg_range) {
                const long long ro = es.ray_off + k;
                A.dbg_range[ro] = range;
                A.dbg_hit[ro] = hit;
                A.dbg_vis[ro] = vis;
            }
        }
        put_range(A, row, k, K, range, rid < total);
        if (A.stats) {
            unsigned v = vis;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            const int nr = min(32, total - base);
            if (lane == 0) {
                atomicAdd(&A.stats[0], (unsigned long long)v);
                atomicAdd(&A.stats[1], (unsigned long long)nr);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Ray phase with refilled lanes (distance-byte views, no moving discs, exact
// traversal).  The tile's rays form one range [0, envs x K + finals x K);
// every lane walks its own ray with a branch-free iteration (the lanes of a
// warp never diverge), and when enough lanes of a warp are idle the warp
// writes their results and takes as many new rays as it has idle lanes with
// one shared-memory atomic, so lanes do not idle until the slowest ray of a
// fixed 32-ray chunk ends.  The arithmetic of a ray is cast_ray's.
// ---------------------------------------------------------------------------
constexpr int kTileRefill = 16; // idle lanes that make a warp take new rays

// Byte offset of element (row, col) of the fused act-step kernel's actor
// input tile: 128 rows, 64-wide K chunks of 16 KiB, 128-byte swizzle (the
// tensor cores' K-major operand layout).
__device__ __forceinline__ unsigned act_swz(int row, int col) { return swz(row, col, 128u * 128u); }

// 8 floats as 8 BF16 in one 16-byte word
__device__ __forceinline__ uint4 act_pack8(const float *v) {
    uint4 u;
    unsigned *w = reinterpret_cast<unsigned *>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<const unsigned *>(&h);
    }
    return u;
}

// TMEM columns for the CTA (warp 0 allocates; every thread gets the base).
__device__ __forceinline__ unsigned tmem_alloc_cols(unsigned *slot, unsigned ncols) {
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

__device__ __forceinline__ void tmem_free_cols(unsigned tmem, unsigned ncols) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ncols)
                     : "memory");
}

struct TileRay {
    float tM, tm, tdM, tdm, tM0, tm0, kM, km, adm, offm, nM, t;
    int b, b0, sbM, sbm, d, tie;
    int o, k;  // origin record and beam of the ray
    bool stopped;
};

// Quotient by K of a ray index 0 <= r < 2^31 for 1 <= K < 2^16: a
// multiply-high by m = ceil(2^(32+s) / K) with s = ceil(log2 K) - 1, so
// m < 2^32; m K exceeds 2^(32+s) by e < K <= 2^(s+1), and r e < 2^(32+s)
// keeps floor(r m / 2^(32+s)) equal to floor(r / K).
struct DivK {
    unsigned m;
    int s;
    bool one;
    __device__ __forceinline__ explicit DivK(int K) {
        one = K == 1;
        s = one ? 0 : 31 - __clz(K - 1);
        m = one ? 0u
                : (unsigned)((((unsigned long long)1 << (32 + s)) + (unsigned long long)K - 1ull) /
                             (unsigned long long)K);
    }
    __device__ __forceinline__ int operator()(int r) const {
        return one ? r : (int)(__umulhi((unsigned)r, m) >> s);
    }
};

// Sets up ray rid of the tile (cast_ray's set-up from the origin record;
// a blocked or off-map origin ends the ray at once, at its cell or at a
// padding cell).  Rays [0, n_main) are the envs' own scans (origin q), the
// rest the final scans (origin fin_base + q).  Branch-free: the lanes of a
// warp set up rays of any direction together.
__device__ __forceinline__ void tile_ray_init(int pb, int rid, int n_main, int K, DivK divk,
                                              int fin_base, float rmax_c, const float2 *beams,
                                              const RayOrigin *org, TileRay &R) {
    const bool fin = rid >= n_main;
    const int rr = fin ? rid - n_main : rid;
    const int q = divk(rr);
    const int k = rr - q * K;
    R.o = fin ? fin_base + q : q;
    R.k = k;
    const float4 o0 = *reinterpret_cast<const float4 *>(&org[R.o].xc);
    const float4 o1 = *reinterpret_cast<const float4 *>(&org[R.o].flx);
    const float xc = o0.x, yc = o0.y, sx = o0.z, cx = o0.w;
    const float fx = o1.x, fy = o1.y;
    const int b0 = __float_as_int(o1.z), d0 = __float_as_int(o1.w);
    const float2 ab = beams[k];
    // Eq. 4: direction of theta + alpha_k by angle addition
    const float dx = cx * ab.x - sx * ab.y;
    const float dy = sx * ab.x + cx * ab.y;
    R.kM = R.km = 0.0f;
    R.t = 0.0f;
    R.b = R.b0 = b0;
    R.d = d0;
    R.stopped = d0 == 0;
    const float rx = __frcp_rn(fabsf(dx)), ry = __frcp_rn(fabsf(dy));
    const float tdx = dx != 0.0f ? rx : 0.0f, tdy = dy != 0.0f ? ry : 0.0f;
    const float tx0 = dx > 0.0f ? ((fx + 1.0f) - xc) * rx : (dx < 0.0f ? (xc - fx) * rx : INFINITY);
    const float ty0 = dy > 0.0f ? ((fy + 1.0f) - yc) * ry : (dy < 0.0f ? (yc - fy) * ry : INFINITY);
    const int sbx = dx > 0.0f ? 1 : (dx < 0.0f ? -1 : 0);
    const int sby = dy > 0.0f ? pb : (dy < 0.0f ? -pb : 0);
    const bool xmaj = fabsf(dx) >= fabsf(dy);
    R.tdM = xmaj ? tdx : tdy;
    R.tM0 = xmaj ? tx0 : ty0;
    R.tdm = xmaj ? tdy : tdx;
    R.tm0 = xmaj ? ty0 : tx0;
    R.sbM = xmaj ? sbx : sby;
    R.sbm = xmaj ? sby : sbx;
    const float adM = xmaj ? fabsf(dx) : fabsf(dy), adm = xmaj ? fabsf(dy) : fabsf(dx);
    R.adm = adm;
    R.tie = xmaj ? 1 : 0;
    R.offm = adm > 0.0f ? 1.0f - R.tm0 * adm : 0.0f;
    R.nM = floorf(__fmaf_rn(rmax_c, adM, 1.0f - R.tM0 * adM));
    R.tM = R.stopped ? INFINITY : R.tM0;
    R.tm = R.stopped ? INFINITY : R.tm0;
}

// One iteration for the lanes with act set (cast_ray's step or jump),
// branch-free; a lane whose ray ends moves from act to res.  Idle lanes
// re-read their own cell, which lies inside the view.
template <class V>
__device__ __forceinline__ void tile_ray_step(const V &view, float rmax_c, TileRay &R, bool &act,
                                              bool &res) {
    const bool sM = __float_as_int(R.tM) < __float_as_int(R.tm) + R.tie;
    const float tn = sM ? R.tM : R.tm;
    const bool go = act && tn <= rmax_c;
    const float n = fminf((float)R.d - 1.0f, R.nM - R.kM);
    const float kM2 = R.kM + n;
    const float T = __fmaf_rn(kM2 - 1.0f, R.tdM, R.tM0);
    const float km2 = fmaxf(R.km, floorf(__fmaf_rn(T, R.adm, R.offm)));
    const bool jump = n >= 1.0f && T <= rmax_c && km2 - R.km <= n &&
                      __fmaf_rn(km2, R.tdm, R.tm0) > T &&
                      (km2 == R.km || __fmaf_rn(km2 - 1.0f, R.tdm, R.tm0) <= T);
    const float kMn = jump ? kM2 : (sM ? R.kM + 1.0f : R.kM);
    const float kmn = jump ? km2 : (sM ? R.km : R.km + 1.0f);
    const int bn = R.b0 + (int)kMn * R.sbM + (int)kmn * R.sbm;
    const int dn = view.dist_at(go ? bn : R.b);
    if (go) {
        R.kM = kMn;
        R.km = kmn;
        R.tM = __fmaf_rn(kMn, R.tdM, R.tM0);
        R.tm = __fmaf_rn(kmn, R.tdm, R.tm0);
        R.b = bn;
        R.t = tn;
        R.d = dn;
    }
    const bool cont = go && dn != 0;
    R.stopped = R.stopped || (go && dn == 0);
    res = res || (act && !cont);
    act = cont;
}

// With xt set (the fused act-step kernel), each range also goes, times
// xscale[k] (if set) and rounded to BF16, into row q (the env's place in the
// tile), column k of the actor's swizzled input tile at xt.
template <class V>
__device__ void ray_phase_refill(const StepArgs &A, const V &view, const MapDev &M,
                                 const TileDev &T, int K, const float2 *beams,
                                 const RayOrigin *org, int fin_base, int n_fin, int *next_ray,
                                 unsigned char *xt = nullptr, const float *xscale = nullptr) {
    const int lane = threadIdx.x & 31;
    const int n_main = T.env_count * K;
    const int total = n_main + n_fin * K;
    const float rmax_c = A.max_range * M.inv_res;
    const DivK divk(K);
    const int m = A.p.n_sectors;
    TileRay R;
    R.tM = R.tm = INFINITY;
    R.tdM = R.tdm = R.tM0 = R.tm0 = R.kM = R.km = R.adm = R.offm = R.nM = R.t = 0.0f;
    R.b = R.b0 = R.sbM = R.sbm = R.d = R.tie = R.o = R.k = 0;
    R.stopped = false;
    bool act = false, res = false, more = true;
    unsigned vis = 0, nrays = 0;
    int thr = kTileRefill;
    for (;;) {
        if (__any_sync(kFull, act)) {
            for (;;) {
                tile_ray_step(view, rmax_c, R, act, res);
                tile_ray_step(view, rmax_c, R, act, res);
                tile_ray_step(view, rmax_c, R, act, res);
                tile_ray_step(view, rmax_c, R, act, res);
                if (__popc(__ballot_sync(kFull, !act)) >= thr) break;
            }
        }
        if (res) {
            // cast_ray's results: range, hit cell, visits
            const bool fin = R.o >= fin_base;
            const int k = R.k;
            const float range = R.stopped ? R.t * M.res : A.max_range;
            const float c = fminf(range, A.max_range);
            float *row = (fin ? A.final_obs : A.obs) + org[R.o].obs_off;
            if (m == 0) row[k] = c;
            else atomicMin(reinterpret_cast<int *>(row + k / (K / m)), __float_as_int(c));
            if (xt && !fin)
                *reinterpret_cast<__nv_bfloat16 *>(xt + act_swz(R.o, k)) =
                    __float2bfloat16_rn(xscale ? c * __ldg(xscale + k) : c);
            // visits (exact: both counts are integers below 2^24), only when
            // counted or captured
            const unsigned v = (A.stats || A.dbg_range) ? 1u + (unsigned)(R.kM + R.km) : 0u;
            if (!fin && A.dbg_range) {
                int hit = -2;
                if (R.stopped) {
                    const int jj = R.b / view.stride, ii = R.b - jj * view.stride;
                    const int i = ii - kPad, j = jj - kPad;
                    hit = (i < 0 || j < 0 || i >= M.w || j >= M.h) ? -1 : j * M.w + i;
                }
                const long long ro = org[R.o].ray_off + k;
                A.dbg_range[ro] = range;
                A.dbg_hit[ro] = hit;
                A.dbg_vis[ro] = v;
            }
            vis += v;
            nrays += 1u;
            res = false;
        }
        const unsigned want = __ballot_sync(kFull, !act);
        if (more && want) {
            int base = 0;
            if (lane == 0) base = atomicAdd(next_ray, __popc(want));
            base = __shfl_sync(kFull, base, 0);
            const int r = base + __popc(want & ((1u << lane) - 1u));
            if (((want >> lane) & 1u) && r < total) {
                tile_ray_init(view.stride, r, n_main, K, divk, fin_base, rmax_c, beams, org, R);
                act = !R.stopped;
                res = R.stopped;
            }
            if (base + __popc(want) >= total) more = false;
        }
        if (!more) {
            if (!__any_sync(kFull, act || res)) break;
            thr = 32;
        }
    }
    if (A.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vis += __shfl_xor_sync(kFull, vis, o);
            nrays += __shfl_xor_sync(kFull, nrays, o);
        }
        if (lane == 0 && nrays) {
            atomicAdd(&A.stats[0], (unsigned long long)vis);
            atomicAdd(&A.stats[1], (unsigned long long)nrays);
        }
    }
}

template <bool DYN, bool MARCH, bool REFILL, class V>
__device__ __forceinline__ void run_tile(const StepArgs &A, const V &view, const MapDev &M,
                                         const TileDev &T, int K, const float2 *sbeam,
                                         EnvSlot *slots, int *fin_slot, int *n_fin, DynEnv *sdyn,
                                         RayOrigin *org, int *next_chunk, const EnvIn &pre) {
    const int tid = threadIdx.x;
    constexpr bool kRefill = REFILL && !DYN && !MARCH && has_dist<V>::value;
    if constexpr (DYN) {
        // with moving discs, one thread per env (`pre`: that env's inputs):
        // the discs' motion and stamps would otherwise run on every lane
        if (tid < T.env_count)
            env_phase<DYN>(A, view, M, K, tid, slots[tid], &sdyn[2 * tid], &sdyn[2 * tid + 1], pre);
    } else {
        // one warp per env (its lanes test the footprint's rows in parallel;
        // `pre` holds the inputs of the warp's first env)
        const int warp = tid >> 5, nw = (int)(blockDim.x >> 5);
        for (int q = warp; q < T.env_count; q += nw) {
            if (q == warp) {
                env_phase<DYN, true>(A, view, M, K, q, slots[q], nullptr, nullptr, pre);
            } else {
                // tiles with more envs than warps: the later envs load their own
                const EnvIn in = A.mode == 0 ? load_env(A, slots[q].env) : EnvIn{};
                env_phase<DYN, true>(A, view, M, K, q, slots[q], nullptr, nullptr, in);
            }
            if constexpr (kRefill) {
                const EnvSlot &es = slots[q];
                set_origin(view, M, es.xc, es.yc, es.st, es.ct, es.obs_off, es.ray_off, org[q]);
            }
        }
    }
    __syncthreads();
    if (tid < 32) {
        const bool f = tid < T.env_count && slots[tid].fin;
        const unsigned m = __ballot_sync(kFull, f);
        const int fi = __popc(m & ((1u << tid) - 1u));
        if (f) {
            fin_slot[fi] = tid;
            if constexpr (kRefill) {
                const EnvSlot &es = slots[tid];
                set_origin(view, M, es.fxc, es.fyc, es.fst, es.fct, es.obs_off, es.ray_off,
                           org[kMaxTileEnvs + fi]);
            }
        }
        if (tid == 0) *n_fin = __popc(m);
    }
    __syncthreads();
    // next-episode records of the envs that reset, written by warp 0 while
    // the other warps start on the rays
    if (tid < T.env_count && slots[tid].prep) prep_next(A, M, slots[tid].env, slots[tid].ep);
    if constexpr (kRefill)
        ray_phase_refill(A, view, M, T, K, sbeam, org, kMaxTileEnvs, *n_fin, next_chunk);
    else
        ray_phase<DYN, MARCH>(A, view, M, T, K, sbeam, slots, fin_slot, *n_fin, sdyn, next_chunk);
}

// Persistent CTAs: each CTA takes tiles from a global queue until none are
// left.  A tile's map is staged into shared memory (its distance bytes or
// its packed bits, by bulk TMA copies) only when the CTA's previous tile used
// another map.  The CTA that draws the launch's last index zeroes the queue
// for the next launch on the stream.
// MINB: resident 512-thread CTAs per SM the register allocation must allow
// (4, 3, 2 -> at most 32, 40, 64 registers per thread).
template <bool DYN, int MINB, bool MARCH, bool REFILL>
__global__ void __launch_bounds__(512, MINB) step_kernel(const StepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ EnvSlot slots[kMaxTileEnvs];
    __shared__ RayOrigin org[REFILL ? 2 * kMaxTileEnvs : 1];
    __shared__ int fin_slot[kMaxTileEnvs];
    __shared__ int n_fin;
    __shared__ int next_chunk;
    __shared__ int tile_id;
    __shared__ int staged_map;
    __shared__ __align__(8) unsigned long long bar;

    uint32_t *sbits = reinterpret_cast<uint32_t *>(smem);
    uint8_t *sbytes = smem;
    float2 *sbeam = reinterpret_cast<float2 *>(smem + (size_t)A.smem_region_bytes);
    DynEnv *sdyn = reinterpret_cast<DynEnv *>(smem + (size_t)A.smem_region_bytes +
                                              (size_t)A.max_k * sizeof(float2));
    const int tid = threadIdx.x;
    unsigned parity = 0;
    int beam_tab = -1;
    // Every CTA draws tile indices until it gets one past the last tile, so a
    // launch makes exactly n_tiles + gridDim draws; the CTA holding the last
    // one zeroes the queue for the next launch (nobody draws after it).
    const int last_draw = A.n_tiles + (int)gridDim.x - 1;
    // exactly one tile per CTA (a full wave): CTA b takes tile b and the
    // queue is not touched (its first draw, an atomic that waits on L2, is
    // off the path to the tile's map)
    const bool one_each = A.n_tiles == (int)gridDim.x;
    int cur = 0;
    if (tid == 0) {
        init_copy_barrier(&bar);
        staged_map = -1;
        cur = one_each ? (int)blockIdx.x : atomicAdd(&A.tile_queue[0], 1);
    }
    // a CTA runs at most n_tiles tiles: a queue left non-zero by a failed
    // launch ends the loop with a status bit instead of running on
    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            tile_id = cur;
            next_chunk = 0;
            if (cur == last_draw) A.tile_queue[0] = 0;
            if (iter >= A.n_tiles && cur < A.n_tiles) {
                atomicOr(A.status, kStatusQueue);
                tile_id = A.n_tiles;
            }
        }
        __syncthreads();
        const int tile = tile_id;
        if (tile >= A.n_tiles) break;
        // the tile's env (read with its record: one dependent load less)
        const int e_tile = A.tile_env && tid < kMaxTileEnvs ? A.tile_env[tile * kMaxTileEnvs + tid] : -1;
        // the tile's staging record, read with the tile's (the copy starts
        // before the map's own record has arrived)
        const int4 ts = A.tile_stage ? A.tile_stage[tile] : make_int4(-1, 0, 0, 0);
        const TileDev T = A.tiles[tile];
        const MapDev M = A.maps[T.map];
        const int K = A.tab_k[T.tab];
        const uint32_t *gbits = A.bits + M.word_off;
        const bool fresh = staged_map != T.map;
        const int smode = ts.x >= 0 ? ts.x : M.mode;
        const bool copy = (smode == kMapSharedBits || smode == kMapSharedBytes) && fresh;
        if (copy && tid == 0) {
            if (ts.x >= 0) {
                const long long off = ((long long)(unsigned)ts.w << 32) | (long long)(unsigned)ts.z;
                const unsigned char *src = smode == kMapSharedBits
                                               ? reinterpret_cast<const unsigned char *>(A.bits)
                                               : A.dist;
                stage_map(smode == kMapSharedBits ? static_cast<void *>(sbits)
                                                  : static_cast<void *>(sbytes),
                          src + off, (unsigned)ts.y, &bar);
            } else if (smode == kMapSharedBits) {
                stage_map(sbits, gbits, (unsigned)M.n_words * 4u, &bar);
            } else {
                stage_map(sbytes, A.dist + M.dist_off, (unsigned)M.n_bytes, &bar);
            }
        }
        if (T.tab != beam_tab) {
            const int toff = A.tab_off[T.tab];
            for (int k = tid; k < K; k += blockDim.x)
                sbeam[k] = make_float2(A.beam_c[toff + k], A.beam_s[toff + k]);
            beam_tab = T.tab;
        }
        if (tid < T.env_count) {
            const int e = A.tile_env ? e_tile : A.perm[T.env_begin + tid];
            slots[tid].env = e;
            slots[tid].obs_off = A.obs_off[e];
            slots[tid].ray_off = A.ray_off[e];
        }
        // the inputs of the env whose phase this thread's warp (or, with
        // moving discs, this thread) runs first, loaded before the map has
        // landed so that their latency overlaps it
        EnvIn pre{};
        if ((DYN ? tid : tid >> 5) < T.env_count && A.mode == 0) {
            const int q = DYN ? tid : tid >> 5;
            pre = load_env(A, A.tile_env ? A.tile_env[tile * kMaxTileEnvs + q] : A.perm[T.env_begin + q]);
        }
        bool ok = true;
        if (copy) {
            ok = wait_bitmap(&bar, parity);
            parity ^= 1u;
        }
        // the block agrees on one outcome so that all threads take one path
        const bool failed = __syncthreads_or(!ok) != 0;
        if (failed) {
            // the copy did not land in time: report it, wait (bounded) for the
            // copy in flight, and read this tile's bitmap from global memory
            if (tid == 0) atomicOr(A.status, kStatusCopyTimeout);
            if (!ok) wait_bitmap(&bar, parity ^ 1u);
        }
        const int mode = failed ? (int)kMapGlobal : smode;
        if (tid == 0) staged_map = mode == kMapGlobal || mode == kMapGlobalBytes ? -1 : T.map;
        if (mode == kMapSharedBytes)
            run_tile<DYN, MARCH, REFILL>(A, BytesShared{sbytes, M.byte_stride}, M, T, K, sbeam, slots, fin_slot,
                          &n_fin, sdyn, org, &next_chunk, pre);
        else if (mode == kMapSharedBits)
            run_tile<DYN, MARCH, REFILL>(A, BitsShared{sbits, M.pitch * 32}, M, T, K, sbeam, slots, fin_slot,
                          &n_fin, sdyn, org, &next_chunk, pre);
        else if (mode == kMapGlobalBytes)
            run_tile<DYN, MARCH, REFILL>(A, BytesGlobal{A.dist + M.dist_off, M.byte_stride}, M, T, K, sbeam,
                                 slots, fin_slot, &n_fin, sdyn, org, &next_chunk, pre);
        else
            run_tile<DYN, MARCH, REFILL>(A, BitsGlobal{gbits, M.pitch * 32}, M, T, K, sbeam, slots, fin_slot,
                          &n_fin, sdyn, org, &next_chunk, pre);
        __syncthreads();
        if (tid == 0) cur = one_each ? A.n_tiles : atomicAdd(&A.tile_queue[0], 1);
    }
}

// ---------------------------------------------------------------------------
// Fused act-step kernel: the step of a tile of up to 128 envs (env phase,
// refilled ray phase) and then the FastDSAC actor (Sec. 2.3; Sec. 2.1 MLP)
// on the tile's new observations, on the tensor cores, from shared memory:
// the observation rows the ray and env phases produce are written, scaled
// and rounded to BF16, straight into the actor's swizzled input tile; the
// three layers (in -> H -> H -> 4, LeakyReLU) stream their weights one
// 64-wide K chunk of all of a layer's output rows at a time (up to 32 KiB),
// pre-swizzled in global memory (bulk copies issued by one thread into
// 32 KiB slots that reuse the staged map's region), accumulate in TMEM
// (tcgen05.mma, M 128, N up to 256, one thread issuing) and are read
// back by every warp (tcgen05.ld) for bias, LeakyReLU and the next layer's
// BF16 tile, written in place; the head turns the last layer's
// (mean, raw log-std) into the action of each env for the next step,
// a = tanh(u + sigma eps) with sigma = exp(-5 + 5 (tanh(r) + 1) / 2) and eps
// from the counter-hash Box-Muller draw keyed by (seed, env, step), or
// tanh(u) when deterministic.  The step's observations are still written to
// obs (the replay needs them), but the policy never reads them back.
// ---------------------------------------------------------------------------
constexpr int kActThreads = 1024;
constexpr int kActMaxEnvs = 128;                 // rows of the MMA tile
constexpr unsigned kActChunk = 128u * 128u;      // a 64-wide K chunk of the input tile
constexpr int kActKChunks = 6;                   // input features <= 384
constexpr unsigned kActSlot = 2u * kActChunk;    // a weight slot: one K chunk of 256 rows
constexpr int kActMaxSlots = 4;

__device__ __forceinline__ unsigned long long act_mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Input feature of a tail value (goal distance, bearing, v, w) of row q.
__device__ __forceinline__ void act_tail(unsigned char *xt, const ActArgs &P, int q, int K,
                                         const float *obs_row) {
    for (int i = 0; i < 4; ++i) {
        const float x = obs_row[K + i];
        *reinterpret_cast<__nv_bfloat16 *>(xt + act_swz(q, K + i)) =
            __float2bfloat16_rn(P.scale ? x * __ldg(P.scale + K + i) : x);
    }
    for (int c = K + 4; c < kActKChunks * 64; ++c)
        *reinterpret_cast<__nv_bfloat16 *>(xt + act_swz(q, c)) = __float2bfloat16_rn(0.0f);
}

// Weight unit u of the actor: layer l, 64-wide K chunk c, output half h
// (rows 128 h ..), and its rows (the layer's width rounded up to 16, at most
// 128).  Units run over the layers in order, K chunks outer, halves inner.
__device__ __forceinline__ void act_unit(const ActArgs &P, int u, int &l, int &c, int &h,
                                         int &rows) {
    l = 0;
    for (;;) {
        const int nk = (P.in[l] + 63) >> 6, nh = P.out[l] > 128 ? 2 : 1;
        if (u < nk * nh || l == 2) {
            c = u / nh;
            h = u % nh;
            rows = min(128, ((P.out[l] + 15) & ~15) - 128 * h);
            return;
        }
        u -= nk * nh;
        ++l;
    }
}

// Weight item i of the actor: layer l, 64-wide K chunk c, the first of its
// units (u0: both halves of the chunk, units u0 and u0 + 1, when the layer
// has more than 128 outputs; they lie next to each other in the unit array)
// and the layer's rows rounded up to 16 (the MMA's N).  Items run over the
// layers in order, K chunks inner; the last layer, when all of its K chunks
// fit one slot (the head's 4 outputs: 2 KiB a chunk), is one item of nc
// chunks (each commit drains the tensor pipe, so one instead of nc).
__device__ __forceinline__ bool act_last_whole(const ActArgs &P) {
    return P.out[2] <= 128 &&
           (unsigned)((P.in[2] + 63) >> 6) * (unsigned)((P.out[2] + 15) & ~15) * 128u <= kActSlot;
}

__device__ __forceinline__ int act_items(const ActArgs &P) {
    return ((P.in[0] + 63) >> 6) + ((P.in[1] + 63) >> 6) +
           (act_last_whole(P) ? 1 : (P.in[2] + 63) >> 6);
}

__device__ __forceinline__ void act_item(const ActArgs &P, int i, int &l, int &c, int &u0,
                                         int &np, int &nc) {
    l = 0;
    u0 = 0;
    for (;;) {
        const int nk = (P.in[l] + 63) >> 6, nh = P.out[l] > 128 ? 2 : 1;
        if (i < nk || l == 2) {
            const bool whole = l == 2 && act_last_whole(P);
            c = whole ? 0 : i;
            nc = whole ? nk : 1;
            u0 += c * nh;
            np = (P.out[l] + 15) & ~15;
            return;
        }
        i -= nk;
        u0 += nk * nh;
        ++l;
    }
}

// One thread per 16-byte piece (8 BF16) of a unit: the weights W[l] [out][ld]
// rearranged into the 128-byte-swizzled K-major tile the MMAs read (zero
// beyond the layer's rows and inputs), so that one bulk copy stages a unit.
__global__ void act_swizzle_kernel(const ActArgs P, unsigned char *dst, int nunits) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int u = t >> 10, r = (t >> 3) & 127, p = t & 7;
    if (u >= nunits) return;
    int l, c, h, rows;
    act_unit(P, u, l, c, h, rows);
    if (r >= rows) return;
    const int row = 128 * h + r, k = 64 * c + 8 * p;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        v[e] = (row < P.out[l] && k + e < P.in[l]) ? P.W[l][(size_t)row * P.ld[l] + k + e]
                                                   : __float2bfloat16_rn(0.0f);
    *reinterpret_cast<uint4 *>(dst + (size_t)u * kActChunk + (r >> 3) * 1024 + (r & 7) * 128 +
                               ((p ^ (r & 7)) << 4)) = *reinterpret_cast<const uint4 *>(v);
}

__device__ __forceinline__ bool act_wait(unsigned bar, unsigned parity, int *status) {
    if (mbar_wait(bar, parity)) return true;
    atomicOr(status, kStatusCopyTimeout);
    return false;
}

__global__ void __launch_bounds__(kActThreads, 1) act_step_kernel(const StepArgs A, const ActArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ EnvSlot slots[kActMaxEnvs];
    __shared__ RayOrigin org[kActMaxEnvs];
    __shared__ int next_ray;
    __shared__ int tile_id;
    __shared__ __align__(8) unsigned long long bar_map;
    __shared__ __align__(8) unsigned long long bar_ld[kActMaxSlots]; // weight item landed, per slot
    __shared__ __align__(8) unsigned long long bar_w[kActMaxSlots];  // MMAs done reading, per slot
    __shared__ unsigned tmem_slot;
    // [0, region): the staged map, or during the actor NS 32 KiB weight slots
    // [region, region + 96 KiB): the actor's input tile (then H1, H2)
    // then the beam table
    // the swizzled tiles need 1024-byte alignment (act_step_smem adds the slack)
    unsigned char *base = smem + ((1024u - (smem_addr(smem) & 1023u)) & 1023u);
    const unsigned region = (unsigned)A.smem_region_bytes; // a multiple of 1024, >= 64 KiB
    uint8_t *sbytes = base;
    unsigned char *xt = base + region;
    float2 *sbeam = reinterpret_cast<float2 *>(base + region + kActKChunks * kActChunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, grp = warp >> 2; // TMEM lane quarter, column group (8 of 32)
    unsigned map_parity = 0;
    int beam_tab = -1;
    // The weights stream from their swizzled copy as items (act_item: one
    // 64-wide K chunk of all of a layer's output rows, up to 32 KiB) by bulk
    // copies into the NS slots of the map's region (free once the ray phase
    // ends).  A K chunk's MMAs run at N = the layer's rows (up to 256): an
    // MMA costs about the same at N 128 as at 256, and each commit drains the
    // tensor pipe, so one commit per chunk rather than per 128-row half.  A
    // slot is refilled one item after its MMAs were issued (by then they have
    // completed, so the refill does not wait on the MMAs just issued).
    // Thread 0 alone issues the copies and the MMAs and tracks, per slot, the
    // phase bits of its two mbarriers and whether an MMA commit on it is
    // still to be waited for.
    unsigned ph_ld = 0u, ph_w = 0u, pend_w = 0u;
    const int nitems = act_items(P);
    const bool last_whole = act_last_whole(P);
    const int NS = min(kActMaxSlots, (int)(region / kActSlot)); // >= 2: region >= 64 KiB
    int next_item = 0;
    if (tid == 0) {
        init_copy_barrier(&bar_map);
        for (int b = 0; b < NS; ++b) {
            init_copy_barrier(&bar_ld[b]);
            init_copy_barrier(&bar_w[b]);
        }
    }
    const unsigned tmem = tmem_alloc_cols(&tmem_slot, 256);
    const unsigned tlane = (unsigned)(quad * 32) << 16;
    const unsigned xt_a = smem_addr(xt);
    const unsigned wb0 = smem_addr(base); // slot b at wb0 + b * 32 KiB
    // (thread 0) waits for the outstanding MMA commit on buffer b, if any
    auto wait_mma = [&](int b) {
        if ((pend_w >> b) & 1u) {
            act_wait(smem_addr(&bar_w[b]), (ph_w >> b) & 1u, A.status);
            ph_w ^= 1u << b;
            pend_w &= ~(1u << b);
        }
    };
    // (thread 0) stages item i once its slot's previous MMAs have completed
    auto issue_item = [&](int i) {
        int l, c, u0, np, nc;
        act_item(P, i, l, c, u0, np, nc);
        const int s = i % NS;
        wait_mma(s);
        if (nc == 1) {
            stage_map(base + (size_t)s * kActSlot, P.Wu + (size_t)u0 * kActChunk,
                      (unsigned)np * 128u, &bar_ld[s]);
        } else {
            // nc chunks of np rows, each from its own unit, packed in the slot
            const unsigned b = smem_u32(&bar_ld[s]), part = (unsigned)np * 128u;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                         "r"(part * (unsigned)nc)
                         : "memory");
            for (int q = 0; q < nc; ++q)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                    "%2, [%3];" ::"r"(wb0 + (unsigned)s * kActSlot + (unsigned)q * part),
                    "l"(P.Wu + (size_t)(u0 + q) * kActChunk), "r"(part), "r"(b)
                    : "memory");
        }
    };
    // (thread 0) stages every item not yet staged whose slot held item x or
    // an earlier one
    auto refill = [&](int x) {
        while (next_item < nitems && next_item - NS <= x) issue_item(next_item++);
    };
    for (;;) {
        if (tid == 0) {
            tile_id = atomicAdd(&A.tile_queue[0], 1);
            next_ray = 0;
        }
        __syncthreads();
        const int tile = tile_id;
        if (tile >= A.n_tiles) break;
        const TileDev T = A.tiles[tile];
        const MapDev M = A.maps[T.map];
        const int K = A.tab_k[T.tab];
        // the map region held weights during the previous tile: restage
        if (tid == 0) stage_map(sbytes, A.dist + M.dist_off, (unsigned)M.n_bytes, &bar_map);
        if (T.tab != beam_tab) {
            const int toff = A.tab_off[T.tab];
            for (int k = tid; k < K; k += blockDim.x)
                sbeam[k] = make_float2(A.beam_c[toff + k], A.beam_s[toff + k]);
            beam_tab = T.tab;
        }
        EnvIn pre{};
        if (tid < T.env_count) {
            const int e = A.perm[T.env_begin + tid];
            slots[tid].env = e;
            slots[tid].obs_off = A.obs_off[e];
            slots[tid].ray_off = A.ray_off[e];
            if (A.mode == 0) pre = load_env(A, e); // overlaps the map's staging
        }
        // rows beyond the tile's envs: zero (their outputs are not used)
        for (int p = tid; p < (kActMaxEnvs - T.env_count) * kActKChunks * 8; p += blockDim.x) {
            const int r = T.env_count + p / (kActKChunks * 8), c = (p % (kActKChunks * 8)) * 8;
            *reinterpret_cast<uint4 *>(xt + act_swz(r, c)) = make_uint4(0u, 0u, 0u, 0u);
        }
        bool ok = true;
        if (tid == 0) {
            ok = wait_bitmap(&bar_map, map_parity);
            if (!ok) {
                atomicOr(A.status, kStatusCopyTimeout);
                wait_bitmap(&bar_map, map_parity); // the copy in flight, bounded
            }
        }
        map_parity ^= 1u;
        if (__syncthreads_or(!ok)) break;
        const BytesShared view{sbytes, M.byte_stride};
        if (tid < T.env_count) {
            env_phase<false>(A, view, M, K, tid, slots[tid], nullptr, nullptr, pre);
            const EnvSlot &es = slots[tid];
            set_origin(view, M, es.xc, es.yc, es.st, es.ct, es.obs_off, es.ray_off, org[tid]);
            act_tail(xt, P, tid, K, A.obs + es.obs_off);
        }
        __syncthreads();
        // next-episode records of the envs that reset (their warps cast later)
        if (tid < T.env_count && slots[tid].prep) prep_next(A, M, slots[tid].env, slots[tid].ep);
        ray_phase_refill(A, view, M, T, K, sbeam, org, kActMaxEnvs, 0, &next_ray, xt, P.scale);
        // ---- the actor on the tile's observations ----
        // the input tile, written by generic stores, is read by the MMAs
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads(); // the map's region is free: the weight buffers
        int it = 0;
        if (tid == 0) {
            next_item = 0;
            refill(-1);
        }
        for (int l = 0; l < 3; ++l) {
            const int out = P.out[l], np = (out + 15) & ~15;
            const bool last = l == 2;
            const int nk = (P.in[l] + 63) >> 6;
            // chunks per item: all of them for a last layer that is one item
            const int per = last && last_whole ? nk : 1;
            if (tid == 0) {
                const unsigned idesc = instr_desc(128, np);
                for (int c = 0; c < nk; c += per, ++it) {
                    const int b = it % NS;
                    act_wait(smem_addr(&bar_ld[b]), (ph_ld >> b) & 1u, A.status);
                    ph_ld ^= 1u << b;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int q = 0; q < per; ++q) {
                        const unsigned a = xt_a + (c + q) * kActChunk;
                        const unsigned wbuf = wb0 + (unsigned)b * kActSlot + (unsigned)(q * np * 128);
#pragma unroll
                        for (int k16 = 0; k16 < 4; ++k16)
                            mma_f16(tmem, smem_desc(a + 32u * k16), smem_desc(wbuf + 32u * k16),
                                    idesc, (c + q > 0 || k16 > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_addr(&bar_w[b]));
                    pend_w |= 1u << b;
                    refill(it - 1);
                }
                // the layer's last MMAs (and so every one of its MMAs) have
                // completed; the slots they read take the next items
                wait_mma((it - 1) % NS);
                refill(it - 1);
            }
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = quad * 32 + lane;
            if (!last) {
                // bias, LeakyReLU, BF16, in place into the input tile (its
                // columns [out, in) zeroed for the next layer)
                const int j0 = 32 * grp;
                for (int j = j0; j < j0 + 32; j += 16) {
                    float v[16];
                    tmem_ld16(tmem + tlane + (unsigned)j, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float x = j + i < out ? v[i] + __ldg(P.b[l] + j + i) : 0.0f;
                        v[i] = x > 0.0f ? x : 0.01f * x;
                    }
                    if (j < np) {
                        *reinterpret_cast<uint4 *>(xt + act_swz(row, j)) = act_pack8(v);
                        *reinterpret_cast<uint4 *>(xt + act_swz(row, j + 8)) = act_pack8(v + 8);
                    }
                }
                // the next layer reads whole 64-wide chunks: columns [np, 64
                // ceil(out / 64)) must be zero too
                if (grp == 0)
                    for (int c0 = np; c0 < ((out + 63) & ~63); c0 += 8)
                        *reinterpret_cast<uint4 *>(xt + act_swz(row, c0)) = make_uint4(0u, 0u, 0u, 0u);
            } else if (grp == 0) {
                // the head: (mean u, raw log-std r) -> the env's next action
                float v[16];
                tmem_ld16(tmem + tlane, v);
                if (row < T.env_count) {
                    const int e = slots[row].env;
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        const float u = v[d] + __ldg(P.b[2] + d);
                        const float r = v[2 + d] + __ldg(P.b[2] + 2 + d);
                        const float ls = -5.0f + 5.0f * 0.5f * (tanhf(r) + 1.0f);
                        float ep = 0.0f;
                        if (P.mode == 1) {
                            const unsigned long long h =
                                act_mix64(P.seed ^ ((unsigned long long)e * 0xD1B54A32D192ED03ull) ^
                                          ((unsigned long long)P.step << 32) ^ (unsigned)d);
                            const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
                            const float u2 = (float)((h >> 8) & 0xFFFFFFull) * (1.0f / 16777216.0f);
                            ep = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
                        }
                        P.act[(size_t)e * 2 + d] = tanhf(u + expf(ls) * ep);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    tmem_free_cols(tmem, 256);
    if (tid == 0) {
        __threadfence();
        const int done = atomicAdd(&A.tile_queue[1], 1);
        if (done == (int)gridDim.x - 1) {
            A.tile_queue[0] = 0;
            A.tile_queue[1] = 0;
            __threadfence();
        }
    }
}

// Uniform actions in [-1, 1]^2 from the counter hash keyed by (seed, env, step):
// an input generator for autotuning and throughput runs (not part of a step).
__global__ void uniform_actions_kernel(float2 *out, int n_envs, unsigned long long seed,
                                       unsigned step) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    const unsigned long long h = draw64(seed, (unsigned)e, step, 0x5EEDu);
    const float a = draw_unit((unsigned)(h >> 40)) * 2.0f - 1.0f;
    const float b = draw_unit((unsigned)((h >> 8) & 0xFFFFFFull)) * 2.0f - 1.0f;
    out[e] = make_float2(a, b);
}

// ---------------------------------------------------------------------------
// Split step.  env_kernel: one thread per env runs the env phase (decode,
// arc, footprint, reward, flags, reset) against the packed bits in L1/L2 and
// records the ray origin of the obs scan (and of the final scan, appending
// the env to the final list).  ray_kernel: persistent CTAs stage every map
// and every beam table into shared memory once; each warp then takes 32-ray
// chunks from a global queue and casts them with no CTA-wide barrier, then
// takes the pending final scans env by env.  The last CTA resets the queues.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) prep_all_kernel(const StepArgs A, int n_envs) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    prep_next(A, A.maps[A.env_map[e]], e, A.episode[e]);
}

__global__ void __launch_bounds__(128) env_kernel(const StepArgs A, int n_envs) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_envs) return;
    const MapDev M = A.maps[A.env_map[e]];
    const int K = A.tab_k[A.env_tab[e]];
    EnvSlot slot;
    slot.env = e;
    slot.obs_off = A.obs_off[e];
    slot.ray_off = A.ray_off[e];
    const EnvIn pre = A.mode == 0 ? load_env(A, e) : EnvIn{};
    env_phase<false>(A, BitsGlobal{A.bits + M.word_off, M.pitch * 32}, M, K, 0, slot, nullptr,
                     nullptr, pre);
    if (slot.prep) prep_next(A, M, e, slot.ep);
    A.ray_main[e] = make_float4(slot.xc, slot.yc, slot.st, slot.ct);
    if (slot.fin) {
        A.ray_fin[e] = make_float4(slot.fxc, slot.fyc, slot.fst, slot.fct);
        A.fin_list[atomicAdd(&A.split_q[3], 1)] = e;
    }
}

// Casts one ray of the split step (no moving discs) and returns its range;
// the caller stores it with put_range.
template <bool MARCH, class V>
__device__ __forceinline__ float cast_one(const StepArgs &A, const V &view, const MapDev &M,
                                          float4 o, float2 ab, int e, int k, bool fin,
                                          unsigned &vis) {
    const float dx = o.w * ab.x - o.z * ab.y;
    const float dy = o.z * ab.x + o.w * ab.y;
    const float rmax_c = A.max_range * M.inv_res;
    int hit;
    const float range =
        MARCH ? march_ray<false>(view, M, o.x, o.y, dx, dy, A.p.march_step * M.inv_res, rmax_c,
                                 A.max_range, nullptr, hit, vis)
              : cast_ray<false>(view, M, o.x, o.y, dx, dy, rmax_c, A.max_range, nullptr, hit,
                                vis);
    if (!fin && A.dbg_range) {
        const long long ro = A.ray_off[e] + k;
        A.dbg_range[ro] = range;
        A.dbg_hit[ro] = hit;
        A.dbg_vis[ro] = vis;
    }
    return range;
}

__device__ __forceinline__ void add_stats(const StepArgs &A, unsigned vis, int nr) {
    if (!A.stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vis += __shfl_xor_sync(kFull, vis, o);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&A.stats[0], (unsigned long long)vis);
        atomicAdd(&A.stats[1], (unsigned long long)nr);
    }
}

template <bool MARCH>
__global__ void __launch_bounds__(1024, 1) ray_kernel(const StepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar;
    uint32_t *sbits = reinterpret_cast<uint32_t *>(smem);
    float2 *sbeam = reinterpret_cast<float2 *>(smem + (size_t)A.all_words * 4);
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        init_copy_barrier(&bar);
        // every map in one transaction count: the copies of all maps complete
        // phase 0 of the barrier
        const unsigned b = smem_u32(&bar);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                     "r"((unsigned)A.all_words * 4u)
                     : "memory");
        for (int m = 0; m < A.n_maps_split; ++m) {
            const MapDev M = A.maps[m];
            const unsigned bytes = (unsigned)M.n_words * 4u;
            for (unsigned off = 0; off < bytes; off += 32768u) {
                const unsigned n = bytes - off < 32768u ? bytes - off : 32768u;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                    "%2, [%3];" ::"r"(smem_u32(sbits + M.all_off) + off),
                    "l"((const char *)(A.bits + M.word_off) + off), "r"(n), "r"(b)
                    : "memory");
            }
        }
    }
    for (int i = tid; i < A.n_beams_total; i += blockDim.x)
        sbeam[i] = make_float2(A.beam_c[i], A.beam_s[i]);
    __syncthreads();
    const bool ok = wait_bitmap(&bar, 0);
    const bool failed = __syncthreads_or(!ok) != 0;
    if (failed) {
        if (tid == 0) atomicOr(A.status, kStatusCopyTimeout);
        if (!ok) wait_bitmap(&bar, 0);
        __syncthreads();
    }
    // obs scans: each warp takes 32-ray chunks from the queue
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&A.split_q[0], 1);
        c = __shfl_sync(kFull, c, 0);
        if (c >= A.n_chunks) break;
        const int2 ch = A.chunks[c];
        const TileDev T = A.tiles[ch.x];
        const MapDev M = A.maps[T.map];
        const int K = A.tab_k[T.tab];
        const int r = ch.y + lane;
        const bool active = r < T.env_count * K;
        unsigned vis = 0;
        float range = 0.0f, *row = nullptr;
        int k = 0;
        if (active) {
            const int el = r / K;
            k = r - el * K;
            const int e = A.perm[T.env_begin + el];
            const float4 o = A.ray_main[e];
            const float2 ab = sbeam[A.tab_off[T.tab] + k];
            if (!failed)
                range = cast_one<MARCH>(A, BitsShared{sbits + M.all_off, M.pitch * 32}, M, o, ab,
                                        e, k, false, vis);
            else
                range = cast_one<MARCH>(A, BitsGlobal{A.bits + M.word_off, M.pitch * 32}, M, o,
                                        ab, e, k, false, vis);
            row = A.obs + A.obs_off[e];
        }
        put_range(A, row, k, K, range, active);
        add_stats(A, vis, min(32, T.env_count * K - ch.y));
    }
    // final scans of the envs that finished this step
    if (A.final_obs) {
        const int n_fin = *(volatile int *)&A.split_q[3];
        for (;;) {
            int f = 0;
            if (lane == 0) f = atomicAdd(&A.split_q[1], 1);
            f = __shfl_sync(kFull, f, 0);
            if (f >= n_fin) break;
            const int e = A.fin_list[f];
            const MapDev M = A.maps[A.env_map[e]];
            const int K = A.tab_k[A.env_tab[e]];
            const int toff = A.tab_off[A.env_tab[e]];
            const float4 o = A.ray_fin[e];
            float *row = A.final_obs + A.obs_off[e];
            for (int k0 = 0; k0 < K; k0 += 32) {
                const int k = k0 + lane;
                unsigned vis = 0;
                float range = 0.0f;
                if (k < K) {
                    if (!failed)
                        range = cast_one<MARCH>(A, BitsShared{sbits + M.all_off, M.pitch * 32}, M,
                                                o, sbeam[toff + k], e, k, true, vis);
                    else
                        range = cast_one<MARCH>(A, BitsGlobal{A.bits + M.word_off, M.pitch * 32},
                                                M, o, sbeam[toff + k], e, k, true, vis);
                }
                put_range(A, row, k, K, range, k < K);
                add_stats(A, vis, min(32, K - k0));
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const int done = atomicAdd(&A.split_q[2], 1);
        if (done == (int)gridDim.x - 1) {
            A.split_q[0] = 0;
            A.split_q[1] = 0;
            A.split_q[2] = 0;
            A.split_q[3] = 0;
            __threadfence();
        }
    }
}

template <bool DYN, bool MARCH, bool REFILL> const void *pick_kernel(int max_regs) {
    if (max_regs <= 32) return (const void *)step_kernel<DYN, 4, MARCH, REFILL>;
    if (max_regs <= 40) return (const void *)step_kernel<DYN, 3, MARCH, REFILL>;
    return (const void *)step_kernel<DYN, 2, MARCH, REFILL>;
}

} // namespace

// (kernel, device, shared bytes, block) -> (SMs, resident CTAs per SM): the
// attribute call and the occupancy query cost microseconds of host time, which
// matters when a step is split into several launches
struct OccKey {
    const void *fn;
    int dev;
    size_t smem;
    int block;
};
struct OccVal {
    int n_sm, per_sm;
};

int occupancy(const void *fn, size_t smem, int block, int &n_sm, int &per_sm) {
    static std::mutex mu;
    static std::vector<std::pair<OccKey, OccVal>> cache;
    // the dynamic shared-memory limit only ever rises, so that a cached
    // launch never meets a limit lowered by another shape's launch
    static std::vector<std::pair<std::pair<const void *, int>, size_t>> limit;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return (int)err;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &kv : cache)
        if (kv.first.fn == fn && kv.first.dev == dev && kv.first.smem == smem &&
            kv.first.block == block) {
            n_sm = kv.second.n_sm;
            per_sm = kv.second.per_sm;
            return 0;
        }
    size_t *lim = nullptr;
    for (auto &kv : limit)
        if (kv.first.first == fn && kv.first.second == dev) lim = &kv.second;
    if (!lim) {
        limit.push_back({{fn, dev}, 0});
        lim = &limit.back().second;
    }
    if (smem > *lim) {
        err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return (int)err;
        *lim = smem;
    }
    err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
    if (err != cudaSuccess) return (int)err;
    cache.push_back({OccKey{fn, dev, smem, block}, OccVal{n_sm, per_sm}});
    return 0;
}

// The tiled step kernel launch_step runs for (a, cfg), and its dynamic
// shared memory.
const void *step_fn(const StepArgs &a, const LaunchCfg &cfg, size_t &smem) {
    const bool dyn = a.p.n_dyn > 0;
    smem = (size_t)a.smem_region_bytes + (size_t)a.max_k * sizeof(float2) +
           (dyn ? (size_t)2 * a.max_tile_envs * sizeof(DynEnv) : 0);
    const bool march = a.p.sensor == 1;
    // lane refill applies to the exact traversal without moving discs
    return dyn ? (march ? pick_kernel<true, true, false>(cfg.max_regs)
                        : pick_kernel<true, false, false>(cfg.max_regs))
               : (march ? pick_kernel<false, true, false>(cfg.max_regs)
                        : cfg.refill ? pick_kernel<false, false, true>(cfg.max_regs)
                                     : pick_kernel<false, false, false>(cfg.max_regs));
}

int step_resident(const StepArgs &a, const LaunchCfg &cfg) {
    size_t smem = 0;
    const void *fn = step_fn(a, cfg, smem);
    int n_sm = 0, per_sm = 0;
    if (occupancy(fn, smem, cfg.block_threads, n_sm, per_sm) != 0) return 0;
    return n_sm * per_sm;
}

int launch_step(const StepArgs &a, const LaunchCfg &cfg, void *stream) {
    if (a.n_tiles <= 0) return 0;
    size_t smem = 0;
    const void *fn = step_fn(a, cfg, smem);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int n_sm = 0, per_sm = 0;
    cudaError_t err = (cudaError_t)occupancy(fn, smem, cfg.block_threads, n_sm, per_sm);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    int grid = std::min(a.n_tiles, n_sm * per_sm);
    if (cfg.max_ctas > 0) grid = std::min(grid, cfg.max_ctas);
    void *args[] = {const_cast<StepArgs *>(&a)};
    err = cudaLaunchKernel(fn, dim3(grid), dim3(cfg.block_threads), args, smem, s);
    if (err != cudaSuccess) return (int)err;
    return (int)cudaGetLastError();
}

int launch_step_split(const StepArgs &a, int n_envs, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    env_kernel<<<(n_envs + 127) / 128, 128, 0, s>>>(a, n_envs);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return (int)err;
    const size_t smem = (size_t)a.all_words * 4 + (size_t)a.n_beams_total * sizeof(float2);
    const void *fn = a.p.sensor == 1 ? (const void *)ray_kernel<true> : (const void *)ray_kernel<false>;
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    int dev = 0, n_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return (int)err;
    void *args[] = {const_cast<StepArgs *>(&a)};
    err = cudaLaunchKernel(fn, dim3(n_sm), dim3(1024), args, smem, s);
    if (err != cudaSuccess) return (int)err;
    return (int)cudaGetLastError();
}

size_t act_step_smem(const StepArgs &a) {
    return 1024 + (size_t)a.smem_region_bytes + (size_t)kActKChunks * kActChunk +
           (size_t)a.max_k * sizeof(float2);
}

int launch_act_step(const StepArgs &a, const ActArgs &p, void *stream) {
    if (a.n_tiles <= 0) return 0;
    const size_t smem = act_step_smem(a);
    const void *fn = (const void *)act_step_kernel;
    int n_sm = 0, per_sm = 0;
    cudaError_t err = (cudaError_t)occupancy(fn, smem, kActThreads, n_sm, per_sm);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    const int grid = std::min(a.n_tiles, n_sm);
    void *args[] = {const_cast<StepArgs *>(&a), const_cast<ActArgs *>(&p)};
    err = cudaLaunchKernel(fn, dim3(grid), dim3(kActThreads), args, smem,
                           static_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return (int)err;
    return (int)cudaGetLastError();
}

int act_units(const ActArgs &p) {
    int n = 0;
    for (int l = 0; l < 3; ++l) n += ((p.in[l] + 63) >> 6) * (p.out[l] > 128 ? 2 : 1);
    return n;
}

int launch_act_swizzle(const ActArgs &p, unsigned char *dst, void *stream) {
    const int n = act_units(p);
    act_swizzle_kernel<<<(n * 1024 + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(p, dst,
                                                                                          n);
    return (int)cudaGetLastError();
}

int launch_prep_all(const StepArgs &a, int n_envs, void *stream) {
    prep_all_kernel<<<(n_envs + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a, n_envs);
    return (int)cudaGetLastError();
}

int launch_uniform_actions(float *out, int n_envs, unsigned long long seed, unsigned step,
                           void *stream) {
    const int bs = 256;
    uniform_actions_kernel<<<(n_envs + bs - 1) / bs, bs, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<float2 *>(out), n_envs, seed, step);
    return (int)cudaGetLastError();
}

} // namespace flashnav
