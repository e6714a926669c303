// Device code shared by the step kernels (nav_step.cu, nav_flow.cu): scalar
// geometry and RNG, map views, grid traversal and march, footprints, the
// env phase (Sec. 2.2.3) and the bulk-copy staging helpers.
//
// Both translation units are compiled with FMA contraction off
// (-fmad=false) and IEEE division and square root, so every binary32
// operation here rounds once and the results are a fixed function of the
// inputs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "nav_internal.h"

namespace flashnav {
namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Scalar building blocks
// ---------------------------------------------------------------------------

// sin and cos of a binary32 angle.  x = k (pi/2) + r with pi/2 split into
// three binary32 parts (Cody-Waite; the first two have 12 significant bits so
// k times them is exact for small k), then the Taylor series of sin through
// r^11 and of cos through r^12 on |r| <= pi/4, Horner form, coefficients
// (-1)^n / n! rounded from binary64; the quadrant k mod 4 selects signs.
__device__ __forceinline__ void sincos_taylor(float x, float &s, float &c) {
    const float k = rintf(x * 0.636619772367581343076f);
    float r = x - k * 0x1.92p+0f;
    r = r - k * 0x1.fb4p-12f;
    r = r - k * 0x1.4442d2p-24f;
    const float r2 = r * r;
    float p = (float)(-1.0 / 39916800.0);
    p = p * r2 + (float)(1.0 / 362880.0);
    p = p * r2 + (float)(-1.0 / 5040.0);
    p = p * r2 + (float)(1.0 / 120.0);
    p = p * r2 + (float)(-1.0 / 6.0);
    const float sr = r + (r * r2) * p;
    float q = (float)(1.0 / 479001600.0);
    q = q * r2 + (float)(-1.0 / 3628800.0);
    q = q * r2 + (float)(1.0 / 40320.0);
    q = q * r2 + (float)(-1.0 / 720.0);
    q = q * r2 + (float)(1.0 / 24.0);
    q = q * r2 + (float)(-1.0 / 2.0);
    const float cr = 1.0f + r2 * q;
    switch (((int)k) & 3) {
    case 0: s = sr; c = cr; break;
    case 1: s = cr; c = -sr; break;
    case 2: s = -sr; c = -cr; break;
    default: s = -cr; c = sr; break;
    }
}

__device__ __forceinline__ float wrap_angle(float a) {
    if (a >= kPi) return a - kTwoPi;
    if (a < -kPi) return a + kTwoPi;
    return a;
}

// Counter-based RNG: SplitMix64's finaliser applied to the key
// seed ^ env*G ^ episode*P2 ^ draw*P3 (G the golden gamma, P2/P3 odd 64-bit
// multipliers), so a reset draw depends only on (seed, env, episode, draw).
__device__ __forceinline__ unsigned long long draw64(unsigned long long seed, unsigned env,
                                                     unsigned episode, unsigned k) {
    unsigned long long z = seed ^ ((unsigned long long)env * 0x9E3779B97F4A7C15ull) ^
                           ((unsigned long long)episode * 0xC2B2AE3D27D4EB4Full) ^
                           ((unsigned long long)k * 0x165667B19E3779F9ull);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// index in [0, n) from the high word (multiply-shift)
__device__ __forceinline__ int draw_index(unsigned long long h, int n) {
    return (int)__umulhi((unsigned)(h >> 32), (unsigned)n);
}

// [0, 1) from 24 bits
__device__ __forceinline__ float draw_unit(unsigned bits24) {
    return (float)bits24 * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// Map views.  Each view indexes the padded map (kPad blocked cells around the
// W x H map) linearly: idx(i, j) = (j + kPad) * stride + (i + kPad), so a
// step in x is +-1 and a step in y is +-stride.
//   BitsShared  packed free bits staged in shared memory (bulk TMA copy)
//   BitsGlobal  packed free bits read through L1/L2
//   BytesShared distance bytes staged in shared memory (bulk TMA copy): a
//               lookup is one byte load, and the value lets a ray jump
//               through the free square around the cell
//   BytesGlobal distance bytes read through L1/L2
// ---------------------------------------------------------------------------
struct BitsShared {
    const uint32_t *w;
    int stride; // pitch * 32
    __device__ __forceinline__ bool free_at(int b) const {
        return (__funnelshift_r(w[b >> 5], 0u, (unsigned)b) & 1u) != 0u;
    }
    __device__ __forceinline__ uint32_t word(int i) const { return w[i]; }
};
struct BitsGlobal {
    const uint32_t *__restrict__ w;
    int stride;
    __device__ __forceinline__ bool free_at(int b) const {
        return (__funnelshift_r(__ldg(w + (b >> 5)), 0u, (unsigned)b) & 1u) != 0u;
    }
    __device__ __forceinline__ uint32_t word(int i) const { return __ldg(w + i); }
};
// One byte per cell: 0 = blocked, else the chessboard distance (cells,
// capped at 255) to the nearest blocked or off-map cell.
struct BytesShared {
    static constexpr bool kDist = true;
    const uint8_t *c;
    int stride; // byte pitch
    __device__ __forceinline__ bool free_at(int b) const { return c[b] != 0; }
    __device__ __forceinline__ int dist_at(int b) const { return c[b]; }
};

// Distance bytes read through L1/L2 (maps too large to stage).
struct BytesGlobal {
    static constexpr bool kDist = true;
    const uint8_t *__restrict__ c;
    int stride; // byte pitch
    __device__ __forceinline__ bool free_at(int b) const { return __ldg(c + b) != 0; }
    __device__ __forceinline__ int dist_at(int b) const { return __ldg(c + b); }
};

template <class V> __device__ __forceinline__ int cell_index(const V &v, int i, int j) {
    return (j + kPad) * v.stride + (i + kPad);
}

// Is any cell of row j, columns [i0, i1] (all inside the map), blocked?
template <class V>
__device__ __forceinline__ bool span_blocked(const V &v, int j, int i0, int i1) {
    const int c0 = cell_index(v, i0, j), c1 = c0 + (i1 - i0);
    const int w0 = c0 >> 5, w1 = c1 >> 5;
    for (int wd = w0; wd <= w1; ++wd) {
        uint32_t m = kFull;
        if (wd == w0) m &= kFull << (c0 & 31);
        if (wd == w1) m &= kFull >> (31 - (c1 & 31));
        if (~v.word(wd) & m) return true;
    }
    return false;
}
// With distance bytes: a cell at distance d has every cell within d - 1
// columns of it free, so the span's middle cell is read first (d beyond the
// half-span clears the whole span with one lookup), and otherwise the scan
// steps d cells at a time from the span's first cell; both give the answer
// of the cell-by-cell test.
template <class V> __device__ __forceinline__ bool dist_span_blocked(const V &v, int c0, int n) {
    const int h = n >> 1;
    const int dm = v.dist_at(c0 + h);
    if (dm == 0) return true;
    if (dm > n - h) return false;
    for (int k = 0; k <= n;) {
        const int d = v.dist_at(c0 + k);
        if (d == 0) return true;
        k += d;
    }
    return false;
}
template <>
__device__ __forceinline__ bool span_blocked<BytesShared>(const BytesShared &v, int j, int i0,
                                                          int i1) {
    return dist_span_blocked(v, cell_index(v, i0, j), i1 - i0);
}
template <>
__device__ __forceinline__ bool span_blocked<BytesGlobal>(const BytesGlobal &v, int j, int i0,
                                                          int i1) {
    return dist_span_blocked(v, cell_index(v, i0, j), i1 - i0);
}

// Is any cell of row j, columns [i0, i1], blocked (occupied or off-map)?
template <class V>
__device__ bool row_blocked(const V &v, const MapDev &M, int j, int i0, int i1) {
    if (i0 > i1) return false;
    if (j < 0 || j >= M.h || i0 < 0 || i1 >= M.w) return true;
    return span_blocked(v, j, i0, i1);
}

// Cells of row j whose closed square meets the open disc (centre xc, yc,
// radius rc, cell units): [i0, i1]; false if the row's slab is out of reach.
__device__ __forceinline__ bool disc_row(float xc, float yc, float rc, int j, int &i0, int &i1) {
    const float fj = (float)j;
    float dy = 0.0f;
    if (yc < fj) dy = fj - yc;
    else if (yc > fj + 1.0f) dy = yc - (fj + 1.0f);
    if (!(dy < rc)) return false;
    const float hh = sqrtf(rc * rc - dy * dy);
    i0 = (int)floorf(xc - hh);
    i1 = (int)ceilf(xc + hh) - 1;
    return true;
}

// ---------------------------------------------------------------------------
// Moving-disc layer (per env, per step): stamped row spans in shared memory
// ---------------------------------------------------------------------------
struct DynEnv {
    short j0[kMaxDyn], nr[kMaxDyn], bi0[kMaxDyn], bi1[kMaxDyn];
    short lo[kMaxDyn][kMaxDynRows], hi[kMaxDyn][kMaxDynRows];
    int n; // stamps kept (those within reach of the robot), entries [0, n)
};

// Stamps the nd discs (cells whose closed square meets the open disc, per
// row) and keeps, in order, those whose stamp comes within `reach` cells of
// the robot at (xc, yc): rays (t <= r_max) and the footprint only enter
// cells that close to it, so the others cannot change any result.
__device__ void stamp_discs(const float4 *ob, int nd, float inv_res, float rdc, float xc, float yc,
                            float reach, DynEnv &de) {
    int k = 0;
    for (int q = 0; q < nd; ++q) {
        const float oxc = ob[q].x * inv_res, oyc = ob[q].y * inv_res;
        const int j0 = (int)floorf(oyc - rdc);
        const int j1 = (int)ceilf(oyc + rdc) - 1;
        int nr = j1 - j0 + 1;
        if (nr > kMaxDynRows) nr = kMaxDynRows; // bounded by the create-time check
        int bmin = 1 << 30, bmax = -(1 << 30);
        for (int r = 0; r < nr; ++r) {
            int a, b;
            if (!disc_row(oxc, oyc, rdc, j0 + r, a, b)) { a = 1; b = 0; }
            de.lo[k][r] = (short)a;
            de.hi[k][r] = (short)b;
            if (a <= b) { bmin = min(bmin, a); bmax = max(bmax, b); }
        }
        if (bmin > bmax) continue; // the disc covers no cell
        const float gx = fmaxf(0.0f, fmaxf((float)bmin - xc, xc - (float)(bmax + 1)));
        const float gy = fmaxf(0.0f, fmaxf((float)j0 - yc, yc - (float)(j0 + nr)));
        if (gx * gx + gy * gy > reach * reach) continue;
        de.j0[k] = (short)j0;
        de.nr[k] = (short)nr;
        de.bi0[k] = (short)bmin;
        de.bi1[k] = (short)bmax;
        ++k;
    }
    de.n = k;
}

__device__ __forceinline__ bool dyn_cell(const DynEnv &de, int i, int j) {
    for (int q = 0; q < de.n; ++q) {
        const int r = j - de.j0[q];
        if ((unsigned)r < (unsigned)de.nr[q] && i >= de.lo[q][r] && i <= de.hi[q][r]) return true;
    }
    return false;
}

__device__ __forceinline__ bool dyn_row(const DynEnv &de, int j, int i0, int i1) {
    if (i0 > i1) return false;
    for (int q = 0; q < de.n; ++q) {
        const int r = j - de.j0[q];
        if ((unsigned)r < (unsigned)de.nr[q] && max(i0, (int)de.lo[q][r]) <= min(i1, (int)de.hi[q][r]))
            return true;
    }
    return false;
}

// Parameter interval along the ray in which it can enter a stamped cell: the
// union of its crossings of every stamp's bounding box grown by one cell
// (the margin also covers the rounding of the crossings, computed with the
// reciprocals rdx = 1 / dx, rdy = 1 / dy).  Outside it the per-cell disc test
// is skipped (it could not succeed).
__device__ void dyn_gate(const DynEnv &de, float xc, float yc, float dx, float dy, float &glo,
                         float &ghi) {
    glo = INFINITY;
    ghi = -INFINITY;
    const float rdx = dx != 0.0f ? __frcp_rn(dx) : 0.0f, rdy = dy != 0.0f ? __frcp_rn(dy) : 0.0f;
    for (int q = 0; q < de.n; ++q) {
        const float x0 = (float)(de.bi0[q] - 1), x1 = (float)(de.bi1[q] + 2);
        const float y0 = (float)(de.j0[q] - 1), y1 = (float)(de.j0[q] + de.nr[q] + 1);
        float ta = 0.0f, tb = INFINITY;
        if (dx != 0.0f) {
            const float u = (x0 - xc) * rdx, v = (x1 - xc) * rdx;
            ta = fmaxf(ta, fminf(u, v));
            tb = fminf(tb, fmaxf(u, v));
        } else if (xc < x0 || xc > x1) {
            continue;
        }
        if (dy != 0.0f) {
            const float u = (y0 - yc) * rdy, v = (y1 - yc) * rdy;
            ta = fmaxf(ta, fminf(u, v));
            tb = fminf(tb, fmaxf(u, v));
        } else if (yc < y0 || yc > y1) {
            continue;
        }
        if (ta <= tb) {
            glo = fminf(glo, ta);
            ghi = fmaxf(ghi, tb);
        }
    }
}

// ---------------------------------------------------------------------------
// Ray cast: Amanatides-Woo traversal over a padded map view (Eq. 4-5).
// Starting cell (floor xc, floor yc); per step the axis whose next boundary
// is nearer is stepped (a tie steps x first), the entry parameter t of the
// new cell is checked against r_max, then the cell is looked up.  After k
// steps on an axis its next boundary lies at t0 + k tDelta, evaluated as one
// fused multiply-add.  Leaving the map stops the walk at a padding cell
// without a bounds test.  The walk ends within 2 r_max/res + 3 steps: each
// step raises tMaxX or tMaxY by tDelta >= 1.
//
// Views that carry a distance (one byte per cell: the chessboard distance
// to the nearest blocked cell) also jump: from a cell at distance d the
// next n = d - 1 columns (rows, for a ray closer to the y axis) of the ray
// are free, so every event up to the n-th major-axis boundary is taken at
// once.  The minor-axis count at that parameter is estimated, and the jump
// is kept only if exact comparisons of the same fused multiply-adds confirm
// the count and it stays within the free square (minor advance <= n);
// otherwise the iteration takes one ordinary step.  Either way the state
// afterwards is one the plain walk passes through: same cell, same boundary
// parameters, same visit count.  Jump and step are one branch-free
// iteration, so the lanes of a warp do not diverge between them.
// Returns the range in metres; hit = j*W+i, -1 off-map, -2 r_max.
// ---------------------------------------------------------------------------
template <class V, class = void> struct has_dist { static constexpr bool value = false; };
template <class V>
struct has_dist<V, decltype((void)V::kDist)> { static constexpr bool value = V::kDist; };

template <bool DYN, class V>
__device__ __forceinline__ float cast_ray(const V &view, const MapDev &M, float xc, float yc,
                                          float dx, float dy, float rmax_c, float max_range,
                                          const DynEnv *de, int &hit, unsigned &vis) {
    const int pb = view.stride;
    if (!(xc >= 0.0f && yc >= 0.0f)) { hit = -1; vis = 1; return 0.0f; }
    const float fx = floorf(xc), fy = floorf(yc);
    const int i0 = (int)fx, j0 = (int)fy;
    if (i0 >= M.w || j0 >= M.h) { hit = -1; vis = 1; return 0.0f; }
    int b = cell_index(view, i0, j0);
    if (!view.free_at(b) || (DYN && dyn_cell(*de, i0, j0))) {
        hit = j0 * M.w + i0;
        vis = 1;
        return 0.0f;
    }
    // per axis: cell-index step, tDelta and the first boundary parameter t0
    // (tDelta 0 and t0 = inf on an axis the ray does not move along);
    // __frcp_rn is the correctly rounded reciprocal, the value of 1 / d
    // without the general division's code
    int sbx = 0, sby = 0;
    float tdx = 0.0f, tdy = 0.0f, tx0 = INFINITY, ty0 = INFINITY;
    if (dx > 0.0f) { sbx = 1; tdx = __frcp_rn(dx); tx0 = ((fx + 1.0f) - xc) * tdx; }
    else if (dx < 0.0f) { sbx = -1; tdx = __frcp_rn(-dx); tx0 = (xc - fx) * tdx; }
    if (dy > 0.0f) { sby = pb; tdy = __frcp_rn(dy); ty0 = ((fy + 1.0f) - yc) * tdy; }
    else if (dy < 0.0f) { sby = -pb; tdy = __frcp_rn(-dy); ty0 = (yc - fy) * tdy; }
    float glo = INFINITY, ghi = -INFINITY;
    if (DYN) dyn_gate(*de, xc, yc, dx, dy, glo, ghi);
    float t = 0.0f, kx, ky;
    bool stopped = false;
    if constexpr (has_dist<V>::value) {
        // major axis M (the larger direction component), minor axis m
        const bool xmaj = fabsf(dx) >= fabsf(dy);
        const float tdM = xmaj ? tdx : tdy, tM0 = xmaj ? tx0 : ty0;
        const float tdm = xmaj ? tdy : tdx, tm0 = xmaj ? ty0 : tx0;
        const int sbM = xmaj ? sbx : sby, sbm = xmaj ? sby : sbx;
        const float adM = xmaj ? fabsf(dx) : fabsf(dy), adm = xmaj ? fabsf(dy) : fabsf(dx);
        // on a tie the x step comes first: the major axis wins ties iff it is x
        const int tie = xmaj ? 1 : 0;
        // minor boundaries at or before T: about T |d_m| + 1 - t0_m |d_m|
        const float offm = adm > 0.0f ? 1.0f - tm0 * adm : 0.0f;
        // about the number of major-axis events at or before r_max (a jump
        // past r_max is refused by an exact test)
        const float nM = floorf(__fmaf_rn(rmax_c, adM, 1.0f - tM0 * adM));
        float kM = 0.0f, km = 0.0f, tM = tM0, tm = tm0;
        int d = view.dist_at(b);
        const int b0 = b;
        for (;;) {
            // the next event (tie: x first; parameters are >= 0, so their
            // bit patterns order like the floats)
            const bool sM = __float_as_int(tM) < __float_as_int(tm) + tie;
            const float tn = sM ? tM : tm;
            if (tn > rmax_c) break;
            // jump candidate: every event up to the n-th next major event,
            // n = d - 1 (capped at r_max); the minor count at that parameter
            // is estimated and kept only if the comparisons confirm it
            const float n = fminf((float)d - 1.0f, nM - kM);
            const float kM2 = kM + n;
            const float T = __fmaf_rn(kM2 - 1.0f, tdM, tM0);
            const float km2 = fmaxf(km, floorf(__fmaf_rn(T, adm, offm)));
            bool jump = n >= 1.0f && T <= rmax_c && km2 - km <= n &&
                        __fmaf_rn(km2, tdm, tm0) > T &&
                        (km2 == km || __fmaf_rn(km2 - 1.0f, tdm, tm0) <= T);
            if (DYN) jump = jump && (T < glo || tn > ghi);
            kM = jump ? kM2 : (sM ? kM + 1.0f : kM);
            km = jump ? km2 : (sM ? km : km + 1.0f);
            tM = __fmaf_rn(kM, tdM, tM0);
            tm = __fmaf_rn(km, tdm, tm0);
            b = b0 + (int)kM * sbM + (int)km * sbm;
            t = tn;
            d = view.dist_at(b);
            if (d == 0) { stopped = true; break; } // only a single step reaches a blocked cell
            if (DYN && !jump && t >= glo && t <= ghi) {
                const float ax = xmaj ? kM : km, ay = xmaj ? km : kM;
                const int ci = i0 + (sbx < 0 ? -(int)ax : (int)ax);
                const int cj = j0 + (sby < 0 ? -(int)ay : (int)ay);
                if (dyn_cell(*de, ci, cj)) { stopped = true; break; }
            }
        }
        kx = xmaj ? kM : km;
        ky = xmaj ? km : kM;
    } else {
        float tmx = tx0, tmy = ty0;
        kx = 0.0f;
        ky = 0.0f;
        for (;;) {
            const bool sx = tmx <= tmy;
            t = sx ? tmx : tmy;
            if (t > rmax_c) break;
            b += sx ? sbx : sby;
            if (sx) { kx += 1.0f; tmx = __fmaf_rn(kx, tdx, tx0); }
            else { ky += 1.0f; tmy = __fmaf_rn(ky, tdy, ty0); }
            if (!view.free_at(b)) { stopped = true; break; }
            if (DYN && t >= glo && t <= ghi) {
                const int ci = i0 + (sbx < 0 ? -(int)kx : (int)kx);
                const int cj = j0 + (sby < 0 ? -(int)ky : (int)ky);
                if (dyn_cell(*de, ci, cj)) { stopped = true; break; }
            }
        }
    }
    const int i = i0 + (sbx < 0 ? -(int)kx : (int)kx);
    const int j = j0 + (sby < 0 ? -(int)ky : (int)ky);
    vis = 1u + (unsigned)kx + (unsigned)ky;
    if (!stopped) { hit = -2; return max_range; }
    hit = (i < 0 || j < 0 || i >= M.w || j >= M.h) ? -1 : j * M.w + i;
    return t * M.res;
}

// ---------------------------------------------------------------------------
// Fixed-step march (Sec. 2.2.2): the ray of Eq. 4 is sampled at
// tau_s = s * step_c cells (s = 0, 1, ...); the first sample whose cell is
// blocked or off the map ends the ray at range tau_s, and a ray whose next
// sample lies beyond r_max returns r_max.  Every sample is one visit.  The
// off-map test is explicit, so any step length is valid.  Same outputs as
// cast_ray: range in metres, hit = j*W+i, -1 off-map, -2 r_max.
// With a distance view, a sample in a cell at chessboard distance d is
// followed by q samples that stay within d - 1 - 1/16 cells of it along
// both axes (q step_c max(|dx|, |dy|) <= d - 1 - 1/16; the 1/16 cell covers
// the rounding of the sample positions), hence in free cells, and the march
// resumes after them; jumps stop at the first sample past r_max.
// ---------------------------------------------------------------------------
template <bool DYN, class V>
__device__ __forceinline__ float march_ray(const V &view, const MapDev &M, float xc, float yc,
                                           float dx, float dy, float step_c, float rmax_c,
                                           float max_range, const DynEnv *de, int &hit,
                                           unsigned &vis) {
    if (!(xc >= 0.0f && yc >= 0.0f)) { hit = -1; vis = 1; return 0.0f; }
    int i = (int)floorf(xc), j = (int)floorf(yc);
    if (i >= M.w || j >= M.h) { hit = -1; vis = 1; return 0.0f; }
    int b0 = cell_index(view, i, j);
    if (!view.free_at(b0) || (DYN && dyn_cell(*de, i, j))) {
        hit = j * M.w + i;
        vis = 1;
        return 0.0f;
    }
    float glo = INFINITY, ghi = -INFINITY;
    if (DYN) dyn_gate(*de, xc, yc, dx, dy, glo, ghi);
    if constexpr (has_dist<V>::value) {
        // s_end: the first sample past r_max
        float s_end = fmaxf(1.0f, floorf(rmax_c / step_c));
        while (s_end > 1.0f && (s_end - 1.0f) * step_c > rmax_c) s_end -= 1.0f;
        while (s_end * step_c <= rmax_c) s_end += 1.0f;
        const float per = __frcp_rn(step_c * fmaxf(fabsf(dx), fabsf(dy)));
        float s = 0.0f;
        int d = view.dist_at(b0);
        for (;;) {
            float q = floorf(((float)d - 1.0625f) * per);
            q = fmaxf(q, 0.0f);
            if (DYN && q > 0.0f && !((s + q) * step_c < glo || (s + 1.0f) * step_c > ghi)) q = 0.0f;
            s = fminf(s + q + 1.0f, s_end);
            const float tc = s * step_c;
            if (tc > rmax_c) { hit = -2; vis = (unsigned)s; return max_range; }
            const float px = xc + tc * dx, py = yc + tc * dy;
            i = (int)floorf(px);
            j = (int)floorf(py);
            if ((unsigned)i >= (unsigned)M.w || (unsigned)j >= (unsigned)M.h) {
                hit = -1;
                vis = (unsigned)s + 1u;
                return tc * M.res;
            }
            d = view.dist_at(cell_index(view, i, j));
            if (d == 0 || (DYN && tc >= glo && tc <= ghi && dyn_cell(*de, i, j))) {
                hit = j * M.w + i;
                vis = (unsigned)s + 1u;
                return tc * M.res;
            }
        }
    } else {
        for (unsigned s = 1;; ++s) {
            const float tc = (float)s * step_c;
            if (tc > rmax_c) { hit = -2; vis = s; return max_range; }
            const float px = xc + tc * dx, py = yc + tc * dy;
            i = (int)floorf(px);
            j = (int)floorf(py);
            if ((unsigned)i >= (unsigned)M.w || (unsigned)j >= (unsigned)M.h) {
                hit = -1;
                vis = s + 1u;
                return tc * M.res;
            }
            if (!view.free_at(cell_index(view, i, j)) ||
                (DYN && tc >= glo && tc <= ghi && dyn_cell(*de, i, j))) {
                hit = j * M.w + i;
                vis = s + 1u;
                return tc * M.res;
            }
        }
    }
}

// Writes beam k's clipped range into its observation row, or, with sectors
// (Eq. 6), folds it into the minimum of sector k / (K / m) by an atomic min
// on the float's bits (ranges are >= 0, so integer order is float order).
// Warp-collective: every lane of the warp calls it, `active` or not.  The
// lanes of one sector are contiguous in a warp, so a segmented min over the
// shuffle tree leaves each sector's minimum in its first lane, which alone
// issues the atomic.  The sector slots hold r_max before the scan.
__device__ __forceinline__ void put_range(const StepArgs &A, float *row, int k, int K,
                                          float range, bool active) {
    const float c = fminf(range, A.max_range);
    const int m = A.p.n_sectors;
    if (m == 0) {
        if (active) row[k] = c;
        return;
    }
    const int lane = threadIdx.x & 31;
    unsigned long long key = active ? (unsigned long long)(row + k / (K / m)) : 0ull;
    int v = active ? __float_as_int(c) : 0x7fffffff;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ov = __shfl_down_sync(kFull, v, o);
        const unsigned long long ok = __shfl_down_sync(kFull, key, o);
        if (lane + o < 32 && ok == key) v = min(v, ov);
    }
    const unsigned long long pk = __shfl_up_sync(kFull, key, 1);
    if (active && (lane == 0 || pk != key)) atomicMin(reinterpret_cast<int *>(key), v);
}

// ---------------------------------------------------------------------------
// Footprints (Sec. 2.2.3 collision check; Tables 8-9 presets)
// ---------------------------------------------------------------------------
// WARP: the 32 lanes of a warp call it together for one env (same
// arguments) and test its rows in parallel, lane l the rows j0 + l, j0 + l
// + 32, ...; the answer (any row blocked) is the same.
template <bool DYN, bool WARP = false, class B>
__device__ bool disc_blocked(const B &bits, const MapDev &M, float xc, float yc, float rc,
                             const DynEnv *de, bool static_clear = false) {
    const int j0 = (int)floorf(yc - rc);
    const int j1 = (int)ceilf(yc + rc) - 1;
    bool hit = false;
    for (int j = j0 + (WARP ? (int)(threadIdx.x & 31) : 0); j <= j1 && !hit; j += WARP ? 32 : 1) {
        int a, b;
        if (!disc_row(xc, yc, rc, j, a, b)) continue;
        if (!static_clear && row_blocked(bits, M, j, a, b)) hit = true;
        else if (DYN && dyn_row(*de, j, a, b)) hit = true;
    }
    return WARP ? __any_sync(kFull, hit) : hit;
}

// Open rectangle (half-length hl along the heading (ct, st), half-width hw,
// cell units) against closed cells: per row slab [j, j+1], the x-extent of
// the polygon within the slab is the hull of its vertices inside the slab
// and its edges' crossings of y = j and y = j + 1.
template <bool DYN, bool WARP = false, class B>
__device__ bool rect_blocked(const B &bits, const MapDev &M, float xc, float yc, float st,
                             float ct, float hl, float hw, const DynEnv *de,
                             bool static_clear = false) {
    const float ax = hl * ct, ay = hl * st;
    const float bx = -(hw * st), by = hw * ct;
    float px[4], py[4];
    px[0] = (xc + ax) + bx; py[0] = (yc + ay) + by;
    px[1] = (xc - ax) + bx; py[1] = (yc - ay) + by;
    px[2] = (xc - ax) - bx; py[2] = (yc - ay) - by;
    px[3] = (xc + ax) - bx; py[3] = (yc + ay) - by;
    float ymin = py[0], ymax = py[0];
#pragma unroll
    for (int v = 1; v < 4; ++v) {
        ymin = py[v] < ymin ? py[v] : ymin;
        ymax = py[v] > ymax ? py[v] : ymax;
    }
    const int j0 = (int)floorf(ymin);
    const int j1 = (int)ceilf(ymax) - 1;
    bool hit = false;
    for (int j = j0 + (WARP ? (int)(threadIdx.x & 31) : 0); j <= j1 && !hit; j += WARP ? 32 : 1) {
        const float lo = (float)j, hi = (float)j + 1.0f;
        float xlo = INFINITY, xhi = -INFINITY;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (py[v] >= lo && py[v] <= hi) {
                xlo = px[v] < xlo ? px[v] : xlo;
                xhi = px[v] > xhi ? px[v] : xhi;
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int u = (v + 1) & 3;
            const float ya = py[v], yb = py[u];
            if (ya == yb) continue;
            const float ylo = ya < yb ? ya : yb, yhi = ya < yb ? yb : ya;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float yl = s ? hi : lo;
                if (yl > ylo && yl < yhi) {
                    const float xx = px[v] + (yl - ya) * (px[u] - px[v]) / (yb - ya);
                    xlo = xx < xlo ? xx : xlo;
                    xhi = xx > xhi ? xx : xhi;
                }
            }
        }
        if (!(xlo <= xhi)) continue;
        const int a = (int)floorf(xlo), b = (int)ceilf(xhi) - 1;
        if (!static_clear && row_blocked(bits, M, j, a, b)) hit = true;
        else if (DYN && dyn_row(*de, j, a, b)) hit = true;
    }
    return WARP ? __any_sync(kFull, hit) : hit;
}

// ---------------------------------------------------------------------------
// Env phase
// ---------------------------------------------------------------------------
struct EnvSlot {
    float xc, yc, st, ct;     // pose of the scan written to obs
    float fxc, fyc, fst, fct; // pre-reset pose (final observation)
    long long obs_off, ray_off;
    int env;
    int fin;
    int prep;     // 1: the env started episode ep; its next-episode record is due
    unsigned ep;
};

// Origin of one scan for the refilled ray phase, set up once per env
// instead of once per ray: pose in cells, heading's sin and cos, floors of
// the position, the origin cell's view index (0, a padding cell, when off
// the map) and its distance byte (0: every ray stops at once), and the
// env's row offsets.
struct __align__(16) RayOrigin {
    float xc, yc, st, ct;
    float flx, fly;
    int b0, d0;
    long long obs_off, ray_off;
};

// cast_ray's set-up before its first step, for a scan from (xc, yc) cells.
template <class V>
__device__ __forceinline__ void set_origin(const V &view, const MapDev &M, float xc, float yc,
                                           float st, float ct, long long obs_off,
                                           long long ray_off, RayOrigin &o) {
    RayOrigin r;
    r.xc = xc;
    r.yc = yc;
    r.st = st;
    r.ct = ct;
    r.flx = r.fly = 0.0f;
    r.b0 = r.d0 = 0;
    r.obs_off = obs_off;
    r.ray_off = ray_off;
    if (xc >= 0.0f && yc >= 0.0f) {
        const float fx = floorf(xc), fy = floorf(yc);
        const int i0 = (int)fx, j0 = (int)fy;
        if (i0 < M.w && j0 < M.h) {
            r.b0 = cell_index(view, i0, j0);
            r.d0 = view.dist_at(r.b0);
            r.flx = fx;
            r.fly = fy;
        }
    }
    o = r;
}

template <class V>
__device__ __forceinline__ bool static_blocked(const V &v, const MapDev &M, int i, int j) {
    if (i < 0 || j < 0 || i >= M.w || j >= M.h) return true;
    return !v.free_at(cell_index(v, i, j));
}

// Sparse reset of env e for `episode` (Sec. 2.2.3): spawn cell uniform over
// the map's spawnable cells (draw 0), heading uniform (draw 1), goal from the
// spawn cell's component with distance in [dmin, dmax] (draws 2..65; after
// 64 misses the draw nearest the band, first on ties), moving discs from
// spawnable cells at least dyn_min_sep away (draws 1024 + 64 q + a, a < 16)
// with speed and heading from draw 1024 + 64 q + 48.
// Spawn pose and goal of env e for `episode` (draws 0..65).
__device__ void reset_pose(const StepArgs &A, const MapDev &M, int e, unsigned episode, float &x,
                           float &y, float &th, float &gx, float &gy, float &dprev) {
    const CsDev cs = A.cs[A.env_cs[e]];
    if (cs.n_spawn <= 0) {
        atomicOr(A.status, kStatusNoSpawn);
        x = y = th = gx = gy = dprev = 0.0f;
        return;
    }
    const unsigned long long h0 = draw64(A.seed, (unsigned)e, episode, 0);
    const int si = cs.spawn_off + draw_index(h0, cs.n_spawn);
    const int cell = A.spawn[si];
    const int comp = A.spawn_comp[si];
    x = ((float)(cell % M.w) + 0.5f) * M.res;
    y = ((float)(cell / M.w) + 0.5f) * M.res;
    th = draw_unit((unsigned)(draw64(A.seed, (unsigned)e, episode, 1) >> 40)) * kTwoPi - kPi;
    const int cstart = cs.cells_off + A.comp_start[cs.comp_off + comp];
    const int ccount = A.comp_count[cs.comp_off + comp];
    const float dmin = A.p.goal_dmin, dmax = A.p.goal_dmax;
    float bx = x, by = y, berr = INFINITY;
    // draws taken in batches of 8: the 8 cell loads are issued together, then
    // examined in draw order (same result as one draw at a time)
    bool found = false;
    for (int a0 = 0; a0 < 64 && !found; a0 += 8) {
        int gcs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const unsigned long long hg =
                draw64(A.seed, (unsigned)e, episode, 2u + (unsigned)(a0 + q));
            gcs[q] = __ldg(A.comp_cells + cstart + draw_index(hg, ccount));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (found) break;
            const int gc = gcs[q];
            const float cx = ((float)(gc % M.w) + 0.5f) * M.res;
            const float cy = ((float)(gc / M.w) + 0.5f) * M.res;
            const float ddx = cx - x, ddy = cy - y;
            const float d = sqrtf(ddx * ddx + ddy * ddy);
            const float err = d < dmin ? dmin - d : (d > dmax ? d - dmax : 0.0f);
            if (err < berr) { berr = err; bx = cx; by = cy; }
            if (err == 0.0f) found = true;
        }
    }
    gx = bx;
    gy = by;
    {
        const float ddx = bx - x, ddy = by - y;
        dprev = sqrtf(ddx * ddx + ddy * ddy);
    }
}

// Moving discs of env e for `episode`, spawned around the robot's spawn
// point (x, y) (draws 1024 + 64 q + a).
__device__ void reset_discs(const StepArgs &A, const MapDev &M, int e, unsigned episode, float x,
                            float y, float4 *ob) {
    const int nd = A.p.n_dyn;
    if (nd <= 0) return;
    const CsDev cs = A.cs[A.env_cs[e]];
    if (cs.n_spawn <= 0) {
        for (int q = 0; q < nd; ++q) ob[q] = make_float4(x, y, 0.0f, 0.0f);
        return;
    }
    for (int q = 0; q < nd; ++q) {
        float ox = x, oy = y;
        for (int a = 0; a < 16; ++a) {
            const unsigned long long hp =
                draw64(A.seed, (unsigned)e, episode, 1024u + 64u * (unsigned)q + (unsigned)a);
            const int oc = A.spawn[cs.spawn_off + draw_index(hp, cs.n_spawn)];
            ox = ((float)(oc % M.w) + 0.5f) * M.res;
            oy = ((float)(oc / M.w) + 0.5f) * M.res;
            const float ddx = ox - x, ddy = oy - y;
            if (sqrtf(ddx * ddx + ddy * ddy) >= A.p.dyn_min_sep) break;
        }
        const unsigned long long hv = draw64(A.seed, (unsigned)e, episode, 1024u + 64u * (unsigned)q + 48u);
        const float sp = draw_unit((unsigned)(hv >> 40)) * A.p.dyn_speed_max;
        const float hd = draw_unit((unsigned)((hv >> 8) & 0xFFFFFFull)) * kTwoPi - kPi;
        float sh, ch;
        sincos_taylor(hd, sh, ch);
        ob[q] = make_float4(ox, oy, sp * ch, sp * sh);
    }
}

template <class B>
__device__ void reset_env(const StepArgs &A, const B &, const MapDev &M, int e, unsigned episode,
                          float &x, float &y, float &th, float &gx, float &gy, float &dprev,
                          float4 *ob) {
    reset_pose(A, M, e, episode, x, y, th, gx, gy, dprev);
    reset_discs(A, M, e, episode, x, y, ob);
}

// The next-episode record of env e: spawn pose, goal and initial goal
// distance of episode ep + 1, a function of (seed, e, ep + 1) alone.  A step
// that ends an episode takes the env's record and has the record of the
// episode after it written here, off the path of the step's scan.
__device__ void prep_next(const StepArgs &A, const MapDev &M, int e, unsigned ep) {
    float x, y, th, gx, gy, dprev;
    reset_pose(A, M, e, ep + 1u, x, y, th, gx, gy, dprev);
    A.nxt_pose[e] = make_float4(x, y, th, dprev);
    A.nxt_goal[e] = make_float2(gx, gy);
}

// Observation tail (Eq. 1): goal distance, bearing in the body frame, v, w.
__device__ __forceinline__ void write_tail(float *row, float x, float y, float th, float gx,
                                           float gy, float v, float w) {
    const float ddx = gx - x, ddy = gy - y;
    row[0] = sqrtf(ddx * ddx + ddy * ddy);
    float phi = atan2f(ddy, ddx) - th;
    if (phi >= kPi) phi -= kTwoPi;
    else if (phi < -kPi) phi += kTwoPi;
    row[1] = phi;
    row[2] = v;
    row[3] = w;
}

// An env's inputs to a step (state, next-episode record, action, robot),
// loaded before the tile's map has landed so that their DRAM latency
// overlaps the staging.
struct EnvIn {
    float x, y, th, gx, gy, dprev;
    int step;
    unsigned episode;
    float4 np;
    float2 ng, act;
    RobotDev rb;
};

__device__ __forceinline__ EnvIn load_env(const StepArgs &A, int e) {
    EnvIn in;
    in.x = A.x[e]; in.y = A.y[e]; in.th = A.th[e];
    in.gx = A.gx[e]; in.gy = A.gy[e]; in.dprev = A.dprev[e];
    in.step = A.step[e];
    in.episode = A.episode[e];
    in.np = A.nxt_pose[e];
    in.ng = A.nxt_goal[e];
    in.act = reinterpret_cast<const float2 *>(A.actions)[e];
    in.rb = A.env_rb[e];
    return in;
}

// WARP: all 32 lanes of a warp run the same env (same values, so their
// stores agree) and test the footprint's rows in parallel.
template <bool DYN, bool WARP = false, class B>
__device__ void env_phase(const StepArgs &A, const B &bits, const MapDev &M, int K, int slot_id,
                          EnvSlot &slot, DynEnv *dmain, DynEnv *dfin, const EnvIn &in) {
    const int e = slot.env;
    const int nd = DYN ? A.p.n_dyn : 0;
    const int D = A.p.n_sectors > 0 ? A.p.n_sectors : K; // range features per row
    float4 ob[kMaxDyn];
    const float rdc = A.p.dyn_radius * M.inv_res;
    // stamps farther than this (cells) from the robot can meet neither a
    // ray (t <= r_max) nor the footprint, and are dropped
    float reach = 0.0f;
    if (DYN) {
        const RobotDev rb0 = A.robots[A.env_robot[e]];
        const float hl = 0.5f * rb0.length, hw = 0.5f * rb0.width;
        const float foot = rb0.shape == 0 ? rb0.radius : sqrtf(hl * hl + hw * hw);
        reach = (A.max_range + foot) * M.inv_res + 2.0f;
    }
    float x, y, th, v, w, gx, gy, dprev;
    int step;
    unsigned episode;
    bool restamp = true; // spans in dmain must describe the discs after this step
    slot.fin = 0;
    slot.prep = 0;
    if (A.mode == 1) {
        episode = 0;
        reset_env(A, bits, M, e, episode, x, y, th, gx, gy, dprev, ob);
        v = w = 0.0f;
        step = 0;
        slot.prep = 1;
        slot.ep = 0;
    } else {
        x = in.x; y = in.y; th = in.th;
        gx = in.gx; gy = in.gy; dprev = in.dprev;
        step = in.step;
        episode = in.episode;
        // the next episode's start, read with the state (used on a reset)
        const float4 np = in.np;
        const float2 ng = in.ng;
        if (DYN)
            for (int q = 0; q < nd; ++q) ob[q] = A.dyn[(size_t)e * nd + q];
        const RobotDev rb = in.rb;
        // a1: clamp and map the normalised action onto the preset's bounds
        const float2 act = in.act;
        const float a0 = fminf(fmaxf(act.x, -1.0f), 1.0f);
        const float a1 = fminf(fmaxf(act.y, -1.0f), 1.0f);
        v = rb.v_min + ((a0 + 1.0f) * 0.5f) * (rb.v_max - rb.v_min);
        w = rb.w_min + ((a1 + 1.0f) * 0.5f) * (rb.w_max - rb.w_min);
        // a2: exact arc over dt (chord length v dt sinc(w dt / 2) along the
        // mid-step heading), heading wrapped to [-pi, pi)
        const float dt = A.p.dt;
        const float hd = (w * dt) * 0.5f;
        float sc;
        if (fabsf(hd) < 0.1f) {
            const float h2 = hd * hd;
            float p = (float)(-1.0 / 5040.0);
            p = p * h2 + (float)(1.0 / 120.0);
            p = p * h2 + (float)(-1.0 / 6.0);
            sc = 1.0f + h2 * p;
        } else {
            float sh, ch;
            sincos_taylor(hd, sh, ch);
            sc = sh / hd;
        }
        float sm, cm;
        sincos_taylor(th + hd, sm, cm);
        const float chord = (v * dt) * sc;
        x = x + chord * cm;
        y = y + chord * sm;
        th = wrap_angle(th + w * dt);
        // a5: moving discs, constant velocity, reflect off blocked cells
        if (DYN) {
            for (int q = 0; q < nd; ++q) {
                float4 o = ob[q];
                const float nx = o.x + o.z * dt;
                if (static_blocked(bits, M, (int)floorf(nx * M.inv_res), (int)floorf(o.y * M.inv_res)))
                    o.z = -o.z;
                else
                    o.x = nx;
                const float ny = o.y + o.w * dt;
                if (static_blocked(bits, M, (int)floorf(o.x * M.inv_res), (int)floorf(ny * M.inv_res)))
                    o.w = -o.w;
                else
                    o.y = ny;
                ob[q] = o;
            }
            stamp_discs(ob, nd, M.inv_res, rdc, x * M.inv_res, y * M.inv_res, reach, *dmain);
            restamp = false;
        }
        // a6: footprint against the bitmap (and the moving-disc layer)
        const float xc = x * M.inv_res, yc = y * M.inv_res;
        float st, ct;
        sincos_taylor(th, st, ct);
        // With a distance view: the footprint lies within R cells of a point
        // of the centre's cell, so it can only meet cells fewer than R + 1
        // rows or columns away; when the centre cell's chessboard distance d
        // has d - 2 >= R (R rounded up a little), all of those are free in
        // the static map: its row scan is skipped (same result), and only
        // the moving discs' stamps (in shared memory) are tested.
        bool clear = false;
        if constexpr (has_dist<B>::value) {
            const float hl = (0.5f * rb.length) * M.inv_res, hw = (0.5f * rb.width) * M.inv_res;
            const float R = rb.shape == 0 ? rb.radius * M.inv_res : sqrtf(hl * hl + hw * hw);
            if (xc >= 0.0f && yc >= 0.0f && xc < (float)M.w && yc < (float)M.h) {
                const int d = bits.dist_at(cell_index(bits, (int)xc, (int)yc));
                clear = (float)(d - 2) >= R * 1.0001f + 0.001f;
            }
        }
        bool coll = false;
        if (clear && (!DYN || dmain->n == 0))
            coll = false;
        else if (rb.shape == 0)
            coll = disc_blocked<DYN, WARP>(bits, M, xc, yc, rb.radius * M.inv_res, dmain, clear);
        else
            coll = rect_blocked<DYN, WARP>(bits, M, xc, yc, st, ct, (0.5f * rb.length) * M.inv_res,
                                     (0.5f * rb.width) * M.inv_res, dmain, clear);
        // a7: goal test, reward, flags
        const float ddx = gx - x, ddy = gy - y;
        const float d = sqrtf(ddx * ddx + ddy * ddy);
        const bool goal = d <= A.p.goal_tol;
        float r;
        if (A.p.reward_mode == 0) {
            r = A.p.c_progress * (dprev - d);
            r = r - A.p.step_penalty;
            if (goal) r = r + A.p.r_goal;
            if (coll) r = r - A.p.r_coll;
        } else {
            r = goal ? A.p.r_goal : (coll ? -A.p.r_coll : A.p.c_progress * (dprev - d));
        }
        dprev = d;
        step += 1;
        const bool term = goal || coll;
        const bool trunc = !term && step >= A.p.horizon;
        A.reward[e] = r;
        A.done[e] = (unsigned char)((term ? 1 : 0) | (trunc ? 2 : 0) | (goal ? 4 : 0) | (coll ? 8 : 0));
        if (term || trunc) {
            // a9 (final): O_{t+1} before the reset, scanned in phase 2
            if (A.final_obs) {
                write_tail(A.final_obs + slot.obs_off + D, x, y, th, gx, gy, v, w);
                for (int q = 0; q < A.p.n_sectors; ++q) A.final_obs[slot.obs_off + q] = A.max_range;
                slot.fin = 1;
                slot.fxc = xc; slot.fyc = yc; slot.fst = st; slot.fct = ct;
                if (DYN) *dfin = *dmain;
            }
            // a8: sparse reset in place, from the next-episode record (the
            // record of the episode after it is written by prep_next)
            episode += 1;
            x = np.x; y = np.y; th = np.z; dprev = np.w;
            gx = ng.x; gy = ng.y;
            if (DYN) reset_discs(A, M, e, episode, x, y, ob);
            v = w = 0.0f;
            step = 0;
            restamp = true;
            slot.prep = 1;
            slot.ep = episode;
        }
    }
    A.x[e] = x; A.y[e] = y; A.th[e] = th; A.v[e] = v; A.w[e] = w;
    A.gx[e] = gx; A.gy[e] = gy; A.dprev[e] = dprev;
    A.step[e] = step;
    A.episode[e] = episode;
    if (DYN) {
        for (int q = 0; q < nd; ++q) A.dyn[(size_t)e * nd + q] = ob[q];
        if (restamp)
            stamp_discs(ob, nd, M.inv_res, rdc, x * M.inv_res, y * M.inv_res, reach, *dmain);
    }
    // a9: observation tail of the scan written to obs (sector minima start at r_max)
    write_tail(A.obs + slot.obs_off + D, x, y, th, gx, gy, v, w);
    for (int q = 0; q < A.p.n_sectors; ++q) A.obs[slot.obs_off + q] = A.max_range;
    float st, ct;
    sincos_taylor(th, st, ct);
    slot.xc = x * M.inv_res;
    slot.yc = y * M.inv_res;
    slot.st = st;
    slot.ct = ct;
}

// ---------------------------------------------------------------------------
// Staging of a map into shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void init_copy_barrier(unsigned long long *bar) {
    const unsigned b = smem_u32(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issued by one thread: one arrive that expects `bytes` bytes (a multiple of
// 16, both addresses 16-byte aligned), then the bulk copies (global ->
// shared, completion counted on the mbarrier).
__device__ __forceinline__ void stage_map(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    const unsigned b = smem_u32(bar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                 : "memory");
    const unsigned chunk = 32768u;
    for (unsigned off = 0; off < bytes; off += chunk) {
        const unsigned n = bytes - off < chunk ? bytes - off : chunk;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst) + off),
            "l"((const char *)src + off), "r"(n), "r"(b)
            : "memory");
    }
}

// Bounded wait for the copy whose completion completes mbarrier phase `parity`.
__device__ __forceinline__ bool wait_bitmap(unsigned long long *bar, unsigned parity) {
    const unsigned b = smem_u32(bar);
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}


} // namespace
} // namespace flashnav
