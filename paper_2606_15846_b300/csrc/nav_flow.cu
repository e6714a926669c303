// Pipelined simulator step for sm_103a (FlashNav Sec. 2.2, Eq. 7): the same
// step as step_kernel (action decode, arc, footprint, reward and flags,
// sparse reset, the scan of Eq. 4-5 and the observation of Eq. 1), organised
// so that no warp waits for another except when there is no work at all.
//
// One persistent CTA of 32 warps per SM.  Warp 0 is the producer: it claims
// a few envs at a time from a (map, beam table) group, stages the group's
// distance bytes into one of two shared-memory buffers by bulk copies
// (cp.async.bulk, completion on an mbarrier) while it runs the env phase of
// the claimed envs (one lane per env, map read through L1/L2), and publishes
// one scan record per observation scan (and per final-observation scan)
// into a ring in shared memory.  Warps 1-31 cast rays: every lane walks its
// own ray, and when enough lanes of a warp have finished, the warp writes
// their ranges and takes as many new rays as it has idle lanes from a shared
// (scan, beam) cursor advanced by compare-and-swap, so lanes do not idle
// until the slowest ray of a fixed 32-ray chunk ends.  Each CTA starts on a
// home group sized by the group's estimated ray cost; when its group is
// exhausted it takes envs of the group with the most left (restaging that
// map).  After its last claim the producer casts rays too.
//
// Every wait is bounded: on a timeout the kernel sets a status bit, stops
// taking work, finishes the rays it holds and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "nav_geom.cuh"
#include "nav_internal.h"

namespace flashnav {
namespace {

constexpr int kRing = 64;          // scan records in flight per CTA (power of two)
constexpr int kFlowThreads = 1024; // warp 0 produces, warps 1-31 cast rays
constexpr int kFlowWarps = kFlowThreads / 32;
constexpr int kRefill = 16;        // idle lanes that make a warp take new rays
constexpr int kSpin = 1 << 22;     // bound of every spin wait (iterations)

// One published scan: an env's observation scan or the scan of its final
// observation.  Everything a lane needs to set up a ray of it.
struct FlowScan {
    float st, ct;         // heading (sin, cos)
    float px, nx, py, ny; // origin to its cell's +x, -x, +y, -y sides (cells)
    int b0;               // origin cell in the padded map view (a padding cell if off-map)
    int d0;               // its distance byte (0: blocked or off-map origin)
    int K;                // beams
    int beam_off;         // first entry of the beam table in shared memory
    int stride;           // view row stride (bytes)
    int base;             // view: byte offset of the shared buffer (>= 0), or -1 - map
    int env;              // env index (row of obs / final_obs)
    int fin;              // 1: final-observation scan
    int map;              // map index
    float res, rmax_c;    // metres per cell, r_max in cells
};

struct FlowShared {
    unsigned long long cursor; // (scan << 32) | beam: the next ray to hand out
    unsigned long long bar[2]; // copy completion of each map buffer
    int n_pub;                 // scans published
    int done;                  // 1: the producer has published its last scan
    int abort;                 // 1: a wait timed out; stop
    int reading[kFlowWarps];   // scan whose record the warp may be reading (INT_MAX: none)
    int buf_map[2];            // map in each buffer (-1: none)
    int rays_done[2];          // rays of each buffer finished by the casters
};

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st_volatile(int *p, int v) { *(volatile int *)p = v; }

__device__ __forceinline__ void flow_fail(const StepArgs &A, FlowShared &F) {
    atomicOr(A.status, kStatusFlowTimeout);
    st_volatile(&F.abort, 1);
}

// Ray state of one lane (exact traversal with distance jumps, as cast_ray).
struct FlowRay {
    float tM, tm, tdM, tdm, tM0, tm0, kM, km, adm, offm, nM, t, rmax_c, res;
    int b, b0, sbM, sbm, d, tie;
    int voff;            // padded map view: byte offset of its shared buffer
    const uint8_t *view; // the same view as an address (shared buffer or global bytes)
    int out;             // beam index k
    int envf;            // env * 2 + fin
    int bufm;            // (shared buffer + 1, 0 for global) | map << 2
    bool stopped;
};

// Sets up beam k of scan S: the direction of theta + alpha_k by angle
// addition (Eq. 4), per axis the cell step, tDelta and the first boundary
// parameter, and the major / minor split of the distance jumps.  The
// arithmetic and its order are those of cast_ray; the per-scan parts (the
// origin's cell and its side distances) come precomputed in S.
__device__ __forceinline__ void ray_init(const StepArgs &A, const FlowScan &S,
                                         const float2 *beams, const uint8_t *smap, int region,
                                         int k, FlowRay &R) {
    const float2 ab = beams[S.beam_off + k];
    const float dx = S.ct * ab.x - S.st * ab.y;
    const float dy = S.st * ab.x + S.ct * ab.y;
    int sbx = 0, sby = 0;
    float tdx = 0.0f, tdy = 0.0f, tx0 = INFINITY, ty0 = INFINITY;
    if (dx > 0.0f) { sbx = 1; tdx = __frcp_rn(dx); tx0 = S.px * tdx; }
    else if (dx < 0.0f) { sbx = -1; tdx = __frcp_rn(-dx); tx0 = S.nx * tdx; }
    if (dy > 0.0f) { sby = S.stride; tdy = __frcp_rn(dy); ty0 = S.py * tdy; }
    else if (dy < 0.0f) { sby = -S.stride; tdy = __frcp_rn(-dy); ty0 = S.ny * tdy; }
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
    R.nM = floorf(__fmaf_rn(S.rmax_c, adM, 1.0f - R.tM0 * adM));
    R.kM = 0.0f;
    R.km = 0.0f;
    R.tM = R.tM0;
    R.tm = R.tm0;
    R.b = S.b0;
    R.b0 = S.b0;
    R.d = S.d0;
    R.t = 0.0f;
    R.rmax_c = S.rmax_c;
    R.res = S.res;
    R.out = k;
    R.envf = S.env * 2 + S.fin;
    if (S.base >= 0) {
        R.voff = S.base;
        R.view = smap + S.base;
        R.bufm = (S.base / region + 1) | (S.map << 2);
    } else {
        R.voff = 0;
        R.view = A.dist + A.maps[S.map].dist_off;
        R.bufm = S.map << 2;
    }
    R.stopped = S.d0 == 0;
}

// One iteration of the traversal: an ordinary step or a distance jump (see
// cast_ray).  Returns false when the ray has ended (r_max passed, or a
// blocked cell entered: R.stopped).  SH: the view is in shared memory.
template <bool SH> __device__ __forceinline__ bool ray_iter(const uint8_t *smap, FlowRay &R) {
    const bool sM = __float_as_int(R.tM) < __float_as_int(R.tm) + R.tie;
    const float tn = sM ? R.tM : R.tm;
    if (tn > R.rmax_c) return false;
    const float n = fminf((float)R.d - 1.0f, R.nM - R.kM);
    const float kM2 = R.kM + n;
    const float T = __fmaf_rn(kM2 - 1.0f, R.tdM, R.tM0);
    const float km2 = fmaxf(R.km, floorf(__fmaf_rn(T, R.adm, R.offm)));
    const bool jump = n >= 1.0f && T <= R.rmax_c && km2 - R.km <= n &&
                      __fmaf_rn(km2, R.tdm, R.tm0) > T &&
                      (km2 == R.km || __fmaf_rn(km2 - 1.0f, R.tdm, R.tm0) <= T);
    R.kM = jump ? kM2 : (sM ? R.kM + 1.0f : R.kM);
    R.km = jump ? km2 : (sM ? R.km : R.km + 1.0f);
    R.tM = __fmaf_rn(R.kM, R.tdM, R.tM0);
    R.tm = __fmaf_rn(R.km, R.tdm, R.tm0);
    R.b = R.b0 + (int)R.kM * R.sbM + (int)R.km * R.sbm;
    R.t = tn;
    // every view staged: a shared-memory load; else a generic load (shared
    // buffer or global distance bytes, per lane)
    R.d = SH ? smap[R.voff + R.b] : R.view[R.b];
    if (R.d == 0) {
        R.stopped = true;
        return false;
    }
    return true;
}

// Writes the finished ray's range into its observation row (or folds it into
// its sector minimum, Eq. 6), and the debug outputs.
__device__ __forceinline__ void ray_write(const StepArgs &A, const FlowRay &R) {
    const int env = R.envf >> 1, fin = R.envf & 1;
    const float range = R.stopped ? R.t * R.res : A.max_range;
    const float c = fminf(range, A.max_range);
    float *row = (fin ? A.final_obs : A.obs) + A.obs_off[env];
    const int m = A.p.n_sectors;
    if (m == 0) {
        row[R.out] = c;
    } else {
        // each lane folds its own ray (ranges >= 0: integer order is float order)
        const int K = A.tab_k[A.env_tab[env]];
        atomicMin(reinterpret_cast<int *>(row + R.out / (K / m)), __float_as_int(c));
    }
    if (!fin && A.dbg_range) {
        const MapDev M = A.maps[R.bufm >> 2];
        int hit = -2;
        if (R.stopped) {
            const int jj = R.b / M.byte_stride, ii = R.b - jj * M.byte_stride;
            const int i = ii - kPad, j = jj - kPad;
            hit = (i < 0 || j < 0 || i >= M.w || j >= M.h) ? -1 : j * M.w + i;
        }
        const long long ro = A.ray_off[env] + R.out;
        A.dbg_range[ro] = range;
        A.dbg_hit[ro] = hit;
        A.dbg_vis[ro] = 1u + (unsigned)R.kM + (unsigned)R.km;
    }
}

// Fills the scan record of a scan from (xc, yc) (cells) with heading (st, ct).
__device__ __forceinline__ void make_scan(const StepArgs &A, const MapDev &M, int map, int K,
                                          int beam_off, int base, int env, int fin, float xc,
                                          float yc, float st, float ct, FlowScan &S) {
    S.st = st;
    S.ct = ct;
    S.K = K;
    S.beam_off = beam_off;
    S.stride = M.byte_stride;
    S.base = base;
    S.env = env;
    S.fin = fin;
    S.map = map;
    S.res = M.res;
    S.rmax_c = A.max_range * M.inv_res;
    S.b0 = 0; // a padding cell: an off-map origin reports hit -1
    S.d0 = 0;
    S.px = S.nx = S.py = S.ny = 0.0f;
    if (xc >= 0.0f && yc >= 0.0f) {
        const float fx = floorf(xc), fy = floorf(yc);
        const int i0 = (int)fx, j0 = (int)fy;
        if (i0 < M.w && j0 < M.h) {
            S.b0 = (j0 + kPad) * M.byte_stride + (i0 + kPad);
            S.d0 = A.dist[M.dist_off + S.b0];
            S.px = (fx + 1.0f) - xc;
            S.nx = xc - fx;
            S.py = (fy + 1.0f) - yc;
            S.ny = yc - fy;
        }
    }
}

// Claims up to A.flow_claim envs of group g (warp-collective): a share of
// what is left, so that the group's CTAs end together.  When g is empty the
// warp looks at up to 32 groups at a time and moves to the one with the most
// envs left.  Returns the count (0: no envs left anywhere) and the first
// position in perm.
__device__ int flow_claim(const StepArgs &A, int &g, int &e0) {
    const int lane = threadIdx.x & 31;
    for (int round = 0; round <= A.n_groups + 1; ++round) {
        if (g >= 0) {
            int c = 0, start = 0;
            if (lane == 0) {
                const int beg = A.grp_beg[g], size = A.grp_end[g] - beg;
                const int rem = size - ld_volatile(&A.grp_next[g]);
                if (rem > 0) {
                    const int share = 2 * max(1, A.grp_ncta[g]);
                    const int want = max(1, min((rem + share - 1) / share, A.flow_claim));
                    const int got = atomicAdd(&A.grp_next[g], want);
                    if (got < size) {
                        start = beg + got;
                        c = min(want, size - got);
                    }
                }
            }
            c = __shfl_sync(kFull, c, 0);
            if (c > 0) {
                e0 = __shfl_sync(kFull, start, 0);
                return c;
            }
        }
        // the group with the most envs left
        int best = -1, best_rem = 0;
        for (int q0 = 0; q0 < A.n_groups; q0 += 32) {
            const int q = q0 + lane;
            int rem = 0;
            if (q < A.n_groups) rem = A.grp_end[q] - A.grp_beg[q] - ld_volatile(&A.grp_next[q]);
            int bq = q;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int r2 = __shfl_xor_sync(kFull, rem, o), q2 = __shfl_xor_sync(kFull, bq, o);
                if (r2 > rem || (r2 == rem && q2 < bq)) { rem = r2; bq = q2; }
            }
            if (rem > best_rem) { best_rem = rem; best = bq; }
        }
        if (best < 0) return 0;
        g = best;
    }
    return 0;
}

// Bounded wait (lane 0) until scans <= last have been handed out and no warp
// reads their records: their ring entries may then be overwritten.
__device__ bool ring_space(FlowShared &F, int last) {
    if (last < 0) return true;
    for (int it = 0; it < kSpin; ++it) {
        const unsigned long long c = ld_volatile64(&F.cursor);
        __threadfence_block();
        bool ok = (int)(c >> 32) > last;
        for (int w = 0; w < kFlowWarps && ok; ++w) ok = ld_volatile(&F.reading[w]) > last;
        if (ok) return true;
        if (ld_volatile(&F.abort)) return false;
        __nanosleep(32);
    }
    return false;
}

// The producer (warp 0): claims, stages, runs the env phase, publishes.
template <bool SH>
__device__ void produce(const StepArgs &A, FlowShared &F, uint8_t *smap, FlowScan *ring) {
    const int lane = threadIdx.x & 31;
    int g = A.cta_grp[blockIdx.x];
    int next_scan = 0;
    int issued[2] = {0, 0};
    unsigned parity[2] = {0u, 0u};
    int lru = 0;
    for (;;) {
        int e0 = 0;
        const int c = flow_claim(A, g, e0);
        if (c == 0) break;
        const int map = A.grp_map[g], tab = A.grp_tab[g];
        const MapDev M = A.maps[map];
        const int K = A.tab_k[tab], beam_off = A.tab_off[tab];
        // the map's shared buffer: already staged, or staged now into the buffer
        // used least recently once every ray published on it has finished
        int buf = -1;
        bool copying = false;
        if (M.n_bytes <= A.flow_region && A.flow_bufs > 0) {
            if (F.buf_map[0] == map) buf = 0;
            else if (A.flow_bufs > 1 && F.buf_map[1] == map) buf = 1;
            else {
                buf = A.flow_bufs > 1 ? lru : 0;
                bool free_ok = true;
                if (lane == 0) {
                    free_ok = false;
                    for (int it = 0; it < kSpin; ++it) {
                        if (ld_volatile(&F.rays_done[buf]) == issued[buf]) { free_ok = true; break; }
                        if (ld_volatile(&F.abort)) break;
                        __nanosleep(32);
                    }
                    if (free_ok) {
                        stage_map(smap + (size_t)buf * A.flow_region, A.dist + M.dist_off,
                                  (unsigned)M.n_bytes, &F.bar[buf]);
                        F.buf_map[buf] = map;
                    } else {
                        flow_fail(A, F);
                    }
                }
                if (!__shfl_sync(kFull, free_ok ? 1 : 0, 0)) break;
                copying = true;
            }
            lru = buf ^ 1;
        }
        // env phase of the claimed envs, one lane each (map through L1/L2)
        EnvSlot slot;
        const bool mine = lane < c;
        if (mine) {
            const int e = A.perm[e0 + lane];
            slot.env = e;
            slot.obs_off = A.obs_off[e];
            slot.ray_off = A.ray_off[e];
            env_phase<false>(A, BytesGlobal{A.dist + M.dist_off, M.byte_stride}, M, K, lane, slot,
                             nullptr, nullptr);
        }
        if (copying) {
            bool landed = true;
            if (lane == 0) {
                landed = wait_bitmap(&F.bar[buf], parity[buf]);
                if (!landed) {
                    flow_fail(A, F);
                    wait_bitmap(&F.bar[buf], parity[buf]); // the copy in flight, bounded
                    F.buf_map[buf] = -1;
                }
            }
            parity[buf] ^= 1u;
            if (!__shfl_sync(kFull, landed ? 1 : 0, 0)) break;
        }
        // publish the observation scans, then the final-observation scans
        const unsigned finm = __ballot_sync(kFull, mine && slot.fin);
        const int n_new = c + __popc(finm);
        bool room = true;
        if (lane == 0) {
            room = ring_space(F, next_scan + n_new - 1 - kRing);
            if (!room) flow_fail(A, F);
        }
        if (!__shfl_sync(kFull, room ? 1 : 0, 0)) break;
        const int base = buf >= 0 ? buf * A.flow_region : -1 - map;
        if (mine) {
            make_scan(A, M, map, K, beam_off, base, slot.env, 0, slot.xc, slot.yc, slot.st, slot.ct,
                      ring[(next_scan + lane) & (kRing - 1)]);
            if (slot.fin) {
                const int r = c + __popc(finm & ((1u << lane) - 1u));
                make_scan(A, M, map, K, beam_off, base, slot.env, 1, slot.fxc, slot.fyc, slot.fst,
                          slot.fct, ring[(next_scan + r) & (kRing - 1)]);
            }
        }
        if (buf >= 0) issued[buf] += n_new * K;
        next_scan += n_new;
        __threadfence_block();
        __syncwarp();
        if (lane == 0) st_volatile(&F.n_pub, next_scan);
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) st_volatile(&F.done, 1);
}

// Takes up to R rays for warp `warp` (lane 0): from the cursor's scan and,
// when that scan ends first, from the next published one.  st = 0 rays
// taken, 1 none published yet, 2 no more scans, 3 stop (timeout).
__device__ void flow_take(FlowShared &F, const FlowScan *ring, int warp, int R, int &s, int &k0,
                          int &n1, int &n2, int &st) {
    for (int it = 0; it < kSpin; ++it) {
        const int fin = ld_volatile(&F.done);
        __threadfence_block();
        const int np = ld_volatile(&F.n_pub);
        const unsigned long long c = ld_volatile64(&F.cursor);
        const int cs = (int)(c >> 32), ck = (int)(unsigned)c;
        if (ld_volatile(&F.abort)) { st = 3; return; }
        if (cs >= np) { st = fin ? 2 : 1; return; }
        st_volatile(&F.reading[warp], cs);
        __threadfence_block();
        // a record read here may be stale only if the cursor moved on, in which
        // case the compare-and-swap below fails
        const int K1 = ring[cs & (kRing - 1)].K;
        int t1 = min(R, K1 - ck), t2 = 0, ns, nk;
        if (ck + t1 < K1) {
            ns = cs;
            nk = ck + t1;
        } else if (t1 < R && cs + 1 < np) {
            const int K2 = ring[(cs + 1) & (kRing - 1)].K;
            t2 = min(R - t1, K2);
            if (t2 < K2) { ns = cs + 1; nk = t2; }
            else { ns = cs + 2; nk = 0; }
        } else {
            ns = cs + 1;
            nk = 0;
        }
        const unsigned long long nc = ((unsigned long long)(unsigned)ns << 32) | (unsigned)nk;
        if (t1 > 0 && atomicCAS(&F.cursor, c, nc) == c) {
            s = cs;
            k0 = ck;
            n1 = t1;
            n2 = t2;
            st = 0;
            return;
        }
        st_volatile(&F.reading[warp], INT_MAX);
    }
    st = 3;
}

// The casters (every warp; warp 0 after producing).
template <bool SH>
__device__ void cast(const StepArgs &A, FlowShared &F, const uint8_t *smap, const float2 *sbeam,
                     const FlowScan *ring) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FlowRay R;
    R.stopped = false;
    bool act = false, res = false;
    unsigned vis = 0, nrays = 0;
    int thr = kRefill;
    int spins = 0;
    for (;;) {
        if (__any_sync(kFull, act)) {
            for (;;) {
                if (act && !ray_iter<SH>(smap, R)) {
                    act = false;
                    res = true;
                }
                if (__popc(__ballot_sync(kFull, !act)) >= thr) break;
            }
        }
        // finished rays: ranges out, finished counts per map buffer
        const unsigned wrote0 = __ballot_sync(kFull, res && (R.bufm & 3) == 1);
        const unsigned wrote1 = __ballot_sync(kFull, res && (R.bufm & 3) == 2);
        if (res) {
            ray_write(A, R);
            vis += 1u + (unsigned)R.kM + (unsigned)R.km;
            nrays += 1u;
            res = false;
        }
        if (lane == 0 && (wrote0 | wrote1)) {
            __threadfence_block();
            if (wrote0) atomicAdd(&F.rays_done[0], __popc(wrote0));
            if (wrote1) atomicAdd(&F.rays_done[1], __popc(wrote1));
        }
        // refill the idle lanes
        const unsigned want = __ballot_sync(kFull, !act);
        int s = 0, k0 = 0, n1 = 0, n2 = 0, st = 1;
        if (want && lane == 0) flow_take(F, ring, warp, __popc(want), s, k0, n1, n2, st);
        st = __shfl_sync(kFull, st, 0);
        if (st == 0) {
            s = __shfl_sync(kFull, s, 0);
            k0 = __shfl_sync(kFull, k0, 0);
            n1 = __shfl_sync(kFull, n1, 0);
            n2 = __shfl_sync(kFull, n2, 0);
            const int rank = __popc(want & ((1u << lane) - 1u));
            if ((want >> lane) & 1u) {
                if (rank < n1) {
                    ray_init(A, ring[s & (kRing - 1)], sbeam, smap, A.flow_region, k0 + rank, R);
                    act = !R.stopped;
                    res = R.stopped;
                } else if (rank < n1 + n2) {
                    ray_init(A, ring[(s + 1) & (kRing - 1)], sbeam, smap, A.flow_region, rank - n1, R);
                    act = !R.stopped;
                    res = R.stopped;
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                st_volatile(&F.reading[warp], INT_MAX);
            }
            thr = kRefill;
            spins = 0;
        } else if (!want) {
            thr = kRefill;
        } else if (st >= 2) {
            // no more scans: finish the rays held
            if (!__any_sync(kFull, act || res)) break;
            thr = 32;
        } else {
            // nothing published yet
            if (!__any_sync(kFull, act || res)) {
                if (++spins > kSpin) {
                    if (lane == 0) flow_fail(A, F);
                    break;
                }
                __nanosleep(64);
            } else {
                thr = min(32, __popc(want) + 1);
            }
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

template <bool SH> __global__ void __launch_bounds__(kFlowThreads, 1) flow_kernel(const StepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ FlowShared F;
    uint8_t *smap = smem;
    const size_t maps_bytes = (size_t)A.flow_bufs * A.flow_region;
    float2 *sbeam = reinterpret_cast<float2 *>(smem + maps_bytes);
    FlowScan *ring = reinterpret_cast<FlowScan *>(
        smem + maps_bytes + (((size_t)A.n_beams_total * sizeof(float2) + 127) & ~(size_t)127));
    const int tid = threadIdx.x;
    if (tid == 0) {
        F.cursor = 0ull;
        F.n_pub = 0;
        F.done = 0;
        F.abort = 0;
        F.buf_map[0] = F.buf_map[1] = -1;
        F.rays_done[0] = F.rays_done[1] = 0;
        init_copy_barrier(&F.bar[0]);
        init_copy_barrier(&F.bar[1]);
    }
    if (tid < kFlowWarps) F.reading[tid] = INT_MAX;
    for (int i = tid; i < A.n_beams_total; i += blockDim.x)
        sbeam[i] = make_float2(A.beam_c[i], A.beam_s[i]);
    __syncthreads();
    if (tid < 32) produce<SH>(A, F, smap, ring);
    cast<SH>(A, F, smap, sbeam, ring);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const int done = atomicAdd(&A.flow_q[0], 1);
        if (done == (int)gridDim.x - 1) {
            // every CTA has made its last claim: reset for the next launch
            for (int q = 0; q < A.n_groups; ++q) A.grp_next[q] = 0;
            A.flow_q[0] = 0;
            __threadfence();
        }
    }
}

} // namespace

size_t flow_smem_bytes(const StepArgs &a) {
    return (size_t)a.flow_bufs * a.flow_region +
           (((size_t)a.n_beams_total * sizeof(float2) + 127) & ~(size_t)127) +
           (size_t)kRing * sizeof(FlowScan);
}

int launch_step_flow(const StepArgs &a, void *stream) {
    if (a.n_groups <= 0) return 0;
    const size_t smem = flow_smem_bytes(a);
    const void *fn = a.flow_all_shared ? (const void *)flow_kernel<true> : (const void *)flow_kernel<false>;
    int n_sm = 0, per_sm = 0;
    cudaError_t err = (cudaError_t)occupancy(fn, smem, kFlowThreads, n_sm, per_sm);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    void *args[] = {const_cast<StepArgs *>(&a)};
    err = cudaLaunchKernel(fn, dim3(a.flow_grid), dim3(kFlowThreads), args, smem,
                           static_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return (int)err;
    return (int)cudaGetLastError();
}

} // namespace flashnav
