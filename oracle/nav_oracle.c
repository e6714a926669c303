/*
 * nav_oracle.c -- plain, slow CPU reference of the FlashNav batched bitmap
 * simulator step (Sec. 2.2 of the paper, Eq. 1-7, Tables 7-9).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path: every routine here is written from
 * the paper and from the textbook definitions it names (Amanatides-Woo grid
 * traversal, the exact unicycle arc, SplitMix64's finaliser).
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * Every FP32 expression is written in the order it is evaluated; with
 * contraction off each operation is one IEEE-754 binary32 rounding, so the
 * results are a fixed function of the inputs.
 *
 * Coordinates (the paper maps world coordinates to bitmap indices, Sec. 2.2.1):
 *   world metres (x, y); cell units xc = x * inv_res, inv_res = (float)(1/res);
 *   cell (i, j) is the closed square [i, i+1] x [j, j+1]; i = column, j = row;
 *   occ[j*W + i] != 0 means occupied; any cell outside [0,W)x[0,H) is an
 *   obstacle (Sec. 2.2.1: out-of-bounds positions are treated as obstacles).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "nav_oracle.h"

/* ------------------------------------------------------------------ */
/* Constants                                                            */
/* ------------------------------------------------------------------ */
static const float OR_PI = 3.14159265358979323846f;
static const float OR_TWO_PI = 6.28318530717958647692f;
static const float OR_TWO_OVER_PI = 0.636619772367581343076f;
/* pi/2 = P1 + P2 + P3: P1 and P2 carry 12 significant bits each so that
 * k*P1 and k*P2 are exact for |k| < 2^12 (Cody & Waite, 1980). */
static const float OR_P1 = 0x1.92p+0f;
static const float OR_P2 = 0x1.fb4p-12f;
static const float OR_P3 = 0x1.4442d2p-24f;

/* ------------------------------------------------------------------ */
/* sin / cos in binary32 from the Taylor series                         */
/* ------------------------------------------------------------------ */
/* Reduction x = k*pi/2 + r, |r| <= pi/4, then the Taylor polynomials of sin
 * (through r^11) and cos (through r^12), coefficients (-1)^n/(2n+1)! and
 * (-1)^n/(2n)! rounded from binary64.  Used for the heading and the arc
 * integration; Eq. 4 needs cos/sin of theta + alpha_k. */
void or_sincosf(float x, float *s_out, float *c_out)
{
    float k = rintf(x * OR_TWO_OVER_PI);
    float r = x - k * OR_P1;
    r = r - k * OR_P2;
    r = r - k * OR_P3;
    float r2 = r * r;
    /* sin: r + r^3 * (-1/3! + r^2 (1/5! + r^2 (-1/7! + r^2 (1/9! - r^2/11!)))) */
    float ps = (float)(-1.0 / 39916800.0);
    ps = ps * r2 + (float)(1.0 / 362880.0);
    ps = ps * r2 + (float)(-1.0 / 5040.0);
    ps = ps * r2 + (float)(1.0 / 120.0);
    ps = ps * r2 + (float)(-1.0 / 6.0);
    float s = r + (r * r2) * ps;
    /* cos: 1 + r^2 * (-1/2! + r^2 (1/4! + ... + r^2/12!)) */
    float pc = (float)(1.0 / 479001600.0);
    pc = pc * r2 + (float)(-1.0 / 3628800.0);
    pc = pc * r2 + (float)(1.0 / 40320.0);
    pc = pc * r2 + (float)(-1.0 / 720.0);
    pc = pc * r2 + (float)(1.0 / 24.0);
    pc = pc * r2 + (float)(-1.0 / 2.0);
    float c = 1.0f + r2 * pc;
    int q = ((int)k) & 3;
    float so, co;
    if (q == 0) { so = s; co = c; }
    else if (q == 1) { so = c; co = -s; }
    else if (q == 2) { so = -s; co = -c; }
    else { so = -c; co = s; }
    *s_out = so;
    *c_out = co;
}

/* Wrap an angle that is at most one turn outside [-pi, pi) back into it. */
static float or_wrap(float a)
{
    if (a >= OR_PI) a = a - OR_TWO_PI;
    else if (a < -OR_PI) a = a + OR_TWO_PI;
    return a;
}

/* ------------------------------------------------------------------ */
/* Counter-based RNG: SplitMix64 finaliser (Steele, Lea & Flood 2014)   */
/* ------------------------------------------------------------------ */
uint64_t or_hash(uint64_t seed, uint64_t env, uint64_t episode, uint64_t k)
{
    uint64_t z = seed ^ (env * 0x9E3779B97F4A7C15ull) ^ (episode * 0xC2B2AE3D27D4EB4Full)
                 ^ (k * 0x165667B19E3779F9ull);
    z = z + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform index in [0, n) from the high 32 bits (multiply-shift). */
static uint32_t or_pick(uint64_t h, uint32_t n)
{
    return (uint32_t)(((h >> 32) * (uint64_t)n) >> 32);
}

/* Uniform float in [0, 1) from the top 24 bits. */
static float or_unit24(uint64_t h)
{
    return (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f);
}

/* ------------------------------------------------------------------ */
/* Maps                                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int w, h;
    float res, inv_res;
    uint8_t *occ; /* w*h, nonzero = occupied */
} or_mapc;

static int or_blocked(const or_mapc *m, int i, int j)
{
    if (i < 0 || j < 0 || i >= m->w || j >= m->h) return 1;
    return m->occ[(size_t)j * m->w + i] != 0;
}

/* Row span of the cells whose closed square meets the open disc of radius rc
 * (cells) centred at (xc, yc): rows [*j0, *j1]; for row j the columns are
 * [floor(xc - h), ceil(xc + h) - 1] with h = sqrt(rc^2 - dy^2) and dy the
 * distance from yc to the row's slab [j, j+1].  Returns 0 if the row is not
 * reached. */
static int or_disc_row(float xc, float yc, float rc, int j, int *i0, int *i1)
{
    float fj = (float)j;
    float dy;
    if (yc < fj) dy = fj - yc;
    else if (yc > fj + 1.0f) dy = yc - (fj + 1.0f);
    else dy = 0.0f;
    if (!(dy < rc)) return 0;
    float hh = sqrtf(rc * rc - dy * dy);
    *i0 = (int)floorf(xc - hh);
    *i1 = (int)ceilf(xc + hh) - 1;
    return 1;
}

/* Collision of an open disc with the closed occupied cells (Sec. 2.2.3, the
 * footprint check; out-of-map counts as occupied). */
static int or_disc_hits(const or_mapc *m, float xc, float yc, float rc)
{
    int j0 = (int)floorf(yc - rc);
    int j1 = (int)ceilf(yc + rc) - 1;
    for (int j = j0; j <= j1; ++j) {
        int i0, i1;
        if (!or_disc_row(xc, yc, rc, j, &i0, &i1)) continue;
        for (int i = i0; i <= i1; ++i)
            if (or_blocked(m, i, j)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dynamic disc obstacles (moving discs stamped into a per-env layer)   */
/* ------------------------------------------------------------------ */
typedef struct { float x, y, vx, vy; } or_dyn;

/* Cell (i,j) belongs to obstacle o's stamp iff its closed square meets the
 * open disc of radius rdc (cells) around the obstacle centre. */
static int or_dyn_covers(const or_dyn *o, float inv_res, float rdc, int i, int j)
{
    float oxc = o->x * inv_res;
    float oyc = o->y * inv_res;
    int j0 = (int)floorf(oyc - rdc);
    int j1 = (int)ceilf(oyc + rdc) - 1;
    if (j < j0 || j > j1) return 0;
    int i0, i1;
    if (!or_disc_row(oxc, oyc, rdc, j, &i0, &i1)) return 0;
    return i >= i0 && i <= i1;
}

/* Static map OR the dynamic layer. */
static int or_blocked_dyn(const or_mapc *m, const or_dyn *d, int nd, float rdc, int i, int j)
{
    if (or_blocked(m, i, j)) return 1;
    for (int q = 0; q < nd; ++q)
        if (or_dyn_covers(&d[q], m->inv_res, rdc, i, j)) return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ray cast: exact grid traversal (Amanatides & Woo, 1987)              */
/* ------------------------------------------------------------------ */
/* Eq. 4 ray from (xc, yc) along the unit vector (dx, dy), both in cell units;
 * returns the range in metres (the entry distance into the first blocked
 * cell, Eq. 5, capped at r_max) and the hit id: j*W+i for an occupied cell,
 * -1 for leaving the map, -2 for reaching r_max.  *visits counts the cells
 * whose occupancy was looked up.
 * Ties tMaxX == tMaxY step X first (then Y on the next iteration).
 * The ray meets the axis-x cell boundaries at t = tMaxX0 + k * tDeltaX
 * (k = 0, 1, ...; Eq. 4 solved for each boundary): after k steps in x the
 * next boundary's parameter is that expression evaluated once, as one fused
 * multiply-add (a single rounding), rather than tDeltaX added k times (k
 * roundings).  Likewise for y. */
static float or_cast(const or_mapc *m, const or_dyn *dyn, int nd, float rdc,
                     float xc, float yc, float dx, float dy, float max_range,
                     int32_t *hit, uint32_t *visits)
{
    float rmax_c = max_range * m->inv_res;
    int i = (int)floorf(xc);
    int j = (int)floorf(yc);
    uint32_t nv = 1;
    if (i < 0 || j < 0 || i >= m->w || j >= m->h) {
        *hit = -1; *visits = nv; return 0.0f;
    }
    if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) {
        *hit = j * m->w + i; *visits = nv; return 0.0f;
    }
    int sx = 0, sy = 0;
    float tdx = INFINITY, tdy = INFINITY, tmx = INFINITY, tmy = INFINITY;
    if (dx > 0.0f) { sx = 1; tdx = 1.0f / dx; tmx = ((floorf(xc) + 1.0f) - xc) * tdx; }
    else if (dx < 0.0f) { sx = -1; tdx = 1.0f / -dx; tmx = (xc - floorf(xc)) * tdx; }
    if (dy > 0.0f) { sy = 1; tdy = 1.0f / dy; tmy = ((floorf(yc) + 1.0f) - yc) * tdy; }
    else if (dy < 0.0f) { sy = -1; tdy = 1.0f / -dy; tmy = (yc - floorf(yc)) * tdy; }
    const float tmx0 = tmx, tmy0 = tmy;
    int kx = 0, ky = 0; /* steps taken in x and in y */
    for (;;) {
        float t;
        if (tmx <= tmy) {
            t = tmx; if (t > rmax_c) break;
            i += sx; kx += 1; tmx = fmaf((float)kx, tdx, tmx0);
        } else {
            t = tmy; if (t > rmax_c) break;
            j += sy; ky += 1; tmy = fmaf((float)ky, tdy, tmy0);
        }
        nv += 1;
        if (i < 0 || j < 0 || i >= m->w || j >= m->h) {
            *hit = -1; *visits = nv; return t * m->res;
        }
        if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) {
            *hit = j * m->w + i; *visits = nv; return t * m->res;
        }
    }
    *hit = -2;
    *visits = nv;
    return max_range;
}

/* Fixed-step ray march (Sec. 2.2.2 as printed in the paper): sample the ray
 * of Eq. 4 at tau = s * step (s = 0, 1, 2, ...) and stop at the first sample
 * whose cell is occupied or off the map (range tau), or once tau exceeds
 * r_max (range r_max).  In cell units with step_c = step * inv_res.  Every
 * sample counts as a visit. */
static float or_march(const or_mapc *m, const or_dyn *dyn, int nd, float rdc, float xc, float yc,
                      float dx, float dy, float step_c, float max_range, int32_t *hit,
                      uint32_t *visits)
{
    float rmax_c = max_range * m->inv_res;
    uint32_t nv = 1;
    int i = (int)floorf(xc);
    int j = (int)floorf(yc);
    if (!(xc >= 0.0f && yc >= 0.0f) || i >= m->w || j >= m->h) {
        *hit = -1; *visits = nv; return 0.0f;
    }
    if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) {
        *hit = j * m->w + i; *visits = nv; return 0.0f;
    }
    for (int s = 1;; ++s) {
        float tc = (float)s * step_c;
        if (tc > rmax_c) break;
        float px = xc + tc * dx;
        float py = yc + tc * dy;
        nv += 1;
        if (!(px >= 0.0f && py >= 0.0f)) { *hit = -1; *visits = nv; return tc * m->res; }
        i = (int)floorf(px);
        j = (int)floorf(py);
        if (i >= m->w || j >= m->h) { *hit = -1; *visits = nv; return tc * m->res; }
        if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) {
            *hit = j * m->w + i; *visits = nv; return tc * m->res;
        }
    }
    *hit = -2;
    *visits = nv;
    return max_range;
}

float or_march_ray(const uint8_t *occ, int w, int h, float res, float x, float y, float dx,
                   float dy, float step, float max_range, int32_t *hit, uint32_t *visits)
{
    or_mapc m;
    m.w = w; m.h = h; m.res = res; m.inv_res = (float)(1.0 / (double)res);
    m.occ = (uint8_t *)occ;
    return or_march(&m, NULL, 0, 0.0f, x * m.inv_res, y * m.inv_res, dx, dy, step * m.inv_res,
                    max_range, hit, visits);
}

float or_cast_ray(const uint8_t *occ, int w, int h, float res, float x, float y,
                  float dx, float dy, float max_range, int32_t *hit, uint32_t *visits)
{
    or_mapc m;
    m.w = w; m.h = h; m.res = res; m.inv_res = (float)(1.0 / (double)res);
    m.occ = (uint8_t *)occ;
    return or_cast(&m, NULL, 0, 0.0f, x * m.inv_res, y * m.inv_res, dx, dy, max_range, hit, visits);
}

/* ------------------------------------------------------------------ */
/* Footprints                                                           */
/* ------------------------------------------------------------------ */
/* Rectangle footprint (Go2-like, Table 9): open rectangle of length L along
 * the heading and width Wd, centred at (xc, yc) in cell units.  For each row
 * slab [j, j+1] the polygon's x-extent comes from its vertices inside the
 * slab and its edges' crossings of y = j and y = j+1; the cells met are
 * those with i < xhi and i + 1 > xlo. */
static int or_rect_hits(const or_mapc *m, const or_dyn *dyn, int nd, float rdc,
                        float xc, float yc, float st, float ct, float hl, float hw)
{
    float ax = hl * ct, ay = hl * st;   /* half-length along heading */
    float bx = -(hw * st), by = hw * ct; /* half-width along the normal */
    float px[4], py[4];
    px[0] = (xc + ax) + bx; py[0] = (yc + ay) + by;
    px[1] = (xc - ax) + bx; py[1] = (yc - ay) + by;
    px[2] = (xc - ax) - bx; py[2] = (yc - ay) - by;
    px[3] = (xc + ax) - bx; py[3] = (yc + ay) - by;
    float ymin = py[0], ymax = py[0];
    for (int v = 1; v < 4; ++v) {
        if (py[v] < ymin) ymin = py[v];
        if (py[v] > ymax) ymax = py[v];
    }
    int j0 = (int)floorf(ymin);
    int j1 = (int)ceilf(ymax) - 1;
    for (int j = j0; j <= j1; ++j) {
        float lo = (float)j, hi = (float)j + 1.0f;
        float xlo = INFINITY, xhi = -INFINITY;
        for (int v = 0; v < 4; ++v) {
            if (py[v] >= lo && py[v] <= hi) {
                if (px[v] < xlo) xlo = px[v];
                if (px[v] > xhi) xhi = px[v];
            }
        }
        for (int v = 0; v < 4; ++v) {
            int u = (v + 1) & 3;
            float ya = py[v], yb = py[u];
            if (ya == yb) continue;
            float ylo = ya < yb ? ya : yb;
            float yhi = ya < yb ? yb : ya;
            for (int s = 0; s < 2; ++s) {
                float yl = s ? hi : lo;
                if (yl > ylo && yl < yhi) {
                    float xx = px[v] + (yl - ya) * (px[u] - px[v]) / (yb - ya);
                    if (xx < xlo) xlo = xx;
                    if (xx > xhi) xhi = xx;
                }
            }
        }
        if (!(xlo <= xhi)) continue;
        int i0 = (int)floorf(xlo);
        int i1 = (int)ceilf(xhi) - 1;
        for (int i = i0; i <= i1; ++i)
            if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) return 1;
    }
    return 0;
}

static int or_disc_hits_dyn(const or_mapc *m, const or_dyn *dyn, int nd, float rdc,
                            float xc, float yc, float rc)
{
    int j0 = (int)floorf(yc - rc);
    int j1 = (int)ceilf(yc + rc) - 1;
    for (int j = j0; j <= j1; ++j) {
        int i0, i1;
        if (!or_disc_row(xc, yc, rc, j, &i0, &i1)) continue;
        for (int i = i0; i <= i1; ++i)
            if (or_blocked_dyn(m, dyn, nd, rdc, i, j)) return 1;
    }
    return 0;
}

int or_footprint(const uint8_t *occ, int w, int h, float res, int shape, float radius,
                 float length, float width, float x, float y, float theta)
{
    or_mapc m;
    m.w = w; m.h = h; m.res = res; m.inv_res = (float)(1.0 / (double)res);
    m.occ = (uint8_t *)occ;
    float xc = x * m.inv_res, yc = y * m.inv_res;
    if (shape == 0) return or_disc_hits(&m, xc, yc, radius * m.inv_res);
    float st, ct;
    or_sincosf(theta, &st, &ct);
    return or_rect_hits(&m, NULL, 0, 0.0f, xc, yc, st, ct, (0.5f * length) * m.inv_res,
                        (0.5f * width) * m.inv_res);
}

/* ------------------------------------------------------------------ */
/* Unicycle integration (Sec. 2.2.3) -- exact arc over dt               */
/* ------------------------------------------------------------------ */
/* theta' = wrap(theta + w dt); the displacement is the chord of the arc:
 * x' = x + v dt sinc(w dt / 2) cos(theta + w dt / 2), same with sin for y. */
void or_integrate(float x, float y, float th, float v, float w, float dt,
                  float *xo, float *yo, float *tho)
{
    float hd = (w * dt) * 0.5f;
    float sc;
    if (fabsf(hd) < 0.1f) {
        float x2 = hd * hd;
        float p = (float)(-1.0 / 5040.0);
        p = p * x2 + (float)(1.0 / 120.0);
        p = p * x2 + (float)(-1.0 / 6.0);
        sc = 1.0f + x2 * p;
    } else {
        float sh, ch;
        or_sincosf(hd, &sh, &ch);
        sc = sh / hd;
    }
    float sm, cm;
    or_sincosf(th + hd, &sm, &cm);
    float chord = (v * dt) * sc;
    *xo = x + chord * cm;
    *yo = y + chord * sm;
    *tho = or_wrap(th + w * dt);
}

/* ------------------------------------------------------------------ */
/* Simulator                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int *spawn;      /* spawnable cells, ascending j*W+i */
    int n_spawn;
    int *comp_of;    /* W*H: component id of a spawnable cell, else -1 */
    int *comp_start; /* per component: offset into comp_cells */
    int *comp_count;
    int *comp_cells; /* cells grouped by component, ascending within a group */
    int n_comp;
} or_cspace;

struct or_sim {
    int n_maps, n_envs, n_robots, max_k, threads;
    or_mapc *maps;
    or_robot *robots;
    or_params par;
    float max_range;
    int *env_map, *env_k, *env_robot;
    int64_t *obs_off, *ray_off;
    /* per (map, robot) C-space */
    or_cspace *cs;
    /* beam tables per env beam count: host FP64 -> FP32 (cos a_k, sin a_k) */
    float **tab_c, **tab_s;
    int *tab_k;
    int n_tab;
    int *env_tab;
    uint64_t seed;
    /* state */
    float *x, *y, *th, *v, *w, *gx, *gy, *dprev;
    int32_t *step;
    uint32_t *episode;
    or_dyn *dyn;     /* n_envs * n_dyn */
    /* debug */
    float *ranges;   /* ray_off layout */
    int32_t *hits;
    uint32_t *ray_visits;
    uint64_t visits_total;
};

void or_default_params(or_params *p)
{
    p->dt = 0.1f;
    p->goal_tol = 0.2f;
    p->c_progress = 2.0f;
    p->step_penalty = 0.01f;
    p->r_goal = 10.0f;
    p->r_coll = 10.0f;
    p->horizon = 200;
    p->goal_dmin = 2.0f;
    p->goal_dmax = 8.0f;
    p->fov_deg = 360.0f;
    p->n_dyn = 0;
    p->dyn_radius = 0.18f;
    p->dyn_speed_max = 0.5f;
    p->dyn_min_sep = 1.0f;
    p->reward_mode = 0;
    p->sensor = 0;
    p->march_step = 0.03f;
    p->n_sectors = 0;
}

static float or_circ_radius(const or_robot *r)
{
    if (r->shape == 0) return r->radius;
    return 0.5f * sqrtf(r->length * r->length + r->width * r->width);
}

/* Spawnable cells: the circumscribed disc of the footprint, centred at the
 * cell centre, touches no blocked cell.  Components: 4-connected spawnable
 * cells (goals are drawn from the spawn cell's component so they are
 * reachable; Sec. 2.2.3 samples poses and goals from free locations). */
static void or_build_cspace(const or_mapc *m, float rcirc_m, or_cspace *cs)
{
    int W = m->w, H = m->h;
    size_t n = (size_t)W * H;
    uint8_t *ok = (uint8_t *)calloc(n, 1);
    float rc = rcirc_m * m->inv_res;
    int ns = 0;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            float x = ((float)i + 0.5f) * m->res;
            float y = ((float)j + 0.5f) * m->res;
            if (!or_disc_hits(m, x * m->inv_res, y * m->inv_res, rc)) {
                ok[(size_t)j * W + i] = 1;
                ns++;
            }
        }
    cs->n_spawn = ns;
    cs->spawn = (int *)malloc(sizeof(int) * (ns ? ns : 1));
    cs->comp_of = (int *)malloc(sizeof(int) * n);
    int k = 0;
    for (size_t c = 0; c < n; ++c) {
        cs->comp_of[c] = -1;
        if (ok[c]) cs->spawn[k++] = (int)c;
    }
    /* BFS labelling in row-major discovery order */
    int *queue = (int *)malloc(sizeof(int) * (ns ? ns : 1));
    int ncomp = 0;
    for (int s = 0; s < ns; ++s) {
        int c0 = cs->spawn[s];
        if (cs->comp_of[c0] >= 0) continue;
        int qh = 0, qt = 0;
        queue[qt++] = c0;
        cs->comp_of[c0] = ncomp;
        while (qh < qt) {
            int c = queue[qh++];
            int ci = c % W, cj = c / W;
            int nb[4][2] = {{ci - 1, cj}, {ci + 1, cj}, {ci, cj - 1}, {ci, cj + 1}};
            for (int t = 0; t < 4; ++t) {
                int a = nb[t][0], b = nb[t][1];
                if (a < 0 || b < 0 || a >= W || b >= H) continue;
                int cc = b * W + a;
                if (ok[cc] && cs->comp_of[cc] < 0) {
                    cs->comp_of[cc] = ncomp;
                    queue[qt++] = cc;
                }
            }
        }
        ncomp++;
    }
    free(queue);
    cs->n_comp = ncomp;
    cs->comp_count = (int *)calloc(ncomp ? ncomp : 1, sizeof(int));
    cs->comp_start = (int *)calloc(ncomp ? ncomp : 1, sizeof(int));
    for (int s = 0; s < ns; ++s) cs->comp_count[cs->comp_of[cs->spawn[s]]]++;
    int acc = 0;
    for (int c = 0; c < ncomp; ++c) { cs->comp_start[c] = acc; acc += cs->comp_count[c]; }
    cs->comp_cells = (int *)malloc(sizeof(int) * (ns ? ns : 1));
    int *fill = (int *)calloc(ncomp ? ncomp : 1, sizeof(int));
    for (int s = 0; s < ns; ++s) {
        int c = cs->spawn[s];
        int id = cs->comp_of[c];
        cs->comp_cells[cs->comp_start[id] + fill[id]++] = c;
    }
    free(fill);
    free(ok);
}

or_sim *or_create(const or_map *maps, int n_maps, const int *env_map, const int *env_k,
                  const int *env_robot, int n_envs, float max_range, const or_robot *robots,
                  int n_robots, const or_params *params)
{
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->n_maps = n_maps;
    s->n_envs = n_envs;
    s->n_robots = n_robots;
    s->threads = 1;
    s->max_range = max_range;
    if (params) s->par = *params; else or_default_params(&s->par);
    s->maps = (or_mapc *)calloc(n_maps, sizeof(or_mapc));
    for (int i = 0; i < n_maps; ++i) {
        or_mapc *m = &s->maps[i];
        m->w = maps[i].width; m->h = maps[i].height; m->res = maps[i].resolution;
        m->inv_res = (float)(1.0 / (double)m->res);
        size_t n = (size_t)m->w * m->h;
        m->occ = (uint8_t *)malloc(n);
        memcpy(m->occ, maps[i].occ, n);
    }
    s->robots = (or_robot *)malloc(sizeof(or_robot) * n_robots);
    memcpy(s->robots, robots, sizeof(or_robot) * n_robots);
    s->env_map = (int *)malloc(sizeof(int) * n_envs);
    s->env_k = (int *)malloc(sizeof(int) * n_envs);
    s->env_robot = (int *)malloc(sizeof(int) * n_envs);
    s->obs_off = (int64_t *)malloc(sizeof(int64_t) * (n_envs + 1));
    s->ray_off = (int64_t *)malloc(sizeof(int64_t) * (n_envs + 1));
    s->obs_off[0] = 0; s->ray_off[0] = 0;
    s->max_k = 0;
    for (int e = 0; e < n_envs; ++e) {
        s->env_map[e] = env_map ? env_map[e] : e % n_maps;
        s->env_k[e] = env_k[e];
        s->env_robot[e] = env_robot ? env_robot[e] : 0;
        if (env_k[e] > s->max_k) s->max_k = env_k[e];
        s->obs_off[e + 1] = s->obs_off[e] + (s->par.n_sectors > 0 ? s->par.n_sectors : env_k[e]) + 4;
        s->ray_off[e + 1] = s->ray_off[e] + env_k[e];
    }
    /* beam tables: alpha_k = -FOV/2 + (k + 1/2) FOV / K (Eq. 4's alpha_k) */
    s->tab_k = (int *)malloc(sizeof(int) * n_envs);
    s->tab_c = (float **)malloc(sizeof(float *) * n_envs);
    s->tab_s = (float **)malloc(sizeof(float *) * n_envs);
    s->env_tab = (int *)malloc(sizeof(int) * n_envs);
    s->n_tab = 0;
    double fov = (double)s->par.fov_deg * (3.14159265358979323846 / 180.0);
    for (int e = 0; e < n_envs; ++e) {
        int K = s->env_k[e], t;
        for (t = 0; t < s->n_tab; ++t) if (s->tab_k[t] == K) break;
        if (t == s->n_tab) {
            s->tab_k[t] = K;
            s->tab_c[t] = (float *)malloc(sizeof(float) * K);
            s->tab_s[t] = (float *)malloc(sizeof(float) * K);
            for (int k = 0; k < K; ++k) {
                double a = -0.5 * fov + ((double)k + 0.5) * fov / (double)K;
                s->tab_c[t][k] = (float)cos(a);
                s->tab_s[t][k] = (float)sin(a);
            }
            s->n_tab++;
        }
        s->env_tab[e] = t;
    }
    s->cs = (or_cspace *)calloc((size_t)n_maps * n_robots, sizeof(or_cspace));
    for (int mi = 0; mi < n_maps; ++mi)
        for (int r = 0; r < n_robots; ++r) {
            int used = 0;
            for (int e = 0; e < n_envs && !used; ++e)
                used = s->env_map[e] == mi && s->env_robot[e] == r;
            if (used) or_build_cspace(&s->maps[mi], or_circ_radius(&s->robots[r]),
                                      &s->cs[(size_t)mi * n_robots + r]);
        }
    size_t E = (size_t)n_envs;
    s->x = (float *)calloc(E, 4); s->y = (float *)calloc(E, 4); s->th = (float *)calloc(E, 4);
    s->v = (float *)calloc(E, 4); s->w = (float *)calloc(E, 4);
    s->gx = (float *)calloc(E, 4); s->gy = (float *)calloc(E, 4); s->dprev = (float *)calloc(E, 4);
    s->step = (int32_t *)calloc(E, 4);
    s->episode = (uint32_t *)calloc(E, 4);
    s->dyn = (or_dyn *)calloc(E * (s->par.n_dyn > 0 ? s->par.n_dyn : 1), sizeof(or_dyn));
    s->ranges = (float *)calloc((size_t)s->ray_off[n_envs] + 1, 4);
    s->hits = (int32_t *)calloc((size_t)s->ray_off[n_envs] + 1, 4);
    s->ray_visits = (uint32_t *)calloc((size_t)s->ray_off[n_envs] + 1, 4);
    return s;
}

int or_spawn_count(const or_sim *s, int map, int robot)
{
    return s->cs[(size_t)map * s->n_robots + robot].n_spawn;
}

int or_comp_count(const or_sim *s, int map, int robot)
{
    return s->cs[(size_t)map * s->n_robots + robot].n_comp;
}

void or_comp_labels(const or_sim *s, int map, int robot, int *out)
{
    const or_cspace *cs = &s->cs[(size_t)map * s->n_robots + robot];
    memcpy(out, cs->comp_of, sizeof(int) * (size_t)s->maps[map].w * s->maps[map].h);
}

void or_free(or_sim *s)
{
    if (!s) return;
    for (int i = 0; i < s->n_maps; ++i) free(s->maps[i].occ);
    for (size_t c = 0; c < (size_t)s->n_maps * s->n_robots; ++c) {
        free(s->cs[c].spawn); free(s->cs[c].comp_of); free(s->cs[c].comp_start);
        free(s->cs[c].comp_count); free(s->cs[c].comp_cells);
    }
    for (int t = 0; t < s->n_tab; ++t) { free(s->tab_c[t]); free(s->tab_s[t]); }
    free(s->tab_c); free(s->tab_s); free(s->tab_k); free(s->env_tab);
    free(s->cs); free(s->maps); free(s->robots);
    free(s->env_map); free(s->env_k); free(s->env_robot); free(s->obs_off); free(s->ray_off);
    free(s->x); free(s->y); free(s->th); free(s->v); free(s->w);
    free(s->gx); free(s->gy); free(s->dprev); free(s->step); free(s->episode); free(s->dyn);
    free(s->ranges); free(s->hits); free(s->ray_visits);
    free(s);
}

void or_set_threads(or_sim *s, int n) { s->threads = n > 0 ? n : 1; }

/* Sparse reset of env e (Sec. 2.2.3): new pose and goal from free cells of
 * the map, counters cleared, obstacles re-drawn.  RNG draws are indexed by
 * (seed, env, episode, k): k = 0 spawn cell, 1 heading, 2..65 goal draws,
 * 1024 + 64 q + a obstacle q position draw a (a < 16), 1024 + 64 q + 48 its
 * speed and heading. */
static int or_reset_env(or_sim *s, int e)
{
    const or_mapc *m = &s->maps[s->env_map[e]];
    const or_cspace *cs = &s->cs[(size_t)s->env_map[e] * s->n_robots + s->env_robot[e]];
    if (cs->n_spawn == 0) return -4;
    uint32_t ep = s->episode[e];
    uint64_t h0 = or_hash(s->seed, (uint64_t)e, ep, 0);
    int cell = cs->spawn[or_pick(h0, (uint32_t)cs->n_spawn)];
    int ci = cell % m->w, cj = cell / m->w;
    float x = ((float)ci + 0.5f) * m->res;
    float y = ((float)cj + 0.5f) * m->res;
    float th = or_unit24(or_hash(s->seed, (uint64_t)e, ep, 1)) * OR_TWO_PI - OR_PI;
    int comp = cs->comp_of[cell];
    int cstart = cs->comp_start[comp], ccount = cs->comp_count[comp];
    float dmin = s->par.goal_dmin, dmax = s->par.goal_dmax;
    float best_gx = x, best_gy = y, best_err = INFINITY;
    for (int a = 0; a < 64; ++a) {
        uint64_t hg = or_hash(s->seed, (uint64_t)e, ep, 2 + (uint64_t)a);
        int gc = cs->comp_cells[cstart + (int)or_pick(hg, (uint32_t)ccount)];
        float gx = ((float)(gc % m->w) + 0.5f) * m->res;
        float gy = ((float)(gc / m->w) + 0.5f) * m->res;
        float ddx = gx - x, ddy = gy - y;
        float d = sqrtf(ddx * ddx + ddy * ddy);
        float err;
        if (d < dmin) err = dmin - d;
        else if (d > dmax) err = d - dmax;
        else err = 0.0f;
        if (err < best_err) { best_err = err; best_gx = gx; best_gy = gy; }
        if (err == 0.0f) break;
    }
    s->x[e] = x; s->y[e] = y; s->th[e] = th;
    s->v[e] = 0.0f; s->w[e] = 0.0f;
    s->gx[e] = best_gx; s->gy[e] = best_gy;
    {
        float ddx = best_gx - x, ddy = best_gy - y;
        s->dprev[e] = sqrtf(ddx * ddx + ddy * ddy);
    }
    s->step[e] = 0;
    int nd = s->par.n_dyn;
    for (int q = 0; q < nd; ++q) {
        or_dyn *o = &s->dyn[(size_t)e * nd + q];
        float ox = x, oy = y;
        for (int a = 0; a < 16; ++a) {
            uint64_t hp = or_hash(s->seed, (uint64_t)e, ep, 1024 + 64 * (uint64_t)q + (uint64_t)a);
            int oc = cs->spawn[or_pick(hp, (uint32_t)cs->n_spawn)];
            ox = ((float)(oc % m->w) + 0.5f) * m->res;
            oy = ((float)(oc / m->w) + 0.5f) * m->res;
            float ddx = ox - x, ddy = oy - y;
            if (sqrtf(ddx * ddx + ddy * ddy) >= s->par.dyn_min_sep) break;
        }
        uint64_t hv = or_hash(s->seed, (uint64_t)e, ep, 1024 + 64 * (uint64_t)q + 48);
        float sp = or_unit24(hv) * s->par.dyn_speed_max;
        float hd = (float)(uint32_t)((hv >> 8) & 0xFFFFFFu) * (1.0f / 16777216.0f) * OR_TWO_PI - OR_PI;
        float sh, ch;
        or_sincosf(hd, &sh, &ch);
        o->x = ox; o->y = oy; o->vx = sp * ch; o->vy = sp * sh;
    }
    return 0;
}

/* Moving-disc update: constant velocity; a velocity component flips sign when
 * the cell that would contain the moved centre is blocked (static layer). */
static void or_move_dyn(or_sim *s, int e)
{
    const or_mapc *m = &s->maps[s->env_map[e]];
    int nd = s->par.n_dyn;
    float dt = s->par.dt;
    for (int q = 0; q < nd; ++q) {
        or_dyn *o = &s->dyn[(size_t)e * nd + q];
        float nx = o->x + o->vx * dt;
        if (or_blocked(m, (int)floorf(nx * m->inv_res), (int)floorf(o->y * m->inv_res)))
            o->vx = -o->vx;
        else
            o->x = nx;
        float ny = o->y + o->vy * dt;
        if (or_blocked(m, (int)floorf(o->x * m->inv_res), (int)floorf(ny * m->inv_res)))
            o->vy = -o->vy;
        else
            o->y = ny;
    }
}

/* Cast all K beams of env e at its current pose; fills the debug arrays and
 * writes min(range, r_max) into obs[0..K-1]. */
static uint64_t or_scan(or_sim *s, int e, float *obs)
{
    const or_mapc *m = &s->maps[s->env_map[e]];
    int t = s->env_tab[e], K = s->env_k[e];
    const float *ca = s->tab_c[t], *sa = s->tab_s[t];
    float st, ct;
    or_sincosf(s->th[e], &st, &ct);
    float xc = s->x[e] * m->inv_res, yc = s->y[e] * m->inv_res;
    int nd = s->par.n_dyn;
    const or_dyn *dyn = nd ? &s->dyn[(size_t)e * nd] : NULL;
    float rdc = s->par.dyn_radius * m->inv_res;
    uint64_t vis = 0;
    int64_t ro = s->ray_off[e];
    for (int k = 0; k < K; ++k) {
        /* Eq. 4: direction of theta + alpha_k by the angle-addition formulas */
        float dx = ct * ca[k] - st * sa[k];
        float dy = st * ca[k] + ct * sa[k];
        int32_t hit;
        uint32_t nv;
        float r = s->par.sensor == 1
                      ? or_march(m, dyn, nd, rdc, xc, yc, dx, dy, s->par.march_step * m->inv_res,
                                 s->max_range, &hit, &nv)
                      : or_cast(m, dyn, nd, rdc, xc, yc, dx, dy, s->max_range, &hit, &nv);
        s->ranges[ro + k] = r;
        s->hits[ro + k] = hit;
        s->ray_visits[ro + k] = nv;
        vis += nv;
        if (obs && s->par.n_sectors == 0) obs[k] = r < s->max_range ? r : s->max_range;
    }
    /* Eq. 6: sector j = min over its K / m consecutive beams */
    if (obs && s->par.n_sectors > 0) {
        int per = K / s->par.n_sectors;
        for (int q = 0; q < s->par.n_sectors; ++q) {
            float mn = s->max_range;
            for (int k = q * per; k < (q + 1) * per; ++k) {
                float r = s->ranges[ro + k];
                if (r < mn) mn = r;
            }
            obs[q] = mn;
        }
    }
    return vis;
}

/* Observation tail (Eq. 1): goal distance, goal bearing in the body frame
 * wrapped to [-pi, pi), applied linear and angular velocity. */
static void or_obs_tail(const or_sim *s, int e, float *tail)
{
    float ddx = s->gx[e] - s->x[e], ddy = s->gy[e] - s->y[e];
    tail[0] = sqrtf(ddx * ddx + ddy * ddy);
    double phi = atan2((double)ddy, (double)ddx) - (double)s->th[e];
    while (phi >= 3.14159265358979323846) phi -= 2.0 * 3.14159265358979323846;
    while (phi < -3.14159265358979323846) phi += 2.0 * 3.14159265358979323846;
    tail[1] = (float)phi;
    tail[2] = s->v[e];
    tail[3] = s->w[e];
}

int or_reset(or_sim *s, uint64_t seed, float *obs)
{
    s->seed = seed;
    s->visits_total = 0;
    int err = 0;
    for (int e = 0; e < s->n_envs; ++e) {
        s->episode[e] = 0;
        if (or_reset_env(s, e)) err = -4;
    }
    if (err) return err;
    for (int e = 0; e < s->n_envs; ++e) {
        float *o = obs ? obs + s->obs_off[e] : NULL;
        s->visits_total += or_scan(s, e, o);
        if (o) or_obs_tail(s, e, o + (s->par.n_sectors > 0 ? s->par.n_sectors : s->env_k[e]));
    }
    return 0;
}

/* One step of env e along Eq. 7: A_t -> X_{t+1} -> R_{t+1} -> (c, r, delta)
 * -> O_{t+1} -> O~_{t+1}. */
static uint64_t or_step_env(or_sim *s, int e, const float *act, float *obs, float *reward,
                            uint8_t *done, float *final_obs, int *err)
{
    const or_mapc *m = &s->maps[s->env_map[e]];
    const or_robot *rb = &s->robots[s->env_robot[e]];
    const or_params *p = &s->par;
    int K = s->env_k[e];
    uint64_t vis = 0;
    /* a1: action decode -- clamp to [-1, 1] and map affinely onto the preset's
     * velocity bounds (Sec. 2.2.3, Table 7 action interface) */
    float a0 = fminf(fmaxf(act[2 * e + 0], -1.0f), 1.0f);
    float a1 = fminf(fmaxf(act[2 * e + 1], -1.0f), 1.0f);
    float v = rb->v_min + ((a0 + 1.0f) * 0.5f) * (rb->v_max - rb->v_min);
    float w = rb->w_min + ((a1 + 1.0f) * 0.5f) * (rb->w_max - rb->w_min);
    /* a2: pose integration */
    float nx, ny, nth;
    or_integrate(s->x[e], s->y[e], s->th[e], v, w, p->dt, &nx, &ny, &nth);
    s->x[e] = nx; s->y[e] = ny; s->th[e] = nth; s->v[e] = v; s->w[e] = w;
    /* a5: moving obstacles */
    if (p->n_dyn > 0) or_move_dyn(s, e);
    /* a3/a4: range scan at the new pose (R_{t+1}) */
    float *fo = final_obs ? final_obs + s->obs_off[e] : NULL;
    float *ob = obs + s->obs_off[e];
    vis += or_scan(s, e, ob);
    /* a6: footprint collision at the new pose */
    int nd = p->n_dyn;
    const or_dyn *dyn = nd ? &s->dyn[(size_t)e * nd] : NULL;
    float rdc = p->dyn_radius * m->inv_res;
    float xc = nx * m->inv_res, yc = ny * m->inv_res;
    int coll;
    if (rb->shape == 0) {
        coll = or_disc_hits_dyn(m, dyn, nd, rdc, xc, yc, rb->radius * m->inv_res);
    } else {
        float st, ct;
        or_sincosf(nth, &st, &ct);
        coll = or_rect_hits(m, dyn, nd, rdc, xc, yc, st, ct, (0.5f * rb->length) * m->inv_res,
                            (0.5f * rb->width) * m->inv_res);
    }
    /* a7: goal distance, reward (Eq. 3 plus a per-step penalty), flags */
    float ddx = s->gx[e] - nx, ddy = s->gy[e] - ny;
    float d = sqrtf(ddx * ddx + ddy * ddy);
    int goal = d <= p->goal_tol;
    float r;
    if (p->reward_mode == 0) {
        r = p->c_progress * (s->dprev[e] - d);
        r = r - p->step_penalty;
        if (goal) r = r + p->r_goal;
        if (coll) r = r - p->r_coll;
    } else {
        if (goal) r = p->r_goal;
        else if (coll) r = -p->r_coll;
        else r = p->c_progress * (s->dprev[e] - d);
    }
    s->dprev[e] = d;
    s->step[e] = s->step[e] + 1;
    int term = goal || coll;
    int trunc = !term && s->step[e] >= p->horizon;
    reward[e] = r;
    done[e] = (uint8_t)((term ? 1 : 0) | (trunc ? 2 : 0) | (goal ? 4 : 0) | (coll ? 8 : 0));
    /* a9: O_{t+1}, kept as the final observation of a finished episode */
    int D = s->par.n_sectors > 0 ? s->par.n_sectors : K;
    or_obs_tail(s, e, ob + D);
    if (term || trunc) {
        if (fo) memcpy(fo, ob, sizeof(float) * (size_t)(D + 4));
        /* a8: sparse reset, then a fresh scan (O~_{t+1}) */
        s->episode[e] = s->episode[e] + 1;
        if (or_reset_env(s, e)) *err = -4;
        vis += or_scan(s, e, ob);
        or_obs_tail(s, e, ob + D);
    }
    return vis;
}

int or_step(or_sim *s, const float *actions, float *obs, float *reward, uint8_t *done,
            float *final_obs)
{
    int err = 0;
    uint64_t vis = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(s->threads) schedule(dynamic, 16) reduction(+ : vis)
#endif
    for (int e = 0; e < s->n_envs; ++e) {
        int le = 0;
        vis += or_step_env(s, e, actions, obs, reward, done, final_obs, &le);
        if (le) err = le;
    }
    s->visits_total += vis;
    return err;
}

uint64_t or_visits(const or_sim *s) { return s->visits_total; }

void or_get_state(const or_sim *s, float *f8, int32_t *i2, float *dyn)
{
    for (int e = 0; e < s->n_envs; ++e) {
        float *f = f8 + 8 * (size_t)e;
        f[0] = s->x[e]; f[1] = s->y[e]; f[2] = s->th[e]; f[3] = s->v[e];
        f[4] = s->w[e]; f[5] = s->gx[e]; f[6] = s->gy[e]; f[7] = s->dprev[e];
        i2[2 * e] = s->step[e];
        i2[2 * e + 1] = (int32_t)s->episode[e];
    }
    if (dyn && s->par.n_dyn > 0)
        memcpy(dyn, s->dyn, sizeof(or_dyn) * (size_t)s->n_envs * s->par.n_dyn);
}

void or_set_state(or_sim *s, uint64_t seed, const float *f8, const int32_t *i2, const float *dyn)
{
    s->seed = seed;
    for (int e = 0; e < s->n_envs; ++e) {
        const float *f = f8 + 8 * (size_t)e;
        s->x[e] = f[0]; s->y[e] = f[1]; s->th[e] = f[2]; s->v[e] = f[3];
        s->w[e] = f[4]; s->gx[e] = f[5]; s->gy[e] = f[6]; s->dprev[e] = f[7];
        s->step[e] = i2[2 * e];
        s->episode[e] = (uint32_t)i2[2 * e + 1];
    }
    if (dyn && s->par.n_dyn > 0)
        memcpy(s->dyn, dyn, sizeof(or_dyn) * (size_t)s->n_envs * s->par.n_dyn);
}

/* Ranges, hit ids and visit counts of the last scan of each env (the
 * post-reset scan for envs that were reset). */
void or_get_debug(const or_sim *s, float *ranges, int32_t *hits, uint32_t *visits)
{
    size_t n = (size_t)s->ray_off[s->n_envs];
    if (ranges) memcpy(ranges, s->ranges, 4 * n);
    if (hits) memcpy(hits, s->hits, 4 * n);
    if (visits) memcpy(visits, s->ray_visits, 4 * n);
}
