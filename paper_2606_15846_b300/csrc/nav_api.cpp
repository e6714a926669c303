// Host runtime of the C ABI declared in include/flashnav.h: argument checks,
// bit-packing of the maps, per-(map, robot) spawn tables, beam tables, the
// env -> tile schedule, device memory and the launches.
//
// Compiled with -ffp-contract=off: the spawnability test below decides which
// cells a reset may draw, so its binary32 arithmetic must round exactly like
// the device footprint test it stands for.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nav_internal.h"
#include "nav_policy.h"

using namespace flashnav;

namespace {

struct DevArena {
    std::vector<void *> ptrs;
    ~DevArena() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T> cudaError_t alloc(T **out, size_t count) {
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        *out = static_cast<T *>(p);
        return cudaSuccess;
    }
    template <class T> cudaError_t upload(T **out, const std::vector<T> &v) {
        cudaError_t e = alloc(out, v.size());
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
};

struct CsHost {
    std::vector<int> spawn, spawn_comp, comp_start, comp_count, comp_cells;
};

// Cells of row j met by the open disc (xc, yc, rc) in cell units.
bool disc_row_host(float xc, float yc, float rc, int j, int &i0, int &i1) {
    const float fj = (float)j;
    float dy = 0.0f;
    if (yc < fj) dy = fj - yc;
    else if (yc > fj + 1.0f) dy = yc - (fj + 1.0f);
    if (!(dy < rc)) return false;
    const float hh = std::sqrt(rc * rc - dy * dy);
    i0 = (int)std::floor(xc - hh);
    i1 = (int)std::ceil(xc + hh) - 1;
    return true;
}

// Spawnable cells: the circumscribed disc of the footprint at the cell centre
// meets no blocked cell.  Components are 4-connected sets of spawnable cells;
// goals are drawn from the spawn cell's component.  Row prefix counts make
// each row-span test O(1).
void build_cspace(const uint8_t *occ, int W, int H, float res, float inv_res, float rcirc_m,
                  CsHost &cs) {
    std::vector<int> pref((size_t)H * (W + 1), 0);
    for (int j = 0; j < H; ++j) {
        int *p = &pref[(size_t)j * (W + 1)];
        for (int i = 0; i < W; ++i) p[i + 1] = p[i] + (occ[(size_t)j * W + i] != 0);
    }
    const float rc = rcirc_m * inv_res;
    std::vector<uint8_t> ok((size_t)W * H, 0);
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            const float xc = (((float)i + 0.5f) * res) * inv_res;
            const float yc = (((float)j + 0.5f) * res) * inv_res;
            const int r0 = (int)std::floor(yc - rc);
            const int r1 = (int)std::ceil(yc + rc) - 1;
            bool blocked = false;
            for (int r = r0; r <= r1 && !blocked; ++r) {
                int a, b;
                if (!disc_row_host(xc, yc, rc, r, a, b) || a > b) continue;
                if (r < 0 || r >= H || a < 0 || b >= W) blocked = true;
                else blocked = pref[(size_t)r * (W + 1) + b + 1] - pref[(size_t)r * (W + 1) + a] > 0;
            }
            ok[(size_t)j * W + i] = !blocked;
        }
    std::vector<int> comp((size_t)W * H, -1);
    std::vector<int> stack;
    int ncomp = 0;
    for (size_t c0 = 0; c0 < ok.size(); ++c0) {
        if (!ok[c0]) continue;
        cs.spawn.push_back((int)c0);
        if (comp[c0] >= 0) continue;
        comp[c0] = ncomp;
        stack.assign(1, (int)c0);
        while (!stack.empty()) {
            const int c = stack.back();
            stack.pop_back();
            const int ci = c % W, cj = c / W;
            const int nb[4] = {ci > 0 ? c - 1 : -1, ci + 1 < W ? c + 1 : -1, cj > 0 ? c - W : -1,
                               cj + 1 < H ? c + W : -1};
            for (int t = 0; t < 4; ++t)
                if (nb[t] >= 0 && ok[nb[t]] && comp[nb[t]] < 0) {
                    comp[nb[t]] = ncomp;
                    stack.push_back(nb[t]);
                }
        }
        ++ncomp;
    }
    cs.comp_count.assign(ncomp, 0);
    for (int c : cs.spawn) cs.comp_count[comp[c]]++;
    cs.comp_start.assign(ncomp, 0);
    for (int k = 1; k < ncomp; ++k) cs.comp_start[k] = cs.comp_start[k - 1] + cs.comp_count[k - 1];
    cs.comp_cells.assign(cs.spawn.size(), 0);
    std::vector<int> fill(ncomp, 0);
    cs.spawn_comp.resize(cs.spawn.size());
    for (size_t s = 0; s < cs.spawn.size(); ++s) {
        const int id = comp[cs.spawn[s]];
        cs.spawn_comp[s] = id;
        cs.comp_cells[cs.comp_start[id] + fill[id]++] = cs.spawn[s];
    }
}

float circ_radius(const nav_robot &r) {
    if (r.shape == 0) return r.radius;
    return 0.5f * std::sqrt(r.length * r.length + r.width * r.width);
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

} // namespace

struct nav_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_envs = 0, n_maps = 0, n_robots = 0, max_k = 0;
    float max_range = 0.0f;
    nav_params par{};
    std::vector<int64_t> obs_off, ray_off;
    std::vector<int> env_map, env_tab, env_k;
    std::vector<MapDev> maps;
    std::vector<float> map_ray_cost; // mean cells per ray of a host sample, per map
    LaunchCfg cfg;
    int smem_map_bytes = 160 * 1024;
    int byte_cells = 1;
    MapDev *d_maps = nullptr;
    int debug = 0, stats = 0;
    uint64_t seed = 0;
    std::string err;
    DevArena arena;
    StepArgs a{};
    TileDev *d_tiles = nullptr;
    int *d_perm = nullptr;
    int tiles_cap = 0;
    int *d_tile_env = nullptr; // [tile][kMaxTileEnvs]: the envs of each tile (-1 past its count)
    int tile_env_cap = 0;
    std::vector<TileDev> tiles_host;  // the main tiles, in queue order
    int4 *d_tile_stage = nullptr;     // [tile] how its map is staged (refresh_tile_stage)
    int tile_stage_cap = 0;
    unsigned long long *d_stats = nullptr;
    int2 *d_chunks = nullptr;
    int chunks_cap = 0;
    bool split_ok = false; // every map (and beam table) fits in one CTA's shared memory
    float *d_dbg_range = nullptr;
    int *d_dbg_hit = nullptr;
    unsigned *d_dbg_vis = nullptr;
    // state snapshot (autotuner), graph, tuning buffers
    float *snap = nullptr;
    cudaGraphExec_t graph = nullptr;
    float *tune_act = nullptr, *tune_obs = nullptr, *tune_rew = nullptr;
    unsigned char *tune_flush = nullptr; // written between the autotuner's final timings
    unsigned char *tune_done = nullptr;
    // nav_step_host staging
    float *h_act = nullptr, *h_obs = nullptr, *h_rew = nullptr, *h_fin = nullptr;
    unsigned char *h_done = nullptr;
    // nav_step_host pipeline: the step runs as host_parts launches over env
    // ranges, each part's results copied out while the next part computes
    int host_parts = 3; // 4096 envs: 171.5 us per call against 177.9 (2) and 195.0 (1)
    TileDev *d_ptiles = nullptr; // tiles of every part, part p at part_tile_off[p]
    int *d_pperm = nullptr;      // envs ordered by (part, map, beam table)
    int ptiles_cap = 0;
    std::vector<int> part_tile_off, part_env_off;
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> part_ev;
    // fused act-step rollout: tiles of up to 128 envs
    TileDev *d_act_tiles = nullptr;
    int act_tiles_cap = 0, act_n_tiles = 0, act_tile_envs = 0;
    unsigned char *d_act_w = nullptr; // the actor's weight units (swizzled copy)
    size_t act_w_cap = 0;
};

namespace {

int fail(nav_handle *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(nav_handle *h, cudaError_t e, const char *what) {
    return fail(h, NAV_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Chessboard distance of every cell of a padded map (rows of `stride`
// bytes, map cell (i, j) at row j + kPad, column i + kPad) to the nearest
// blocked cell, padding included, capped at 255: two raster passes with
// the unit 3x3 mask (Rosenfeld & Pfaltz, 1966), exact for this metric.
void chessboard_distance(const nav_map &mp, int stride, uint8_t *out) {
    const int rows = mp.height + 2 * kPad, cols = mp.width + 2 * kPad;
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < stride; ++c) {
            const int i = c - kPad, j = r - kPad;
            const bool free = c < cols && i >= 0 && j >= 0 && i < mp.width && j < mp.height &&
                              !mp.occ[(size_t)j * mp.width + i];
            out[(size_t)r * stride + c] = free ? 255 : 0;
        }
    auto at = [&](int r, int c) -> uint8_t & { return out[(size_t)r * stride + c]; };
    // free cells lie strictly inside the padding ring, so every neighbour exists
    for (int r = kPad; r < rows - kPad; ++r)
        for (int c = kPad; c < cols - kPad; ++c) {
            if (!at(r, c)) continue;
            int v = std::min({(int)at(r, c - 1), (int)at(r - 1, c - 1), (int)at(r - 1, c),
                              (int)at(r - 1, c + 1)}) + 1;
            at(r, c) = (uint8_t)std::min(v, (int)at(r, c));
        }
    for (int r = rows - kPad - 1; r >= kPad; --r)
        for (int c = cols - kPad - 1; c >= kPad; --c) {
            if (!at(r, c)) continue;
            int v = std::min({(int)at(r, c + 1), (int)at(r + 1, c + 1), (int)at(r + 1, c),
                              (int)at(r + 1, c - 1)}) + 1;
            at(r, c) = (uint8_t)std::min(v, (int)at(r, c));
        }
}

// Relative cost of one ray on this map, in iterations of the ray loop, over
// a fixed sample of rays from free cells in seeded directions: a fixed
// per-ray part (set-up, result, refill: about as much as kRayFixedIters
// iterations, measured with rays cut to one cell) plus the iterations of
// the walk to a blocked cell, the map edge or r_max.  With distance bytes
// (dist, rows of `stride` bytes, padded like the device copy) an iteration
// at a cell of distance d >= 2 covers the next d - 1 boundaries of the
// ray's major axis, as the device's jumps do; without, every cell is one.
constexpr double kRayFixedIters = 8.0;

float sample_ray_cost(const nav_map &mp, float rmax_c, const uint8_t *dist, int stride) {
    const int W = mp.width, H = mp.height;
    auto blocked = [&](int i, int j) {
        return i < 0 || j < 0 || i >= W || j >= H || mp.occ[(size_t)j * W + i] != 0;
    };
    unsigned long long z = 0x2545F4914F6CDD1Dull ^ ((unsigned long long)W << 32) ^ (unsigned)H;
    auto next = [&]() {
        z ^= z << 13;
        z ^= z >> 7;
        z ^= z << 17;
        return z;
    };
    double total = 0.0;
    int n = 0;
    for (int tries = 0; tries < 16384 && n < 1024; ++tries) {
        const int i0 = (int)(next() % (unsigned long long)W), j0 = (int)(next() % (unsigned long long)H);
        if (blocked(i0, j0)) continue;
        const double a = (double)(next() >> 11) * (6.283185307179586 / 9007199254740992.0);
        const double dx = std::cos(a), dy = std::sin(a);
        const bool xmaj = std::fabs(dx) >= std::fabs(dy);
        double x = i0 + 0.5, y = j0 + 0.5;
        int i = i0, j = j0;
        const int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1;
        const double tdx = dx != 0 ? std::fabs(1.0 / dx) : 1e30, tdy = dy != 0 ? std::fabs(1.0 / dy) : 1e30;
        double tx = dx > 0 ? (i + 1 - x) * tdx : dx < 0 ? (x - i) * tdx : 1e30;
        double ty = dy > 0 ? (j + 1 - y) * tdy : dy < 0 ? (y - j) * tdy : 1e30;
        // cover: the major-axis count at which the current jump ends; -1: the
        // next cell starts an iteration; -2: a single step is under way
        int iters = 0, major = 0, cover = -1;
        for (;;) {
            if (cover == -1 || (cover >= 0 && major >= cover)) {
                ++iters;
                const int d = dist ? dist[(size_t)(j + kPad) * stride + (i + kPad)] : 1;
                cover = d >= 2 ? major + d - 1 : -2;
            }
            const double t = std::min(tx, ty);
            if (t > rmax_c) break;
            const bool stepx = tx <= ty;
            if (stepx) { i += sx; tx += tdx; } else { j += sy; ty += tdy; }
            if (stepx == xmaj) ++major;
            if (cover == -2) cover = -1;
            if (blocked(i, j)) break;
        }
        total += kRayFixedIters + iters;
        ++n;
    }
    return n ? (float)(total / n) : 1.0f;
}

// One step (or reset) of the envs that A covers, on the kernel the handle's
// launch configuration selects.
int launch_args(nav_handle *h, const StepArgs &A) {
    if (h->cfg.split && h->split_ok) return launch_step_split(A, h->n_envs, h->stream);
    return launch_step(A, h->cfg, h->stream);
}

// Sizes of the (map, beam table) groups of the handle's envs.
std::vector<int> group_sizes(const nav_handle *h) {
    std::vector<std::pair<int, int>> keys;
    for (int e = 0; e < h->n_envs; ++e) keys.push_back({h->env_map[e], h->env_tab[e]});
    std::sort(keys.begin(), keys.end());
    std::vector<int> n;
    for (size_t i = 0; i < keys.size(); ++i)
        if (i == 0 || keys[i] != keys[i - 1]) n.push_back(1);
        else ++n.back();
    return n;
}

// The smallest tile size (<= te_max) whose balanced tiles (cut_group) number
// at most `slots` (whole waves of resident CTAs), else -1.
int fit_tile(const nav_handle *h, long long slots, int te_max) {
    const std::vector<int> n = group_sizes(h);
    for (int te = 1; te <= te_max; ++te) {
        long long tiles = 0;
        for (int g : n) tiles += (g + te - 1) / te;
        if (tiles <= slots) return te;
    }
    return -1;
}

// Cuts the envs perm[s, t) of one (map, beam table) group into
// ceil((t - s) / te) tiles of nearly equal size (sizes differ by at most
// one), so that no tile is a small remainder.
void cut_group_n(int s, int t, int k, int map, int tab, std::vector<TileDev> &out) {
    const int n = t - s;
    for (int i = 0; i < k; ++i) {
        const int b = s + (int)((long long)n * i / k), e = s + (int)((long long)n * (i + 1) / k);
        out.push_back(TileDev{map, tab, b, e - b});
    }
}

void cut_group(int s, int t, int te, int map, int tab, std::vector<TileDev> &out) {
    cut_group_n(s, t, (t - s + te - 1) / te, map, tab, out);
}

// Tiles per (map, beam table) group: `total` tiles in all, shared out in
// proportion to each group's sampled ray cost (envs x beams x cost per ray
// on its map), so that the tiles of cheap and dear maps take about equal
// time; each group gets at least ceil(n_g / kMaxTileEnvs) and at most n_g
// tiles.
std::vector<int> weighted_tile_counts(const nav_handle *h, const std::vector<int> &perm,
                                      const std::vector<std::pair<int, int>> &groups,
                                      long long total) {
    const size_t G = groups.size();
    std::vector<int> k(G), lo(G), hi(G);
    std::vector<double> want(G);
    double cost = 0.0;
    for (size_t g = 0; g < G; ++g) {
        const int n = groups[g].second - groups[g].first;
        const int e = perm[groups[g].first];
        want[g] = (double)n * h->env_k[e] * h->map_ray_cost[h->env_map[e]];
        cost += want[g];
        lo[g] = (n + kMaxTileEnvs - 1) / kMaxTileEnvs;
        hi[g] = n;
    }
    long long used = 0;
    std::vector<std::pair<double, int>> frac;
    for (size_t g = 0; g < G; ++g) {
        want[g] = want[g] / cost * (double)total;
        k[g] = std::min(hi[g], std::max(lo[g], (int)std::floor(want[g])));
        used += k[g];
        frac.push_back({want[g] - std::floor(want[g]), (int)g});
    }
    std::stable_sort(frac.begin(), frac.end(),
                     [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
                         return a.first > b.first;
                     });
    for (size_t r = 0; used < total && r < 4 * G + 4; ++r) {
        const int g = frac[r % G].second;
        if (k[g] < hi[g]) {
            ++k[g];
            ++used;
        }
    }
    return k;
}

// Groups envs by (map, beam table) and cuts each group into nearly equal
// tiles, as many per group as weighted_tile_counts gives (tile_envs sets
// their number).  The queue runs over the largest tiles first so that the
// longest CTAs start early: by map size x beams (order 0, ties in map order)
// or by envs x beams x sampled cells per ray (order 1, ties by map size).
int refresh_tile_stage(nav_handle *h);

int build_tiles(nav_handle *h) {
    const int E = h->n_envs;
    std::vector<int> perm(E);
    for (int e = 0; e < E; ++e) perm[e] = e;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        const long long ka = (long long)h->env_map[a] * 4096 + h->env_tab[a];
        const long long kb = (long long)h->env_map[b] * 4096 + h->env_tab[b];
        return ka < kb;
    });
    std::vector<TileDev> tiles;
    std::vector<std::pair<int, int>> groups;
    for (int s = 0; s < E;) {
        int t = s;
        while (t < E && h->env_map[perm[t]] == h->env_map[perm[s]] &&
               h->env_tab[perm[t]] == h->env_tab[perm[s]])
            ++t;
        groups.push_back({s, t});
        s = t;
    }
    // as many tiles in all as tiles of at most tile_envs envs make; a count
    // just short of one wave of resident CTAs (within 10 %) is raised to
    // the full wave, so that no SM holds fewer tiles than the others (the
    // tiles shrink a little instead)
    long long total = 0;
    for (const auto &gr : groups)
        total += (gr.second - gr.first + h->cfg.tile_envs - 1) / h->cfg.tile_envs;
    if (h->par.n_dyn == 0 && !(h->cfg.split && h->split_ok)) {
        const long long R = step_resident(h->a, h->cfg);
        if (R > 0 && total < R && 10 * total >= 9 * R) total = std::min<long long>(R, E);
    }
    const std::vector<int> counts = weighted_tile_counts(h, perm, groups, total);
    for (size_t g = 0; g < groups.size(); ++g) {
        const int s = groups[g].first;
        cut_group_n(s, groups[g].second, counts[g], h->env_map[perm[s]], h->env_tab[perm[s]],
                    tiles);
    }
    std::stable_sort(tiles.begin(), tiles.end(), [&](const TileDev &x, const TileDev &y) {
        const long long wx = (long long)h->maps[x.map].n_words * h->env_k[perm[x.env_begin]];
        const long long wy = (long long)h->maps[y.map].n_words * h->env_k[perm[y.env_begin]];
        if (h->cfg.order == 1) {
            const double cx = (double)x.env_count * h->env_k[perm[x.env_begin]] * h->map_ray_cost[x.map];
            const double cy = (double)y.env_count * h->env_k[perm[y.env_begin]] * h->map_ray_cost[y.map];
            if (cx != cy) return cx > cy;
        }
        return wx > wy;
    });
    cudaError_t e;
    if ((int)tiles.size() > h->tiles_cap) {
        e = h->arena.alloc(&h->d_tiles, tiles.size());
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(tiles)");
        h->tiles_cap = (int)tiles.size();
    }
    if (!h->d_perm) {
        e = h->arena.alloc(&h->d_perm, (size_t)E);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(perm)");
    }
    // each tile's envs at a fixed stride, so that a CTA reads them with its
    // tile record instead of after it (one dependent load less per tile)
    std::vector<int> tile_env(tiles.size() * kMaxTileEnvs, -1);
    for (size_t t = 0; t < tiles.size(); ++t)
        for (int i = 0; i < tiles[t].env_count; ++i)
            tile_env[t * kMaxTileEnvs + i] = perm[tiles[t].env_begin + i];
    if ((int)tiles.size() > h->tile_env_cap) {
        e = h->arena.alloc(&h->d_tile_env, tile_env.size());
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(tile envs)");
        h->tile_env_cap = (int)tiles.size();
    }
    e = cudaMemcpy(h->d_tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_perm, perm.data(), (size_t)E * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_tile_env, tile_env.data(), tile_env.size() * sizeof(int),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(tiles)");
    h->a.tiles = h->d_tiles;
    h->a.perm = h->d_perm;
    h->a.tile_env = h->d_tile_env;
    h->tiles_host = tiles;
    {
        const int rs = refresh_tile_stage(h);
        if (rs != NAV_OK) return rs;
    }
    h->a.n_tiles = (int)tiles.size();
    h->a.max_tile_envs = 1;
    for (const TileDev &t : tiles) h->a.max_tile_envs = std::max(h->a.max_tile_envs, t.env_count);
    // tiles of the host-step pipeline: the same grouping within each env range
    std::vector<int> pperm;
    {
        const int P = std::max(1, std::min(h->host_parts, E));
        // smaller tiles keep each part's launch as wide as the whole step's
        const int pt = std::max(1, (h->cfg.tile_envs + P - 1) / P);
        std::vector<TileDev> ptiles;
        h->part_tile_off.assign(1, 0);
        h->part_env_off.assign(1, 0);
        for (int p = 0; p < P; ++p) {
            const int e0 = (int)((long long)E * p / P), e1 = (int)((long long)E * (p + 1) / P);
            const int base = (int)pperm.size();
            for (int e = e0; e < e1; ++e) pperm.push_back(e);
            std::stable_sort(pperm.begin() + base, pperm.end(), [&](int a, int b) {
                const long long ka = (long long)h->env_map[a] * 4096 + h->env_tab[a];
                const long long kb = (long long)h->env_map[b] * 4096 + h->env_tab[b];
                return ka < kb;
            });
            const size_t t0 = ptiles.size();
            int q = base;
            while (q < (int)pperm.size()) {
                int r = q;
                while (r < (int)pperm.size() && h->env_map[pperm[r]] == h->env_map[pperm[q]] &&
                       h->env_tab[pperm[r]] == h->env_tab[pperm[q]])
                    ++r;
                cut_group(q, r, pt, h->env_map[pperm[q]], h->env_tab[pperm[q]], ptiles);
                q = r;
            }
            std::stable_sort(ptiles.begin() + t0, ptiles.end(), [&](const TileDev &x, const TileDev &y) {
                const long long wx = (long long)h->maps[x.map].n_words * h->env_k[pperm[x.env_begin]];
                const long long wy = (long long)h->maps[y.map].n_words * h->env_k[pperm[y.env_begin]];
                return wx > wy;
            });
            for (size_t i = t0; i < ptiles.size(); ++i)
                h->a.max_tile_envs = std::max(h->a.max_tile_envs, ptiles[i].env_count);
            h->part_tile_off.push_back((int)ptiles.size());
            h->part_env_off.push_back(e1);
        }
        if ((int)ptiles.size() > h->ptiles_cap) {
            e = h->arena.alloc(&h->d_ptiles, ptiles.size());
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(part tiles)");
            h->ptiles_cap = (int)ptiles.size();
        }
        if (!h->d_pperm) {
            e = h->arena.alloc(&h->d_pperm, (size_t)E);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(part perm)");
        }
        e = cudaMemcpy(h->d_ptiles, ptiles.data(), ptiles.size() * sizeof(TileDev),
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->d_pperm, pperm.data(), (size_t)E * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(part tiles)");
    }
    // 32-ray chunks of every tile for the split step
    std::vector<int2> chunks;
    for (size_t t = 0; t < tiles.size(); ++t) {
        const int n = tiles[t].env_count * h->env_k[perm[tiles[t].env_begin]];
        for (int r = 0; r < n; r += 32) chunks.push_back(make_int2((int)t, r));
    }
    if ((int)chunks.size() > h->chunks_cap) {
        e = h->arena.alloc(&h->d_chunks, chunks.size());
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(chunks)");
        h->chunks_cap = (int)chunks.size();
    }
    e = cudaMemcpy(h->d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(chunks)");
    h->a.chunks = h->d_chunks;
    h->a.n_chunks = (int)chunks.size();
    return NAV_OK;
}

// Chooses each map's staging under the shared-memory cap.  byte_cells 1:
// distance bytes, in shared memory when they fit, else through L1/L2;
// 2: packed bits, in shared memory when they fit, else through L1/L2;
// 3: distance bytes in shared memory when they fit, else packed bits in
// shared memory when they fit, else distance bytes through L1/L2.  Maps
// without distance bytes use packed bits.  The shared region is sized for
// the largest staged map.
// Per main tile, how its map is staged, so that a CTA starts the copy from
// the tile's own record instead of after a second load of the map's:
// {map mode, bytes to copy, byte offset into the bitmap or distance-byte
// buffer (low, high 32 bits)}.  Rebuilt whenever tiles or map modes change.
int refresh_tile_stage(nav_handle *h) {
    const size_t n = h->tiles_host.size();
    if (n == 0) return NAV_OK;
    std::vector<int4> st(n);
    for (size_t t = 0; t < n; ++t) {
        const MapDev &m = h->maps[h->tiles_host[t].map];
        long long off = 0;
        int bytes = 0;
        if (m.mode == kMapSharedBits) {
            off = m.word_off * 4;
            bytes = m.n_words * 4;
        } else if (m.mode == kMapSharedBytes) {
            off = m.dist_off;
            bytes = m.n_bytes;
        }
        st[t] = make_int4(m.mode, bytes, (int)(off & 0xffffffffll), (int)(off >> 32));
    }
    cudaError_t e = cudaSuccess;
    if ((int)n > h->tile_stage_cap) {
        e = h->arena.alloc(&h->d_tile_stage, n);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(tile stage)");
        h->tile_stage_cap = (int)n;
    }
    e = cudaMemcpy(h->d_tile_stage, st.data(), n * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(tile stage)");
    h->a.tile_stage = h->d_tile_stage;
    return NAV_OK;
}

int set_map_modes(nav_handle *h) {
    int region = 0;
    for (MapDev &m : h->maps) {
        const bool dist = m.dist_off >= 0 && h->byte_cells != 2;
        const bool bytes_fit = m.n_bytes <= h->smem_map_bytes;
        const bool bits_fit = m.n_words * 4 <= h->smem_map_bytes;
        if (dist && bytes_fit) m.mode = kMapSharedBytes;
        else if (dist && h->byte_cells == 1) m.mode = kMapGlobalBytes;
        else if (bits_fit) m.mode = kMapSharedBits;
        else m.mode = dist ? kMapGlobalBytes : kMapGlobal;
        const int need = m.mode == kMapSharedBytes ? m.n_bytes
                         : m.mode == kMapSharedBits ? m.n_words * 4 : 0;
        region = std::max(region, need);
    }
    h->a.smem_region_bytes = region;
    if (h->d_maps) {
        cudaError_t e = cudaMemcpy(h->d_maps, h->maps.data(), h->maps.size() * sizeof(MapDev),
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(maps)");
    }
    return refresh_tile_stage(h);
}

int launch(nav_handle *h) {
    const int rc = launch_args(h, h->a);
    if (rc != 0) return cuda_fail(h, (cudaError_t)rc, "step kernel launch");
    return NAV_OK;
}

} // namespace

namespace flashnav {

int handle_view(const nav_handle *h, HandleView *out) {
    if (!h || !out) return NAV_E_INVAL;
    out->device = h->device;
    out->stream = h->stream;
    out->n_envs = h->n_envs;
    out->obs_floats = h->obs_off.back();
    out->uniform_d = h->env_k.empty() ? -1 : h->env_k[0];
    for (int k : h->env_k)
        if (k != out->uniform_d) out->uniform_d = -1;
    if (h->par.n_sectors > 0) out->uniform_d = h->par.n_sectors;
    return NAV_OK;
}

int handle_fail(nav_handle *h, int code, const char *msg) { return fail(h, code, msg); }

} // namespace flashnav

extern "C" {

void nav_default_params(nav_params *p) {
    if (!p) return;
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

int nav_create_ex(const nav_map *maps, int n_maps, const int *env_map, const int *env_beams,
                  const int *env_robot, int n_envs, float max_range, const nav_robot *robots,
                  int n_robots, const nav_params *params, nav_handle **out) {
    if (!out) return NAV_E_INVAL;
    *out = nullptr;
    if (!maps || n_maps <= 0 || !env_beams || n_envs <= 0 || !robots || n_robots <= 0 ||
        !finite_pos(max_range))
        return NAV_E_INVAL;
    nav_handle *h = new (std::nothrow) nav_handle();
    if (!h) return NAV_E_NOMEM;
    auto bail = [&](int code) {
        if (code != NAV_OK) {
            // keep the message for the caller only through stderr: the handle dies
            std::fprintf(stderr, "nav_create: %s\n", h->err.c_str());
            delete h;
        }
        return code;
    };
    h->n_envs = n_envs;
    h->n_maps = n_maps;
    h->n_robots = n_robots;
    h->max_range = max_range;
    if (params) h->par = *params;
    else nav_default_params(&h->par);
    const nav_params &P = h->par;
    if (!finite_pos(P.dt) || !(P.goal_tol >= 0.0f) || P.horizon <= 0 || P.n_dyn < 0 ||
        P.n_dyn > kMaxDyn || !finite_pos(P.fov_deg) || P.fov_deg > 360.0f ||
        !(P.goal_dmin <= P.goal_dmax) || (P.reward_mode != 0 && P.reward_mode != 1))
        return bail(fail(h, NAV_E_INVAL, "bad nav_params"));
    if (P.n_dyn > 0 && (!finite_pos(P.dyn_radius) || !(P.dyn_speed_max >= 0.0f)))
        return bail(fail(h, NAV_E_INVAL, "bad moving-disc parameters"));
    if ((P.sensor != 0 && P.sensor != 1) || P.n_sectors < 0 || P.n_sectors > kMaxBeams)
        return bail(fail(h, NAV_E_INVAL, "bad sensor or n_sectors"));
    if (P.sensor == 1 && (!finite_pos(P.march_step) ||
                          (double)max_range / (double)P.march_step > (double)(1 << 22)))
        return bail(fail(h, NAV_E_INVAL, "march_step must be > 0 with max_range / step <= 2^22"));
    for (int r = 0; r < n_robots; ++r) {
        const nav_robot &rb = robots[r];
        const bool shape_ok = (rb.shape == 0 && finite_pos(rb.radius)) ||
                              (rb.shape == 1 && finite_pos(rb.length) && finite_pos(rb.width));
        if (!shape_ok || !(rb.v_min <= rb.v_max) || !(rb.w_min <= rb.w_max) ||
            !std::isfinite(rb.v_min) || !std::isfinite(rb.v_max) || !std::isfinite(rb.w_min) ||
            !std::isfinite(rb.w_max))
            return bail(fail(h, NAV_E_INVAL, "bad nav_robot " + std::to_string(r)));
    }
    // maps: validate and pack (free bits, one blocked padding cell per side;
    // distance bytes for maps small enough to be staged as bytes)
    std::vector<uint32_t> words;
    std::vector<uint8_t> dist_all;
    for (int m = 0; m < n_maps; ++m) {
        const nav_map &mp = maps[m];
        if (!mp.occ || mp.width <= 0 || mp.height <= 0 || mp.width > 16384 || mp.height > 16384 ||
            !finite_pos(mp.resolution))
            return bail(fail(h, NAV_E_INVAL, "bad nav_map " + std::to_string(m)));
        if (max_range / mp.resolution > 65536.0f)
            return bail(fail(h, NAV_E_INVAL, "max_range spans more than 65536 cells"));
        if (P.n_dyn > 0 &&
            std::ceil(2.0f * P.dyn_radius / mp.resolution) + 1.0f > (float)kMaxDynRows)
            return bail(fail(h, NAV_E_INVAL, "dyn_radius too large for the map resolution"));
        MapDev md;
        md.w = mp.width;
        md.h = mp.height;
        int pitch = (mp.width + 2 * kPad + 31) / 32;
        if ((pitch & 1) == 0) pitch += 1;
        md.pitch = pitch;
        const long long nw = (long long)(mp.height + 2 * kPad) * pitch;
        int bstride = (mp.width + 2 * kPad + 3) / 4 * 4;
        if (((bstride / 4) & 1) == 0) bstride += 4;
        md.byte_stride = bstride;
        const long long nb = (long long)(mp.height + 2 * kPad) * bstride;
        md.n_bytes = nb > (1 << 30) ? (1 << 30) : (int)((nb + 15) / 16 * 16);
        md.mode = kMapGlobal;
        md.n_words = (int)((nw + 3) / 4 * 4);
        md.word_off = (long long)words.size();
        md.res = mp.resolution;
        md.inv_res = (float)(1.0 / (double)mp.resolution);
        words.resize(words.size() + md.n_words, 0u);
        uint32_t *base = words.data() + md.word_off;
        for (int j = 0; j < mp.height; ++j)
            for (int i = 0; i < mp.width; ++i)
                if (!mp.occ[(size_t)j * mp.width + i]) {
                    const long long b = (long long)(j + kPad) * pitch * 32 + (i + kPad);
                    base[b >> 5] |= 1u << (b & 31);
                }
        md.all_off = 0;
        md.dist_off = -1;
        if (nb <= kMaxDistBytes) {
            md.dist_off = (long long)dist_all.size();
            dist_all.resize(dist_all.size() + md.n_bytes, 0);
            chessboard_distance(mp, bstride, dist_all.data() + md.dist_off);
        }
        h->maps.push_back(md);
        h->map_ray_cost.push_back(sample_ray_cost(
            mp, max_range * md.inv_res,
            md.dist_off >= 0 ? dist_all.data() + md.dist_off : nullptr, bstride));
    }
    // envs
    h->env_map.resize(n_envs);
    h->env_k.resize(n_envs);
    h->env_tab.resize(n_envs);
    std::vector<int> env_robot_v(n_envs), env_cs(n_envs);
    h->obs_off.assign(n_envs + 1, 0);
    h->ray_off.assign(n_envs + 1, 0);
    std::vector<int> tab_k;
    for (int e = 0; e < n_envs; ++e) {
        const int m = env_map ? env_map[e] : e % n_maps;
        const int k = env_beams[e];
        const int r = env_robot ? env_robot[e] : 0;
        if (m < 0 || m >= n_maps || k <= 0 || k > kMaxBeams || r < 0 || r >= n_robots)
            return bail(fail(h, NAV_E_INVAL, "bad per-env entry at env " + std::to_string(e)));
        if (P.n_sectors > 0 && k % P.n_sectors != 0)
            return bail(fail(h, NAV_E_INVAL, "beam count not a multiple of n_sectors at env " +
                                                 std::to_string(e)));
        h->env_map[e] = m;
        h->env_k[e] = k;
        env_robot_v[e] = r;
        int t = (int)(std::find(tab_k.begin(), tab_k.end(), k) - tab_k.begin());
        if (t == (int)tab_k.size()) tab_k.push_back(k);
        h->env_tab[e] = t;
        h->max_k = std::max(h->max_k, k);
        h->obs_off[e + 1] = h->obs_off[e] + (P.n_sectors > 0 ? P.n_sectors : k) + 4;
        h->ray_off[e + 1] = h->ray_off[e] + k;
    }
    // every map side by side in one shared-memory region (split step)
    {
        long long off = 0;
        for (MapDev &m : h->maps) {
            m.all_off = (int)std::min<long long>(off, 1 << 30);
            off += m.n_words;
        }
        h->a.all_words = (int)std::min<long long>(off, 1 << 30);
        h->a.n_maps_split = n_maps;
    }
    // beam tables: alpha_k = -FOV/2 + (k + 1/2) FOV / K, cos and sin in binary64
    // rounded to binary32 (Eq. 4)
    std::vector<float> beam_c, beam_s;
    std::vector<int> tab_off;
    h->a.n_beams_total = 0;
    const double fov = (double)P.fov_deg * (3.14159265358979323846 / 180.0);
    for (int K : tab_k) {
        tab_off.push_back((int)beam_c.size());
        for (int k = 0; k < K; ++k) {
            const double a = -0.5 * fov + ((double)k + 0.5) * fov / (double)K;
            beam_c.push_back((float)std::cos(a));
            beam_s.push_back((float)std::sin(a));
        }
    }
    // spawn tables per used (map, robot)
    std::vector<CsDev> cs_dev;
    std::vector<int> spawn, spawn_comp, comp_start, comp_count, comp_cells;
    std::vector<int> cs_index((size_t)n_maps * n_robots, -1);
    for (int e = 0; e < n_envs; ++e) {
        const size_t key = (size_t)h->env_map[e] * n_robots + env_robot_v[e];
        if (cs_index[key] < 0) {
            const int m = h->env_map[e];
            const MapDev &md = h->maps[m];
            CsHost c;
            build_cspace(maps[m].occ, md.w, md.h, md.res, md.inv_res,
                         circ_radius(robots[env_robot_v[e]]), c);
            if (c.spawn.empty()) {
                fail(h, NAV_E_NOSPAWN,
                     "map " + std::to_string(m) + " has no cell where robot " +
                         std::to_string(env_robot_v[e]) + " fits");
                return bail(NAV_E_NOSPAWN);
            }
            CsDev d;
            d.n_spawn = (int)c.spawn.size();
            d.spawn_off = (int)spawn.size();
            d.comp_off = (int)comp_start.size();
            d.cells_off = (int)comp_cells.size();
            spawn.insert(spawn.end(), c.spawn.begin(), c.spawn.end());
            spawn_comp.insert(spawn_comp.end(), c.spawn_comp.begin(), c.spawn_comp.end());
            comp_start.insert(comp_start.end(), c.comp_start.begin(), c.comp_start.end());
            comp_count.insert(comp_count.end(), c.comp_count.begin(), c.comp_count.end());
            comp_cells.insert(comp_cells.end(), c.comp_cells.begin(), c.comp_cells.end());
            cs_index[key] = (int)cs_dev.size();
            cs_dev.push_back(d);
        }
        env_cs[e] = cs_index[key];
    }
    std::vector<RobotDev> rdev(n_robots);
    for (int r = 0; r < n_robots; ++r) {
        rdev[r] = RobotDev{robots[r].shape, robots[r].radius, robots[r].length, robots[r].width,
                           robots[r].v_min, robots[r].v_max, robots[r].w_min, robots[r].w_max};
    }
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaGetDevice"));
    StepArgs &A = h->a;
    std::vector<long long> obs_off_ll(h->obs_off.begin(), h->obs_off.end());
    std::vector<long long> ray_off_ll(h->ray_off.begin(), h->ray_off.end());
    uint32_t *bits;
    uint8_t *d_dist = nullptr;
    MapDev *d_maps;
    CsDev *d_cs;
    RobotDev *d_rob, *d_env_rb;
    int *d_spawn, *d_spawn_comp, *d_comp_start, *d_comp_count, *d_comp_cells, *d_tab_off, *d_tab_k;
    int *d_env_map, *d_env_tab, *d_env_robot, *d_env_cs;
    float *d_bc, *d_bs;
    long long *d_obs_off, *d_ray_off;
#define NAV_UP(ptr, vec)                                                          \
    do {                                                                          \
        ce = h->arena.upload(&ptr, vec);                                          \
        if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "upload " #vec));     \
    } while (0)
    NAV_UP(bits, words);
    if (!dist_all.empty()) NAV_UP(d_dist, dist_all);
    NAV_UP(d_maps, h->maps);
    h->d_maps = d_maps;
    NAV_UP(d_cs, cs_dev);
    NAV_UP(d_rob, rdev);
    std::vector<RobotDev> env_rb(h->n_envs);
    for (int e = 0; e < h->n_envs; ++e) env_rb[e] = rdev[env_robot_v[e]];
    NAV_UP(d_env_rb, env_rb);
    NAV_UP(d_spawn, spawn);
    NAV_UP(d_spawn_comp, spawn_comp);
    NAV_UP(d_comp_start, comp_start);
    NAV_UP(d_comp_count, comp_count);
    NAV_UP(d_comp_cells, comp_cells);
    NAV_UP(d_tab_off, tab_off);
    NAV_UP(d_tab_k, tab_k);
    NAV_UP(d_env_map, h->env_map);
    NAV_UP(d_env_tab, h->env_tab);
    NAV_UP(d_env_robot, env_robot_v);
    NAV_UP(d_env_cs, env_cs);
    h->a.n_beams_total = (int)beam_c.size();
    h->split_ok = P.n_dyn == 0 &&
                  (long long)h->a.all_words * 4 + (long long)beam_c.size() * 8 <= 200 * 1024;
    NAV_UP(d_bc, beam_c);
    NAV_UP(d_bs, beam_s);
    NAV_UP(d_obs_off, obs_off_ll);
    NAV_UP(d_ray_off, ray_off_ll);
#undef NAV_UP
    A.bits = bits;
    A.dist = d_dist;
    A.maps = d_maps;
    A.cs = d_cs;
    A.robots = d_rob;
    A.env_rb = d_env_rb;
    A.spawn = d_spawn;
    A.spawn_comp = d_spawn_comp;
    A.comp_start = d_comp_start;
    A.comp_count = d_comp_count;
    A.comp_cells = d_comp_cells;
    A.tab_off = d_tab_off;
    A.tab_k = d_tab_k;
    A.beam_c = d_bc;
    A.beam_s = d_bs;
    A.env_map = d_env_map;
    A.env_tab = d_env_tab;
    A.env_robot = d_env_robot;
    A.env_cs = d_env_cs;
    A.obs_off = d_obs_off;
    A.ray_off = d_ray_off;
    const size_t E = (size_t)n_envs;
    float *f[8];
    for (int i = 0; i < 8; ++i) {
        ce = h->arena.alloc(&f[i], E);
        if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMalloc(state)"));
        cudaMemset(f[i], 0, E * sizeof(float));
    }
    A.x = f[0]; A.y = f[1]; A.th = f[2]; A.v = f[3]; A.w = f[4];
    A.gx = f[5]; A.gy = f[6]; A.dprev = f[7];
    ce = h->arena.alloc(&A.step, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.episode, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.dyn, E * std::max(P.n_dyn, 1));
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.nxt_pose, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.nxt_goal, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.status, 1);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.tile_queue, 2);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.split_q, 4);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.ray_main, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.ray_fin, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&A.fin_list, E);
    if (ce == cudaSuccess) ce = h->arena.alloc(&h->d_stats, 2);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaMalloc(state)"));
    cudaMemset(A.step, 0, E * sizeof(int));
    cudaMemset(A.episode, 0, E * sizeof(unsigned));
    cudaMemset(A.nxt_pose, 0, E * sizeof(float4));
    cudaMemset(A.nxt_goal, 0, E * sizeof(float2));
    cudaMemset(A.status, 0, sizeof(int));
    cudaMemset(A.tile_queue, 0, 2 * sizeof(int));
    cudaMemset(A.split_q, 0, 4 * sizeof(int));
    cudaMemset(h->d_stats, 0, 2 * sizeof(unsigned long long));
    A.stats = nullptr;
    A.p = ParamsDev{P.dt, P.goal_tol, P.c_progress, P.step_penalty, P.r_goal, P.r_coll,
                    P.horizon, P.goal_dmin, P.goal_dmax, P.n_dyn, P.dyn_radius,
                    P.dyn_speed_max, P.dyn_min_sep, P.reward_mode, P.sensor, P.march_step,
                    P.n_sectors};
    A.max_range = max_range;
    A.max_k = h->max_k;
    int rc = set_map_modes(h);
    if (rc == NAV_OK) rc = build_tiles(h);
    if (rc != NAV_OK) return bail(rc);
    ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "create"));
    *out = h;
    return NAV_OK;
}

int nav_create(const nav_map *maps, int n_maps, int n_envs, int n_beams, float max_range,
               const nav_robot *robot, const nav_params *params, nav_handle **out) {
    if (n_envs <= 0 || n_beams <= 0) return NAV_E_INVAL;
    std::vector<int> beams((size_t)n_envs, n_beams);
    return nav_create_ex(maps, n_maps, nullptr, beams.data(), nullptr, n_envs, max_range, robot,
                         1, params, out);
}

int nav_set_stream(nav_handle *h, void *cuda_stream) {
    if (!h) return NAV_E_INVAL;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return NAV_OK;
}

int nav_obs_offsets(const nav_handle *h, int64_t *offsets_host) {
    if (!h || !offsets_host) return NAV_E_INVAL;
    std::memcpy(offsets_host, h->obs_off.data(), sizeof(int64_t) * h->obs_off.size());
    return NAV_OK;
}

int nav_num_envs(const nav_handle *h) { return h ? h->n_envs : NAV_E_INVAL; }

int64_t nav_obs_size(const nav_handle *h) { return h ? h->obs_off.back() : NAV_E_INVAL; }

int nav_reset(nav_handle *h, uint64_t seed, float *obs_dev) {
    if (!h || !obs_dev) return fail(h, NAV_E_INVAL, "nav_reset: null argument");
    h->seed = seed;
    StepArgs &A = h->a;
    A.seed = seed;
    A.mode = 1;
    A.actions = nullptr;
    A.obs = obs_dev;
    A.reward = nullptr;
    A.done = nullptr;
    A.final_obs = nullptr;
    return launch(h);
}

int nav_step(nav_handle *h, const float *actions_dev, float *obs_dev, float *reward_dev,
             uint8_t *done_dev, float *final_obs_dev) {
    if (!h || !actions_dev || !obs_dev || !reward_dev || !done_dev)
        return fail(h, NAV_E_INVAL, "nav_step: null argument");
    if ((reinterpret_cast<uintptr_t>(actions_dev) & 7u) != 0)
        return fail(h, NAV_E_INVAL, "nav_step: actions must be 8-byte aligned");
    StepArgs &A = h->a;
    A.seed = h->seed;
    A.mode = 0;
    A.actions = actions_dev;
    A.obs = obs_dev;
    A.reward = reward_dev;
    A.done = done_dev;
    A.final_obs = final_obs_dev;
    return launch(h);
}

int nav_step_host(nav_handle *h, const float *actions_host, float *obs_host, float *reward_host,
                  uint8_t *done_host, float *final_obs_host) {
    if (!h || !actions_host || !obs_host || !reward_host || !done_host)
        return fail(h, NAV_E_INVAL, "nav_step_host: null argument");
    const size_t E = (size_t)h->n_envs, O = (size_t)h->obs_off.back();

    cudaError_t e = cudaSuccess;
    if (!h->h_act) {
        e = h->arena.alloc(&h->h_act, 2 * E);
        if (e == cudaSuccess) e = h->arena.alloc(&h->h_obs, O);
        if (e == cudaSuccess) e = h->arena.alloc(&h->h_rew, E);
        if (e == cudaSuccess) e = h->arena.alloc(&h->h_done, E);
        if (e == cudaSuccess) e = h->arena.alloc(&h->h_fin, O);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(staging)");
    }
    e = cudaMemcpyAsync(h->h_act, actions_host, 2 * E * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync(actions)");
    const int P = (int)h->part_tile_off.size() - 1;
    if (P > 1 && !(h->cfg.split && h->split_ok)) {
        // pipeline: part p's results leave the device while part p + 1 computes
        if (!h->copy_stream) {
            e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate(copy)");
        }
        while ((int)h->part_ev.size() < P) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate(part)");
            h->part_ev.push_back(ev);
        }
        StepArgs &A = h->a;
        A.seed = h->seed;
        A.mode = 0;
        A.actions = h->h_act;
        A.obs = h->h_obs;
        A.reward = h->h_rew;
        A.done = h->h_done;
        A.final_obs = final_obs_host ? h->h_fin : nullptr;
        for (int p = 0; p < P; ++p) {
            StepArgs Ap = A;
            Ap.tiles = h->d_ptiles + h->part_tile_off[p];
            Ap.n_tiles = h->part_tile_off[p + 1] - h->part_tile_off[p];
            Ap.perm = h->d_pperm;
            Ap.tile_env = nullptr;
            Ap.tile_stage = nullptr;
            const int lrc = launch_args(h, Ap);
            if (lrc != 0) return cuda_fail(h, (cudaError_t)lrc, "step kernel launch (part)");
            e = cudaEventRecord(h->part_ev[p], h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->part_ev[p], 0);
            const int e0 = h->part_env_off[p], e1 = h->part_env_off[p + 1];
            const size_t o0 = (size_t)h->obs_off[e0], o1 = (size_t)h->obs_off[e1];
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(obs_host + o0, h->h_obs + o0, (o1 - o0) * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->copy_stream);
            // rewards and flags of every part in two copies after the last
            // part (each small copy costs the queue a few microseconds)
            if (e == cudaSuccess && p == P - 1)
                e = cudaMemcpyAsync(reward_host, h->h_rew, E * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->copy_stream);
            if (e == cudaSuccess && p == P - 1)
                e = cudaMemcpyAsync(done_host, h->h_done, E, cudaMemcpyDeviceToHost, h->copy_stream);
            if (e == cudaSuccess && final_obs_host)
                e = cudaMemcpyAsync(final_obs_host + o0, h->h_fin + o0, (o1 - o0) * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->copy_stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "nav_step_host (part)");
        }
        e = cudaStreamSynchronize(h->copy_stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize(copy)");
        return NAV_OK;
    }
    int rc = nav_step(h, h->h_act, h->h_obs, h->h_rew, h->h_done, final_obs_host ? h->h_fin : nullptr);
    if (rc != NAV_OK) return rc;
    e = cudaMemcpyAsync(obs_host, h->h_obs, O * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(reward_host, h->h_rew, E * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(done_host, h->h_done, E, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && final_obs_host)
        e = cudaMemcpyAsync(final_obs_host, h->h_fin, O * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync(results)");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return NAV_OK;
}

int nav_set_host_pipeline(nav_handle *h, int parts) {
    if (!h || parts < 1 || parts > 64) return NAV_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    h->host_parts = parts;
    return build_tiles(h);
}

int nav_set_grid_cap(nav_handle *h, int max_ctas) {
    if (!h || max_ctas < 0) return NAV_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    h->cfg.max_ctas = max_ctas;
    return NAV_OK;
}

int nav_get_grid_cap(const nav_handle *h, int *max_ctas) {
    if (!h || !max_ctas) return NAV_E_INVAL;
    *max_ctas = h->cfg.max_ctas;
    return NAV_OK;
}

int nav_sync(nav_handle *h, int timeout_ms) {
    if (!h) return NAV_E_INVAL;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    e = cudaEventRecord(ev, h->stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return cuda_fail(h, e, "cudaEventRecord");
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e != cudaErrorNotReady) break;
        if (timeout_ms > 0 &&
            std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
            cudaEventDestroy(ev);
            return fail(h, NAV_E_TIMEOUT, "nav_sync: deadline passed");
        }
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream");
    int status = 0;
    e = cudaMemcpy(&status, h->a.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(status)");
    if (status != 0) {
        cudaMemset(h->a.status, 0, sizeof(int));
        return fail(h, NAV_E_INTERNAL, "device status word " + std::to_string(status));
    }
    return NAV_OK;
}

int nav_get_state(nav_handle *h, float *f8_host, int32_t *i2_host, float *dyn_host) {
    if (!h || !f8_host || !i2_host) return fail(h, NAV_E_INVAL, "nav_get_state: null argument");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    const size_t E = (size_t)h->n_envs;
    std::vector<float> col(E);
    float *src[8] = {h->a.x, h->a.y, h->a.th, h->a.v, h->a.w, h->a.gx, h->a.gy, h->a.dprev};
    for (int c = 0; c < 8; ++c) {
        e = cudaMemcpy(col.data(), src[c], E * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(state)");
        for (size_t i = 0; i < E; ++i) f8_host[8 * i + c] = col[i];
    }
    std::vector<int32_t> st(E), ep(E);
    e = cudaMemcpy(st.data(), h->a.step, E * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ep.data(), h->a.episode, E * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(counters)");
    for (size_t i = 0; i < E; ++i) {
        i2_host[2 * i] = st[i];
        i2_host[2 * i + 1] = ep[i];
    }
    if (dyn_host && h->par.n_dyn > 0) {
        e = cudaMemcpy(dyn_host, h->a.dyn, E * h->par.n_dyn * sizeof(float4), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(dyn)");
    }
    return NAV_OK;
}

int nav_set_state(nav_handle *h, uint64_t seed, const float *f8_host, const int32_t *i2_host,
                  const float *dyn_host) {
    if (!h || !f8_host || !i2_host) return fail(h, NAV_E_INVAL, "nav_set_state: null argument");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    const size_t E = (size_t)h->n_envs;
    std::vector<float> col(E);
    float *dst[8] = {h->a.x, h->a.y, h->a.th, h->a.v, h->a.w, h->a.gx, h->a.gy, h->a.dprev};
    for (int c = 0; c < 8; ++c) {
        for (size_t i = 0; i < E; ++i) col[i] = f8_host[8 * i + c];
        e = cudaMemcpy(dst[c], col.data(), E * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(state)");
    }
    std::vector<int32_t> st(E), ep(E);
    for (size_t i = 0; i < E; ++i) {
        st[i] = i2_host[2 * i];
        ep[i] = i2_host[2 * i + 1];
    }
    e = cudaMemcpy(h->a.step, st.data(), E * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->a.episode, ep.data(), E * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && dyn_host && h->par.n_dyn > 0)
        e = cudaMemcpy(h->a.dyn, dyn_host, E * h->par.n_dyn * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(state)");
    h->seed = seed;
    // the next-episode records follow from (seed, env, episode + 1)
    StepArgs A = h->a;
    A.seed = seed;
    e = (cudaError_t)launch_prep_all(A, h->n_envs, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "next-episode records");
    return NAV_OK;
}

int nav_set_debug(nav_handle *h, int enable) {
    if (!h) return NAV_E_INVAL;
    if (enable && !h->d_dbg_range) {
        const size_t n = (size_t)h->ray_off.back();
        cudaError_t e = h->arena.alloc(&h->d_dbg_range, n);
        if (e == cudaSuccess) e = h->arena.alloc(&h->d_dbg_hit, n);
        if (e == cudaSuccess) e = h->arena.alloc(&h->d_dbg_vis, n);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(debug)");
    }
    h->debug = enable ? 1 : 0;
    h->a.dbg_range = h->debug ? h->d_dbg_range : nullptr;
    h->a.dbg_hit = h->debug ? h->d_dbg_hit : nullptr;
    h->a.dbg_vis = h->debug ? h->d_dbg_vis : nullptr;
    return NAV_OK;
}

int nav_get_debug(nav_handle *h, float *ranges_host, int32_t *hits_host, uint32_t *visits_host) {
    if (!h) return NAV_E_INVAL;
    if (!h->debug) return fail(h, NAV_E_INVAL, "nav_get_debug: debug capture is off");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    const size_t n = (size_t)h->ray_off.back();
    if (ranges_host) e = cudaMemcpy(ranges_host, h->d_dbg_range, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hits_host)
        e = cudaMemcpy(hits_host, h->d_dbg_hit, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && visits_host)
        e = cudaMemcpy(visits_host, h->d_dbg_vis, n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(debug)");
    return NAV_OK;
}

int nav_set_stats(nav_handle *h, int enable) {
    if (!h) return NAV_E_INVAL;
    h->stats = enable ? 1 : 0;
    h->a.stats = h->stats ? h->d_stats : nullptr;
    if (enable) {
        cudaError_t e = cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(unsigned long long), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync(stats)");
    }
    return NAV_OK;
}

int nav_get_stats(nav_handle *h, uint64_t *visits, uint64_t *rays) {
    if (!h) return NAV_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    unsigned long long v[2];
    e = cudaMemcpy(v, h->d_stats, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(stats)");
    if (visits) *visits = v[0];
    if (rays) *rays = v[1];
    return NAV_OK;
}

int nav_set_launch(nav_handle *h, int tile_envs, int block_threads, int smem_map_bytes,
                   int max_regs, int byte_cells, int split) {
    if (!h) return NAV_E_INVAL;
    if (tile_envs < 0 || tile_envs > kMaxTileEnvs || block_threads < 0 || block_threads > 512 ||
        (block_threads % 32) != 0 || (block_threads > 0 && block_threads < 64) ||
        smem_map_bytes < 0 || smem_map_bytes > kMaxSmemMapBytes ||
        !(max_regs == 0 || max_regs == 32 || max_regs == 40 || max_regs == 64) ||
        byte_cells < 0 || byte_cells > 3 || split < 0 || split > 4 || split == 3)
        return fail(h, NAV_E_INVAL, "nav_set_launch: out of range");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    if (block_threads) h->cfg.block_threads = block_threads;
    if (max_regs) h->cfg.max_regs = max_regs;
    if (smem_map_bytes) h->smem_map_bytes = smem_map_bytes;
    if (byte_cells) h->byte_cells = byte_cells;
    if (split) {
        h->cfg.split = split == 1 ? 1 : 0;
        h->cfg.refill = split == 4 ? 1 : 0;
    }
    int rc = set_map_modes(h);
    if (rc != NAV_OK) return rc;
    if (tile_envs && tile_envs != h->cfg.tile_envs) {
        h->cfg.tile_envs = tile_envs;
        return build_tiles(h);
    }
    return NAV_OK;
}

int nav_set_tile_order(nav_handle *h, int order) {
    if (!h) return NAV_E_INVAL;
    if (order != 0 && order != 1) return fail(h, NAV_E_INVAL, "nav_set_tile_order: order 0 or 1");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    if (order == h->cfg.order) return NAV_OK;
    h->cfg.order = order;
    return build_tiles(h);
}

int nav_get_tile_order(const nav_handle *h, int *order) {
    if (!h || !order) return NAV_E_INVAL;
    *order = h->cfg.order;
    return NAV_OK;
}

int nav_get_launch(const nav_handle *h, int *tile_envs, int *block_threads, int *smem_map_bytes,
                   int *max_regs, int *byte_cells, int *split) {
    if (!h) return NAV_E_INVAL;
    if (tile_envs) *tile_envs = h->cfg.tile_envs;
    if (block_threads) *block_threads = h->cfg.block_threads;
    if (smem_map_bytes) *smem_map_bytes = h->smem_map_bytes;
    if (max_regs) *max_regs = h->cfg.max_regs;
    if (byte_cells) *byte_cells = h->byte_cells;
    if (split)
        *split = (h->cfg.split && h->split_ok) ? 1 : h->cfg.refill ? 4 : 2;
    return NAV_OK;
}

namespace {

// Device-to-device copy of the per-env state (save = true keeps a copy in the
// handle's snapshot buffer, false restores it).
int copy_state(nav_handle *h, bool save) {
    const size_t E = (size_t)h->n_envs;
    const size_t nd = (size_t)std::max(h->par.n_dyn, 1);
    cudaError_t e = cudaSuccess;
    if (!h->snap) {
        e = h->arena.alloc(&h->snap, 10 * E + 4 * nd * E + 6 * E);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(snapshot)");
    }
    StepArgs &A = h->a;
    void *cols[10] = {A.x, A.y, A.th, A.v, A.w, A.gx, A.gy, A.dprev, A.step, A.episode};
    for (int c = 0; c < 10 && e == cudaSuccess; ++c) {
        float *sn = h->snap + c * E;
        e = save ? cudaMemcpyAsync(sn, cols[c], E * 4, cudaMemcpyDeviceToDevice, h->stream)
                 : cudaMemcpyAsync(cols[c], sn, E * 4, cudaMemcpyDeviceToDevice, h->stream);
    }
    if (e == cudaSuccess) {
        float *sn = h->snap + 10 * E;
        e = save ? cudaMemcpyAsync(sn, A.dyn, nd * E * 16, cudaMemcpyDeviceToDevice, h->stream)
                 : cudaMemcpyAsync(A.dyn, sn, nd * E * 16, cudaMemcpyDeviceToDevice, h->stream);
    }
    if (e == cudaSuccess) {
        float *sn = h->snap + 10 * E + 4 * nd * E;
        e = save ? cudaMemcpyAsync(sn, A.nxt_pose, E * 16, cudaMemcpyDeviceToDevice, h->stream)
                 : cudaMemcpyAsync(A.nxt_pose, sn, E * 16, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess)
            e = save ? cudaMemcpyAsync(sn + 4 * E, A.nxt_goal, E * 8, cudaMemcpyDeviceToDevice,
                                       h->stream)
                     : cudaMemcpyAsync(A.nxt_goal, sn + 4 * E, E * 8, cudaMemcpyDeviceToDevice,
                                       h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "state snapshot copy");
    return NAV_OK;
}

// bytes written between timed steps of the autotuner's final comparison:
// more than the L2 holds, so that each step starts from DRAM as a step of a
// long rollout with other work in between does
constexpr size_t kTuneFlushBytes = 160ull << 20;

int ensure_tune_buffers(nav_handle *h) {
    if (h->tune_act) return NAV_OK;
    const size_t E = (size_t)h->n_envs, O = (size_t)h->obs_off.back();
    cudaError_t e = h->arena.alloc(&h->tune_act, 2 * E);
    if (e == cudaSuccess) e = h->arena.alloc(&h->tune_obs, O);
    if (e == cudaSuccess) e = h->arena.alloc(&h->tune_rew, E);
    if (e == cudaSuccess) e = h->arena.alloc(&h->tune_done, E);
    if (e == cudaSuccess) e = h->arena.alloc(&h->tune_flush, kTuneFlushBytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(tuning buffers)");
    return NAV_OK;
}

// Mean device time of `steps` steps (after 2 untimed) from the snapshot state
// with hash-uniform actions; +inf if a launch fails.
float time_config(nav_handle *h, int steps, cudaEvent_t e0, cudaEvent_t e1, bool flush = false) {
    StepArgs A = h->a;
    A.mode = 0;
    A.obs = h->tune_obs;
    A.reward = h->tune_rew;
    A.done = h->tune_done;
    A.final_obs = nullptr;
    A.actions = h->tune_act;
    A.stats = nullptr;
    A.dbg_range = nullptr;
    A.dbg_hit = nullptr;
    A.dbg_vis = nullptr;
    if (copy_state(h, false) != NAV_OK) return INFINITY;
    float total = 0.0f;
    for (int t = 0; t < steps + 2; ++t) {
        launch_uniform_actions(h->tune_act, h->n_envs, 0x7A11ull, (unsigned)t, h->stream);
        if (flush) cudaMemsetAsync(h->tune_flush, t & 0xFF, kTuneFlushBytes, h->stream);
        cudaEventRecord(e0, h->stream);
        const int lrc = launch_args(h, A);
        if (lrc != 0) {
            cudaGetLastError();
            cudaStreamSynchronize(h->stream);
            return INFINITY;
        }
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return INFINITY;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (t >= 2) total += ms;
    }
    return total / steps;
}

} // namespace

namespace {

// Tiles of `te` envs of one (map, beam table) for the fused act-step kernel
// (and a remainder per group), over the handle's env order (perm), largest
// first.
int build_act_tiles(nav_handle *h, int te) {
    if (te == h->act_tile_envs && h->d_act_tiles) return NAV_OK;
    std::vector<int> perm(h->n_envs);
    cudaError_t e = cudaMemcpy(perm.data(), h->a.perm, perm.size() * sizeof(int),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(perm)");
    std::vector<TileDev> tiles;
    int s = 0;
    const int E = h->n_envs;
    while (s < E) {
        int t = s;
        while (t < E && h->env_map[perm[t]] == h->env_map[perm[s]] &&
               h->env_tab[perm[t]] == h->env_tab[perm[s]])
            ++t;
        for (int b = s; b < t; b += te)
            tiles.push_back(TileDev{h->env_map[perm[s]], h->env_tab[perm[s]], b, std::min(te, t - b)});
        s = t;
    }
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const TileDev &x, const TileDev &y) { return x.env_count > y.env_count; });
    if ((int)tiles.size() > h->act_tiles_cap) {
        e = h->arena.alloc(&h->d_act_tiles, tiles.size());
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(act tiles)");
        h->act_tiles_cap = (int)tiles.size();
    }
    e = cudaMemcpy(h->d_act_tiles, tiles.data(), tiles.size() * sizeof(TileDev),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(act tiles)");
    h->act_n_tiles = (int)tiles.size();
    h->act_tile_envs = te;
    return NAV_OK;
}

} // namespace

int nav_rollout_fused(nav_handle *h, nav_policy *p, int n_steps, int mode, uint64_t seed,
                      uint32_t step0, float *obs_dev, float *actions_dev, float *reward_dev,
                      uint8_t *done_dev, int actions_ready) {
    if (!h || !p || !obs_dev || !actions_dev || !reward_dev || !done_dev || n_steps <= 0 ||
        (mode != 0 && mode != 1))
        return fail(h, NAV_E_INVAL, "nav_rollout_fused: bad argument");
    if ((reinterpret_cast<uintptr_t>(actions_dev) & 7u) != 0)
        return fail(h, NAV_E_INVAL, "nav_rollout_fused: actions must be 8-byte aligned");
    const StepArgs &H = h->a;
    const int K = h->env_k.empty() ? 0 : h->env_k[0];
    bool uniform = true;
    for (int k : h->env_k) uniform = uniform && k == K;
    if (!uniform || h->par.n_sectors != 0 || h->par.sensor != 0 || h->par.n_dyn != 0)
        return fail(h, NAV_E_INVAL,
                    "nav_rollout_fused: needs one beam count, raw beams, the exact traversal "
                    "and no moving discs");
    Mlp *net = policy_actor(p);
    if (!net || net->n_layers != 3 || policy_ipap(p) != 0 || policy_obs_dim(p) != K + 4 ||
        K + 4 > 384 || net->layer[0].in != K + 4 || net->layer[0].out > 256 ||
        net->layer[1].in != net->layer[0].out || net->layer[1].out > 256 ||
        net->layer[2].in != net->layer[1].out || net->layer[2].out != 4 ||
        policy_max_batch(p) < h->n_envs)
        return fail(h, NAV_E_INVAL,
                    "nav_rollout_fused: the policy must be obs_dim = beams + 4 <= 384 -> H -> H "
                    "-> 4 with H <= 256, no Eq. 2 input, max_batch >= n_envs");
    // shared memory: the staged map (or the two 32 KiB weight buffers) and
    // the 96 KiB input tile
    int region = 64 * 1024;
    for (const MapDev &m : h->maps) {
        if (m.dist_off < 0) return fail(h, NAV_E_INVAL, "nav_rollout_fused: a map has no distance bytes");
        region = std::max(region, m.n_bytes);
    }
    region = (region + 1023) & ~1023;
    StepArgs A = H;
    A.smem_region_bytes = region;
    if (act_step_smem(A) + 8 * 1024 > 227 * 1024)
        return fail(h, NAV_E_INVAL, "nav_rollout_fused: the maps are too large to stage");
    // tiles: as many as the SMs take in whole waves, at most 128 envs each
    int n_sm = 0;
    cudaError_t ce = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaDeviceGetAttribute");
    // full tiles of E / (whole waves of one CTA per SM) envs and one smaller
    // remainder tile per group, queued last (largest first): with four waves
    // of 65536 envs 822-830 us per step against 847-854 us with equal tiles
    // (the small tiles fill the last wave's gaps)
    const long long waves = std::max(1LL, ((long long)h->n_envs + 128LL * n_sm - 1) / (128LL * n_sm));
    const int te = (int)std::max(1LL, std::min(128LL, ((long long)h->n_envs + waves * n_sm - 1) /
                                                          (waves * n_sm)));
    int rc = build_act_tiles(h, te);
    if (rc != NAV_OK) return rc;
    // the first action from the current observation (the inference path),
    // unless the previous call left it in actions_dev
    if (!actions_ready) {
        rc = nav_policy_act(p, obs_dev, K + 4, h->n_envs, mode, seed, step0, actions_dev, nullptr,
                            nullptr, h->stream);
        if (rc != NAV_OK) return fail(h, rc, "nav_rollout_fused: first action");
    }
    A.seed = h->seed;
    A.mode = 0;
    A.actions = actions_dev;
    A.obs = obs_dev;
    A.reward = reward_dev;
    A.done = done_dev;
    A.final_obs = nullptr;
    A.tiles = h->d_act_tiles;
    A.n_tiles = h->act_n_tiles;
    A.tile_env = nullptr;
    A.tile_stage = nullptr;
    ActArgs P{};
    for (int l = 0; l < 3; ++l) {
        P.W[l] = static_cast<const __nv_bfloat16 *>(net->layer[l].W16);
        P.b[l] = net->layer[l].b;
        P.ld[l] = net->layer[l].ld_in;
        P.in[l] = net->layer[l].in;
        P.out[l] = net->layer[l].out;
    }
    // the current weights as swizzled units (they change between calls while
    // a trainer syncs the policy)
    const size_t wbytes = (size_t)act_units(P) * 16384;
    if (wbytes > h->act_w_cap) {
        cudaError_t e = h->arena.alloc(&h->d_act_w, wbytes);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(actor weight units)");
        h->act_w_cap = wbytes;
    }
    P.Wu = h->d_act_w;
    rc = launch_act_swizzle(P, h->d_act_w, h->stream);
    if (rc != 0) return cuda_fail(h, (cudaError_t)rc, "actor weight swizzle");
    P.scale = policy_scale(p);
    P.act = actions_dev;
    P.mode = mode;
    P.seed = seed;
    for (int t = 0; t < n_steps; ++t) {
        P.step = step0 + (uint32_t)t + 1u;
        const int lrc = launch_act_step(A, P, h->stream);
        if (lrc != 0) return cuda_fail(h, (cudaError_t)lrc, "act-step kernel launch");
    }
    return NAV_OK;
}

int nav_autotune(nav_handle *h, int steps, float *best_ms) {
    if (!h || steps <= 0) return fail(h, NAV_E_INVAL, "nav_autotune: bad argument");
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamSynchronize");
    int rc = ensure_tune_buffers(h);
    if (rc == NAV_OK) rc = copy_state(h, true);
    if (rc != NAV_OK) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    LaunchCfg best_cfg = h->cfg;
    int best_cap = h->smem_map_bytes, best_bytes = h->byte_cells;
    // every timing, for the final comparison with L2 flushed between steps
    struct Timed {
        float ms;
        LaunchCfg cfg;
        int cap, bytes;
    };
    std::vector<Timed> all;
    auto timed = [&](int n) {
        const float ms = time_config(h, n, e0, e1);
        all.push_back({ms, h->cfg, h->smem_map_bytes, h->byte_cells});
        return ms;
    };
    // pass 1: launch shape with the current staging choice; the three
    // fastest shapes are timed again with three times the steps
    // fixed sizes, and sizes whose tiles fill 1-4 whole waves of one to four
    // resident CTAs per SM
    std::vector<int> tiles = {1, 2, 4, 8, 16, 32};
    {
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess)
            for (int k = 1; k <= 8; ++k) {
                const int te = fit_tile(h, (long long)n_sm * k, kMaxTileEnvs);
                if (te > 0 && std::find(tiles.begin(), tiles.end(), te) == tiles.end())
                    tiles.push_back(te);
            }
    }
    const int blocks[] = {128, 256, 512};
    const int regs[] = {32, 40, 64};
    // refilled lanes apply to the exact traversal without moving discs
    const int n_refill = (h->par.n_dyn == 0 && h->par.sensor == 0) ? 2 : 1;
    std::vector<std::pair<float, LaunchCfg>> cand;
    for (int rf = 0; rf < n_refill && rc == NAV_OK; ++rf)
        for (int te : tiles) {
            if (te > 1 && te > h->n_envs) continue;
            h->cfg.tile_envs = te;
            h->cfg.refill = rf;
            if ((rc = build_tiles(h)) != NAV_OK) break;
            for (int bt : blocks)
                for (int mr : regs) {
                    h->cfg.block_threads = bt;
                    h->cfg.max_regs = mr;
                    cand.push_back({timed(steps), h->cfg});
                }
        }
    if (rc == NAV_OK && !cand.empty()) {
        std::sort(cand.begin(), cand.end(),
                  [](const std::pair<float, LaunchCfg> &a, const std::pair<float, LaunchCfg> &b) {
                      return a.first < b.first;
                  });
        for (size_t c = 0; c < cand.size() && c < 3; ++c) {
            h->cfg = cand[c].second;
            if ((rc = build_tiles(h)) != NAV_OK) break;
            const float ms = timed(3 * steps);
            if (ms < best) {
                best = ms;
                best_cfg = h->cfg;
            }
        }
    }
    // pass 2: staging (byte cells or packed bits) and the shared-memory cap,
    // with every register cap for the best shape (a smaller staged map
    // leaves room for more resident CTAs, which shifts the best cap)
    if (rc == NAV_OK) {
        const LaunchCfg shape = best_cfg;
        h->cfg = shape;
        rc = build_tiles(h);
        const int caps[] = {24 * 1024, 80 * 1024, 160 * 1024};
        for (int mr : regs)
            for (int bc = 1; bc <= 3 && rc == NAV_OK; ++bc)
                for (int cap : caps) {
                    h->cfg.max_regs = mr;
                    h->byte_cells = bc;
                    h->smem_map_bytes = cap;
                    if ((rc = set_map_modes(h)) != NAV_OK) break;
                    const float ms = timed(steps);
                    if (ms < best) {
                        best = ms;
                        best_cap = cap;
                        best_bytes = bc;
                        best_cfg = h->cfg;
                    }
                }
    }
    // pass 2b: the tile queue order
    if (rc == NAV_OK) {
        h->cfg = best_cfg;
        h->smem_map_bytes = best_cap;
        h->byte_cells = best_bytes;
        if ((rc = set_map_modes(h)) == NAV_OK) {
            h->cfg.order = 1 - best_cfg.order;
            if ((rc = build_tiles(h)) == NAV_OK) {
                const float ms = timed(3 * steps);
                if (ms < best) {
                    best = ms;
                    best_cfg = h->cfg;
                }
            }
        }
    }
    // pass 3: the split step (env kernel + all-maps-resident ray kernel)
    if (rc == NAV_OK && h->split_ok) {
        h->cfg = best_cfg;
        h->smem_map_bytes = best_cap;
        h->byte_cells = best_bytes;
        if ((rc = set_map_modes(h)) == NAV_OK) rc = build_tiles(h);
        if (rc == NAV_OK) {
            h->cfg.split = 1;
            const float ms = timed(steps);
            if (ms < best) {
                best = ms;
                best_cfg = h->cfg;
            }
            h->cfg.split = 0;
        }
    }
    // final: the four fastest distinct settings again, each step after an
    // L2 flush and with four times the steps (short unflushed timings rank
    // shapes within a few per cent of each other in either order)
    if (rc == NAV_OK && !all.empty()) {
        std::stable_sort(all.begin(), all.end(),
                         [](const Timed &a, const Timed &b) { return a.ms < b.ms; });
        auto same = [](const Timed &a, const Timed &b) {
            return a.cap == b.cap && a.bytes == b.bytes && a.cfg.tile_envs == b.cfg.tile_envs &&
                   a.cfg.block_threads == b.cfg.block_threads && a.cfg.max_regs == b.cfg.max_regs &&
                   a.cfg.split == b.cfg.split && a.cfg.order == b.cfg.order &&
                   a.cfg.refill == b.cfg.refill;
        };
        std::vector<Timed> top;
        for (const Timed &t : all) {
            if (!(t.ms < INFINITY) || top.size() >= 4) break;
            bool dup = false;
            for (const Timed &u : top) dup = dup || same(t, u);
            if (!dup) top.push_back(t);
        }
        float fbest = INFINITY;
        for (const Timed &t : top) {
            h->cfg = t.cfg;
            h->smem_map_bytes = t.cap;
            h->byte_cells = t.bytes;
            if ((rc = set_map_modes(h)) != NAV_OK || (rc = build_tiles(h)) != NAV_OK) break;
            const float ms = time_config(h, 4 * steps, e0, e1, true);
            if (ms < fbest) {
                fbest = ms;
                best = ms;
                best_cfg = t.cfg;
                best_cap = t.cap;
                best_bytes = t.bytes;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg = best_cfg;
    h->smem_map_bytes = best_cap;
    h->byte_cells = best_bytes;
    int rc2 = set_map_modes(h);
    if (rc2 == NAV_OK) rc2 = build_tiles(h);
    int rc3 = copy_state(h, false);
    ce = cudaStreamSynchronize(h->stream);
    if (rc != NAV_OK) return rc;
    if (rc2 != NAV_OK) return rc2;
    if (rc3 != NAV_OK) return rc3;
    if (ce != cudaSuccess) return cuda_fail(h, ce, "nav_autotune");
    if (!(best < INFINITY)) return fail(h, NAV_E_CUDA, "nav_autotune: no launch shape ran");
    if (best_ms) *best_ms = best;
    return NAV_OK;
}

int nav_uniform_actions(nav_handle *h, uint64_t seed, uint32_t step, float *actions_dev) {
    if (!h || !actions_dev) return fail(h, NAV_E_INVAL, "nav_uniform_actions: null argument");
    int rc = launch_uniform_actions(actions_dev, h->n_envs, seed, step, h->stream);
    if (rc != 0) return cuda_fail(h, (cudaError_t)rc, "uniform actions kernel");
    return NAV_OK;
}

int nav_graph_capture(nav_handle *h, int n_steps, const float *actions_dev, float *obs_dev,
                      float *reward_dev, uint8_t *done_dev, float *final_obs_dev) {
    if (!h || n_steps <= 0 || !actions_dev || !obs_dev || !reward_dev || !done_dev)
        return fail(h, NAV_E_INVAL, "nav_graph_capture: bad argument");
    if (!h->stream) return fail(h, NAV_E_INVAL, "nav_graph_capture: bind a non-default stream");
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    int rc = NAV_OK;
    for (int t = 0; t < n_steps && rc == NAV_OK; ++t)
        rc = nav_step(h, actions_dev + (size_t)t * 2 * h->n_envs, obs_dev, reward_dev, done_dev,
                      final_obs_dev);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->stream, &g);
    if (rc != NAV_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return NAV_OK;
}

int nav_graph_launch(nav_handle *h) {
    if (!h || !h->graph) return fail(h, NAV_E_INVAL, "nav_graph_launch: no graph captured");
    cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    return NAV_OK;
}

const char *nav_last_error(const nav_handle *h) { return h ? h->err.c_str() : "null handle"; }

void nav_free(nav_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    for (cudaEvent_t ev : h->part_ev) cudaEventDestroy(ev);
    delete h;
}

} // extern "C"
