// Private declarations shared by the host runtime (nav_api.cpp) and the
// kernels (nav_step.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>

#include "../../include/flashnav.h"

namespace flashnav {

constexpr int kMaxDyn = 8;      // moving discs per env
constexpr int kMaxDynRows = 16; // rows spanned by one stamped disc
constexpr int kMaxTileEnvs = 32;
constexpr int kMaxBeams = 2048;

// Packed map: free bits (1 = free), one padding cell on every side that reads
// as blocked, rows of `pitch` 32-bit words (odd, to spread smem banks); the
// padded bit index of cell (i, j) is (j + 1) * pitch * 32 + (i + 1).
struct MapDev {
    int w, h, pitch, n_words; // n_words is a multiple of 4 (16-byte copies)
    long long word_off;       // into the concatenated bitmap, multiple of 4
    float res, inv_res;
};

// C-space of one (map, robot) pair: spawnable cells ascending, the component
// of each, and every component's cells grouped and ascending.
struct CsDev {
    int n_spawn, spawn_off; // into spawn / spawn_comp
    int comp_off;           // into comp_start / comp_count
    int cells_off;          // into comp_cells
};

struct RobotDev {
    int shape;
    float radius, length, width, v_min, v_max, w_min, w_max;
};

struct ParamsDev {
    float dt, goal_tol, c_progress, step_penalty, r_goal, r_coll;
    int horizon;
    float goal_dmin, goal_dmax;
    int n_dyn;
    float dyn_radius, dyn_speed_max, dyn_min_sep;
    int reward_mode;
};

// One CTA work unit: up to kMaxTileEnvs envs sharing a map and a beam count.
struct TileDev {
    int map, tab, env_begin, env_count;
};

struct StepArgs {
    const uint32_t *bits;
    const MapDev *maps;
    const int *spawn, *spawn_comp, *comp_start, *comp_count, *comp_cells;
    const CsDev *cs;
    const float *beam_c, *beam_s; // per table, at tab_off
    const int *tab_off, *tab_k;
    const int *env_map, *env_tab, *env_robot, *env_cs;
    const long long *obs_off, *ray_off;
    const RobotDev *robots;
    const TileDev *tiles;
    const int *perm;
    int n_tiles;
    // state (structure of arrays)
    float *x, *y, *th, *v, *w, *gx, *gy, *dprev;
    int *step;
    unsigned *episode;
    float4 *dyn; // [n_envs][n_dyn]
    // io
    const float *actions;
    float *obs, *reward, *final_obs;
    unsigned char *done;
    // debug / stats / status
    float *dbg_range;
    int *dbg_hit;
    unsigned *dbg_vis;
    unsigned long long *stats; // [0] visits, [1] rays
    int *status;
    ParamsDev p;
    unsigned long long seed;
    float max_range;
    int mode; // 0 step, 1 reset all
    int smem_map_words; // capacity of the staged-bitmap region (0 = none)
    int max_k;
};

enum StatusBits { kStatusNoSpawn = 1, kStatusCopyTimeout = 2, kStatusBadPose = 4 };

// Launches one step (or reset) of every tile on `stream`.
int launch_step(const StepArgs &a, int block_threads, int tile_envs, void *stream);

} // namespace flashnav
