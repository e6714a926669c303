// Private declarations shared by the host runtime (nav_api.cpp) and the
// kernels (nav_step.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/flashnav.h"

namespace flashnav {

constexpr int kMaxDyn = 8;      // moving discs per env
constexpr int kMaxDynRows = 16; // rows spanned by one stamped disc
constexpr int kMaxTileEnvs = 32;
constexpr int kMaxBeams = 2048;
constexpr int kMaxSmemMapBytes = 200 * 1024; // largest map staged in shared memory
constexpr long long kMaxDistBytes = 64ll << 20; // largest map given distance bytes

// Packed map: free bits (1 = free), kPad padding cells on every side that
// read as blocked, rows of `pitch` 32-bit words (odd, to spread smem banks);
// the padded bit index of cell (i, j) is (j + kPad) * pitch * 32 + (i + kPad).
// The same padded map as one byte per cell has a row stride of byte_stride
// bytes (a multiple of 4 whose word count is odd); each byte is 0 for a
// blocked cell, else the chessboard distance (in cells, capped at 255) to the
// nearest blocked or padding cell.
constexpr int kPad = 1;
struct MapDev {
    int w, h, pitch, n_words; // n_words is a multiple of 4 (16-byte copies)
    long long word_off;       // into the concatenated bitmap, multiple of 4
    float res, inv_res;
    int byte_stride, n_bytes; // byte view; n_bytes is a multiple of 16
    int mode;                 // staging, one of MapMode
    int all_off;              // word offset when every map is staged together (split step)
    long long dist_off;       // byte offset of the distance bytes (multiple of 16), -1: none
};
// Where a tile reads its map: packed bits through L1/L2, packed bits or
// distance bytes staged in shared memory, or distance bytes through L1/L2.
enum MapMode { kMapGlobal = 0, kMapSharedBits = 1, kMapSharedBytes = 2, kMapGlobalBytes = 3 };

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
    int sensor;       // 0 exact traversal, 1 fixed-step march
    float march_step; // metres
    int n_sectors;    // 0 raw beams, else Eq. 6 sector minima
};

// One CTA work unit: up to kMaxTileEnvs envs sharing a map and a beam count.
struct TileDev {
    int map, tab, env_begin, env_count;
};

struct StepArgs {
    const uint32_t *bits;
    const uint8_t *dist; // distance bytes of the maps that have them, at dist_off
    const MapDev *maps;
    const int *spawn, *spawn_comp, *comp_start, *comp_count, *comp_cells;
    const CsDev *cs;
    const float *beam_c, *beam_s; // per table, at tab_off
    const int *tab_off, *tab_k;
    const int *env_map, *env_tab, *env_robot, *env_cs;
    const long long *obs_off, *ray_off;
    const RobotDev *robots;
    const RobotDev *env_rb; // [n_envs] each env's robot record (robots[env_robot[e]])
    const TileDev *tiles;
    const int *perm;
    const int *tile_env; // [n_tiles][kMaxTileEnvs] envs of each tile, or null: perm
    const int4 *tile_stage; // [n_tiles] {map mode, bytes, byte offset lo, hi}, or null: maps
    int n_tiles;
    int max_tile_envs; // envs of the largest tile
    int *tile_queue; // [0] next tile to hand out, [1] CTAs finished; zero between launches
    // state (structure of arrays)
    float *x, *y, *th, *v, *w, *gx, *gy, *dprev;
    int *step;
    unsigned *episode;
    // next-episode record per env: spawn (x, y, theta, goal distance) and
    // goal of episode + 1 (written by prep_next, read by the env phase)
    float4 *nxt_pose;
    float2 *nxt_goal;
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
    int smem_region_bytes; // shared-memory region holding a staged map (0 = none)
    int max_k;
    // split step (all maps resident in shared memory, no moving discs):
    // env kernel -> per-env ray origins -> ray kernel over 32-ray chunks
    float4 *ray_main, *ray_fin; // [n_envs] (xc, yc, sin, cos) of the obs scan / final scan
    int *fin_list;              // [n_envs] envs whose final scan is pending
    int *split_q;               // [0] next chunk [1] next final env [2] CTAs done [3] final count
    const int2 *chunks;         // [n_chunks] (tile, first ray of the chunk in the tile)
    int n_chunks;
    int all_words;              // words of every map together
    int n_maps_split;           // maps staged by the ray kernel
    int n_beams_total;          // entries of the concatenated beam tables
};

enum StatusBits {
    kStatusNoSpawn = 1,
    kStatusCopyTimeout = 2,
    kStatusBadPose = 4,
    kStatusQueue = 8 // a CTA drew more tiles than a launch holds
};

// Defaults: the autotuner's usual choice for 256 x 256 maps with distance
// bytes staged (three 512-thread CTAs per SM).
struct LaunchCfg {
    int tile_envs = 8;     // envs per CTA tile
    int block_threads = 512;
    int max_regs = 40;     // register cap per thread: 32, 40 or 64
    int split = 0;         // 1: env kernel + all-maps-resident ray kernel when eligible
    int order = 0;         // tile queue order: 0 map size x beams, 1 sampled ray cost
    int refill = 0;        // 1: tiled kernel with refilled lanes (exact traversal, no discs)
    int max_ctas = 0;      // > 0: at most this many persistent CTAs (the rest of the GPU free)
};

// Launches one step (or reset) of every tile on `stream`: persistent CTAs,
// grid = SMs x resident CTAs per SM, capped by the tile count.
int launch_step(const StepArgs &a, const LaunchCfg &cfg, void *stream);

// Resident CTAs of the tiled step kernel launch_step would run (SMs x CTAs
// per SM), 0 if the occupancy query fails.
int step_resident(const StepArgs &a, const LaunchCfg &cfg);

// Split step: env phase for every env, then the ray kernel (all maps staged
// in shared memory once per CTA, warps take 32-ray chunks from a queue).
int launch_step_split(const StepArgs &a, int n_envs, void *stream);

// (SMs, resident CTAs per SM) of a kernel at a shared-memory size and block
// (raises the kernel's dynamic shared-memory limit when needed; cached).
int occupancy(const void *fn, size_t smem, int block, int &n_sm, int &per_sm);

// The actor of the fused act-step kernel: a network in -> H -> H -> 4 with
// H <= 256 and in <= 384 (BF16 W [out][ld] K-major, FP32 bias), the input
// scale (null: none), and the head's noise: act[e] receives the action for
// the next step of env e (mode 1: a = tanh(u + sigma eps), eps keyed by
// (seed, e, step); mode 0: tanh(u)).
struct ActArgs {
    const __nv_bfloat16 *W[3];
    const float *b[3];
    int ld[3], in[3], out[3];
    // the weights as 16 KiB units in the tensor cores' swizzled layout (unit
    // u at Wu + u * 16 KiB: 128 output rows, or the layer's last rows, of
    // one 64-wide K chunk), written by launch_act_swizzle
    const unsigned char *Wu;
    const float *scale;
    float *act;
    int mode;
    unsigned long long seed;
    unsigned step;
};
// One fused step + actor of every tile (tiles of <= 128 envs, exact
// traversal over staged distance bytes, no moving discs, raw beams).
int launch_act_step(const StepArgs &a, const ActArgs &p, void *stream);
// Writes the weight units of p's layers into dst (act_units(p) x 16 KiB).
int launch_act_swizzle(const ActArgs &p, unsigned char *dst, void *stream);
int act_units(const ActArgs &p);
size_t act_step_smem(const StepArgs &a);

// Rewrites every env's next-episode record from its episode counter (after
// the state was set from outside).
int launch_prep_all(const StepArgs &a, int n_envs, void *stream);

// Writes n_envs uniform [-1, 1]^2 actions keyed by (seed, env, step).
int launch_uniform_actions(float *out, int n_envs, unsigned long long seed, unsigned step,
                           void *stream);

// Tensor-core GEMM C = A B^T (BF16 in, FP32 accumulate) with bias, optional
// LeakyReLU, and FP32 / BF16 / transposed-BF16 outputs (each may be null).
int launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                     const float *bias, int act, float *C32, int ldc32, void *C16, int ldc16,
                     void *C16T, int ldct, int *status, void *stream);

// Split-K variant for weight gradients (large K = batch): C32 = A B^T, C32
// zeroed on the stream first, partial products added atomically.
int launch_gemm_bf16_splitk(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                            float *C32, int ldc32, int *status, void *stream);

// Read-only facts about a handle for entry points defined outside nav_api.cpp.
struct HandleView {
    int device;
    void *stream;
    int n_envs;
    long long obs_floats;
    int uniform_d; // range features per observation row if every env has the same count, else -1
};
int handle_view(const nav_handle *h, HandleView *out);
// Records `msg` as the handle's last error and returns `code`.
int handle_fail(nav_handle *h, int code, const char *msg);

} // namespace flashnav
