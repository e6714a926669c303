/*
 * flashnav.h -- C ABI of the B300 batched bitmap navigation simulator
 * (FlashNav, Sec. 2.2: vectorised bitmap simulator; Eq. 1-7; Tables 7-9).
 *
 * One handle simulates n_envs independent goal-navigation environments on
 * one CUDA device.  Every call is asynchronous on the handle's stream unless
 * it says otherwise.  Device pointers ("*_dev") are caller-owned CUDA global
 * memory (for example torch tensors); host pointers ("*_host") are caller-
 * owned host memory.  The library owns the packed bitmaps, the per-map spawn
 * tables and the per-env state (structure of arrays) in device memory.
 *
 * Errors: every int-returning call returns NAV_OK (0) or a negative NAV_E_*
 * code and records a message readable with nav_last_error().  No C++
 * exception crosses this boundary.  Kernels never trap: an anomaly found on
 * the device sets a status word that nav_sync() reports as NAV_E_INTERNAL.
 *
 * Geometry (Sec. 2.2.1): a map is a W x H occupancy bitmap with square cells
 * of `resolution` metres; cell (i, j) covers [i, i+1] x [j, j+1] in cell
 * units, i = column (x), j = row (y); the world origin is the corner of cell
 * (0, 0).  Positions outside the map are obstacles.
 */
#ifndef FLASHNAV_H
#define FLASHNAV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    NAV_OK = 0,
    NAV_E_INVAL = -1,    /* bad argument (null pointer, size, range)        */
    NAV_E_CUDA = -2,     /* a CUDA runtime call failed                       */
    NAV_E_NOMEM = -3,    /* device or host allocation failed                 */
    NAV_E_NOSPAWN = -4,  /* a map has no cell where the robot fits           */
    NAV_E_INTERNAL = -5, /* the device status word reported an anomaly       */
    NAV_E_TIMEOUT = -6   /* nav_sync's deadline passed before the GPU was done */
};

typedef struct nav_handle nav_handle;

/* Occupancy map (Sec. 2.2.1 binary bitmap).  occ: host, row-major H x W,
 * nonzero = occupied.  Copied and packed 1 bit per cell by nav_create. */
typedef struct {
    int width, height;
    float resolution;
    const uint8_t *occ;
} nav_map;

/* Robot preset (Sec. 2.2.1 presets; Tables 8-9).  shape 0 = disc of
 * `radius`; shape 1 = rectangle `length` (along the heading) x `width`.
 * Normalised actions a in [-1, 1]^2 map affinely onto [v_min, v_max] (m/s)
 * and [w_min, w_max] (rad/s). */
typedef struct {
    int shape;
    float radius, length, width;
    float v_min, v_max, w_min, w_max;
} nav_robot;

/* Episode constants (Table 7).  reward_mode 0: r = c_progress (d_prev - d)
 * - step_penalty + r_goal [goal] - r_coll [collision]; reward_mode 1: the
 * exclusive cases of Eq. 3 (goal, else collision, else progress).
 * fov_deg: beam fan, beam k at alpha_k = -fov/2 + (k + 1/2) fov / K (Eq. 4).
 * Goals are drawn with distance in [goal_dmin, goal_dmax] m when possible.
 * n_dyn moving discs per env (radius dyn_radius, speed <= dyn_speed_max,
 * spawned >= dyn_min_sep from the robot) are stamped into a per-env layer.
 * sensor 0: exact grid traversal (range = entry distance of the first
 * blocked cell).  sensor 1: the fixed-step march of Sec. 2.2.2 (samples at
 * s * march_step metres, s = 0, 1, ...; range = distance of the first sample
 * in a blocked or off-map cell, r_max if none within r_max); needs
 * march_step > 0 and max_range / march_step <= 2^22.
 * n_sectors 0: the observation holds every beam's clipped range.
 * n_sectors m > 0: Eq. 6, the observation holds m sector minima, sector q
 * covering beams [q K/m, (q+1) K/m); every env's K must be a multiple of m. */
typedef struct {
    float dt, goal_tol, c_progress, step_penalty, r_goal, r_coll;
    int horizon;
    float goal_dmin, goal_dmax, fov_deg;
    int n_dyn;
    float dyn_radius, dyn_speed_max, dyn_min_sep;
    int reward_mode;
    int sensor;
    float march_step;
    int n_sectors;
} nav_params;

/* Fills the Table 7 defaults: dt 0.1 s, goal 0.2 m, c1 = 2, penalty 0.01,
 * +10 / -10, horizon 200, goals 2-8 m, 360 deg, no moving discs, exact
 * traversal (march_step 0.03 m for sensor 1), raw beams (no sectors). */
void nav_default_params(nav_params *p);

/* Creates a simulator (Sec. 2.2.1 batched state).  All envs use n_beams beams
 * and robots[0]; env e uses map e mod n_maps.  max_range in metres (Eq. 5's
 * r_max).  params may be NULL (defaults).  Host arrays are copied.  Returns
 * NAV_E_NOSPAWN if a used map has no free cell for the robot.  Synchronous. */
int nav_create(const nav_map *maps, int n_maps, int n_envs, int n_beams, float max_range,
               const nav_robot *robot, const nav_params *params, nav_handle **out);

/* Like nav_create with per-env arrays (each host, length n_envs, or NULL for
 * the default): env_map (default e mod n_maps), env_beams (required),
 * env_robot index into robots[0..n_robots) (default 0).  Envs of one handle
 * may mix map sizes, beam counts and robot shapes (one launch steps them). */
int nav_create_ex(const nav_map *maps, int n_maps, const int *env_map, const int *env_beams,
                  const int *env_robot, int n_envs, float max_range, const nav_robot *robots,
                  int n_robots, const nav_params *params, nav_handle **out);

/* Binds a cudaStream_t (NULL = the legacy default stream). */
int nav_set_stream(nav_handle *h, void *cuda_stream);

/* Observation layout: env e's row starts at offsets[e] and holds
 * [D_e range features, goal distance, goal bearing, v, w] (Eq. 1), where
 * the range features are the K_e clipped ranges (D_e = K_e) or, with
 * n_sectors = m, the m sector minima of Eq. 6 (D_e = m).  offsets has
 * n_envs + 1 entries (host); offsets[n_envs] is the total float count.
 * With one beam count K and no sectors, offsets[e] = e (K + 4). */
int nav_obs_offsets(const nav_handle *h, int64_t *offsets_host);
int nav_num_envs(const nav_handle *h);
int64_t nav_obs_size(const nav_handle *h);

/* Resets every env (episode 0) from the counter RNG keyed by seed and writes
 * the first observation to obs_dev (nav_obs_size floats); also writes each
 * env's next-episode record (episode 1), which a step that ends an episode
 * takes instead of drawing the reset on its critical path. */
int nav_reset(nav_handle *h, uint64_t seed, float *obs_dev);

/* One simulator step (Eq. 7): A_t -> X_{t+1} -> R_{t+1} -> (c, r, delta)
 * -> O_{t+1} -> O~_{t+1}.
 *   actions_dev   [n_envs][2] float, normalised, clamped to [-1, 1]
 *   obs_dev       [nav_obs_size] float, post-reset observation O~_{t+1}
 *   reward_dev    [n_envs] float
 *   done_dev      [n_envs] uint8: bit0 terminated (goal or collision),
 *                 bit1 truncated (horizon reached without a terminal event),
 *                 bit2 goal, bit3 collision
 *   final_obs_dev NULL, or [nav_obs_size] float: for envs that finished this
 *                 step the pre-reset observation O_{t+1}; other rows untouched.
 * Finished envs are reset in place (Sec. 2.2.3 sparse reset). */
int nav_step(nav_handle *h, const float *actions_dev, float *obs_dev, float *reward_dev,
             uint8_t *done_dev, float *final_obs_dev);

/* nav_step with host buffers, synchronous; results identical to nav_step.
 * Device staging buffers are allocated on the first call and kept.  The step
 * runs as nav_set_host_pipeline's number of launches over consecutive env
 * ranges (3 by default), each range's observations copied out on a second
 * stream while the next range computes, the rewards and flags of all ranges
 * after the last one; host buffers should be pinned for the copies to
 * overlap. */
int nav_step_host(nav_handle *h, const float *actions_host, float *obs_host,
                  float *reward_host, uint8_t *done_host, float *final_obs_host);

/* Number of env ranges nav_step_host pipelines (1..64; 1 = one launch, then
 * the copies).  Synchronises the handle's stream. */
int nav_set_host_pipeline(nav_handle *h, int parts);

/* Cap on the persistent CTAs of the fused tiled step kernels (no paper
 * counterpart): max_ctas > 0 launches at most that many (each still takes
 * tiles from the queue until none are left, so every env is stepped and the
 * results are unchanged); 0 (the default) fills every SM.  For a collector
 * that runs beside other kernels (the overlapped collector / learner of
 * Sec. 3.3): a capped step leaves SMs to the learner instead of holding the
 * whole GPU while it runs.  The split step ignores the cap.  Synchronises
 * the handle's stream. */
int nav_set_grid_cap(nav_handle *h, int max_ctas);
int nav_get_grid_cap(const nav_handle *h, int *max_ctas);

/* nav_step_host without any device allocation (the paper has no counterpart;
 * this is for callers that may not allocate device memory after start-up,
 * such as a robot control loop or embedded process that sizes its GPU memory
 * once, or an application whose own allocator must own every allocation --
 * nav_step_host allocates its staging buffers on its first call).  Same
 * arguments and results as nav_step_host, except that rows of final_obs_host
 * for envs that did not finish this step come back as zeros.  The staging
 * lives in one fixed 8 MiB device array inside the library, present on every
 * GPU that loads it until the process exits: 8 n_envs + 4 obs_size + 5 n_envs
 * bytes (plus 4 obs_size with final_obs_host), each part rounded up to 256,
 * must fit, else NAV_E_INVAL (4096 envs x 360 beams fit without final_obs_host;
 * 2048 envs x 360 beams fit with it).  The handle's device
 * must be current.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); with CUDA's default lazy module loading
 * that lookup is also when the library's module holding the array is loaded
 * and the 8 MiB array is placed on the device, which allocates device memory
 * at that moment.  So make one call on each device during start-up (a
 * warm-up step of any handle on that device), before any stream capture and
 * before the phase in which the caller may not allocate; later calls, on any
 * handle of that device, allocate nothing.  All calls on a device share the
 * array: calls that overlap on the GPU (other threads, other handles, other
 * streams) race.  Synchronous. */
int nav_step_host_noalloc(nav_handle *h, const float *actions_host, float *obs_host,
                          float *reward_host, uint8_t *done_host, float *final_obs_host);

/* Waits for the handle's stream for at most timeout_ms (<= 0: no limit), then
 * checks the device status word.  NAV_E_TIMEOUT if the deadline passed. */
int nav_sync(nav_handle *h, int timeout_ms);

/* State exchange for parity checks and checkpoints (synchronous, host):
 *   f8  [n_envs][8] float: x, y, theta, v, w, goal_x, goal_y, d_prev
 *   i2  [n_envs][2] int32: step counter, episode counter
 *   dyn [n_envs][n_dyn][4] float (x, y, vx, vy) or NULL
 * nav_set_state also sets the RNG seed used by later resets, and rewrites
 * every env's next-episode record (the spawn pose, goal and initial goal
 * distance its next reset takes, a function of seed, env and episode + 1)
 * from the new episode counters. */
int nav_get_state(nav_handle *h, float *f8_host, int32_t *i2_host, float *dyn_host);
int nav_set_state(nav_handle *h, uint64_t seed, const float *f8_host, const int32_t *i2_host,
                  const float *dyn_host);

/* Debug capture of the last scan of each env (the post-reset scan for envs
 * reset this step): enable once, then after a step read (synchronous) the
 * unclipped ranges (m), hit ids (j*W+i occupied cell, -1 left the map, -2
 * reached r_max) and cell visits per beam, each [sum_e K_e] (host). */
int nav_set_debug(nav_handle *h, int enable);
int nav_get_debug(nav_handle *h, float *ranges_host, int32_t *hits_host,
                  uint32_t *visits_host);

/* Work counters: with stats enabled every step adds the number of bitmap
 * cells the ray casts looked up (one visit = one cell of Amanatides-Woo
 * traversal) and the number of rays cast.  nav_get_stats is synchronous. */
int nav_set_stats(nav_handle *h, int enable);
int nav_get_stats(nav_handle *h, uint64_t *visits, uint64_t *rays);

/* Launch shape.  One persistent grid per step (SMs x resident CTAs, each CTA
 * taking tiles of envs that share a map and a beam count from a queue):
 *   tile_envs      envs per CTA tile (1..32)
 *   block_threads  threads per CTA (64..512, multiple of 32)
 *   smem_map_bytes shared-memory budget for the staged map (<= 200 KiB); a
 *                  map that does not fit is read through L1/L2 (see
 *                  byte_cells)
 *   max_regs       register cap per thread: 32, 40 or 64 (more resident CTAs
 *                  against fewer registers)
 *   byte_cells     map representation: 1 distance bytes (one byte per cell,
 *                  0 blocked, else the chessboard distance to the nearest
 *                  blocked cell; ray casts jump through free space), staged
 *                  in shared memory when they fit, else read through L1/L2;
 *                  2 packed bits, staged when they fit (bulk TMA copy), else
 *                  read through L1/L2; 3 distance bytes when they fit in
 *                  shared memory, else packed bits when they fit, else
 *                  distance bytes through L1/L2.  Maps above 64 MiB as bytes
 *                  always use packed bits
 *   split          1: when every map and beam table fits in one CTA's shared
 *                  memory (<= 200 KiB) and there are no moving discs, run the
 *                  step as an env-phase kernel then a ray kernel whose CTAs
 *                  keep every map resident and whose warps take 32-ray chunks
 *                  from a queue (no per-tile barriers); 2: the fused tiled
 *                  kernel; 4: the fused tiled kernel whose ray phase
 *                  refills lanes (exact traversal over distance bytes,
 *                  without moving discs; otherwise as 2): a tile's rays
 *                  form one range, every lane walks its own ray and a warp
 *                  with idle lanes takes as many new rays as it has idle
 *                  lanes from a shared counter, instead of retiring 32-ray
 *                  chunks when their slowest ray ends.  3 is rejected.
 *                  nav_get_launch reports the path in use (1, 2 or 4).
 * 0 keeps the current value.  A new handle starts at tile_envs 8, 512
 * threads, 160 KiB, 40 registers, byte_cells 1, fused kernel.  Synchronises
 * the handle's stream. */
int nav_set_launch(nav_handle *h, int tile_envs, int block_threads, int smem_map_bytes,
                   int max_regs, int byte_cells, int split);
int nav_get_launch(const nav_handle *h, int *tile_envs, int *block_threads,
                   int *smem_map_bytes, int *max_regs, int *byte_cells, int *split);

/* Order of the tile queue (no paper counterpart): 0 largest map x beam count
 * first (ties in map order), 1 most expensive tiles first, by envs x beams x
 * the mean cells per ray of a fixed host-side sample of rays on the map.
 * The autotuner tries both.  Synchronises the handle's stream. */
int nav_set_tile_order(nav_handle *h, int order);
int nav_get_tile_order(const nav_handle *h, int *order);

/* Autotuner (no paper counterpart; it picks the launch shape for this
 * handle's mix of map sizes, beam counts and robots).  From a device copy of
 * the current state it times `steps` steps of each candidate with uniform
 * random actions: first tile_envs x block_threads x max_regs, with chunked
 * and (when eligible) refilled lanes, then the
 * staging mode and shared-memory budget for the best shape, then the tile
 * order, then the split step when eligible; last, the four fastest distinct
 * settings again with four times the steps and the L2 flushed between steps
 * (a 160 MiB device scratch, allocated on the first call and kept by the
 * handle).  It restores the state and keeps the fastest candidate of that
 * last pass.  Synchronous.  best_ms (host, may be NULL) receives the
 * winner's mean step time with the L2 flushed. */
int nav_autotune(nav_handle *h, int steps, float *best_ms);

/* Writes n_envs uniform [-1, 1]^2 actions keyed by (seed, env, step) to
 * actions_dev ([n_envs][2] float) on the handle's stream: a seeded input
 * generator for throughput runs. */
int nav_uniform_actions(nav_handle *h, uint64_t seed, uint32_t step, float *actions_dev);

/* CUDA graph of n_steps consecutive nav_step calls: step t reads
 * actions_dev + t * 2 * n_envs ([n_steps][n_envs][2] float) and overwrites
 * obs_dev, reward_dev, done_dev (and final_obs_dev if not NULL).  The graph is
 * owned by the handle (a new capture replaces it) and needs a non-default
 * stream bound with nav_set_stream.  nav_graph_launch replays it. */
int nav_graph_capture(nav_handle *h, int n_steps, const float *actions_dev, float *obs_dev,
                      float *reward_dev, uint8_t *done_dev, float *final_obs_dev);
int nav_graph_launch(nav_handle *h);

/* Tensor-core GEMM of the policy and critic MLPs (Sec. 2.1 LeakyReLU MLPs;
 * the learner of Sec. 2.3): C = act(A B^T + bias) on the stream `stream`
 * (cudaStream_t, NULL = default).
 *   a_dev [m][lda] BF16, b_dev [n][ldb] BF16 (both K-major: k contiguous),
 *         16-byte aligned, lda and ldb multiples of 8 and >= k
 *   bias_dev [n] float or NULL; act 0 = none, 1 = LeakyReLU (slope 0.01)
 *   outputs (each optional): c32_dev [m][ldc32] float, c16_dev [m][ldc16]
 *         BF16, c16t_dev [n][ldct] BF16 (the transpose, for the next GEMM's
 *         K-major operand)
 *   status_dev int or NULL: bit 0 set if a tensor-core completion wait timed out
 * FP32 accumulation; tcgen05 MMA with TMEM accumulators, 128 x <=256 tiles. */
int nav_gemm_bf16(const void *a_dev, int lda, const void *b_dev, int ldb, int m, int n, int k,
                  const float *bias_dev, int act, float *c32_dev, int ldc32, void *c16_dev,
                  int ldc16, void *c16t_dev, int ldct, int *status_dev, void *stream);

/* Random-gather rate probe: the memory ceiling of the beam traversal of
 * Sec. 2.2.1, whose lanes read single map bytes at unrelated addresses.
 * n_blocks CTAs of 256 threads; each thread keeps 8 generators
 * s <- 1664525 s + 1013904223 (uint32), the generator for thread g of the
 * launch (g = block * 256 + thread) and chain c starting at
 * s = (8 g + c) * 2654435761 + 0x9E3779B9; per iteration each chain steps
 * once and reads the byte at offset s >> (32 - log2(bytes)) of the table.
 *   where 0: the table is the CTA's own shared memory (bytes <= 196608),
 *            byte j = (j * 2654435761) >> 24 (uint32 arithmetic);
 *            table_dev is ignored
 *   where 1: the table is table_dev (device memory of at least `bytes`
 *            bytes, caller-owned), read through the read-only data path
 *   bytes: a power of two in [1024, 2^31]; iters >= 0 iterations per thread
 *   sums_dev [n_blocks] uint32 (caller-owned): each CTA's sum of the bytes
 *            it read (wrapping), written, not accumulated
 * Launches one kernel on `stream` (cudaStream_t, NULL = default); the caller
 * times it.  NAV_E_INVAL for an argument outside these ranges. */
int nav_gather_probe(int where, const void *table_dev, int64_t bytes, int n_blocks, int iters,
                     uint32_t *sums_dev, void *stream);

/* Tensor-pipe rate probe (measurement, no paper counterpart: the costs that
 * set how the fused actor of nav_rollout_fused stages its weights).  Each of
 * n_blocks CTAs has one thread issue n_mma back-to-back tcgen05.mma
 * (kind::f16, M 128, N n, K 16, BF16 zero operands in shared memory) into
 * its own 256 TMEM columns, with a tcgen05.commit after every commit_every
 * MMAs (0: none but the final one) that the thread waits on when wait is 1,
 * and a final commit it waits on; ns_dev[b] (uint64, caller-owned, n_blocks
 * entries) receives CTA b's %globaltimer nanoseconds from its first issue
 * to the final completion.  At most two CTAs share an SM.
 *   n: a multiple of 16 in [16, 256]; n_mma in [1, 2^20]; commit_every >= 0;
 *   wait 0 or 1; n_blocks in [1, 1024]
 *   status_dev (int, caller-owned): bit 0 set when a bounded wait gave up
 *   (the CTA then waits once more, frees its TMEM and returns)
 * Launches one kernel on `stream`; NAV_E_INVAL for an argument outside these
 * ranges. */
int nav_mma_probe(int n, int n_mma, int commit_every, int wait, int n_blocks,
                  unsigned long long *ns_dev, int *status_dev, void *stream);

/* Policy network (Sec. 2.1 policy MLP; the FastDSAC actor of Sec. 2.3): a
 * tanh-squashed Gaussian actor obs_dim -> hidden -> hidden -> 4 (mean 2, raw
 * log-std 2) with LeakyReLU (slope 0.01); log sigma = -5 + 5 (tanh(r) + 1)/2,
 * action a = tanh(mean + sigma eps).  FP32 master weights initialised
 * U(-1/sqrt(in), 1/sqrt(in)) from a counter hash of `seed`, BF16 copies for
 * the tensor cores.  max_batch bounds the rows of one nav_policy_act call.
 * Weights in host order [W1 (hidden x obs_dim, row-major), b1, W2, b2, W3, b3]. */
typedef struct nav_policy nav_policy;
int nav_policy_create(int obs_dim, int hidden, int max_batch, uint64_t seed, nav_policy **out);

/* Like nav_policy_create with n_hidden (1..4) hidden layers of `hidden`
 * units (any width; Table 3's actor is (100) x 4) and, if ipap_features > 0,
 * the IPAPRec input transform of Eq. 2 on the first ipap_features
 * observation features (the range readings): x = 1 / (l - beta), with
 * beta = ipap_beta (< 0) until a trainer's nav_trainer_sync_policy copies
 * its trained beta.  Any per-feature input scale multiplies after it. */
int nav_policy_create_ex(int obs_dim, int hidden, int n_hidden, int ipap_features,
                         float ipap_beta, int max_batch, uint64_t seed, nav_policy **out);
/* The policy's current beta of Eq. 2 (synchronous). */
int nav_policy_get_beta(const nav_policy *p, float *beta_host);
void nav_policy_free(nav_policy *p);
int64_t nav_policy_num_params(const nav_policy *p);
int nav_policy_get_weights(nav_policy *p, float *host);       /* synchronous */
int nav_policy_set_weights(nav_policy *p, const float *host); /* synchronous */

/* Actions for n observation rows (obs_dev row r at r * obs_stride floats):
 * mode 0 deterministic a = tanh(mean), mode 1 sampled with eps from the
 * counter hash of (seed, row, step).  actions_dev [n][2] float; logp_dev [n]
 * and out_dev [n][4] (the network's raw outputs) may be NULL.  BF16 tensor
 * cores (tcgen05) with FP32 accumulation; asynchronous on `stream`.
 * nav_policy_act_fp32 is the same in plain FP32 on CUDA cores. */
int nav_policy_act(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n, int mode,
                   uint64_t seed, uint32_t step, float *actions_dev, float *logp_dev,
                   float *out_dev, void *stream);
int nav_policy_act_fp32(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n, int mode,
                        uint64_t seed, uint32_t step, float *actions_dev, float *logp_dev,
                        float *out_dev, void *stream);
/* nav_policy_act with the noise step read from the device counter step_dev
 * (one uint64, caller-owned; the low 32 bits are the step) and incremented
 * after the read, so that a CUDA graph holding the call draws fresh noise on
 * every replay. */
int nav_policy_act_counted(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n,
                           int mode, uint64_t seed, uint64_t *step_dev, float *actions_dev,
                           float *logp_dev, float *out_dev, void *stream);

/* Per-feature input scale (host, obs_dim floats) multiplied into the
 * observation before the network (NULL removes it).  Synchronous. */
int nav_policy_set_input_scale(nav_policy *p, const float *scale_host);

/* Reactive goal-seeking controller, a hand-written baseline policy without learning
 * (no paper counterpart): among beams whose range and both neighbours' exceed
 * 0.6 m, head for the one closest to the goal bearing; turn rate 2 x heading
 * error, speed scaled by the heading error's cosine and the range straight
 * ahead; rotate in place when no beam is clear.  obs rows as nav_step writes
 * them (n_beams beams over fov_deg), actions_dev [n][2] normalised for a
 * robot with speeds [0, v_max] and turn rates [-w_max, w_max]. */
int nav_reactive_act(const float *obs_dev, int64_t obs_stride, int n, int n_beams, float fov_deg,
                     float v_max, float w_max, float *actions_dev, void *stream);

/* Rollout with the policy in the loop (Sec. 2.3 collector side): n_steps of
 * [policy actions from obs_dev -> nav_step], all on the handle's stream (so a
 * CUDA graph can capture it).  obs_dev must hold the current observation
 * (from nav_reset or the previous step); every env must use the same beam
 * count.  actions_dev [n_envs][2], reward_dev, done_dev as for nav_step hold
 * the last step's values.  fp32_path 1 uses nav_policy_act_fp32. */
int nav_rollout(nav_handle *h, nav_policy *p, int n_steps, int mode, uint64_t seed,
                uint32_t step0, float *obs_dev, float *actions_dev, float *reward_dev,
                uint8_t *done_dev, int fp32_path);

/* The same rollout with the actor evaluated inside the step kernel (Sec. 2.3
 * collector, Eq. 7 with the policy in the loop): the actions for obs_dev come
 * from nav_policy_act once (or, with actions_ready set, are already in
 * actions_dev: the actions a previous call left there for this obs_dev),
 * then each of the n_steps launches steps a tile of
 * up to 128 envs (env phase, ray casts), writes the new observation rows to
 * obs_dev and, scaled and rounded to BF16, into a tile in shared memory, runs
 * the actor on that tile on the tensor cores (weights streamed from L2 by
 * 64-wide chunks, FP32 accumulation in tensor memory) and writes each env's
 * next action to actions_dev: the policy never reads the observations back
 * from global memory and there is no separate policy launch.  Step t's
 * actions use the noise step step0 + t as in nav_rollout (mode 0:
 * deterministic tanh(mean)).  On return obs_dev, reward_dev and done_dev hold
 * the last step's values and actions_dev the actions for obs_dev.
 * Requirements (else NAV_E_INVAL): one beam count K, raw beams (no sectors),
 * the exact traversal, no moving discs, every map's distance bytes within
 * ~120 KiB; an actor (K + 4) -> H -> H -> 4 with H <= 256, K + 4 <= 384, no
 * Eq. 2 input, max_batch >= n_envs. */
int nav_rollout_fused(nav_handle *h, nav_policy *p, int n_steps, int mode, uint64_t seed,
                      uint32_t step0, float *obs_dev, float *actions_dev, float *reward_dev,
                      uint8_t *done_dev, int actions_ready);

/* FastDSAC learner (Sec. 2.3, FastDSAC paragraph; hyperparameters of Table 4,
 * workload overrides for batch, gamma and the optimiser).  Actor as in
 * nav_policy; twin critics (obs_dim + 2) -> hidden -> hidden -> (mean, raw
 * scale) with sigma = softplus(raw) + 0.1; target critics by Polyak
 * averaging (tau).  Critic loss w Huber(m - y_mean) + Gaussian NLL of the
 * sampled target y (clipped double Q, draw clipped to +-3 sigma) with the
 * uncertainty weight w = clip(sbar^2 / sigma^2, 0.5, 2); actor loss
 * alpha logpi - min_i m_i every policy_freq critic updates; log alpha by Adam
 * towards target_entropy.  BF16 tensor-core GEMMs (tcgen05) with FP32 master
 * weights and FP32 Adam. */
/* algo 1 (Sec. 2.3 FastSAC; Table 5): twin categorical critics with n_atoms
 * logits on the support z_i = v_min + i (v_max - v_min) / (n_atoms - 1); the
 * target takes, per sample, the target critic with the smaller expected
 * value, moves its atoms to rs r + gamma (1 - term) (z - alpha logpi') (clipped
 * to the support) and projects them back by linear interpolation; both
 * critics descend the cross-entropy to it; the actor descends
 * mean(alpha logpi - min_j E[Q_j]); alpha as for FastDSAC.  Needs networks on
 * the fused passes (every width <= 128).  Gaussian-critic fields (tau_b,
 * huber_delta) are unused.
 * n_hidden hidden layers of `hidden` units in every network (1..4).
 * weight_decay: decoupled (AdamW, Table 3) decay of weights and biases,
 * p <- p (1 - lr wd) before each Adam step; 0 = Adam.
 * ipap_features > 0: Eq. 2 on the first ipap_features observation features
 * of every network's input, x = 1 / (l - beta) with one trainable beta
 * (initial ipap_beta_init), stored raw in the replay and transformed when a
 * batch is drawn; beta descends the actor loss by Adam (lr_actor) and is
 * kept <= ipap_beta_max < 0 so that l - beta > 0 for every range l >= 0. */
typedef struct {
    int obs_dim, hidden, batch;
    long long replay_capacity;
    float lr_actor, lr_critic, lr_alpha, beta1, beta2, gamma, tau, tau_b, reward_scale,
        huber_delta, alpha_init, target_entropy;
    int policy_freq;
    uint64_t seed;
    int n_hidden;
    float weight_decay;
    int ipap_features;
    float ipap_beta_init, ipap_beta_max;
    int algo;           /* 0 FastDSAC (Gaussian critics), 1 FastSAC (C51 critics) */
    int n_atoms;        /* FastSAC: atoms of the categorical critics (2..128) */
    float v_min, v_max; /* FastSAC: support [v_min, v_max] */
} nav_train_cfg;
typedef struct nav_trainer nav_trainer;
void nav_train_default_cfg(nav_train_cfg *c); /* obs 364, hidden 256 x 2, batch 4096, replay
                                                 4 Mi, lr 3e-4, betas (0.9, 0.95), gamma 0.99,
                                                 tau 0.1, tau_b 0.005, reward scale 0.4,
                                                 Huber 50, alpha 0.001, target entropy -1,
                                                 policy freq 2, no weight decay, no Eq. 2
                                                 (beta -0.2 initial, <= -0.01) */
int nav_trainer_create(const nav_train_cfg *cfg, nav_trainer **out); /* synchronous */
void nav_trainer_free(nav_trainer *t);
const char *nav_trainer_last_error(const nav_trainer *t);

/* Appends n_envs transitions to the device replay ring (obs and next obs
 * stored as BF16): next obs = final_obs_dev's row for envs whose done flag
 * has bit0 or bit1 set (final_obs_dev may be NULL), else next_obs_dev's;
 * terminal = bit0 (a truncated episode still bootstraps).  All arrays are
 * device rows of obs_dim floats / [n_envs][2] actions / [n_envs] rewards. */
int nav_train_insert(nav_trainer *t, const float *obs_dev, const float *act_dev,
                     const float *rew_dev, const uint8_t *done_dev, const float *next_obs_dev,
                     const float *final_obs_dev, int n_envs, void *stream);

/* n_updates gradient steps on batches drawn uniformly from the replay (needs
 * at least one batch of transitions), asynchronous on `stream`.  Update
 * indices, replay size and Adam's bias corrections live in device counters,
 * so the launches can be captured in a CUDA graph (by the caller, or by
 * nav_trainer_set_graphs). */
int nav_train_update(nav_trainer *t, int n_updates, void *stream);

/* Overlapped collector / learner (Sec. 3.3's producer-consumer pipeline):
 * before updates that run concurrently with a nav_train_insert of n_pending
 * transitions on another stream, call this on the learner's stream ahead of
 * the fork point; it snapshots the replay's head and size, and the updates'
 * draws then skip the n_pending slots the insert overwrites (so no update
 * reads a slot being written).  n_pending = 0 (after the join) restores the
 * plain draw.  Asynchronous on `stream`. */
int nav_train_overlap(nav_trainer *t, int n_pending, void *stream);

/* on = 1: nav_train_update captures each distinct (n_updates, policy phase)
 * sequence once on its (non-null) stream and replays the graph afterwards
 * (about 180 small launches per update become one graph launch).  Results
 * are those of the launches themselves. */
int nav_trainer_set_graphs(nav_trainer *t, int on);

/* Path of the updates.  Networks whose every width is <= 128 (batch a
 * multiple of 128) run on fused passes by default: one
 * launch runs every layer of a network's forward or backward for 128 batch
 * rows (operands in shared memory, accumulators in TMEM), the twin critics
 * share launches, and one kernel applies AdamW to a whole network; ~25
 * launches per update instead of ~180.  on = 0 selects the per-layer GEMM
 * path (same arithmetic); on = 1 fails with NAV_E_INVAL for wider networks. */
int nav_trainer_set_fused(nav_trainer *t, int on);

/* Per-feature input scale applied to observations as they enter the replay
 * (the same scale must be set on the acting policy).  Synchronous. */
int nav_trainer_set_input_scale(nav_trainer *t, const float *scale_host);

/* Copies the trainer's actor into a policy handle (actor-weight sync). */
int nav_trainer_sync_policy(nav_trainer *t, nav_policy *p, void *stream);

/* Parity hooks (synchronous, host buffers): what 0..4 = parameters of actor,
 * critic 1, critic 2, target 1, target 2 (order as nav_policy weights; set=1
 * writes); 10..12 = last gradients of actor, critic 1, critic 2; 20 batch
 * indices, 21 actor-update noise, 22 next-action noise, 23 target noise,
 * 24 scalars (16 floats: [0] log alpha, [1] sbar, [11] last gradient of Eq. 2's
 * beta, [12] beta), 32 FastSAC target distributions [batch][n_atoms], 25 y,
 * 26 y_mean, 27 critic-1 outputs ([batch][2], FastSAC [batch][n_atoms]),
 * 28 logpi of the actor update, 29 its actions, 30 actor outputs, 31 logpi of
 * the next actions. */
int nav_trainer_io(nav_trainer *t, int what, int set, void *host);
/* Replay size and update counts from the device counters (synchronous). */
int nav_trainer_counts(const nav_trainer *t, int64_t *replay_size, int64_t *critic_updates,
                       int64_t *actor_updates);

/* Evaluation (success-rate protocol of Sec. 3.2): begin clears per-env
 * accumulators, accumulate adds one step's rewards (FP64) to envs whose first
 * episode is still running and records success (goal without collision) when
 * it ends, result reduces success count and return sum in FP64 and copies the
 * two doubles to the host (synchronous). */
int nav_eval_begin(nav_trainer *t, int n_envs, void *stream);
int nav_eval_accumulate(nav_trainer *t, const float *reward_dev, const uint8_t *done_dev,
                        int n_envs, void *stream);
int nav_eval_result(nav_trainer *t, int n_envs, double *successes, double *return_sum,
                    void *stream);

const char *nav_last_error(const nav_handle *h);
void nav_free(nav_handle *h);

#ifdef __cplusplus
}
#endif
#endif
