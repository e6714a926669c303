/*
 * nav_oracle.h -- interface of the CPU oracle of the FlashNav simulator step.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Private to oracle/: the CUDA path never includes it.
 */
#ifndef NAV_ORACLE_H
#define NAV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int width, height;
    float resolution;   /* metres per cell */
    const uint8_t *occ; /* row-major, nonzero = occupied */
} or_map;

typedef struct {
    int shape; /* 0 disc, 1 rectangle */
    float radius, length, width;
    float v_min, v_max, w_min, w_max;
} or_robot;

typedef struct {
    float dt, goal_tol, c_progress, step_penalty, r_goal, r_coll;
    int horizon;
    float goal_dmin, goal_dmax, fov_deg;
    int n_dyn;
    float dyn_radius, dyn_speed_max, dyn_min_sep;
    int reward_mode; /* 0 additive (progress - penalty + goal - collision), 1 exclusive cases of Eq. 3 */
    int sensor;       /* 0 exact grid traversal, 1 fixed-step march (Sec. 2.2.2) */
    float march_step; /* metres between march samples */
    int n_sectors;    /* 0: raw beams in the observation, else min-pooled sectors (Eq. 6) */
} or_params;

typedef struct or_sim or_sim;

void or_default_params(or_params *p);
or_sim *or_create(const or_map *maps, int n_maps, const int *env_map, const int *env_k,
                  const int *env_robot, int n_envs, float max_range, const or_robot *robots,
                  int n_robots, const or_params *params);
void or_free(or_sim *s);
void or_set_threads(or_sim *s, int n);
int or_reset(or_sim *s, uint64_t seed, float *obs);
int or_step(or_sim *s, const float *actions, float *obs, float *reward, uint8_t *done,
            float *final_obs);
uint64_t or_visits(const or_sim *s);
void or_get_state(const or_sim *s, float *f8, int32_t *i2, float *dyn);
void or_set_state(or_sim *s, uint64_t seed, const float *f8, const int32_t *i2, const float *dyn);
void or_get_debug(const or_sim *s, float *ranges, int32_t *hits, uint32_t *visits);
int or_spawn_count(const or_sim *s, int map, int robot);
int or_comp_count(const or_sim *s, int map, int robot);
void or_comp_labels(const or_sim *s, int map, int robot, int *out);

/* primitives, exposed for the pin tests */
void or_sincosf(float x, float *s, float *c);
uint64_t or_hash(uint64_t seed, uint64_t env, uint64_t episode, uint64_t k);
float or_march_ray(const uint8_t *occ, int w, int h, float res, float x, float y, float dx,
                   float dy, float step, float max_range, int32_t *hit, uint32_t *visits);
float or_cast_ray(const uint8_t *occ, int w, int h, float res, float x, float y, float dx,
                  float dy, float max_range, int32_t *hit, uint32_t *visits);
int or_footprint(const uint8_t *occ, int w, int h, float res, int shape, float radius,
                 float length, float width, float x, float y, float theta);
void or_integrate(float x, float y, float th, float v, float w, float dt, float *xo, float *yo,
                  float *tho);

#ifdef __cplusplus
}
#endif
#endif
