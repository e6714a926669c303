"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds input generators only (occupancy maps, robot presets,
episode constants, action streams); none of the simulator's arithmetic lives
here.  The paper trains on occupancy bitmaps it does not describe (Sec. 2.2.1)
and publishes no maps, so every workload is a seeded synthetic stand-in:

* maps: random axis-aligned boxes (sides U[0.2, 1.0] m) and discs
  (radius U[0.1, 0.5] m), plus axis-aligned corridor walls (1-2 cells thick,
  2-6 m long) for the larger workloads, drawn until the occupied fraction
  reaches the target.  A cell is occupied when its closed square meets the
  shape.
* robots: a TurtleBot2-like disc and a Go2-like rectangle (Tables 8-9, with
  the workload's radius, size and velocity bounds).
* actions: i.i.d. uniform [-1, 1]^2 float32 per env and step.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RES = 0.05  # metres per cell


@dataclasses.dataclass(frozen=True)
class Robot:
    shape: int  # 0 disc, 1 rectangle
    radius: float = 0.0
    length: float = 0.0
    width: float = 0.0
    v_min: float = 0.0
    v_max: float = 0.5
    w_min: float = -1.0
    w_max: float = 1.0


DISC = Robot(shape=0, radius=0.18, v_min=0.0, v_max=0.5, w_min=-1.0, w_max=1.0)
RECT = Robot(shape=1, length=0.70, width=0.31, v_min=0.0, v_max=1.0, w_min=-1.5, w_max=1.5)
# The paper's platforms (Tables 8-9): action bounds (0, -pi/4) .. (0.5, pi/4)
TURTLEBOT2 = Robot(shape=0, radius=0.20, v_min=0.0, v_max=0.5, w_min=-math.pi / 4,
                   w_max=math.pi / 4)
GO2 = Robot(shape=1, length=0.80, width=0.41, v_min=0.0, v_max=0.5, w_min=-math.pi / 4,
            w_max=math.pi / 4)


@dataclasses.dataclass(frozen=True)
class Params:
    """Episode constants (Table 7) with the workload's overrides."""
    dt: float = 0.1
    goal_tol: float = 0.2
    c_progress: float = 2.0
    step_penalty: float = 0.01
    r_goal: float = 10.0
    r_coll: float = 10.0
    horizon: int = 200
    goal_dmin: float = 2.0
    goal_dmax: float = 8.0
    fov_deg: float = 360.0
    n_dyn: int = 0
    dyn_radius: float = 0.18
    dyn_speed_max: float = 0.5
    dyn_min_sep: float = 1.0
    reward_mode: int = 0
    sensor: int = 0           # 0 exact grid traversal, 1 fixed-step march (Sec. 2.2.2)
    march_step: float = 0.03  # metres between march samples
    n_sectors: int = 0        # 0 raw beams, else Eq. 6 sector minima in the observation


def _rasterise_box(occ, x0, y0, x1, y1, res):
    h, w = occ.shape
    i0 = max(int(math.floor(x0 / res)), 0)
    i1 = min(int(math.ceil(x1 / res)) - 1, w - 1)
    j0 = max(int(math.floor(y0 / res)), 0)
    j1 = min(int(math.ceil(y1 / res)) - 1, h - 1)
    if i0 > i1 or j0 > j1:
        return 0
    before = int(occ[j0:j1 + 1, i0:i1 + 1].sum())
    occ[j0:j1 + 1, i0:i1 + 1] = 1
    return (j1 - j0 + 1) * (i1 - i0 + 1) - before


def _rasterise_disc(occ, cx, cy, r, res):
    h, w = occ.shape
    i0 = max(int(math.floor((cx - r) / res)), 0)
    i1 = min(int(math.ceil((cx + r) / res)), w - 1)
    j0 = max(int(math.floor((cy - r) / res)), 0)
    j1 = min(int(math.ceil((cy + r) / res)), h - 1)
    if i0 > i1 or j0 > j1:
        return 0
    ii = np.arange(i0, i1 + 1) * res
    jj = np.arange(j0, j1 + 1) * res
    # distance from the centre to each closed cell square
    ddx = np.maximum(np.maximum(ii - cx, cx - (ii + res)), 0.0)
    ddy = np.maximum(np.maximum(jj - cy, cy - (jj + res)), 0.0)
    hit = (ddx[None, :] ** 2 + ddy[:, None] ** 2) <= r * r
    win = occ[j0:j1 + 1, i0:i1 + 1]
    new = int((hit & (win == 0)).sum())
    win[hit] = 1
    return new


def make_map(seed: int, width: int, height: int, occupancy: float, corridors: bool = False,
             res: float = RES) -> np.ndarray:
    """One seeded occupancy map, uint8 [height][width], 1 = occupied."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((height, width), np.uint8)
    wm, hm = width * res, height * res
    target = int(round(occupancy * width * height))
    filled = 0
    kinds = 3 if corridors else 2
    guard = 0
    while filled < target and guard < 1_000_000:
        guard += 1
        kind = int(rng.integers(0, kinds))
        if kind == 0:
            sx, sy = rng.uniform(0.2, 1.0, size=2)
            cx, cy = rng.uniform(0.0, wm), rng.uniform(0.0, hm)
            filled += _rasterise_box(occ, cx - sx / 2, cy - sy / 2, cx + sx / 2, cy + sy / 2, res)
        elif kind == 1:
            r = rng.uniform(0.1, 0.5)
            cx, cy = rng.uniform(0.0, wm), rng.uniform(0.0, hm)
            filled += _rasterise_disc(occ, cx, cy, r, res)
        else:
            length = rng.uniform(2.0, 6.0)
            thick = int(rng.integers(1, 3)) * res
            cx, cy = rng.uniform(0.0, wm), rng.uniform(0.0, hm)
            if rng.integers(0, 2) == 0:
                filled += _rasterise_box(occ, cx, cy, cx + length, cy + thick, res)
            else:
                filled += _rasterise_box(occ, cx, cy, cx + thick, cy + length, res)
    return occ


def uniform_actions(seed: int, n_steps: int, n_envs: int) -> np.ndarray:
    """float32 [n_steps][n_envs][2], i.i.d. uniform on [-1, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_steps, n_envs, 2)).astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    maps: list            # list of uint8 [H][W]
    env_map: np.ndarray   # int32 [E]
    env_beams: np.ndarray  # int32 [E]
    env_robot: np.ndarray  # int32 [E]
    robots: list          # list of Robot
    max_range: float
    params: Params
    res: float = RES

    @property
    def n_envs(self) -> int:
        return int(self.env_map.shape[0])


def config_small(n_envs: int = 64, seed: int = 1) -> Workload:
    """64 envs, one 64x64 map at 15 % occupancy, 180 beams over 360 deg,
    r_max 4 m, disc robot r = 0.18 m; the map (3.2 m) is too small for
    2-8 m goals, so goals are drawn at >= 1 m."""
    occ = make_map(seed, 64, 64, 0.15)
    return Workload(
        name="plain-64env-64x64-180beam",
        maps=[occ],
        env_map=np.zeros(n_envs, np.int32),
        env_beams=np.full(n_envs, 180, np.int32),
        env_robot=np.zeros(n_envs, np.int32),
        robots=[DISC],
        max_range=4.0,
        params=Params(goal_dmin=1.0, goal_dmax=1.0e9),
    )


def config_throughput(n_envs: int = 4096, n_maps: int = 16, size: int = 256,
                      seed0: int = 100) -> Workload:
    """4096 envs over 16 seeded 256x256 maps (10-25 % boxes, discs and
    corridor walls), 360 beams, r_max 6 m, disc robot, goals 2-8 m;
    env e uses map e mod 16."""
    maps = []
    for m in range(n_maps):
        occ_target = np.random.default_rng(seed0 + m + 7919).uniform(0.10, 0.25)
        maps.append(make_map(seed0 + m, size, size, occ_target, corridors=True))
    e = np.arange(n_envs, dtype=np.int32)
    return Workload(
        name="plain-4096env-16x256x256-360beam",
        maps=maps,
        env_map=(e % n_maps).astype(np.int32),
        env_beams=np.full(n_envs, 360, np.int32),
        env_robot=np.zeros(n_envs, np.int32),
        robots=[DISC],
        max_range=6.0,
        params=Params(),
    )


def config_uneven(n_envs: int = 16384, n_maps: int = 64, seed0: int = 200,
                  max_side: int = 1024, n_dyn: int = 8) -> Workload:
    """16384 envs over 64 maps with sides log-uniform in 128..1024, beams
    180/360/720 by e mod 3, disc robots on even envs and rectangles on odd
    ones, 8 moving discs per env, r_max 6 m."""
    maps = []
    for m in range(n_maps):
        r = np.random.default_rng(seed0 + m + 104729)
        side = int(round(math.exp(r.uniform(math.log(128), math.log(max_side)))))
        side = max(32, min(max_side, side))
        occ_target = r.uniform(0.10, 0.25)
        maps.append(make_map(seed0 + m, side, side, occ_target, corridors=True))
    e = np.arange(n_envs, dtype=np.int32)
    beams = np.array([180, 360, 720], np.int32)[e % 3]
    return Workload(
        name="uneven-16384env-64maps-128to1024-mixedbeams-dyn8",
        maps=maps,
        env_map=(e % n_maps).astype(np.int32),
        env_beams=beams.astype(np.int32),
        env_robot=(e % 2).astype(np.int32),
        robots=[DISC, RECT],
        max_range=6.0,
        params=Params(n_dyn=n_dyn),
    )


def paper_params(fov_deg: float, goal_dmax: float = 6.0) -> Params:
    """Table 7's sensing, episode and reward constants: 0.03 m fixed-step
    march, 30 sector minima (of 1080 beams), horizon 200, dt 0.1 s, goal
    0.2 m, the exclusive reward cases of Eq. 3 (+10 / -10 / 2 x progress).
    The paper gives no goal distance band; goals are drawn 1-6 m away in a
    straight line, so that a detour still fits the 10 m an episode can travel
    (200 steps x 0.1 s x 0.5 m/s)."""
    return Params(reward_mode=1, step_penalty=0.0, goal_dmin=1.0, goal_dmax=goal_dmax,
                  fov_deg=fov_deg, sensor=1, march_step=0.03, n_sectors=30)


def config_paper(robot: str = "turtlebot2", n_envs: int = 1024, seed: int = 31,
                 occupancy: float = 0.10, beams: int = 1080,
                 goal_dmax: float = 6.0, corridors: bool = False) -> Workload:
    """The paper's training setting (Sec. 2.2.1, Tables 7-9): every env on
    one shared map, 10 x 10 m for the TurtleBot2 (disc r = 0.20 m, 270 deg
    fan) or 13.5 x 13.5 m for the Go2 (0.80 x 0.41 m rectangle, 360 deg),
    1080 beams marched at 0.03 m to 20 m and pooled into 30 sectors.  The
    map content is not published: a seeded cluttered room of boxes and discs
    at `occupancy` stands in (0.05 m cells; corridor walls optional)."""
    if robot == "turtlebot2":
        side, rb, fov = 200, TURTLEBOT2, 270.0
    elif robot == "go2":
        side, rb, fov = 270, GO2, 360.0
    else:
        raise ValueError(robot)
    occ = make_map(seed, side, side, occupancy, corridors=corridors)
    return Workload(
        name=f"paper-{robot}-{n_envs}env-{side}x{side}-{beams}beam-march-30sector",
        maps=[occ],
        env_map=np.zeros(n_envs, np.int32),
        env_beams=np.full(n_envs, beams, np.int32),
        env_robot=np.zeros(n_envs, np.int32),
        robots=[rb],
        max_range=20.0,
        params=paper_params(fov, goal_dmax),
    )
