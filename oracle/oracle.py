"""ctypes wrapper of the C oracle (nav_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the CPU-baseline leg of
bench.py use it.  It never imports the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nav_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11", "-shared",
          "-fPIC"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nav_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Map(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("resolution", C.c_float),
                ("occ", C.c_void_p)]


class _Robot(C.Structure):
    _fields_ = [("shape", C.c_int), ("radius", C.c_float), ("length", C.c_float),
                ("width", C.c_float), ("v_min", C.c_float), ("v_max", C.c_float),
                ("w_min", C.c_float), ("w_max", C.c_float)]


class _Params(C.Structure):
    _fields_ = [("dt", C.c_float), ("goal_tol", C.c_float), ("c_progress", C.c_float),
                ("step_penalty", C.c_float), ("r_goal", C.c_float), ("r_coll", C.c_float),
                ("horizon", C.c_int), ("goal_dmin", C.c_float), ("goal_dmax", C.c_float),
                ("fov_deg", C.c_float), ("n_dyn", C.c_int), ("dyn_radius", C.c_float),
                ("dyn_speed_max", C.c_float), ("dyn_min_sep", C.c_float),
                ("reward_mode", C.c_int), ("sensor", C.c_int), ("march_step", C.c_float),
                ("n_sectors", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.c_void_p
        L.or_create.restype = P
        L.or_create.argtypes = [P, C.c_int, P, P, P, C.c_int, C.c_float, P, C.c_int, P]
        L.or_free.argtypes = [P]
        L.or_set_threads.argtypes = [P, C.c_int]
        L.or_reset.argtypes = [P, C.c_uint64, P]
        L.or_step.argtypes = [P, P, P, P, P, P]
        L.or_visits.restype = C.c_uint64
        L.or_visits.argtypes = [P]
        L.or_get_state.argtypes = [P, P, P, P]
        L.or_set_state.argtypes = [P, C.c_uint64, P, P, P]
        L.or_get_debug.argtypes = [P, P, P, P]
        L.or_spawn_count.argtypes = [P, C.c_int, C.c_int]
        L.or_comp_count.argtypes = [P, C.c_int, C.c_int]
        L.or_comp_labels.argtypes = [P, C.c_int, C.c_int, P]
        L.or_sincosf.argtypes = [C.c_float, P, P]
        L.or_hash.restype = C.c_uint64
        L.or_hash.argtypes = [C.c_uint64] * 4
        L.or_cast_ray.restype = C.c_float
        L.or_cast_ray.argtypes = [P, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                  C.c_float, C.c_float, C.c_float, P, P]
        L.or_march_ray.restype = C.c_float
        L.or_march_ray.argtypes = [P, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                   C.c_float, C.c_float, C.c_float, C.c_float, P, P]
        L.or_footprint.argtypes = [P, C.c_int, C.c_int, C.c_float, C.c_int, C.c_float,
                                   C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]
        L.or_integrate.argtypes = [C.c_float] * 6 + [P, P, P]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def sincosf(x: float):
    s, c = C.c_float(), C.c_float()
    lib().or_sincosf(C.c_float(x), C.byref(s), C.byref(c))
    return np.float32(s.value), np.float32(c.value)


def hash64(seed, env, episode, k) -> int:
    return int(lib().or_hash(seed, env, episode, k))


def cast_ray(occ: np.ndarray, res: float, x: float, y: float, dx: float, dy: float,
             max_range: float):
    """(range, hit, visits) of one ray; x, y in metres, (dx, dy) a unit vector."""
    occ = np.ascontiguousarray(occ, np.uint8)
    hit, vis = C.c_int32(), C.c_uint32()
    r = lib().or_cast_ray(_ptr(occ), occ.shape[1], occ.shape[0], res, x, y, dx, dy, max_range,
                          C.byref(hit), C.byref(vis))
    return np.float32(r), int(hit.value), int(vis.value)


def march_ray(occ: np.ndarray, res: float, x: float, y: float, dx: float, dy: float,
              step: float, max_range: float):
    """(range, hit, samples) of one fixed-step march (Sec. 2.2.2); step in metres."""
    occ = np.ascontiguousarray(occ, np.uint8)
    hit, vis = C.c_int32(), C.c_uint32()
    r = lib().or_march_ray(_ptr(occ), occ.shape[1], occ.shape[0], res, x, y, dx, dy, step,
                           max_range, C.byref(hit), C.byref(vis))
    return np.float32(r), int(hit.value), int(vis.value)


def footprint(occ: np.ndarray, res: float, robot, x: float, y: float, theta: float) -> bool:
    occ = np.ascontiguousarray(occ, np.uint8)
    return bool(lib().or_footprint(_ptr(occ), occ.shape[1], occ.shape[0], res, robot.shape,
                                   robot.radius, robot.length, robot.width, x, y, theta))


def integrate(x, y, th, v, w, dt):
    xo, yo, to = C.c_float(), C.c_float(), C.c_float()
    lib().or_integrate(x, y, th, v, w, dt, C.byref(xo), C.byref(yo), C.byref(to))
    return np.float32(xo.value), np.float32(yo.value), np.float32(to.value)


class OracleSim:
    """The oracle simulator over a Workload-like description."""

    def __init__(self, maps, env_map, env_beams, env_robot, robots, max_range, params, res,
                 threads: int = 1):
        L = lib()
        self._maps = [np.ascontiguousarray(m, np.uint8) for m in maps]
        marr = (_Map * len(maps))()
        for i, m in enumerate(self._maps):
            marr[i] = _Map(m.shape[1], m.shape[0], res, m.ctypes.data)
        rarr = (_Robot * len(robots))()
        for i, r in enumerate(robots):
            rarr[i] = _Robot(r.shape, r.radius, r.length, r.width, r.v_min, r.v_max, r.w_min,
                             r.w_max)
        p = params
        par = _Params(p.dt, p.goal_tol, p.c_progress, p.step_penalty, p.r_goal, p.r_coll,
                      p.horizon, p.goal_dmin, p.goal_dmax, p.fov_deg, p.n_dyn, p.dyn_radius,
                      p.dyn_speed_max, p.dyn_min_sep, p.reward_mode,
                      getattr(p, "sensor", 0), getattr(p, "march_step", 0.03),
                      getattr(p, "n_sectors", 0))
        self.env_map = np.ascontiguousarray(env_map, np.int32)
        self.env_beams = np.ascontiguousarray(env_beams, np.int32)
        self.env_robot = np.ascontiguousarray(env_robot, np.int32)
        self.n_envs = int(self.env_map.shape[0])
        self.n_dyn = int(p.n_dyn)
        self._h = L.or_create(marr, len(maps), _ptr(self.env_map), _ptr(self.env_beams),
                              _ptr(self.env_robot), self.n_envs, max_range, rarr, len(robots),
                              C.byref(par))
        if not self._h:
            raise RuntimeError("or_create failed")
        L.or_set_threads(self._h, threads)
        m = int(getattr(p, "n_sectors", 0))
        feat = np.full(self.n_envs, m, np.int64) if m > 0 else self.env_beams.astype(np.int64)
        self.obs_off = np.concatenate([[0], np.cumsum(feat + 4)])
        self.ray_off = np.concatenate([[0], np.cumsum(self.env_beams.astype(np.int64))])

    @classmethod
    def from_workload(cls, wl, threads: int = 1):
        return cls(wl.maps, wl.env_map, wl.env_beams, wl.env_robot, wl.robots, wl.max_range,
                   wl.params, wl.res, threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_free(h)
            self._h = None

    def set_threads(self, n):
        lib().or_set_threads(self._h, n)

    def reset(self, seed: int) -> np.ndarray:
        obs = np.zeros(int(self.obs_off[-1]), np.float32)
        rc = lib().or_reset(self._h, seed, _ptr(obs))
        if rc:
            raise RuntimeError(f"or_reset -> {rc}")
        return obs

    def step(self, actions: np.ndarray, want_final: bool = False):
        actions = np.ascontiguousarray(actions, np.float32)
        obs = np.zeros(int(self.obs_off[-1]), np.float32)
        rew = np.zeros(self.n_envs, np.float32)
        done = np.zeros(self.n_envs, np.uint8)
        fin = np.zeros_like(obs) if want_final else None
        rc = lib().or_step(self._h, _ptr(actions), _ptr(obs), _ptr(rew), _ptr(done), _ptr(fin))
        if rc:
            raise RuntimeError(f"or_step -> {rc}")
        return (obs, rew, done, fin) if want_final else (obs, rew, done)

    def visits(self) -> int:
        return int(lib().or_visits(self._h))

    def get_state(self):
        f = np.zeros((self.n_envs, 8), np.float32)
        i = np.zeros((self.n_envs, 2), np.int32)
        d = np.zeros((self.n_envs, max(self.n_dyn, 1), 4), np.float32)
        lib().or_get_state(self._h, _ptr(f), _ptr(i), _ptr(d))
        return f, i, d[:, :self.n_dyn]

    def set_state(self, seed, f, i, d=None):
        f = np.ascontiguousarray(f, np.float32)
        i = np.ascontiguousarray(i, np.int32)
        d = np.ascontiguousarray(d, np.float32) if d is not None and self.n_dyn else None
        lib().or_set_state(self._h, seed, _ptr(f), _ptr(i), _ptr(d))

    def debug(self):
        n = int(self.ray_off[-1])
        r = np.zeros(n, np.float32)
        h = np.zeros(n, np.int32)
        v = np.zeros(n, np.uint32)
        lib().or_get_debug(self._h, _ptr(r), _ptr(h), _ptr(v))
        return r, h, v

    def spawn_count(self, m, r):
        return lib().or_spawn_count(self._h, m, r)

    def comp_labels(self, m):
        occ = self._maps[m]
        out = np.zeros(occ.size, np.int32)
        lib().or_comp_labels(self._h, m, 0, _ptr(out))
        return out.reshape(occ.shape)
