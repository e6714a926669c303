"""Python binding of libflashnav.so (include/flashnav.h): argument marshalling
only.  Every step of the simulator runs in the library's CUDA kernels; this
module converts torch tensors and numpy arrays to pointers and return codes to
exceptions.  It never falls back to another implementation: if the library or
a CUDA device is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflashnav.so")

NAV_OK = 0
_ERR = {-1: "NAV_E_INVAL", -2: "NAV_E_CUDA", -3: "NAV_E_NOMEM", -4: "NAV_E_NOSPAWN",
        -5: "NAV_E_INTERNAL", -6: "NAV_E_TIMEOUT"}

# every symbol include/flashnav.h declares
EXPORTS = [
    "nav_default_params", "nav_create", "nav_create_ex", "nav_set_stream", "nav_obs_offsets",
    "nav_num_envs", "nav_obs_size", "nav_reset", "nav_step", "nav_step_host", "nav_sync",
    "nav_get_state", "nav_set_state", "nav_set_debug", "nav_get_debug", "nav_set_stats",
    "nav_get_stats", "nav_set_host_pipeline", "nav_set_launch", "nav_get_launch",
    "nav_set_tile_order", "nav_get_tile_order", "nav_set_grid_cap", "nav_get_grid_cap",
    "nav_autotune", "nav_uniform_actions",
    "nav_graph_capture", "nav_graph_launch", "nav_step_host_noalloc", "nav_gemm_bf16",
    "nav_gather_probe", "nav_mma_probe",
    "nav_policy_create", "nav_policy_create_ex", "nav_policy_get_beta", "nav_policy_free",
    "nav_policy_num_params", "nav_policy_get_weights",
    "nav_policy_set_weights", "nav_policy_act", "nav_policy_act_fp32", "nav_policy_act_counted",
    "nav_rollout", "nav_rollout_fused", "nav_trainer_set_graphs", "nav_trainer_set_fused", "nav_train_overlap",
    "nav_train_default_cfg", "nav_trainer_create", "nav_trainer_free", "nav_trainer_last_error",
    "nav_train_insert", "nav_train_update", "nav_trainer_sync_policy", "nav_trainer_io",
    "nav_trainer_counts", "nav_eval_begin", "nav_eval_accumulate", "nav_eval_result",
    "nav_policy_set_input_scale", "nav_reactive_act", "nav_trainer_set_input_scale",
    "nav_last_error", "nav_free",
]


class nav_train_cfg(C.Structure):
    _fields_ = [("obs_dim", C.c_int), ("hidden", C.c_int), ("batch", C.c_int),
                ("replay_capacity", C.c_longlong), ("lr_actor", C.c_float),
                ("lr_critic", C.c_float), ("lr_alpha", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("gamma", C.c_float), ("tau", C.c_float),
                ("tau_b", C.c_float), ("reward_scale", C.c_float), ("huber_delta", C.c_float),
                ("alpha_init", C.c_float), ("target_entropy", C.c_float),
                ("policy_freq", C.c_int), ("seed", C.c_uint64), ("n_hidden", C.c_int),
                ("weight_decay", C.c_float), ("ipap_features", C.c_int),
                ("ipap_beta_init", C.c_float), ("ipap_beta_max", C.c_float),
                ("algo", C.c_int), ("n_atoms", C.c_int), ("v_min", C.c_float),
                ("v_max", C.c_float)]


class NavError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


class nav_map(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("resolution", C.c_float),
                ("occ", C.c_void_p)]


class nav_robot(C.Structure):
    _fields_ = [("shape", C.c_int), ("radius", C.c_float), ("length", C.c_float),
                ("width", C.c_float), ("v_min", C.c_float), ("v_max", C.c_float),
                ("w_min", C.c_float), ("w_max", C.c_float)]


class nav_params(C.Structure):
    _fields_ = [("dt", C.c_float), ("goal_tol", C.c_float), ("c_progress", C.c_float),
                ("step_penalty", C.c_float), ("r_goal", C.c_float), ("r_coll", C.c_float),
                ("horizon", C.c_int), ("goal_dmin", C.c_float), ("goal_dmax", C.c_float),
                ("fov_deg", C.c_float), ("n_dyn", C.c_int), ("dyn_radius", C.c_float),
                ("dyn_speed_max", C.c_float), ("dyn_min_sep", C.c_float),
                ("reward_mode", C.c_int), ("sensor", C.c_int), ("march_step", C.c_float),
                ("n_sectors", C.c_int)]


_lib = None


def load():
    """Loads libflashnav.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    P, I, F, U64 = C.c_void_p, C.c_int, C.c_float, C.c_uint64
    sig = {
        "nav_default_params": (None, [P]),
        "nav_create": (I, [P, I, I, I, F, P, P, P]),
        "nav_create_ex": (I, [P, I, P, P, P, I, F, P, I, P, P]),
        "nav_set_stream": (I, [P, P]),
        "nav_obs_offsets": (I, [P, P]),
        "nav_set_host_pipeline": (I, [P, I]),
        "nav_num_envs": (I, [P]),
        "nav_obs_size": (C.c_int64, [P]),
        "nav_reset": (I, [P, U64, P]),
        "nav_step": (I, [P, P, P, P, P, P]),
        "nav_step_host": (I, [P, P, P, P, P, P]),
        "nav_sync": (I, [P, I]),
        "nav_get_state": (I, [P, P, P, P]),
        "nav_set_state": (I, [P, U64, P, P, P]),
        "nav_set_debug": (I, [P, I]),
        "nav_get_debug": (I, [P, P, P, P]),
        "nav_set_stats": (I, [P, I]),
        "nav_get_stats": (I, [P, P, P]),
        "nav_set_launch": (I, [P, I, I, I, I, I, I]),
        "nav_get_launch": (I, [P, P, P, P, P, P, P]),
        "nav_set_tile_order": (I, [P, I]),
        "nav_get_tile_order": (I, [P, P]),
        "nav_set_grid_cap": (I, [P, I]),
        "nav_get_grid_cap": (I, [P, P]),
        "nav_autotune": (I, [P, I, P]),
        "nav_uniform_actions": (I, [P, U64, C.c_uint32, P]),
        "nav_graph_capture": (I, [P, I, P, P, P, P, P]),
        "nav_graph_launch": (I, [P]),
        "nav_step_host_noalloc": (I, [P, P, P, P, P, P]),
        "nav_gemm_bf16": (I, [P, I, P, I, I, I, I, P, I, P, I, P, I, P, I, P, P]),
        "nav_gather_probe": (I, [I, P, C.c_int64, I, I, P, P]),
        "nav_mma_probe": (I, [I, I, I, I, I, P, P, P]),
        "nav_policy_create": (I, [I, I, I, U64, P]),
        "nav_policy_create_ex": (I, [I, I, I, I, C.c_float, I, U64, P]),
        "nav_policy_get_beta": (I, [P, P]),
        "nav_policy_free": (None, [P]),
        "nav_policy_num_params": (C.c_int64, [P]),
        "nav_policy_get_weights": (I, [P, P]),
        "nav_policy_set_weights": (I, [P, P]),
        "nav_policy_act": (I, [P, P, C.c_int64, I, I, U64, C.c_uint32, P, P, P, P]),
        "nav_policy_act_fp32": (I, [P, P, C.c_int64, I, I, U64, C.c_uint32, P, P, P, P]),
        "nav_rollout": (I, [P, P, I, I, U64, C.c_uint32, P, P, P, P, I]),
        "nav_rollout_fused": (I, [P, P, I, I, U64, C.c_uint32, P, P, P, P, I]),
        "nav_train_default_cfg": (None, [P]),
        "nav_trainer_create": (I, [P, P]),
        "nav_trainer_free": (None, [P]),
        "nav_trainer_last_error": (C.c_char_p, [P]),
        "nav_train_insert": (I, [P, P, P, P, P, P, P, I, P]),
        "nav_train_update": (I, [P, I, P]),
        "nav_trainer_set_graphs": (I, [P, I]),
        "nav_trainer_set_fused": (I, [P, I]),
        "nav_train_overlap": (I, [P, I, P]),
        "nav_policy_act_counted": (I, [P, P, C.c_int64, I, I, U64, P, P, P, P, P]),
        "nav_trainer_sync_policy": (I, [P, P, P]),
        "nav_trainer_io": (I, [P, I, I, P]),
        "nav_trainer_counts": (I, [P, P, P, P]),
        "nav_eval_begin": (I, [P, I, P]),
        "nav_eval_accumulate": (I, [P, P, P, I, P]),
        "nav_eval_result": (I, [P, I, P, P, P]),
        "nav_policy_set_input_scale": (I, [P, P]),
        "nav_reactive_act": (I, [P, C.c_int64, I, I, F, F, F, P, P]),
        "nav_trainer_set_input_scale": (I, [P, P]),
        "nav_last_error": (C.c_char_p, [P]),
        "nav_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _t_ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def gather_probe(where: int, table, nbytes: int, n_blocks: int, iters: int, sums,
                 stream: int = 0):
    """nav_gather_probe: random single-byte gathers from shared memory
    (where 0) or from the device tensor `table` (where 1); `sums` is a
    uint32-sized device tensor of n_blocks entries."""
    rc = load().nav_gather_probe(where, _t_ptr(table), nbytes, n_blocks, iters, _t_ptr(sums),
                                 C.c_void_p(stream))
    if rc != 0:
        raise NavError(rc, "nav_gather_probe: argument out of range or launch failed")


def mma_probe(n: int, n_mma: int, commit_every: int, wait: int, ns, status, stream: int = 0):
    """nav_mma_probe: back-to-back tcgen05.mma (M 128, N n, K 16) from one
    thread per CTA; `ns` a device int64 tensor of one entry per CTA (the
    grid is its length), `status` a device int32 tensor of one entry."""
    rc = load().nav_mma_probe(n, n_mma, commit_every, wait, ns.numel(), _t_ptr(ns),
                              _t_ptr(status), C.c_void_p(stream))
    if rc != 0:
        raise NavError(rc, "nav_mma_probe: argument out of range or launch failed")


def params_struct(p) -> nav_params:
    s = nav_params()
    load().nav_default_params(C.byref(s))
    if p is not None:
        for name, _ in nav_params._fields_:
            if hasattr(p, name):
                setattr(s, name, getattr(p, name))
    return s


class NavSim:
    """A handle of the CUDA simulator.  Observations, rewards and flags are
    torch CUDA tensors written by the library on the current torch stream."""

    def __init__(self, maps, env_map, env_beams, env_robot, robots, max_range, params,
                 res: float, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("NavSim needs a CUDA device")
        torch.cuda.set_device(device)
        L = load()
        self._maps = [np.ascontiguousarray(m, np.uint8) for m in maps]
        marr = (nav_map * len(maps))()
        for i, m in enumerate(self._maps):
            marr[i] = nav_map(m.shape[1], m.shape[0], res, m.ctypes.data)
        rarr = (nav_robot * len(robots))()
        for i, r in enumerate(robots):
            rarr[i] = nav_robot(r.shape, r.radius, r.length, r.width, r.v_min, r.v_max, r.w_min,
                                r.w_max)
        self.env_map = np.ascontiguousarray(env_map, np.int32)
        self.env_beams = np.ascontiguousarray(env_beams, np.int32)
        self.env_robot = np.ascontiguousarray(env_robot, np.int32)
        self.n_envs = int(self.env_map.shape[0])
        self.n_dyn = int(getattr(params, "n_dyn", 0))
        self.max_range = float(max_range)
        par = params_struct(params)
        h = C.c_void_p()
        rc = L.nav_create_ex(marr, len(maps), _np_ptr(self.env_map), _np_ptr(self.env_beams),
                             _np_ptr(self.env_robot), self.n_envs, max_range, rarr, len(robots),
                             C.byref(par), C.byref(h))
        if rc != NAV_OK:
            raise NavError(rc, "nav_create_ex failed (see stderr)")
        self._h = h
        self._torch = torch
        self.device = torch.device("cuda", device)
        self.obs_size = int(L.nav_obs_size(h))
        off = np.zeros(self.n_envs + 1, np.int64)
        self._check(L.nav_obs_offsets(h, _np_ptr(off)))
        self.obs_offsets = off
        self.uniform_k = bool((self.env_beams == self.env_beams[0]).all())

    @classmethod
    def from_workload(cls, wl, device: int = 0):
        return cls(wl.maps, wl.env_map, wl.env_beams, wl.env_robot, wl.robots, wl.max_range,
                   wl.params, wl.res, device)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc):
        if rc != NAV_OK:
            msg = load().nav_last_error(self._h)
            raise NavError(rc, msg.decode() if msg else "")

    def _bind_stream(self):
        s = self._torch.cuda.current_stream(self.device).cuda_stream
        self._check(load().nav_set_stream(self._h, C.c_void_p(s)))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().nav_free(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ----------------------------------------------------------------
    def new_obs(self):
        return self._torch.empty(self.obs_size, dtype=self._torch.float32, device=self.device)

    def reset(self, seed: int, obs=None):
        obs = self.new_obs() if obs is None else obs
        self._bind_stream()
        self._check(load().nav_reset(self._h, C.c_uint64(seed), _t_ptr(obs)))
        return obs

    def step(self, actions, obs=None, reward=None, done=None, final_obs=None, want_final=False):
        torch = self._torch
        assert actions.is_cuda and actions.dtype == torch.float32 and actions.is_contiguous()
        assert actions.numel() == 2 * self.n_envs
        obs = self.new_obs() if obs is None else obs
        reward = torch.empty(self.n_envs, dtype=torch.float32, device=self.device) \
            if reward is None else reward
        done = torch.empty(self.n_envs, dtype=torch.uint8, device=self.device) \
            if done is None else done
        if want_final and final_obs is None:
            final_obs = torch.zeros(self.obs_size, dtype=torch.float32, device=self.device)
        self._bind_stream()
        self._check(load().nav_step(self._h, _t_ptr(actions), _t_ptr(obs), _t_ptr(reward),
                                    _t_ptr(done), _t_ptr(final_obs)))
        if want_final or final_obs is not None:
            return obs, reward, done, final_obs
        return obs, reward, done

    def step_host(self, actions: np.ndarray, obs: np.ndarray, reward: np.ndarray,
                  done: np.ndarray, final_obs: np.ndarray | None = None):
        """nav_step_host: host (ideally pinned) buffers in and out, synchronous."""
        self._bind_stream()
        self._check(load().nav_step_host(self._h, _np_ptr(actions), _np_ptr(obs),
                                         _np_ptr(reward), _np_ptr(done), _np_ptr(final_obs)))

    def step_host_ptrs(self, actions_ptr: int, obs_ptr: int, reward_ptr: int, done_ptr: int,
                       final_ptr: int | None = None):
        self._bind_stream()
        self._check(load().nav_step_host(self._h, C.c_void_p(actions_ptr), C.c_void_p(obs_ptr),
                                         C.c_void_p(reward_ptr), C.c_void_p(done_ptr),
                                         C.c_void_p(final_ptr) if final_ptr else None))

    def sync(self, timeout_ms: int = 0):
        self._check(load().nav_sync(self._h, timeout_ms))

    def get_state(self):
        f = np.zeros((self.n_envs, 8), np.float32)
        i = np.zeros((self.n_envs, 2), np.int32)
        d = np.zeros((self.n_envs, max(self.n_dyn, 1), 4), np.float32)
        self._check(load().nav_get_state(self._h, _np_ptr(f), _np_ptr(i), _np_ptr(d)))
        return f, i, d[:, :self.n_dyn]

    def set_state(self, seed, f, i, d=None):
        f = np.ascontiguousarray(f, np.float32)
        i = np.ascontiguousarray(i, np.int32)
        d = np.ascontiguousarray(d, np.float32) if d is not None and self.n_dyn else None
        self._check(load().nav_set_state(self._h, C.c_uint64(seed), _np_ptr(f), _np_ptr(i),
                                         _np_ptr(d)))

    def set_debug(self, on: bool = True):
        self._check(load().nav_set_debug(self._h, 1 if on else 0))

    def debug(self):
        n = int(self.env_beams.astype(np.int64).sum())
        r = np.zeros(n, np.float32)
        h = np.zeros(n, np.int32)
        v = np.zeros(n, np.uint32)
        self._check(load().nav_get_debug(self._h, _np_ptr(r), _np_ptr(h), _np_ptr(v)))
        return r, h, v

    def set_stats(self, on: bool = True):
        self._bind_stream()
        self._check(load().nav_set_stats(self._h, 1 if on else 0))

    def stats(self):
        v, r = C.c_uint64(), C.c_uint64()
        self._check(load().nav_get_stats(self._h, C.byref(v), C.byref(r)))
        return int(v.value), int(r.value)

    def set_launch(self, tile_envs=0, block_threads=0, smem_map_bytes=0, max_regs=0,
                   byte_cells=0, split=0):
        self._bind_stream()
        self._check(load().nav_set_launch(self._h, tile_envs, block_threads, smem_map_bytes,
                                          max_regs, byte_cells, split))

    def set_host_pipeline(self, parts: int):
        self._check(load().nav_set_host_pipeline(self._h, parts))

    def set_grid_cap(self, max_ctas: int):
        """At most max_ctas persistent CTAs for the tiled step (0: every SM)."""
        self._bind_stream()
        self._check(load().nav_set_grid_cap(self._h, max_ctas))

    def get_grid_cap(self) -> int:
        v = C.c_int()
        self._check(load().nav_get_grid_cap(self._h, C.byref(v)))
        return v.value

    def get_launch(self):
        v = [C.c_int() for _ in range(6)]
        self._check(load().nav_get_launch(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_tile_order(self, order: int):
        self._bind_stream()
        self._check(load().nav_set_tile_order(self._h, order))

    def get_tile_order(self) -> int:
        v = C.c_int()
        self._check(load().nav_get_tile_order(self._h, C.byref(v)))
        return v.value

    def autotune(self, steps: int = 5) -> float:
        """Picks the fastest launch shape for this handle; returns its ms/step."""
        self._bind_stream()
        ms = C.c_float()
        self._check(load().nav_autotune(self._h, steps, C.byref(ms)))
        return float(ms.value)

    def uniform_actions(self, seed: int, step: int, out=None):
        out = self._torch.empty(self.n_envs, 2, dtype=self._torch.float32, device=self.device) \
            if out is None else out
        self._bind_stream()
        self._check(load().nav_uniform_actions(self._h, C.c_uint64(seed), C.c_uint32(step),
                                               _t_ptr(out)))
        return out

    def graph_capture(self, actions, obs, reward, done, final_obs=None):
        """Captures actions.shape[0] consecutive steps into a CUDA graph."""
        self._bind_stream()
        self._check(load().nav_graph_capture(self._h, int(actions.shape[0]), _t_ptr(actions),
                                             _t_ptr(obs), _t_ptr(reward), _t_ptr(done),
                                             _t_ptr(final_obs)))

    def graph_launch(self):
        self._bind_stream()
        self._check(load().nav_graph_launch(self._h))
