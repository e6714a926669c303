"""End-to-end FastDSAC training on the batched simulator (Sec. 2.3 and the
time-to-threshold protocol of Sec. 3.2): a thin loop over the C ABI.  Every
computation runs in the library's kernels; this module only orders the calls.

Per environment step: policy actions (sampled, BF16 tensor cores) -> nav_step
(with final observations) -> replay insert -> `utd` learner updates -> actor
weights copied to the acting policy.  Every `eval_every_s` seconds of wall
clock the deterministic policy runs one episode on each held-out map and the
FP64 success count is read back; evaluation time is part of the clock.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import time

import numpy as np

from . import flashnav as F
from . import workloads as W


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


@dataclasses.dataclass
class TrainConfig:
    """setting "maps": training maps and held-out maps (one episode per map
    scores success).  setting "paper": every env on the paper's one shared
    map with its sensing (Sec. 2.2.1-2.2.2, Tables 7-9); success is scored on
    n_eval fresh episodes of that map."""
    robot: str = "disc"  # disc, rect, turtlebot2, go2
    setting: str = "maps"
    n_envs: int = 4096
    n_train_maps: int = 64
    n_eval: int = 1000
    map_size: int = 256
    beams: int = 360
    max_range: float = 6.0
    batch: int = 4096
    replay: int = 4 << 20
    utd: int = 8
    learning_starts: int = 8192
    eval_every_s: float = 1.0
    time_budget_s: float = 60.0
    threshold: float = 1.0
    seed: int = 0
    scale_inputs: bool = True
    hidden: int = 256
    n_hidden: int = 2
    gamma: float = 0.99
    weight_decay: float = 0.0
    ipap: bool = False  # Eq. 2 on the range features, beta trained with the actor
    steps_per_sync: int = 1
    graph: bool = True        # capture collector + updates in one CUDA graph once learning runs
    overlap: bool = False     # collector of step t + 1 on a second stream beside step t's updates
    collector_ctas: int = -1  # overlapped: the step kernel's CTA cap (-1: one per SM, 0: none)
    algo: str = "fastdsac"    # or "fastsac" (C51 critics, Table 5)
    policy_freq: int = 2      # critic updates per actor update
    reward_scale: float = 0.4
    goal_dmax: float = 6.0    # paper setting: straight-line goal distance bound (m)
    occupancy: float = 0.10   # paper setting: occupied fraction of the stand-in map
    corridors: bool = False   # paper setting: corridor walls in the stand-in map
    alpha_init: float = 0.001
    target_entropy: float = -1.0  # of the tanh-squashed actions (2 dims)


def paper_config(robot: str = "turtlebot2", algo: str = "fastdsac", **kw) -> TrainConfig:
    """Tables 3-4 and 7-9: 1024 envs on one shared map, 1080 beams marched at
    0.03 m and pooled into 30 sectors, (100) x 4 networks, batch 1024,
    gamma 0.97, AdamW 1e-3, UTD 40, learning start 8192, Eq. 2 inputs, actor
    sync every 1 (TurtleBot2) or 2 (Go2) env steps, collector and learner
    overlapped (Sec. 3.3).  algo "fastsac": Table 5's C51 critics."""
    base = dict(robot=robot, setting="paper", n_envs=1024, batch=1024, utd=40, hidden=100,
                n_hidden=4, gamma=0.97, weight_decay=1e-3, ipap=True, learning_starts=8192,
                beams=1080, max_range=20.0, steps_per_sync=1 if robot == "turtlebot2" else 2,
                overlap=True, algo=algo)
    if algo == "fastsac":  # Table 5: policy frequency 1 / 2; no reward scale listed
        base.update(policy_freq=1 if robot == "turtlebot2" else 2, reward_scale=1.0)
    base.update(kw)
    return TrainConfig(**base)


def _robot(cfg: TrainConfig):
    return {"disc": W.DISC, "rect": W.RECT, "turtlebot2": W.TURTLEBOT2, "go2": W.GO2}[cfg.robot]


def obs_features(cfg: TrainConfig) -> int:
    """Range features per observation row (sectors in the paper setting)."""
    return 30 if cfg.setting == "paper" else cfg.beams


def make_workloads(cfg: TrainConfig):
    if cfg.setting == "paper":
        kw = dict(beams=cfg.beams, goal_dmax=cfg.goal_dmax, occupancy=cfg.occupancy,
                  corridors=cfg.corridors)
        train = W.config_paper(cfg.robot, n_envs=cfg.n_envs, **kw)
        ev = W.config_paper(cfg.robot, n_envs=cfg.n_eval, **kw)
        return train, ev
    robot = _robot(cfg)
    train_maps = [W.make_map(10_000 + cfg.seed * 1000 + m, cfg.map_size, cfg.map_size,
                             float(np.random.default_rng(10_000 + m).uniform(0.10, 0.25)),
                             corridors=True) for m in range(cfg.n_train_maps)]
    eval_maps = [W.make_map(1_000_000 + m, cfg.map_size, cfg.map_size,
                            float(np.random.default_rng(1_000_000 + m).uniform(0.10, 0.25)),
                            corridors=True) for m in range(cfg.n_eval)]
    e = np.arange(cfg.n_envs, dtype=np.int32)
    train = W.Workload(name="train", maps=train_maps,
                       env_map=(e % cfg.n_train_maps).astype(np.int32),
                       env_beams=np.full(cfg.n_envs, cfg.beams, np.int32),
                       env_robot=np.zeros(cfg.n_envs, np.int32), robots=[robot],
                       max_range=cfg.max_range, params=W.Params())
    ev = W.Workload(name="eval", maps=eval_maps,
                    env_map=np.arange(cfg.n_eval, dtype=np.int32),
                    env_beams=np.full(cfg.n_eval, cfg.beams, np.int32),
                    env_robot=np.zeros(cfg.n_eval, np.int32), robots=[robot],
                    max_range=cfg.max_range, params=W.Params())
    return train, ev


def input_scale(cfg: TrainConfig, robot) -> np.ndarray:
    """Per-feature scale of the observation: ranges by r_max (1 under Eq. 2,
    whose output is already O(1)), goal distance by 8 m, bearing by pi, v and
    w by their bounds."""
    D = obs_features(cfg)
    sc = np.full(D + 4, 1.0 if cfg.ipap else 1.0 / cfg.max_range, np.float32)
    sc[D:] = [1.0 / 8.0, 1.0 / np.pi, 1.0 / robot.v_max,
              1.0 / max(abs(robot.w_min), abs(robot.w_max))]
    return sc


def evaluate_reactive(cfg: TrainConfig, log=print):
    """Success rate of the reactive controller (no learning) on the held-out
    maps, same episodes and FP64 reduction as the policy evaluation."""
    import torch
    lib = F.load()
    _, eval_wl = make_workloads(cfg)
    robot = eval_wl.robots[0]
    ev = F.NavSim.from_workload(eval_wl)
    D = obs_features(cfg)
    tc = F.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(tc))
    tc.obs_dim, tc.batch, tc.replay_capacity = D + 4, 128, 256
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(tc), C.byref(T)) == 0
    S = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    obs = ev.new_obs()
    act = torch.empty(cfg.n_eval, 2, device="cuda")
    rew = torch.empty(cfg.n_eval, device="cuda")
    done = torch.empty(cfg.n_eval, dtype=torch.uint8, device="cuda")
    ev.reset(777, obs)
    assert lib.nav_eval_begin(T, cfg.n_eval, S) == 0
    for t in range(200):
        assert lib.nav_reactive_act(_p(obs), D + 4, cfg.n_eval, D, eval_wl.params.fov_deg,
                                    robot.v_max, max(abs(robot.w_min), abs(robot.w_max)),
                                    _p(act), S) == 0
        ev.step(act, obs, rew, done)
        assert lib.nav_eval_accumulate(T, _p(rew), _p(done), cfg.n_eval, S) == 0
    succ, ret = C.c_double(), C.c_double()
    assert lib.nav_eval_result(T, cfg.n_eval, C.byref(succ), C.byref(ret), S) == 0
    lib.nav_trainer_free(T)
    return succ.value / cfg.n_eval, ret.value / cfg.n_eval


def evaluate_policy(cfg: TrainConfig, pol, fp32: bool = False):
    """Success rate and mean return of a policy handle on the evaluation
    episodes (deterministic actions), through the BF16 tensor-core path or
    the plain FP32 path; same episodes and FP64 reduction as in training."""
    import torch
    lib = F.load()
    _, eval_wl = make_workloads(cfg)
    ev = F.NavSim.from_workload(eval_wl)
    D = obs_features(cfg)
    tc = F.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(tc))
    tc.obs_dim, tc.batch, tc.replay_capacity = D + 4, 128, 256
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(tc), C.byref(T)) == 0
    S = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    obs = ev.new_obs()
    act = torch.empty(cfg.n_eval, 2, device="cuda")
    ev.reset(777, obs)
    assert lib.nav_eval_begin(T, cfg.n_eval, S) == 0
    act_fn = lib.nav_policy_act_fp32 if fp32 else lib.nav_policy_act
    for t in range(200):
        assert act_fn(pol, _p(obs), D + 4, cfg.n_eval, 0, 0, t, _p(act), None, None, S) == 0
        o, r, d = ev.step(act, obs)
        assert lib.nav_eval_accumulate(T, _p(r), _p(d), cfg.n_eval, S) == 0
    succ, ret = C.c_double(), C.c_double()
    assert lib.nav_eval_result(T, cfg.n_eval, C.byref(succ), C.byref(ret), S) == 0
    lib.nav_trainer_free(T)
    return succ.value / cfg.n_eval, ret.value / cfg.n_eval


def evaluate_policy_fused(cfg: TrainConfig, pol):
    """The same evaluation through the actor inside the step kernel
    (nav_rollout_fused, one launch per env step, deterministic actions): the
    collector form of the policy in the loop, scored on the same episodes."""
    import torch
    lib = F.load()
    _, eval_wl = make_workloads(cfg)
    ev = F.NavSim.from_workload(eval_wl)
    D = obs_features(cfg)
    tc = F.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(tc))
    tc.obs_dim, tc.batch, tc.replay_capacity = D + 4, 128, 256
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(tc), C.byref(T)) == 0
    S = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ev._bind_stream()
    obs = ev.new_obs()
    act = torch.empty(cfg.n_eval, 2, device="cuda")
    rew = torch.empty(cfg.n_eval, device="cuda")
    done = torch.empty(cfg.n_eval, dtype=torch.uint8, device="cuda")
    ev.reset(777, obs)
    assert lib.nav_eval_begin(T, cfg.n_eval, S) == 0
    for t in range(200):
        rc = lib.nav_rollout_fused(ev._h, pol, 1, 0, 0, t, _p(obs), _p(act), _p(rew), _p(done),
                                   1 if t else 0)
        if rc:
            raise F.NavError(rc, "nav_rollout_fused")
        assert lib.nav_eval_accumulate(T, _p(rew), _p(done), cfg.n_eval, S) == 0
    succ, ret = C.c_double(), C.c_double()
    assert lib.nav_eval_result(T, cfg.n_eval, C.byref(succ), C.byref(ret), S) == 0
    lib.nav_trainer_free(T)
    return succ.value / cfg.n_eval, ret.value / cfg.n_eval


def train(cfg: TrainConfig, log=print, keep_policy: bool = False):
    """Runs FastDSAC until the threshold or the time budget.  With
    keep_policy the result also holds the trained nav_policy handle
    ("policy", freed by the caller with nav_policy_free)."""
    import torch
    lib = F.load()
    train_wl, eval_wl = make_workloads(cfg)
    sim = F.NavSim.from_workload(train_wl)
    ev = F.NavSim.from_workload(eval_wl)
    D = obs_features(cfg)
    od = D + 4
    ipap = D if cfg.ipap else 0
    tc = F.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(tc))
    tc.obs_dim, tc.batch, tc.replay_capacity, tc.seed = od, cfg.batch, cfg.replay, cfg.seed + 1
    tc.hidden, tc.n_hidden, tc.gamma, tc.weight_decay = cfg.hidden, cfg.n_hidden, cfg.gamma, \
        cfg.weight_decay
    tc.ipap_features = ipap
    tc.alpha_init = cfg.alpha_init
    tc.target_entropy = cfg.target_entropy
    tc.policy_freq, tc.reward_scale = cfg.policy_freq, cfg.reward_scale
    tc.algo = 1 if cfg.algo == "fastsac" else 0
    pol = C.c_void_p()
    assert lib.nav_policy_create_ex(od, cfg.hidden, cfg.n_hidden, ipap,
                                    C.c_float(tc.ipap_beta_init), max(cfg.n_envs, cfg.n_eval),
                                    cfg.seed + 11, C.byref(pol)) == 0
    T = C.c_void_p()
    rc = lib.nav_trainer_create(C.byref(tc), C.byref(T))
    if rc:
        raise F.NavError(rc, "nav_trainer_create failed")
    if cfg.scale_inputs:
        sc = input_scale(cfg, train_wl.robots[0])
        ptr = sc.ctypes.data_as(C.c_void_p)
        assert lib.nav_policy_set_input_scale(pol, ptr) == 0
        assert lib.nav_trainer_set_input_scale(T, ptr) == 0
    dev = torch.device("cuda")
    E = cfg.n_envs
    obs = [sim.new_obs(), sim.new_obs()]
    fin = sim.new_obs()
    act = torch.empty(E, 2, device=dev)
    rew = torch.empty(E, device=dev)
    done = torch.empty(E, dtype=torch.uint8, device=dev)
    ev_obs = ev.new_obs()
    ev_act = torch.empty(cfg.n_eval, 2, device=dev)
    ev_rew = torch.empty(cfg.n_eval, device=dev)
    ev_done = torch.empty(cfg.n_eval, dtype=torch.uint8, device=dev)
    noise_step = torch.zeros(1, dtype=torch.int64, device=dev)  # collector noise counter
    side = torch.cuda.Stream()
    ctx = torch.cuda.stream(side)
    ctx.__enter__()
    stream = side.cuda_stream
    S = C.c_void_p(stream)
    # launch shapes of both simulators tuned before the clock starts
    sim.reset(cfg.seed + 100, obs[0])
    sim.autotune(steps=5)
    ev.reset(777, ev_obs)
    ev.autotune(steps=5)
    if cfg.overlap and cfg.collector_ctas != 0:
        # the overlapped collector's step leaves SMs to the concurrent updates
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sim.set_grid_cap(n_sm if cfg.collector_ctas < 0 else cfg.collector_ctas)
    sim.reset(cfg.seed + 100, obs[0])
    assert lib.nav_trainer_sync_policy(T, pol, S) == 0
    history = []
    cur = 0
    step = 0
    n_transitions = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    next_eval = 0.0
    reached = None

    def evaluate():
        ev.reset(777, ev_obs)
        assert lib.nav_eval_begin(T, cfg.n_eval, S) == 0
        ev._bind_stream()
        for t in range(200):
            assert lib.nav_policy_act(pol, _p(ev_obs), od, cfg.n_eval, 0, 0, t, _p(ev_act), None,
                                      None, S) == 0
            ev.step(ev_act, ev_obs, ev_rew, ev_done)
            assert lib.nav_eval_accumulate(T, _p(ev_rew), _p(ev_done), cfg.n_eval, S) == 0
        succ, ret = C.c_double(), C.c_double()
        assert lib.nav_eval_result(T, cfg.n_eval, C.byref(succ), C.byref(ret), S) == 0
        return succ.value / cfg.n_eval, ret.value / cfg.n_eval

    learning = lambda: n_transitions >= max(cfg.learning_starts, cfg.batch)

    def iteration(cur, sync):
        """One collector step and, once learning has started, utd updates."""
        nxt = 1 - cur
        rc = lib.nav_policy_act_counted(pol, _p(obs[cur]), od, E, 1, cfg.seed, _p(noise_step),
                                        _p(act), None, None, S)
        assert rc == 0
        sim.step(act, obs[nxt], rew, done, final_obs=fin)
        assert lib.nav_train_insert(T, _p(obs[cur]), _p(act), _p(rew), _p(done), _p(obs[nxt]),
                                    _p(fin), E, S) == 0
        if learning():
            rc = lib.nav_train_update(T, cfg.utd, S)
            if rc:
                raise F.NavError(rc, lib.nav_trainer_last_error(T).decode())
            if sync:
                assert lib.nav_trainer_sync_policy(T, pol, S) == 0

    coll = torch.cuda.Stream()
    S_coll = C.c_void_p(coll.cuda_stream)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def iteration_overlapped(cur, sync):
        """Producer-consumer (Sec. 3.3): the collector step on its own stream
        runs beside the updates on the learner's, which draw only replay slots
        the concurrent insert does not write; the actor sync waits for both."""
        nxt = 1 - cur
        assert lib.nav_train_overlap(T, E, S) == 0
        fork.record(side)
        coll.wait_event(fork)
        with torch.cuda.stream(coll):
            assert lib.nav_policy_act_counted(pol, _p(obs[cur]), od, E, 1, cfg.seed,
                                              _p(noise_step), _p(act), None, None, S_coll) == 0
            sim.step(act, obs[nxt], rew, done, final_obs=fin)
            assert lib.nav_train_insert(T, _p(obs[cur]), _p(act), _p(rew), _p(done),
                                        _p(obs[nxt]), _p(fin), E, S_coll) == 0
        rc = lib.nav_train_update(T, cfg.utd, S)
        if rc:
            raise F.NavError(rc, lib.nav_trainer_last_error(T).decode())
        join.record(coll)
        side.wait_event(join)
        assert lib.nav_train_overlap(T, 0, S) == 0
        if sync:
            assert lib.nav_trainer_sync_policy(T, pol, S) == 0

    # once learning runs, two iterations (obs buffers 0 -> 1 -> 0) are one
    # CUDA graph: collector, replay insert, the updates and the actor syncs
    graph = None
    inflight = []
    n_replays = 0
    use_graph = cfg.graph and cfg.utd % tc.policy_freq == 0 and cfg.steps_per_sync in (1, 2)
    while True:
        el = time.perf_counter() - t0
        if el >= next_eval:
            rate, mret = evaluate()
            el = time.perf_counter() - t0
            history.append({"t": el, "success": rate, "return": mret, "env_steps": step * E,
                            "transitions": n_transitions})
            log(f"t={el:6.2f}s env_steps={step * E:>10d} success={rate:.3f} return={mret:8.3f}")
            if rate >= cfg.threshold and reached is None:
                reached = el
                break
            next_eval = el + cfg.eval_every_s
        if el >= cfg.time_budget_s:
            break
        if use_graph and learning() and cur == 0:
            if graph is None:
                graph = torch.cuda.CUDAGraph()
                step_fn = iteration_overlapped if cfg.overlap else iteration
                with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
                    step_fn(0, cfg.steps_per_sync == 1)
                    step_fn(1, True)
            graph.replay()
            n_replays += 1
            # at most two replays in flight, so that the wall clock the loop
            # reads (evaluation cadence, budget) tracks the device
            inflight.append(torch.cuda.Event())
            inflight[-1].record(side)
            if len(inflight) > 2:
                inflight.pop(0).synchronize()
            n_transitions += 2 * E
            step += 2
            continue
        iteration(cur, step % cfg.steps_per_sync == 0)
        n_transitions += E
        cur = 1 - cur
        step += 1
    if reached is None and (not history or history[-1]["t"] < time.perf_counter() - t0 - 1e-3):
        rate, mret = evaluate()
        el = time.perf_counter() - t0
        history.append({"t": el, "success": rate, "return": mret, "env_steps": step * E,
                        "transitions": n_transitions})
        log(f"t={el:6.2f}s env_steps={step * E:>10d} success={rate:.3f} return={mret:8.3f}")
    # training-cycle time (Sec. 3.3): device time of one collector step with
    # its UTD updates, from 10 extra graph replays after the run
    cycle_ms = None
    if graph is not None:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(10):
            graph.replay()
        e1.record(side)
        e1.synchronize()
        cycle_ms = e0.elapsed_time(e1) / 20.0
    torch.cuda.synchronize()
    ctx.__exit__(None, None, None)
    del graph
    lib.nav_trainer_free(T)
    out = {"time_to_threshold_s": reached, "history": history, "env_steps": step * E,
           "cycle_ms": cycle_ms}
    if keep_policy:
        out["policy"] = pol
    else:
        lib.nav_policy_free(pol)
    return out


def reachable_fraction(cfg: TrainConfig, horizon: int = 200, dt: float = 0.1) -> dict:
    """What 100 % success can mean on the held-out episodes: the share of
    them whose goal a perfect planner could reach within the horizon at the
    robot's top speed.  Per episode (the reset the evaluation uses), the
    shortest 8-connected grid path from the start cell to a cell within the
    goal tolerance, through the cells whose centre keeps the robot's
    circumscribed disc clear of every occupied cell square (Dijkstra, scipy),
    is compared with v_max dt horizon.  An 8-connected path is at most
    1.0824 times a straight segment's length, so `upper` (path <= 1.0824 x
    budget) bounds from above the share any policy can reach; `grid` uses
    the budget itself."""
    from scipy import ndimage
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    _, ev_wl = make_workloads(cfg)
    ev = F.NavSim.from_workload(ev_wl)
    ev.reset(777)
    f, _, _ = ev.get_state()
    rb = ev_wl.robots[0]
    rc = rb.radius if rb.shape == 0 else 0.5 * float(np.hypot(rb.length, rb.width))
    budget = rb.v_max * dt * horizon
    res = ev_wl.res
    tol = ev_wl.params.goal_tol / res
    lens = np.full(ev_wl.n_envs, np.inf)
    for e in range(ev_wl.n_envs):
        occ = ev_wl.maps[int(ev_wl.env_map[e])]
        H, Wd = occ.shape
        # distance from a cell centre to the nearest occupied cell square is at
        # least the distance between the centres minus half a cell
        free = ndimage.distance_transform_edt(occ == 0) - 0.5 > rc / res
        sj, si = int(f[e, 1] / res), int(f[e, 0] / res)
        if not (0 <= sj < H and 0 <= si < Wd):
            continue
        free[sj, si] = True
        idx = np.full(occ.shape, -1, np.int64)
        cells = np.flatnonzero(free.ravel())
        idx.ravel()[cells] = np.arange(cells.size)
        rows, cols, wts = [], [], []
        for dj, di, w in ((0, 1, 1.0), (1, 0, 1.0), (1, 1, 2 ** 0.5), (1, -1, 2 ** 0.5)):
            a = free[max(0, -dj):H - max(0, dj), max(0, -di):Wd - max(0, di)]
            b = free[max(0, dj):H - max(0, -dj) if dj < 0 else H, max(0, di):Wd - max(0, -di) if di < 0 else Wd]
            ia = idx[max(0, -dj):H - max(0, dj), max(0, -di):Wd - max(0, di)]
            ib = idx[max(0, dj):H - max(0, -dj) if dj < 0 else H, max(0, di):Wd - max(0, -di) if di < 0 else Wd]
            both = a & b
            rows.append(ia[both])
            cols.append(ib[both])
            wts.append(np.full(int(both.sum()), w))
        r_, c_, w_ = np.concatenate(rows), np.concatenate(cols), np.concatenate(wts)
        G = csr_matrix((np.concatenate([w_, w_]), (np.concatenate([r_, c_]), np.concatenate([c_, r_]))),
                       shape=(cells.size, cells.size))
        d = dijkstra(G, indices=int(idx[sj, si]), limit=1.0824 * budget / res + 1.0)
        jj, ii = np.divmod(cells, Wd)
        near = np.hypot(ii + 0.5 - f[e, 5] / res, jj + 0.5 - f[e, 6] / res) <= tol
        if near.any():
            lens[e] = float(d[near].min()) * res
    return {"grid": float(np.mean(lens <= budget)), "upper": float(np.mean(lens <= 1.0824 * budget)),
            "budget_m": budget, "median_path_m": float(np.median(lens[np.isfinite(lens)]))
            if np.isfinite(lens).any() else None}
