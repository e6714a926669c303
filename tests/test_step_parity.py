"""Parity of the CUDA step (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs.

Bit-exact: done flags, hit cells, per-beam visit counts, step and episode
counters, goals (they come from the reset RNG).  Toleranced (FP32, north
star): ranges 1e-4 m, poses 1e-5; the observation bearing, which the oracle
computes with a binary64 atan2, 1e-4 rad.
"""
import math

import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W

pytestmark = pytest.mark.gpu

RANGE_TOL = 1e-4
POSE_TOL = 1e-5


@pytest.fixture(scope="module")
def mods(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav, oracle, torch


def _ang(a, b):
    d = np.abs(a - b)
    return np.minimum(d, 2 * np.pi - d)


def _features(wl):
    """Range features per observation row: the beams, or Eq. 6's sectors."""
    m = int(getattr(wl.params, "n_sectors", 0))
    return np.full(wl.n_envs, m, np.int32) if m > 0 else wl.env_beams


def _compare_obs(obs, ref, beams, rows=None, what="obs"):
    off = np.concatenate([[0], np.cumsum(beams.astype(np.int64) + 4)])
    env_ids = range(len(beams)) if rows is None else rows
    for e in env_ids:
        k = int(beams[e])
        a, b = obs[off[e]:off[e + 1]], ref[off[e]:off[e + 1]]
        dr = np.abs(a[:k] - b[:k]).max() if k else 0.0
        assert dr <= RANGE_TOL, f"{what} env {e}: range error {dr}"
        assert abs(a[k] - b[k]) <= POSE_TOL * 10, f"{what} env {e}: goal distance"
        assert _ang(a[k + 1], b[k + 1]) <= 1e-4, f"{what} env {e}: bearing"
        assert a[k + 2] == b[k + 2] and a[k + 3] == b[k + 3], f"{what} env {e}: velocity"


def _compare_state(sim, ref, tag):
    f, i, d = sim.get_state()
    rf, ri, rd = ref.get_state()
    assert np.array_equal(i, ri), f"{tag}: step/episode counters differ"
    assert np.array_equal(f[:, 5:7], rf[:, 5:7]), f"{tag}: goals differ"
    assert np.abs(f[:, :2] - rf[:, :2]).max() <= POSE_TOL, f"{tag}: positions"
    assert _ang(f[:, 2], rf[:, 2]).max() <= POSE_TOL, f"{tag}: headings"
    assert np.abs(f[:, 7] - rf[:, 7]).max() <= POSE_TOL, f"{tag}: d_prev"
    if d.size:
        assert np.abs(d - rd).max() <= POSE_TOL, f"{tag}: moving discs"
    return int((f == rf).all())


def _compare_debug(sim, ref, tag):
    r, h, v = sim.debug()
    rr, rh, rv = ref.debug()
    assert np.array_equal(h, rh), f"{tag}: hit cells differ at {np.flatnonzero(h != rh)[:8]}"
    assert np.array_equal(v, rv), f"{tag}: visit counts differ"
    assert np.abs(r - rr).max() <= RANGE_TOL, f"{tag}: ranges"


def run_parity(mods, wl, n_steps, seed=1, want_final=True, launch=None, threads=8,
               check_state_every=1, autotune=False, tile_order=None, grid_cap=0):
    flashnav, oracle, torch = mods
    sim = flashnav.NavSim.from_workload(wl)
    if launch:
        sim.set_launch(*launch)
    if grid_cap:
        sim.set_grid_cap(grid_cap)
        assert sim.get_grid_cap() == grid_cap
    if tile_order is not None:
        sim.set_tile_order(tile_order)
        assert sim.get_tile_order() == tile_order
    ref = oracle.OracleSim.from_workload(wl, threads=threads)
    if autotune:
        sim.reset(seed)
        sim.autotune(steps=3)
    sim.set_debug(True)
    obs = sim.reset(seed)
    robs = ref.reset(seed)
    feat = _features(wl)
    _compare_obs(obs.cpu().numpy(), robs, feat, what="reset obs")
    _compare_state(sim, ref, "reset")
    _compare_debug(sim, ref, "reset")
    acts = W.uniform_actions(seed + 1000, n_steps, wl.n_envs)
    n_done = 0
    for t in range(n_steps):
        a = torch.from_numpy(acts[t]).cuda()
        if want_final:
            o, r, d, fo = sim.step(a, want_final=True)
            ro, rr, rd, rfo = ref.step(acts[t], want_final=True)
        else:
            o, r, d = sim.step(a)
            ro, rr, rd = ref.step(acts[t])
        d = d.cpu().numpy()
        assert np.array_equal(d, rd), f"step {t}: done flags differ at {np.flatnonzero(d != rd)[:8]}"
        assert np.abs(r.cpu().numpy() - rr).max() <= 1e-5, f"step {t}: reward"
        _compare_obs(o.cpu().numpy(), ro, feat, what=f"step {t} obs")
        if want_final:
            ended = np.flatnonzero(d & 3)
            n_done += len(ended)
            if len(ended):
                _compare_obs(fo.cpu().numpy(), rfo, feat, rows=ended,
                             what=f"step {t} final obs")
        _compare_debug(sim, ref, f"step {t}")
        if t % check_state_every == 0 or t == n_steps - 1:
            _compare_state(sim, ref, f"step {t}")
    sim.sync(60000)
    return sim, ref, n_done


def test_reset_and_1000_free_running_steps_small(mods):
    """64 envs, one 64x64 map, 180 beams, 4 m, 1000 steps with auto-reset."""
    wl = W.config_small()
    _, _, n_done = run_parity(mods, wl, 1000, seed=1)
    assert n_done > 100  # resets are exercised


def test_throughput_workload_steps(mods):
    """4096 envs over 16 maps of 256x256, 360 beams, r_max 6 m, with the
    autotuned launch shape, as the benchmark times it."""
    wl = W.config_throughput()
    run_parity(mods, wl, 4, seed=5, want_final=False, autotune=True)


@pytest.mark.parametrize("byte_cells", [1, 2])
def test_throughput_workload_both_staging_modes(mods, byte_cells):
    wl = W.config_throughput(n_envs=1024, n_maps=4)
    run_parity(mods, wl, 3, seed=6, launch=(2, 256, 0, 32, byte_cells))


def test_visit_counter_matches_oracle(mods):
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=512, n_maps=4)
    sim = flashnav.NavSim.from_workload(wl)
    ref = oracle.OracleSim.from_workload(wl, threads=8)
    sim.reset(2)
    ref.reset(2)
    sim.set_stats(True)
    v0 = ref.visits()
    acts = W.uniform_actions(2, 6, wl.n_envs)
    for t in range(6):
        sim.step(torch.from_numpy(acts[t]).cuda(), want_final=True)
        ref.step(acts[t], want_final=True)
    visits, rays = sim.stats()
    assert visits == ref.visits() - v0
    assert rays >= 6 * wl.n_envs * 360


# (tile_envs, block_threads, smem_map_bytes, max_regs, byte_cells): a smem
# cap of 16 bytes forces the L1/L2 paths (distance bytes with byte_cells 1
# or 3, packed bits with 2); byte_cells 2 with room stages packed bits; a
# 4 KiB cap with byte_cells 3 stages the 64 x 64 map's bits (its bytes do
# not fit)
@pytest.mark.parametrize("launch", [(1, 64, 0, 32, 1), (3, 96, 0, 64, 2), (32, 512, 0, 40, 1),
                                    (8, 256, 16, 40, 1), (5, 128, 16, 32, 2),
                                    (2, 224, 0, 64, 2), (6, 192, 16, 40, 3),
                                    (4, 256, 4096, 40, 3)])
def test_launch_shapes_and_ragged_tiles(mods, launch):
    """Ragged env count, a beam count that is not a multiple of 32, tiles of
    1..32 envs, 64..512 threads, register caps, and all four map stagings."""
    wl = W.config_small(n_envs=37)
    wl.env_beams[:] = 37
    run_parity(mods, wl, 60, seed=7, launch=launch)


def test_single_env_single_beam(mods):
    wl = W.config_small(n_envs=1)
    wl.env_beams[:] = 1
    run_parity(mods, wl, 50, seed=3)


def _mixed(n_envs=96, n_dyn=0, sizes=(48, 96, 160, 200), seed0=40):
    maps = [W.make_map(seed0 + i, s, s + 8 * i, 0.12 + 0.03 * i, corridors=True)
            for i, s in enumerate(sizes)]
    e = np.arange(n_envs)
    return W.Workload(
        name="mixed", maps=maps, env_map=(e % len(maps)).astype(np.int32),
        env_beams=np.array([180, 360, 720, 45], np.int32)[(e // 4) % 4],
        env_robot=(e % 2).astype(np.int32), robots=[W.DISC, W.RECT], max_range=6.0,
        params=W.Params(n_dyn=n_dyn, goal_dmin=1.0, goal_dmax=6.0))


def test_mixed_maps_beams_and_rectangles(mods):
    run_parity(mods, _mixed(), 80, seed=11)


def test_mixed_maps_tile_queue_by_ray_cost(mods):
    """The tile queue ordered by sampled ray cost (tiles of four map sizes,
    four beam counts and two robots interleave differently)."""
    run_parity(mods, _mixed(), 40, seed=19, launch=(3, 256, 0, 40, 1), tile_order=1)


def test_moving_discs(mods):
    run_parity(mods, _mixed(n_dyn=8), 80, seed=12)


def test_moving_discs_packed_bits(mods):
    run_parity(mods, _mixed(n_dyn=8), 40, seed=14, launch=(4, 256, 0, 40, 2))


@pytest.mark.parametrize("byte_cells", [1, 2])
def test_moving_discs_l2_path(mods, byte_cells):
    run_parity(mods, _mixed(n_dyn=3), 40, seed=13, launch=(4, 128, 16, 64, byte_cells))


def test_exclusive_reward_and_270_degree_fan(mods):
    wl = W.config_small(n_envs=40)
    wl.params = W.Params(goal_dmin=1.0, goal_dmax=1e9, reward_mode=1, fov_deg=270.0)
    wl.env_beams[:] = 34
    run_parity(mods, wl, 200, seed=4)


def test_cramped_map(mods):
    wl = W.config_small(n_envs=48)
    wl.maps = [W.make_map(77, 96, 96, 0.40)]
    run_parity(mods, wl, 100, seed=8)


def test_lockstep_random_states(mods):
    """Injected states (positions anywhere in free space, any heading, step
    counters at the horizon) give the same single step on both sides."""
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=1024, n_maps=4)
    sim = flashnav.NavSim.from_workload(wl)
    sim.set_debug(True)
    ref = oracle.OracleSim.from_workload(wl, threads=8)
    sim.reset(0)
    ref.reset(0)
    rng = np.random.default_rng(0)
    f = np.zeros((wl.n_envs, 8), np.float32)
    i2 = np.zeros((wl.n_envs, 2), np.int32)
    for e in range(wl.n_envs):
        occ = wl.maps[wl.env_map[e]]
        free = np.argwhere(occ == 0)
        j, i = free[rng.integers(len(free))]
        f[e, 0] = (i + rng.random()) * W.RES
        f[e, 1] = (j + rng.random()) * W.RES
        f[e, 2] = rng.uniform(-math.pi, math.pi)
        j2, i2_ = free[rng.integers(len(free))]
        f[e, 5] = (i2_ + 0.5) * W.RES
        f[e, 6] = (j2 + 0.5) * W.RES
        f[e, 7] = rng.uniform(0, 10)
        i2[e, 0] = rng.integers(0, 201)
        i2[e, 1] = rng.integers(0, 1000)
    sim.set_state(99, f, i2)
    ref.set_state(99, f, i2)
    acts = W.uniform_actions(99, 1, wl.n_envs)[0]
    o, r, d, fo = sim.step(torch.from_numpy(acts).cuda(), want_final=True)
    ro, rr, rd, rfo = ref.step(acts, want_final=True)
    d = d.cpu().numpy()
    assert np.array_equal(d, rd)
    assert np.abs(r.cpu().numpy() - rr).max() <= 1e-5
    _compare_obs(o.cpu().numpy(), ro, wl.env_beams)
    ended = np.flatnonzero(d & 3)
    assert len(ended) > 10
    _compare_obs(fo.cpu().numpy(), rfo, wl.env_beams, rows=ended, what="final obs")
    _compare_debug(sim, ref, "lockstep")
    _compare_state(sim, ref, "lockstep")


@pytest.mark.parametrize("parts,mixed", [(4, False), (1, False), (3, True), (7, True)])
def test_step_host_matches_device_step(mods, parts, mixed):
    """nav_step_host (pipelined over `parts` env ranges, results copied out
    while the next range computes) returns exactly nav_step's results."""
    flashnav, oracle, torch = mods
    wl = _mixed(n_envs=75, n_dyn=4) if mixed else W.config_small(n_envs=64)
    a_sim = flashnav.NavSim.from_workload(wl)
    b_sim = flashnav.NavSim.from_workload(wl)
    b_sim.set_host_pipeline(parts)
    a_sim.reset(5)
    b_sim.reset(5)
    acts = W.uniform_actions(5, 30, wl.n_envs)
    n = a_sim.obs_size
    for t in range(30):
        o, r, d, fo = a_sim.step(torch.from_numpy(acts[t]).cuda(), want_final=True)
        ho = np.zeros(n, np.float32)
        hr = np.zeros(wl.n_envs, np.float32)
        hd = np.zeros(wl.n_envs, np.uint8)
        hf = np.zeros(n, np.float32)
        b_sim.step_host(np.ascontiguousarray(acts[t]), ho, hr, hd, hf)
        dd = d.cpu().numpy()
        assert np.array_equal(o.cpu().numpy(), ho)
        assert np.array_equal(r.cpu().numpy(), hr)
        assert np.array_equal(dd, hd)
        ended = np.flatnonzero(dd & 3)
        off = a_sim.obs_offsets
        fa = fo.cpu().numpy()
        for e in ended:
            assert np.array_equal(fa[off[e]:off[e + 1]], hf[off[e]:off[e + 1]])


@pytest.mark.parametrize("final", [False, True])
def test_step_host_pinned_buffers_match_device_step(mods, final):
    """Pinned host buffers (the copies overlap the second part's kernel):
    results equal nav_step's."""
    flashnav, oracle, torch = mods
    wl = _mixed(n_envs=90)
    a_sim = flashnav.NavSim.from_workload(wl)
    b_sim = flashnav.NavSim.from_workload(wl)
    a_sim.reset(8)
    b_sim.reset(8)
    acts = W.uniform_actions(8, 25, wl.n_envs)
    n = a_sim.obs_size
    h_act = torch.empty(wl.n_envs, 2, pin_memory=True)
    h_obs = torch.full((n,), -7.0, pin_memory=True)
    h_rew = torch.empty(wl.n_envs, pin_memory=True)
    h_done = torch.empty(wl.n_envs, dtype=torch.uint8, pin_memory=True)
    h_fin = torch.zeros(n, pin_memory=True) if final else None
    for t in range(25):
        o, r, d, fo = a_sim.step(torch.from_numpy(acts[t]).cuda(), want_final=True)
        h_act.copy_(torch.from_numpy(acts[t]))
        b_sim.step_host_ptrs(h_act.data_ptr(), h_obs.data_ptr(), h_rew.data_ptr(),
                             h_done.data_ptr(), h_fin.data_ptr() if final else None)
        assert torch.equal(o.cpu(), h_obs)
        assert torch.equal(r.cpu(), h_rew)
        assert torch.equal(d.cpu(), h_done)
        if final:
            off = a_sim.obs_offsets
            fa = fo.cpu()
            for e in np.flatnonzero(d.cpu().numpy() & 3):
                assert torch.equal(fa[off[e]:off[e + 1]], h_fin[off[e]:off[e + 1]])


def test_sync_reports_clean_status(mods):
    flashnav, oracle, torch = mods
    wl = W.config_small(n_envs=8)
    sim = flashnav.NavSim.from_workload(wl)
    sim.reset(1)
    sim.sync(10000)


def test_autotune_keeps_state_and_results(mods):
    """The autotuner times candidate shapes on a copy of the state: the
    trajectory afterwards still matches the oracle."""
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=256, n_maps=2)
    sim = flashnav.NavSim.from_workload(wl)
    ref = oracle.OracleSim.from_workload(wl, threads=8)
    sim.reset(21)
    ref.reset(21)
    assert sim.autotune(steps=2) > 0
    acts = W.uniform_actions(21, 5, wl.n_envs)
    for t in range(5):
        o, r, d = sim.step(torch.from_numpy(acts[t]).cuda())
        ro, rr, rd = ref.step(acts[t])
        assert np.array_equal(d.cpu().numpy(), rd)
        _compare_obs(o.cpu().numpy(), ro, wl.env_beams)
    _compare_state(sim, ref, "after autotune")


def test_graph_replay_matches_eager_steps(mods):
    flashnav, oracle, torch = mods
    wl = W.config_small(n_envs=64)
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    n = 16
    acts = torch.from_numpy(W.uniform_actions(3, n, wl.n_envs)).cuda().contiguous()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a.reset(3)
        b.reset(3)
        obs = b.new_obs()
        rew = torch.empty(wl.n_envs, device="cuda")
        done = torch.empty(wl.n_envs, dtype=torch.uint8, device="cuda")
        b.graph_capture(acts, obs, rew, done)
        b.graph_launch()
        for t in range(n):
            eo, er, ed = a.step(acts[t])
    torch.cuda.synchronize()
    assert torch.equal(eo, obs) and torch.equal(er, rew) and torch.equal(ed, done)
    fa, ia, _ = a.get_state()
    fb, ib, _ = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ia, ib)


def test_uniform_action_generator_range(mods):
    flashnav, oracle, torch = mods
    wl = W.config_small(n_envs=4096)
    sim = flashnav.NavSim.from_workload(wl)
    a = sim.uniform_actions(1, 0)
    torch.cuda.synchronize()
    a = a.cpu().numpy()
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.05
    b = sim.uniform_actions(1, 1).cpu().numpy()
    assert not np.array_equal(a, b)


@pytest.mark.parametrize("byte_cells", [1, 3])
def test_uneven_maps_distance_bytes(mods, byte_cells):
    """The uneven workload's 64 maps of 128..1024 cells with distance bytes:
    maps up to 160 KiB staged in shared memory, larger ones read through
    L1/L2 (byte_cells 1) or staged as packed bits when those fit (3), with
    8 moving discs per env gating the jumps."""
    wl = W.config_uneven(n_envs=1536)
    run_parity(mods, wl, 4, seed=17, launch=(8, 512, 160 * 1024, 64, byte_cells), threads=16)


def test_uneven_workload_full_size(mods):
    """16384 envs over 64 maps of 128..1024 cells, beams 180/360/720, disc and
    rectangle robots, 8 moving discs per env, autotuned launch: reset and two
    steps compared in full (flags, hit cells, visits, observations, state)."""
    wl = W.config_uneven()
    run_parity(mods, wl, 2, seed=3, autotune=True, threads=16)


@pytest.mark.parametrize("n_envs,steps", [(64, 300), (37, 80)])
def test_split_step_small(mods, n_envs, steps):
    """Env-phase kernel + all-maps-resident ray kernel (split step)."""
    wl = W.config_small(n_envs=n_envs)
    run_parity(mods, wl, steps, seed=9, launch=(0, 0, 0, 0, 0, 1))


def test_split_step_throughput_maps(mods):
    wl = W.config_throughput(n_envs=2048, n_maps=16)
    sim, _, _ = run_parity(mods, wl, 4, seed=10, launch=(0, 0, 0, 0, 0, 1))
    assert sim.get_launch()[5] == 1


def test_split_step_mixed_beams_and_robots(mods):
    wl = _mixed()
    wl.maps = [m[:96, :96].copy() for m in wl.maps]
    run_parity(mods, wl, 60, seed=15, launch=(0, 0, 0, 0, 0, 1))


# --------------------------------------------------------------------------
# Paper sensing (Sec. 2.2.2, Eq. 6, Table 7): fixed-step march, sector minima
# --------------------------------------------------------------------------
def test_paper_turtlebot2_march_and_sectors(mods):
    """TurtleBot2 preset: one 10 x 10 m map, 1080 beams over 270 deg marched
    at 0.03 m to 20 m, 30 sector minima; hit cells and sample counts
    bit-exact, 120 steps with resets."""
    wl = W.config_paper("turtlebot2", n_envs=256)
    _, _, n_done = run_parity(mods, wl, 120, seed=4)
    assert n_done > 20


def test_paper_go2_march_and_sectors(mods):
    wl = W.config_paper("go2", n_envs=128)
    run_parity(mods, wl, 60, seed=5)


@pytest.mark.parametrize("launch", [(1, 64, 0, 32, 1), (4, 256, 0, 64, 2), (32, 512, 16, 40, 1),
                                    (8, 256, 16, 40, 2)])
def test_march_launch_shapes_and_staging(mods, launch):
    wl = W.config_paper("turtlebot2", n_envs=97)
    run_parity(mods, wl, 30, seed=6, launch=launch)


def test_march_split_step(mods):
    wl = W.config_paper("turtlebot2", n_envs=300)
    sim, _, _ = run_parity(mods, wl, 40, seed=7, launch=(0, 0, 0, 0, 0, 1))
    assert sim.get_launch()[5] == 1


def test_march_with_moving_discs_raw_beams(mods):
    """March with the moving-disc layer (t-gated per ray), raw 360-beam
    observation, two map sizes."""
    wl = _mixed()
    wl.params = W.Params(sensor=1, march_step=0.03, n_dyn=6, goal_dmin=1.0, goal_dmax=1e9)
    run_parity(mods, wl, 40, seed=8)


def test_march_long_step(mods):
    """A step longer than a cell (samples may skip cells): the explicit
    off-map test keeps the march inside the map."""
    wl = W.config_small()
    wl.params = W.Params(goal_dmin=1.0, goal_dmax=1e9, sensor=1, march_step=0.13)
    run_parity(mods, wl, 100, seed=9)


@pytest.mark.parametrize("m", [1, 12, 360])
def test_exact_traversal_with_sectors(mods, m):
    wl = W.config_throughput(n_envs=512, n_maps=4)
    wl.params = W.Params(n_sectors=m)
    run_parity(mods, wl, 20, seed=10)


def test_sector_count_must_divide_the_beams(mods):
    flashnav, _, _ = mods
    wl = W.config_small()
    wl.params = W.Params(goal_dmin=1.0, goal_dmax=1e9, n_sectors=7)  # 180 % 7 != 0
    with pytest.raises(flashnav.NavError):
        flashnav.NavSim.from_workload(wl)


# --------------------------------------------------------------------------
# Limits and degenerate inputs
# --------------------------------------------------------------------------
def test_maximum_beams_on_a_large_map(mods):
    """2048 beams (the per-env maximum) on one 2048 x 2048 map (102 m, the
    global-memory path), r_max 20 m (400 cells)."""
    occ = W.make_map(91, 2048, 2048, 0.02, corridors=True)
    wl = W.Workload(name="max", maps=[occ], env_map=np.zeros(24, np.int32),
                    env_beams=np.full(24, 2048, np.int32), env_robot=np.zeros(24, np.int32),
                    robots=[W.DISC], max_range=20.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=30.0))
    run_parity(mods, wl, 6, seed=21, threads=16)


@pytest.mark.parametrize("sensor", [0, 1])
def test_distance_jumps_on_a_sparse_map(mods, sensor):
    """Long free stretches (2 % occupancy, 20 m = 400-cell range on a
    20 x 20 m map) staged as distance bytes: most of each ray is covered by
    jumps; hit cells, visit counts and ranges must equal the oracle's
    cell-by-cell walk (exact traversal) or sample-by-sample march."""
    occ = W.make_map(93, 400, 400, 0.02)
    wl = W.Workload(name="sparse", maps=[occ], env_map=np.zeros(64, np.int32),
                    env_beams=np.full(64, 360, np.int32), env_robot=np.zeros(64, np.int32),
                    robots=[W.DISC], max_range=20.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=12.0, sensor=sensor,
                                    march_step=0.03))
    sim, _, _ = run_parity(mods, wl, 30, seed=23, launch=(8, 256, 200 * 1024, 64, 1, 2))
    assert sim.get_launch()[4] == 1


def test_empty_map_every_ray_reaches_max_range(mods):
    flashnav, oracle, torch = mods
    occ = np.zeros((512, 512), np.uint8)
    wl = W.Workload(name="empty", maps=[occ], env_map=np.zeros(16, np.int32),
                    env_beams=np.full(16, 360, np.int32), env_robot=np.zeros(16, np.int32),
                    robots=[W.DISC], max_range=4.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=3.0))
    sim = flashnav.NavSim.from_workload(wl)
    sim.set_debug(True)
    # every env at the map centre (12.8 m from any edge), heading 0
    f = np.zeros((16, 8), np.float32)
    f[:, 0] = f[:, 1] = 12.8
    f[:, 5] = f[:, 6] = 14.0
    f[:, 7] = float(np.hypot(1.2, 1.2))
    sim.reset(1)
    sim.set_state(1, f, np.zeros((16, 2), np.int32))
    obs, _, done = sim.step(torch.full((16, 2), -1.0, device="cuda").contiguous())  # v = 0
    r, h, _ = sim.debug()
    assert (h == -2).all() and (r == np.float32(4.0)).all()
    o = obs.cpu().numpy().reshape(16, 364)
    assert (o[:, :360] == np.float32(4.0)).all() and (done.cpu().numpy() == 0).all()


def test_rollout_workload_full_size(mods):
    """Config 4's simulator at full size: 65536 envs over 16 maps of 256 x 256,
    360 beams, autotuned launch; reset and two steps compared in full."""
    wl = W.config_throughput(n_envs=65536)
    run_parity(mods, wl, 2, seed=31, want_final=False, autotune=True, threads=16)


@pytest.mark.parametrize("cap,launch", [(3, (4, 256, 0, 64, 1, 4)), (5, (8, 512, 0, 40, 1, 2))])
def test_capped_grid(mods, cap, launch):
    """A step kernel capped at a few persistent CTAs (the overlapped
    collector's setting) takes every tile from the queue: same results."""
    run_parity(mods, W.config_small(n_envs=37), 60, seed=12, launch=launch, grid_cap=cap)
