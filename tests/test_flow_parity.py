"""Parity of the pipelined step (nav_set_launch split = 3: one CTA per SM,
a producer warp running the env phase and staging maps, ray-casting warps
that refill idle lanes from a shared cursor) with the CPU oracle, element by
element, through the C ABI.

The same comparisons as test_step_parity: done flags, hit cells, per-beam
visit counts, counters and goals bit-exact; ranges within 1e-4 m, poses
within 1e-5.  The cases cover one and two shared map buffers, maps read
through L1/L2, groups with no home CTA (work taken from other groups), claim
sizes from 1 to 32 envs, final observations, sector minima, the host-buffer
pipeline and graph replay.
"""
import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W
from test_step_parity import _compare_obs, _compare_state, _mixed, mods, run_parity  # noqa: F401

pytestmark = pytest.mark.gpu

FLOW = 3  # nav_set_launch split value of the pipelined step


def flow(claim=16, smem=0):
    """Launch tuple for run_parity: claim size, shared-memory budget."""
    return (claim, 0, smem, 0, 0, FLOW)


def _check_flow(sim):
    assert sim.get_launch()[5] == FLOW, "the pipelined step is not the one in use"


def test_flow_small_1000_steps(mods):
    """64 envs on one 64 x 64 map, 180 beams, 1000 steps with auto-reset and
    final observations."""
    sim, _, n_done = run_parity(mods, W.config_small(), 1000, seed=1, launch=flow())
    _check_flow(sim)
    assert n_done > 100


@pytest.mark.parametrize("claim", [1, 4, 32])
def test_flow_throughput_workload(mods, claim):
    """The benchmark workload (4096 envs over 16 maps of 256 x 256, 360
    beams, 6 m) with two shared map buffers and several claim sizes."""
    wl = W.config_throughput()
    sim, _, _ = run_parity(mods, wl, 3, seed=5, launch=flow(claim), threads=16)
    _check_flow(sim)


def test_flow_one_map_buffer(mods):
    """Maps of 352 x 352 cells (126 KB as distance bytes) leave room for one
    shared buffer: every restage waits for the rays of the previous map
    (16 maps, 512 envs)."""
    wl = W.config_throughput(n_envs=512, n_maps=16, size=352)
    sim, _, _ = run_parity(mods, wl, 6, seed=8, launch=flow(8, 200 * 1024))
    _check_flow(sim)


def test_flow_all_maps_through_l2(mods):
    """A 16-byte budget stages no map: every lane reads distance bytes
    through L1/L2."""
    wl = W.config_throughput(n_envs=512, n_maps=4)
    sim, _, _ = run_parity(mods, wl, 6, seed=9, launch=flow(8, 16))
    _check_flow(sim)


def test_flow_mixed_maps_beams_rectangles(mods):
    """Four map sizes, beams 180/360/720/45, disc and rectangle robots,
    final observations."""
    sim, _, _ = run_parity(mods, _mixed(), 80, seed=11, launch=flow(4))
    _check_flow(sim)


def test_flow_more_groups_than_ctas(mods):
    """More (map, beam table) groups than SMs: most groups have no home CTA
    and are taken by CTAs whose own group ran out."""
    maps = [W.make_map(300 + i, 64 + 8 * (i % 5), 64, 0.15, corridors=False) for i in range(40)]
    e = np.arange(640)
    wl = W.Workload(name="many-groups", maps=maps, env_map=(e % 40).astype(np.int32),
                    env_beams=np.array([90, 180, 270, 360, 33], np.int32)[(e // 40) % 5],
                    env_robot=np.zeros(640, np.int32), robots=[W.DISC], max_range=3.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=1e9))
    sim, _, _ = run_parity(mods, wl, 30, seed=12, launch=flow(2))
    _check_flow(sim)


def test_flow_single_env_single_beam(mods):
    wl = W.config_small(n_envs=1)
    wl.env_beams[:] = 1
    sim, _, _ = run_parity(mods, wl, 50, seed=3, launch=flow(1))
    _check_flow(sim)


def test_flow_cramped_map(mods):
    wl = W.config_small(n_envs=48)
    wl.maps = [W.make_map(77, 96, 96, 0.40)]
    sim, _, _ = run_parity(mods, wl, 100, seed=8, launch=flow(8))
    _check_flow(sim)


@pytest.mark.parametrize("m", [1, 12, 360])
def test_flow_sectors(mods, m):
    """Eq. 6 sector minima folded by per-ray atomic minima."""
    wl = W.config_throughput(n_envs=512, n_maps=4)
    wl.params = W.Params(n_sectors=m)
    sim, _, _ = run_parity(mods, wl, 20, seed=10, launch=flow(16))
    _check_flow(sim)


def test_flow_uneven_maps_mixed_views(mods):
    """64 maps of 128..1024 cells without moving discs: maps within the
    160 KiB budget staged, larger ones read through L1/L2 (generic loads)."""
    wl = W.config_uneven(n_envs=1536, n_dyn=0)
    sim, _, _ = run_parity(mods, wl, 4, seed=17, launch=flow(8, 160 * 1024), threads=16)
    _check_flow(sim)


def test_flow_maximum_beams_on_a_large_map(mods):
    """2048 beams on one 2048 x 2048 map (too large to stage), r_max 20 m."""
    occ = W.make_map(91, 2048, 2048, 0.02, corridors=True)
    wl = W.Workload(name="max", maps=[occ], env_map=np.zeros(24, np.int32),
                    env_beams=np.full(24, 2048, np.int32), env_robot=np.zeros(24, np.int32),
                    robots=[W.DISC], max_range=20.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=30.0))
    sim, _, _ = run_parity(mods, wl, 6, seed=21, threads=16, launch=flow(8))
    _check_flow(sim)


def test_flow_rollout_workload_full_size(mods):
    """65536 envs over 16 maps of 256 x 256, 360 beams: reset and two steps
    compared in full."""
    wl = W.config_throughput(n_envs=65536)
    sim, _, _ = run_parity(mods, wl, 2, seed=31, want_final=False, launch=flow(16), threads=16)
    _check_flow(sim)


@pytest.mark.parametrize("parts", [1, 3])
def test_flow_step_host_matches_device_step(mods, parts):
    """nav_step_host over `parts` env ranges with the pipelined step gives
    nav_step's results exactly."""
    flashnav, oracle, torch = mods
    wl = _mixed(n_envs=75)
    a_sim = flashnav.NavSim.from_workload(wl)
    b_sim = flashnav.NavSim.from_workload(wl)
    a_sim.set_launch(*flow(8))
    b_sim.set_launch(*flow(8))
    b_sim.set_host_pipeline(parts)
    a_sim.reset(5)
    b_sim.reset(5)
    acts = W.uniform_actions(5, 20, wl.n_envs)
    n = a_sim.obs_size
    for t in range(20):
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
        off = a_sim.obs_offsets
        fa = fo.cpu().numpy()
        for e in np.flatnonzero(dd & 3):
            assert np.array_equal(fa[off[e]:off[e + 1]], hf[off[e]:off[e + 1]])
    _check_flow(b_sim)


def test_flow_graph_replay_matches_eager_steps(mods):
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=512, n_maps=4)
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    a.set_launch(*flow(8))
    b.set_launch(*flow(8))
    n = 12
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
    b.sync(10000)


def test_flow_matches_tiled_kernel_without_debug(mods):
    """The timed configuration (no debug outputs, no visit counter): the
    pipelined step's observations, rewards and flags equal the tiled
    kernel's bit for bit over 20 steps of the benchmark workload."""
    flashnav, oracle, torch = mods
    wl = W.config_throughput()
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    b.set_launch(*flow(16))
    a.reset(9)
    b.reset(9)
    for t in range(20):
        act = b.uniform_actions(77, t)
        oa, ra, da = a.step(act)
        ob, rb, db = b.step(act)
        assert torch.equal(oa, ob) and torch.equal(ra, rb) and torch.equal(da, db), f"step {t}"
    b.sync(10000)
    _check_flow(b)


def test_flow_visit_counter(mods):
    """The visit counter of the pipelined step equals the oracle's
    cell-by-cell count, final scans included."""
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=512, n_maps=4)
    sim = flashnav.NavSim.from_workload(wl)
    sim.set_launch(*flow(8))
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
    _check_flow(sim)
