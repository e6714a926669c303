"""Parity of the tiled step kernel with refilled lanes (nav_set_launch split
= 4) with the CPU oracle, element by element, through the C ABI.

In this ray phase a tile's rays form one range; every lane walks its own ray
with a branch-free iteration, and a warp whose lanes have gone idle takes as
many new rays as it has idle lanes from a shared counter.  The comparisons
are test_step_parity's: done flags, hit cells, per-beam visit counts,
counters and goals bit-exact; ranges within 1e-4 m, poses within 1e-5.
"""
import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W
from test_step_parity import _mixed, mods, run_parity  # noqa: F401

pytestmark = pytest.mark.gpu

REFILL = 4


def refill(tile=8, regs=64, smem=0, byte_cells=1):
    return (tile, 512, smem, regs, byte_cells, REFILL)


def _check_refill(sim):
    assert sim.get_launch()[5] == REFILL, "the refilled tiled kernel is not the one in use"


def test_refill_small_1000_steps(mods):
    sim, _, n_done = run_parity(mods, W.config_small(), 1000, seed=1, launch=refill(8))
    _check_refill(sim)
    assert n_done > 100


@pytest.mark.parametrize("tile,regs", [(1, 64), (10, 64), (32, 64), (8, 40), (12, 32)])
def test_refill_throughput_workload(mods, tile, regs):
    wl = W.config_throughput()
    sim, _, _ = run_parity(mods, wl, 3, seed=5, launch=refill(tile, regs), threads=16)
    _check_refill(sim)


def test_refill_mixed_maps_beams_rectangles(mods):
    sim, _, _ = run_parity(mods, _mixed(), 80, seed=11, launch=refill(4))
    _check_refill(sim)


def test_refill_maps_through_l2(mods):
    """A 16-byte budget: distance bytes read through L1/L2."""
    wl = W.config_throughput(n_envs=512, n_maps=4)
    sim, _, _ = run_parity(mods, wl, 6, seed=9, launch=refill(8, 64, 16))
    _check_refill(sim)


@pytest.mark.parametrize("m", [1, 12, 360])
def test_refill_sectors(mods, m):
    wl = W.config_throughput(n_envs=512, n_maps=4)
    wl.params = W.Params(n_sectors=m)
    sim, _, _ = run_parity(mods, wl, 20, seed=10, launch=refill(16))
    _check_refill(sim)


def test_refill_single_env_single_beam_and_cramped(mods):
    wl = W.config_small(n_envs=1)
    wl.env_beams[:] = 1
    run_parity(mods, wl, 50, seed=3, launch=refill(1))
    wl = W.config_small(n_envs=48)
    wl.maps = [W.make_map(77, 96, 96, 0.40)]
    sim, _, _ = run_parity(mods, wl, 100, seed=8, launch=refill(8))
    _check_refill(sim)


def test_refill_maximum_beams_on_a_large_map(mods):
    occ = W.make_map(91, 2048, 2048, 0.02, corridors=True)
    wl = W.Workload(name="max", maps=[occ], env_map=np.zeros(24, np.int32),
                    env_beams=np.full(24, 2048, np.int32), env_robot=np.zeros(24, np.int32),
                    robots=[W.DISC], max_range=20.0,
                    params=W.Params(goal_dmin=1.0, goal_dmax=30.0))
    sim, _, _ = run_parity(mods, wl, 6, seed=21, threads=16, launch=refill(8))
    _check_refill(sim)


def test_refill_visit_counter(mods):
    flashnav, oracle, torch = mods
    wl = W.config_throughput(n_envs=512, n_maps=4)
    sim = flashnav.NavSim.from_workload(wl)
    sim.set_launch(*refill(8))
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
    _check_refill(sim)


def test_refill_step_host_and_graph(mods):
    """nav_step_host and a captured graph with refilled lanes give nav_step's
    results exactly."""
    flashnav, oracle, torch = mods
    wl = _mixed(n_envs=75)
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    a.set_launch(*refill(8))
    b.set_launch(*refill(8))
    b.set_host_pipeline(3)
    a.reset(5)
    b.reset(5)
    acts = W.uniform_actions(5, 15, wl.n_envs)
    n = a.obs_size
    for t in range(15):
        o, r, d = a.step(torch.from_numpy(acts[t]).cuda())
        ho = np.zeros(n, np.float32)
        hr = np.zeros(wl.n_envs, np.float32)
        hd = np.zeros(wl.n_envs, np.uint8)
        b.step_host(np.ascontiguousarray(acts[t]), ho, hr, hd)
        assert np.array_equal(o.cpu().numpy(), ho)
        assert np.array_equal(r.cpu().numpy(), hr)
        assert np.array_equal(d.cpu().numpy(), hd)
    _check_refill(b)
    wl = W.config_throughput(n_envs=512, n_maps=4)
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    a.set_launch(*refill(16))
    b.set_launch(*refill(16))
    steps = 12
    acts = torch.from_numpy(W.uniform_actions(3, steps, wl.n_envs)).cuda().contiguous()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a.reset(3)
        b.reset(3)
        obs = b.new_obs()
        rew = torch.empty(wl.n_envs, device="cuda")
        done = torch.empty(wl.n_envs, dtype=torch.uint8, device="cuda")
        b.graph_capture(acts, obs, rew, done)
        b.graph_launch()
        for t in range(steps):
            eo, er, ed = a.step(acts[t])
    torch.cuda.synchronize()
    assert torch.equal(eo, obs) and torch.equal(er, rew) and torch.equal(ed, done)
    b.sync(10000)


def test_refill_matches_chunked_lanes_without_debug(mods):
    """The timed configuration (no debug outputs, no visit counter): refilled
    lanes give the chunked kernel's observations, rewards and flags bit for
    bit over 20 steps of the benchmark workload."""
    flashnav, oracle, torch = mods
    wl = W.config_throughput()
    a = flashnav.NavSim.from_workload(wl)
    b = flashnav.NavSim.from_workload(wl)
    b.set_launch(*refill(16))
    a.reset(9)
    b.reset(9)
    for t in range(20):
        act = b.uniform_actions(77, t)
        oa, ra, da = a.step(act)
        ob, rb, db = b.step(act)
        assert torch.equal(oa, ob) and torch.equal(ra, rb) and torch.equal(da, db), f"step {t}"
    b.sync(10000)
    _check_refill(b)
