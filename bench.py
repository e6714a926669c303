"""Throughput benchmark of the batched bitmap simulator step.

Workload: 4096 envs over 16 seeded 256x256 maps (10-25 % boxes, discs and
corridor walls, 0.05 m cells), 360 beams over 360 deg, r_max 6 m, disc robot,
goals 2-8 m, uniform random actions, auto-reset.  One step = one fused launch
that advances every env (action decode, arc integration, footprint, reward,
flags, sparse reset, 360-beam scan, observation).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank simulates its own
4096 envs on its own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s (360-beam scan)"
UNIT = "env-steps/s"
SEED = 12345
L2_FLUSH_BYTES = 256 << 20
SM_MAX_MHZ = 2032.0
# ncu counters of the step kernel per launch shape (DRAM bytes and warp
# instructions per launch, cell visits per launch), from the captures whose
# commands profiles/ records; a shape without a capture reports null
COUNTERS = os.path.join(ROOT, "profiles", "step_kernel_counters.json")


def _counters(launch):
    """(DRAM bytes, warp instructions per visit) of the ncu capture of this
    launch shape (tile_envs, block_threads, smem_map_bytes, max_regs,
    byte_cells, split), or (None, None): the same shape, with any
    shared-memory cap that stages the captured workload's maps."""
    try:
        with open(COUNTERS) as f:
            entries = json.load(f)["captures"]
    except (OSError, ValueError, KeyError):
        return None, None
    # byte_cells 1 (distance bytes) and 3 (bytes when they fit in shared
    # memory) stage the same maps when the cap holds the captured bytes
    cells = lambda c: 1 if c == 3 else c
    key = lambda l: (l[0], l[1], l[3], cells(l[4]), l[5])
    for e in entries:
        if key(e["launch"]) == key(launch) and launch[2] >= e.get("smem_min", e["launch"][2]):
            return float(e["dram_bytes_per_launch"]), float(e["warp_inst_per_launch"]) / float(
                e["visits_per_launch"])
    return None, None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Max of a per-rank float over the process group (the job's wall time
    is its slowest rank's); plain value on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, n_envs: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: the env-steps of every rank over the slowest
    rank's time (weak scaling: each rank steps its own n_envs)."""
    return world * n_envs * steps / seconds


def make_workload(rank: int):
    from paper_2606_15846_b300 import workloads as W
    # each rank simulates its own 4096 envs on its own 16 maps (weak scaling)
    return W.config_throughput(seed0=100 + 1000 * rank)


def cpu_baseline(wl, seconds: float = 15.0):
    """The oracle, as it stands, on all host cores over a bounded sample of the
    same workload: full 4096-env steps until ~`seconds` have elapsed."""
    from oracle import oracle
    from paper_2606_15846_b300 import workloads as W
    cores = os.cpu_count() or 1
    ref = oracle.OracleSim.from_workload(wl, threads=cores)
    ref.reset(SEED)
    acts = W.uniform_actions(SEED, 64, wl.n_envs)
    n = 0
    t0 = time.perf_counter()
    while True:
        ref.step(acts[n % 64])
        n += 1
        el = time.perf_counter() - t0
        if (el > seconds and n >= 3) or n >= 512:
            break
    # single-thread rate on the first 512 envs (same maps and actions)
    one = oracle.OracleSim.from_workload(_sub_workload(wl, 512), threads=1)
    one.reset(SEED)
    m = 0
    t1 = time.perf_counter()
    while True:
        one.step(acts[m % 64][:512])
        m += 1
        el1 = time.perf_counter() - t1
        if (el1 > 3.0 and m >= 3) or m >= 256:
            break
    return {"value": wl.n_envs * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": 512 * m / el1,
            "sample": f"{n} full steps of the {wl.n_envs}-env workload (C oracle, OpenMP over "
                      f"envs, {cores} threads), {el:.1f} s; single thread: {m} steps of the "
                      f"first 512 envs, {el1:.1f} s"}


def policy_rollout(steps: int = 20, n_envs: int = 65536, n_maps: int = 16):
    """Rollout with the policy in the loop on 65536 envs over 16 256x256 maps
    (or n_envs over n_maps; 18944 over 4 is one wave of the fused kernel's
    128-env tiles), 360 beams, actor 364-256-256-4 (random init, sampled
    actions): the actor
    inside the step kernel (nav_rollout_fused), the BF16 tensor-core policy
    as separate launches beside the step (nav_rollout), and the plain FP32
    SIMT policy (register-blocked shared-memory GEMM) beside the step."""
    import ctypes as C
    import torch
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import workloads as W
    wl = W.config_throughput(n_envs=n_envs, n_maps=n_maps)
    sim = flashnav.NavSim.from_workload(wl)
    sim.reset(SEED)
    sim.autotune(steps=3)  # one simulator launch shape for the unfused arms
    lib = flashnav.load()
    pol = C.c_void_p()
    assert lib.nav_policy_create(364, 256, wl.n_envs, 7, C.byref(pol)) == 0
    scale = np.ones(364, np.float32)
    scale[:360] = 1.0 / wl.max_range
    scale[360:] = [0.125, 1.0 / np.pi, 2.0, 1.0]
    assert lib.nav_policy_set_input_scale(pol, scale.ctypes.data_as(C.c_void_p)) == 0
    E = wl.n_envs
    obs = sim.new_obs()
    act = torch.empty(E, 2, device="cuda")
    rew = torch.empty(E, device="cuda")
    done = torch.empty(E, dtype=torch.uint8, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())

    def run(name, n, step0):
        sim._bind_stream()
        if name == "fused_actor_in_step":
            return lib.nav_rollout_fused(sim._h, pol, n, 1, 5, step0, P(obs), P(act), P(rew),
                                         P(done), 0)
        return lib.nav_rollout(sim._h, pol, n, 1, 5, step0, P(obs), P(act), P(rew), P(done),
                               1 if name == "fp32_simt_policy" else 0)

    out = {}
    for name in ("fused_actor_in_step", "bf16_tensor_core_policy", "fp32_simt_policy"):
        sim.reset(SEED, obs)
        assert run(name, 3, 0) == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        assert run(name, steps, 3) == 0
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"env_steps_per_s": E / (ms / 1e3), "ms_per_step": ms}
    sim.sync(60000)
    f32 = out["fp32_simt_policy"]["env_steps_per_s"]
    out["speedup_fused_vs_fp32"] = out["fused_actor_in_step"]["env_steps_per_s"] / f32
    out["speedup_bf16_vs_fp32"] = out["bf16_tensor_core_policy"]["env_steps_per_s"] / f32
    out["config"] = (f"{E} envs, {n_maps} maps 256x256, 360 beams, actor 364-256-256-4, "
                     "sampled actions")
    lib.nav_policy_free(pol)
    return out


def policy_forward(rows: int = 65536, calls: int = 20):
    """The actor 364-256-256-4 alone on `rows` observation rows (the policy
    half of the rollout workload): BF16 tensor-core path (observation
    conversion, three products, head) and the plain FP32 path, CUDA events
    over `calls` calls after 6 warm-up calls."""
    import ctypes as C
    import torch
    from paper_2606_15846_b300 import flashnav
    lib = flashnav.load()
    pol = C.c_void_p()
    assert lib.nav_policy_create(364, 256, rows, 7, C.byref(pol)) == 0
    g = torch.Generator(device="cuda")
    g.manual_seed(SEED)
    obs = torch.rand(rows, 364, device="cuda", generator=g) * 6.0
    act = torch.empty(rows, 2, device="cuda")
    logp = torch.empty(rows, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    s = torch.cuda.Stream()
    out = {}
    for name, fn in (("bf16_tensor_cores", lib.nav_policy_act), ("fp32_simt", lib.nav_policy_act_fp32)):
        with torch.cuda.stream(s):
            for it in range(6):
                assert fn(pol, P(obs), 364, rows, 0, 1, it, P(act), P(logp), None,
                          C.c_void_p(s.cuda_stream)) == 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for it in range(calls):
                assert fn(pol, P(obs), 364, rows, 0, 1, it, P(act), P(logp), None,
                          C.c_void_p(s.cuda_stream)) == 0
            e1.record(s)
            e1.synchronize()
        us = e0.elapsed_time(e1) / calls * 1e3
        flop = 2.0 * rows * (364 * 256 + 256 * 256 + 256 * 4)
        out[name] = {"us_per_forward": us, "tflops": flop / us / 1e6}
    lib.nav_policy_free(pol)
    out["config"] = f"{rows} rows of 364 features, actor 364-256-256-4, sampled actions"
    return out


def step_sizes(steps: int = 300, sizes=(1024, 2048, 4096, 8192, 16384, 32768, 65536)):
    """The plain step (16 maps 256x256, 360 beams, uniform actions) at batch
    sizes from 1024 to 65536 envs on one GPU: autotuned launch shape, L2
    flushed before each step, CUDA events around each step."""
    import torch
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import workloads as W
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for n in sizes:
        wl = W.config_throughput(n_envs=n)
        sim = flashnav.NavSim.from_workload(wl)
        obs = sim.new_obs()
        rew = torch.empty(n, device="cuda")
        done = torch.empty(n, dtype=torch.uint8, device="cuda")
        g = torch.Generator(device="cuda")
        g.manual_seed(SEED)
        acts = torch.rand(steps + 20, n, 2, device="cuda", generator=g) * 2 - 1
        sim.reset(SEED, obs)
        sim.autotune(steps=12)
        launch = sim.get_launch()
        sim.reset(SEED, obs)
        for t in range(20):
            sim.step(acts[t], obs, rew, done)
        stream = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        for t in range(steps):
            flush.fill_(float(t))
            ev[t][0].record(stream)
            sim.step(acts[20 + t], obs, rew, done)
            ev[t][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        out[str(n)] = {"us_per_step": ms * 1e3, "env_steps_per_s": n / (ms / 1e3),
                       "launch": list(launch)}
        del sim, obs, acts
    out["config"] = "16 maps 256x256, 360 beams, r_max 6 m, uniform actions, L2 flushed"
    return out


def uneven_batch(steps_per_graph: int = 20, replays: int = 5, eager: bool = False,
                 launch: str = "", tile_order: int = -1):
    """Uneven batch in one persistent launch per step: 16384 envs over 64 maps
    of 128..1024 cells, beams 180/360/720, disc and rectangle robots, 8 moving
    discs per env; autotuned; steps captured in one CUDA graph; L2 flushed
    between graph replays.  eager: the same steps launched one by one (L2
    flushed before each), for profilers that cannot follow graph launches.
    launch / tile_order: a fixed launch shape instead of the autotuner's (to
    profile the shape the benchmark's own run chose)."""
    import torch
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import workloads as W
    wl = W.config_uneven()
    sim = flashnav.NavSim.from_workload(wl)
    E = wl.n_envs
    s = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        obs = sim.reset(SEED)
        if launch:
            sim.set_launch(*[int(v) for v in launch.split(",")])
            if tile_order >= 0:
                sim.set_tile_order(tile_order)
            tune_ms = None
        else:
            tune_ms = sim.autotune(steps=3)
        obs = sim.reset(SEED, obs)
        acts = torch.empty(steps_per_graph, E, 2, device="cuda")
        for t in range(steps_per_graph):
            sim.uniform_actions(SEED, t, acts[t])
        rew = torch.empty(E, device="cuda")
        done = torch.empty(E, dtype=torch.uint8, device="cuda")
        # work count on a graph captured with the visit counter on
        sim.set_stats(True)
        sim.graph_capture(acts, obs, rew, done)
        sim.graph_launch()
        visits, rays = sim.stats()
        sim.set_stats(False)
        tot = 0.0
        if eager:
            for r in range(replays):
                for t in range(steps_per_graph):
                    flush.fill_(float(t))
                    e0, e1 = (torch.cuda.Event(enable_timing=True),
                              torch.cuda.Event(enable_timing=True))
                    e0.record(s)
                    sim.step(acts[t], obs, rew, done)
                    e1.record(s)
                    e1.synchronize()
                    tot += e0.elapsed_time(e1)
        else:
            sim.graph_capture(acts, obs, rew, done)
            sim.graph_launch()
            for r in range(replays):
                flush.fill_(float(r))
                e0, e1 = (torch.cuda.Event(enable_timing=True),
                          torch.cuda.Event(enable_timing=True))
                e0.record(s)
                sim.graph_launch()
                e1.record(s)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
    ms = tot / (replays * steps_per_graph)
    return {"env_steps_per_s": E / (ms / 1e3), "ms_per_step": ms,
            "beam_casts_per_step": rays / steps_per_graph,
            "cell_visits_per_s": visits / steps_per_graph / (ms / 1e3),
            "launch": dict(zip(("tile_envs", "block_threads", "smem_map_bytes", "max_regs",
                                "byte_cells", "split"), sim.get_launch()),
                           tile_order=sim.get_tile_order()),
            "autotune_ms_per_step": tune_ms,
            "config": "16384 envs, 64 maps 128..1024 cells, beams 180/360/720, disc+rect, "
                      "8 moving discs, graph of 20 steps, L2 flushed between replays"}


def gather_rates(reps: int = 10):
    """Random single-byte gather rates of this GPU (nav_gather_probe), in
    G reads/s: the memory ceilings of the beam traversal, whose lanes read
    unrelated cells, with the map in shared memory (a 64 KiB table per CTA,
    three CTAs per SM), in L2 (a 32 MiB table) or in HBM (a 2 GiB table)."""
    import torch
    from paper_2606_15846_b300 import flashnav
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    s = torch.cuda.Stream()
    out = {}
    for name, where, nbytes, blocks, iters in (("shared_64KiB", 0, 1 << 16, 3 * sms, 512),
                                               ("l2_32MiB", 1, 1 << 25, 8 * sms, 64),
                                               ("hbm_2GiB", 1, 1 << 31, 8 * sms, 16)):
        with torch.cuda.stream(s):
            table = (torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device="cuda")
                     if where else None)
            sums = torch.empty(blocks, dtype=torch.int32, device="cuda")
            for _ in range(3):
                flashnav.gather_probe(where, table, nbytes, blocks, iters, sums, s.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                flashnav.gather_probe(where, table, nbytes, blocks, iters, sums, s.cuda_stream)
            e1.record(s)
            e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = blocks * 256 * iters * 8 / (ms / 1e3) / 1e9
        del table
    out["unit"] = "G random byte reads/s"
    return out


def mma_rates(n_mma: int = 1024):
    """Cost of back-to-back tcgen05.mma (M 128, K 16, BF16) on this GPU by N,
    and of tcgen05.commit (nav_mma_probe): one CTA per SM, one thread issuing
    n_mma MMAs with no commit before the last, a commit every 4 MMAs that it
    waits on, a commit every 4 or every MMA that nobody waits on; ns per MMA
    (the slowest CTA) and the dense BF16 rate per SM it implies."""
    import torch
    from paper_2606_15846_b300 import flashnav
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ns = torch.zeros(sms, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {}
    for label, every, wait in (("no_commit", 0, 0), ("commit_every_4_waited", 4, 1),
                               ("commit_every_4", 4, 0), ("commit_every_1", 1, 0)):
        row = {}
        for n in (16, 64, 128, 256):
            for _ in range(2):
                flashnav.mma_probe(n, n_mma, every, wait, ns, status)
            torch.cuda.synchronize()
            per = float(ns.max().item()) / n_mma
            row[str(n)] = {"ns_per_mma": per, "tflops_per_sm": 2.0 * 128 * n * 16 / per / 1e3}
        out[label] = row
    assert int(status.item()) == 0, "a bounded wait in the MMA probe gave up"
    out["config"] = f"{sms} CTAs (one per SM), {n_mma} MMAs each, M 128, K 16, BF16 zero operands"
    return out


def paper_sensing(steps: int = 200, launch: str = ""):
    """The paper's sensing (Sec. 2.2.2, Eq. 6, Table 7) on its TurtleBot2
    setting: one shared 10 x 10 m map, 1080 beams over 270 deg to 20 m,
    30 sector minima.  The 0.03 m fixed-step march against the exact
    traversal on the same trajectories (uniform actions do not depend on the
    observation): env-steps/s at 1024 envs (the paper's count) and 16384
    envs, and the march's range error against the exact range per beam."""
    import dataclasses
    import torch
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import workloads as W
    out = {}
    s = torch.cuda.Stream()
    for n_envs in (1024, 16384):
        wl = W.config_paper("turtlebot2", n_envs=n_envs)
        for name, sensor in (("march_0.03m", 1), ("exact_traversal", 0)):
            w2 = dataclasses.replace(wl, params=dataclasses.replace(wl.params, sensor=sensor))
            sim = flashnav.NavSim.from_workload(w2)
            E = w2.n_envs
            with torch.cuda.stream(s):
                obs = sim.reset(SEED)
                if launch:
                    sim.set_launch(*[int(v) for v in launch.split(",")])
                else:
                    sim.autotune(steps=5)
                obs = sim.reset(SEED, obs)
                acts = torch.empty(steps, E, 2, device="cuda")
                for t in range(steps):
                    sim.uniform_actions(SEED, t, acts[t])
                rew = torch.empty(E, device="cuda")
                done = torch.empty(E, dtype=torch.uint8, device="cuda")
                for t in range(5):
                    sim.step(acts[t], obs, rew, done)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                for t in range(steps):
                    sim.step(acts[t], obs, rew, done)
                e1.record(s)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / steps
                sim.set_stats(True)
                for t in range(20):
                    sim.step(acts[t], obs, rew, done)
                visits, rays = sim.stats()
                sim.set_stats(False)
            out[f"{name}_{n_envs}env"] = {
                "env_steps_per_s": E / (ms / 1e3), "ms_per_step": ms,
                "samples_or_visits_per_ray": visits / max(rays, 1),
                "launch": sim.get_launch()}
            sim.close()
    # range error of the march against the exact traversal, same poses
    wl = W.config_paper("turtlebot2", n_envs=1024)
    sims = []
    for sensor in (1, 0):
        w2 = dataclasses.replace(wl, params=dataclasses.replace(wl.params, sensor=sensor))
        sims.append(flashnav.NavSim.from_workload(w2))
    diffs = []
    acts = W.uniform_actions(SEED + 1, 40, wl.n_envs)
    for sm in sims:
        sm.set_debug(True)
        sm.reset(SEED)
    for t in range(40):
        a = torch.from_numpy(acts[t]).cuda()
        rs = []
        for sm in sims:
            sm.step(a)
            rs.append(sm.debug()[0])
        diffs.append(rs[0] - rs[1])
    d = np.concatenate(diffs).astype(np.float64)
    out["march_minus_exact_range_m"] = {
        "rays": int(d.size), "mean": float(d.mean()), "p50": float(np.percentile(d, 50)),
        "p99": float(np.percentile(d, 99)), "max": float(d.max()), "min": float(d.min()),
        "frac_over_one_step": float(np.mean(d > 0.03 + 1e-6))}
    out["config"] = ("TurtleBot2 preset: one 200x200 map (0.05 m cells), 1080 beams, 270 deg, "
                     "20 m, 30 sectors, uniform actions; autotuned launch per handle")
    return out


def learner_update(n_updates: int = 200, graphs: bool = True):
    """Learner update time (Sec. 2.3) on a filled replay, replayed from a
    captured CUDA graph: the paper's (100) x 4 networks at batch 1024 on the
    fused passes and on the per-layer GEMM path (FastDSAC), FastSAC's C51
    critics on the fused passes, and the benchmark learner (364-256-256,
    batch 4096, per-layer path)."""
    import ctypes as C
    import torch
    from paper_2606_15846_b300 import flashnav
    lib = flashnav.load()
    P = lambda t: C.c_void_p(t.data_ptr())
    cases = {
        "paper_fastdsac_fused": dict(od=34, hidden=100, nh=4, batch=1024, ipap=30, fused=1),
        "paper_fastdsac_per_layer": dict(od=34, hidden=100, nh=4, batch=1024, ipap=30, fused=0),
        "paper_fastsac_fused": dict(od=34, hidden=100, nh=4, batch=1024, ipap=30, fused=1,
                                    algo=1, pf=1),
        "bench_fastdsac_per_layer": dict(od=364, hidden=256, nh=2, batch=4096, ipap=0, fused=0),
    }
    out = {}
    s = torch.cuda.Stream()
    S = C.c_void_p(s.cuda_stream)
    for name, c in cases.items():
        cfg = flashnav.nav_train_cfg()
        lib.nav_train_default_cfg(C.byref(cfg))
        cfg.obs_dim, cfg.hidden, cfg.n_hidden, cfg.batch = c["od"], c["hidden"], c["nh"], c["batch"]
        cfg.replay_capacity, cfg.ipap_features, cfg.algo = 1 << 20, c["ipap"], c.get("algo", 0)
        cfg.policy_freq = c.get("pf", 2)
        T = C.c_void_p()
        assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
        if c["fused"] == 0:
            assert lib.nav_trainer_set_fused(T, 0) == 0
        N = 65536
        g = torch.Generator(device="cuda")
        g.manual_seed(SEED)
        obs = torch.rand(N, c["od"], device="cuda", generator=g) * 5
        act = torch.rand(N, 2, device="cuda", generator=g) * 2 - 1
        rew = torch.randn(N, device="cuda", generator=g)
        done = torch.zeros(N, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(s):
            assert lib.nav_train_insert(T, P(obs), P(act), P(rew), P(done), P(obs), None, N, S) == 0
            assert lib.nav_trainer_set_graphs(T, 1 if graphs else 0) == 0
            assert lib.nav_train_update(T, 40, S) == 0  # capture (or warm-up)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(n_updates // 40):
                assert lib.nav_train_update(T, 40, S) == 0
            e1.record(s)
            e1.synchronize()
        ms = e0.elapsed_time(e1) / (n_updates // 40 * 40)
        out[name] = {"ms_per_update": ms, "updates_per_s": 1e3 / ms, "batch": c["batch"]}
        lib.nav_trainer_free(T)
    out["config"] = ("one critic update (+ actor update every 2nd for FastDSAC, every update for "
                     "FastSAC), " + ("graph-replayed" if graphs else "eager launches") +
                     " in groups of 40, random replay of 65536")
    return out


def training_run(seconds: float, robot: str = "disc"):
    """Config 5's training (FastDSAC from scratch): 16384 envs on 64 seeded
    256x256 training maps, 4 M replay, actor 364-256-256-4 and twin critics,
    batch 4096, 16 updates per env step, for a bounded wall-clock budget;
    the time at which the deterministic policy first reaches each success
    threshold on 1000 held-out maps (evaluation time included), and the share
    of held-out episodes a perfect planner could reach within the horizon."""
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import train as TR
    cfg = TR.TrainConfig(robot=robot, n_envs=16384, utd=16, time_budget_s=seconds, threshold=1.0)
    res = TR.train(cfg, log=lambda *a: None, keep_policy=True)
    hist = res["history"]
    # the final policy on the held-out episodes through the three policy
    # paths: BF16 tensor-core GEMMs, plain FP32, and the actor inside the
    # step kernel (deterministic actions; BF16 and FP32 round differently)
    pol = res["policy"]
    final = {"bf16_tensor_cores": TR.evaluate_policy(cfg, pol, fp32=False)[0],
             "fp32_simt": TR.evaluate_policy(cfg, pol, fp32=True)[0],
             "fused_actor_in_step": TR.evaluate_policy_fused(cfg, pol)[0]}
    flashnav.load().nav_policy_free(pol)
    reach = TR.reachable_fraction(cfg)
    times = {}
    for thr in (0.25, 0.50, 0.75, 1.00):
        hit = [h["t"] for h in hist if h["success"] >= thr]
        times[f"{int(thr * 100)}%"] = hit[0] if hit else None
    best = max(h["success"] for h in hist)
    hit = [h["t"] for h in hist if h["success"] >= reach["upper"]]
    return {"seconds_to_success": times, "best_success": best,
            "final_policy_success": final,
            "reachable_share": reach, "seconds_to_reachable_share": hit[0] if hit else None,
            "budget_s": seconds, "env_steps": res["env_steps"], "cycle_ms": res["cycle_ms"],
            "reactive_controller_success": TR.evaluate_reactive(cfg)[0],
            "config": f"{robot} robot, 16384 envs on 64 training maps 256x256, 1000 held-out "
                      "maps, batch 4096, 16 updates per env step, eval every 1 s"}


def training_cycle(robot: str = "disc", seconds: float = 3.0):
    """Config 5's training cycle (one collector step of 16384 envs and 16
    updates of the 364-256-256 networks, batch 4096), serial and with the
    collector on a second stream beside the updates (Sec. 3.3): device time
    per cycle from graph replays after a short run of each."""
    from paper_2606_15846_b300 import train as TR
    out = {}
    for name, ov, cap in (("serial", False, 0), ("overlapped", True, -1),
                          ("overlapped_uncapped", True, 0), ("overlapped_cap74", True, 74)):
        cfg = TR.TrainConfig(robot=robot, n_envs=16384, utd=16, time_budget_s=seconds,
                             threshold=2.0, overlap=ov, collector_ctas=cap, eval_every_s=1e9)
        out[name + "_ms"] = TR.train(cfg, log=lambda *a: None)["cycle_ms"]
    out["config"] = f"{robot} robot, 16384 envs, 16 updates per env step, batch 4096"
    return out


def compact(extras: dict) -> dict:
    """Headline numbers of the extra measurements (the full records go to
    stderr), short enough to stay in a truncated log's tail."""
    r = lambda v, n=4: None if v is None else float(f"{v:.{n}g}")
    c = {}
    pr = extras.get("policy_rollout")
    if pr:
        c["rollout_65536_Msteps"] = {k: r(pr[k]["env_steps_per_s"] / 1e6) for k in
                                     ("fused_actor_in_step", "bf16_tensor_core_policy",
                                      "fp32_simt_policy")}
        c["rollout_65536_Msteps"]["fused_vs_fp32"] = r(pr["speedup_fused_vs_fp32"], 3)
    ub = extras.get("uneven_batch")
    if ub:
        c["uneven_16384_Msteps"] = r(ub["env_steps_per_s"] / 1e6)
    ps = extras.get("paper_sensing")
    if ps:
        c["paper_sensing_16384_Msteps"] = {"march": r(ps["march_0.03m_16384env"]["env_steps_per_s"] / 1e6),
                                           "exact": r(ps["exact_traversal_16384env"]["env_steps_per_s"] / 1e6)}
    lu = extras.get("learner_update")
    if lu:
        c["learner_ms_per_update"] = {k: r(v["ms_per_update"], 3) for k, v in lu.items()
                                      if isinstance(v, dict)}
    tp = extras.get("training_paper_turtlebot2")
    if tp:
        c["train_turtlebot2_s"] = {**{k: r(v, 3) for k, v in tp["seconds_to_success"].items()},
                                   "best": r(tp["best_success"], 3)}
    for robot in ("disc", "rect"):
        t = extras.get(f"training_config5_{robot}")
        if t:
            c[f"train_cfg5_{robot}_s"] = {**{k: r(v, 3) for k, v in t["seconds_to_success"].items()},
                                          "best": r(t["best_success"], 3),
                                          "reachable": r(t["reachable_share"]["upper"], 3),
                                          "to_reachable": r(t["seconds_to_reachable_share"], 3),
                                          "final_bf16_fp32_fused": [
                                              r(t["final_policy_success"][k], 3) for k in
                                              ("bf16_tensor_cores", "fp32_simt",
                                               "fused_actor_in_step")]}
    tc = extras.get("training_cycle_config5")
    if tc:
        c["cycle_cfg5_ms"] = {"serial": r(tc["serial_ms"]), "overlapped": r(tc["overlapped_ms"])}
    return c


def training_paper(seconds: float, robot: str = "turtlebot2", algo: str = "fastdsac"):
    """The paper's own training setting (Tables 3-4, 7-9; Table 2's protocol):
    FastDSAC from scratch on one shared map, 1024 envs, the 0.03 m march with
    30 sector minima through Eq. 2, (100) x 4 networks, UTD 40, batch 1024;
    wall-clock seconds (evaluation included) to 90 / 95 / 100 % success over
    1000 fresh episodes of that map."""
    from paper_2606_15846_b300 import train as TR
    cfg = TR.paper_config(robot, algo, time_budget_s=seconds, threshold=1.0)
    res = TR.train(cfg, log=lambda *a: None, keep_policy=True)
    # config 4's "equal eval success": the trained policy on both paths
    s16, _ = TR.evaluate_policy(cfg, res["policy"], fp32=False)
    s32, _ = TR.evaluate_policy(cfg, res["policy"], fp32=True)
    import paper_2606_15846_b300.flashnav as FN
    FN.load().nav_policy_free(res["policy"])
    hist = res["history"]
    reach = {}
    for thr in (0.90, 0.95, 1.00):
        hit = [h["t"] for h in hist if h["success"] >= thr]
        reach[f"{int(thr * 100)}%"] = hit[0] if hit else None
    # training-cycle time of the serial graph, for Sec. 3.3's comparison
    serial = TR.train(TR.paper_config(robot, algo, time_budget_s=3.0, threshold=2.0,
                                      overlap=False), log=lambda *a: None)
    return {"seconds_to_success": reach, "best_success": max(h["success"] for h in hist),
            "budget_s": seconds, "env_steps": res["env_steps"],
            "cycle_ms_overlapped": res["cycle_ms"], "cycle_ms_serial": serial["cycle_ms"],
            "final_policy_success_bf16_tensor_cores": s16, "final_policy_success_fp32": s32,
            "reactive_controller_success": TR.evaluate_reactive(cfg)[0],
            "config": f"{robot} preset, {algo}: 1024 envs, one shared map, 1080 beams marched 0.03 m, "
                      "30 sectors, Eq. 2 inputs, (100)x4 nets on the fused passes, batch 1024, "
                      "UTD 40, gamma 0.97, AdamW 1e-3, collector/learner overlapped, one CUDA "
                      "graph per two env steps, eval every 1 s on 1000 fresh episodes"}


def table2(seconds: float, seeds: int):
    """Table 2's protocol on the paper presets: for TurtleBot2 and Go2 with
    FastDSAC and FastSAC, `seeds` training runs of `seconds` each; per
    threshold (90 / 95 / 100 % success) the best and the mean time over the
    seeds that reach it, and how many do (evaluation time included)."""
    from paper_2606_15846_b300 import train as TR
    out = {}
    for robot in ("turtlebot2", "go2"):
        for algo in ("fastdsac", "fastsac"):
            times = {0.90: [], 0.95: [], 1.00: []}
            best = []
            for sd in range(seeds):
                cfg = TR.paper_config(robot, algo, time_budget_s=seconds, threshold=1.0, seed=sd)
                hist = TR.train(cfg, log=lambda *a: None)["history"]
                best.append(max(h["success"] for h in hist))
                for thr in times:
                    hit = [h["t"] for h in hist if h["success"] >= thr]
                    if hit:
                        times[thr].append(hit[0])
            row = {}
            for thr, ts in times.items():
                row[f"{int(thr * 100)}%"] = {
                    "best_s": min(ts) if ts else None,
                    "mean_s": sum(ts) / len(ts) if ts else None,
                    "seeds_reached": len(ts)}
            row["best_success_per_seed"] = best
            out[f"{robot}_{algo}"] = row
    out["config"] = (f"{seeds} seeds x {seconds:.0f} s per preset and learner; paper presets as in "
                     "training_paper; mean over the seeds that reach each threshold")
    return out


def _sub_workload(wl, n):
    """The first n envs of a workload (same maps, beams and robots)."""
    import dataclasses
    return dataclasses.replace(wl, env_map=wl.env_map[:n].copy(),
                               env_beams=wl.env_beams[:n].copy(),
                               env_robot=wl.env_robot[:n].copy())


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only).
    Each step is one oracle step over a bounded sample of the workload's envs,
    sized from a probe so that warm-up plus timed steps take about 2 minutes."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle
    from paper_2606_15846_b300 import workloads as W
    wl = make_workload(0)
    cores = os.cpu_count() or 1
    probe = oracle.OracleSim.from_workload(wl, threads=cores)
    probe.reset(SEED)
    acts = W.uniform_actions(SEED, 64, wl.n_envs)
    t0 = time.perf_counter()
    probe.step(acts[0])
    probe.step(acts[1])
    per_env_s = (time.perf_counter() - t0) / 2 / wl.n_envs
    del probe
    budget_s = 120.0
    n = int(budget_s / max(args.steps + args.warmup, 1) / max(per_env_s, 1e-12))
    n = max(min(n, wl.n_envs), min(64, wl.n_envs))
    sub = _sub_workload(wl, n)
    ref = oracle.OracleSim.from_workload(sub, threads=cores)
    ref.reset(SEED)
    for t in range(args.warmup):
        ref.step(acts[t % 64, :n])
    t0 = time.perf_counter()
    for t in range(args.steps):
        ref.step(acts[(args.warmup + t) % 64, :n])
    el = time.perf_counter() - t0
    value = n * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "n_envs": wl.n_envs, "n_maps": len(wl.maps),
                   "map": "256x256", "beams": 360, "max_range_m": wl.max_range},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: the first {n} of the {wl.n_envs} envs "
                                   f"(C oracle, OpenMP over envs, {cores} threads); "
                                   f"{args.steps} timed steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import workloads as W

    wl = make_workload(rank)
    E = wl.n_envs
    sim = flashnav.NavSim.from_workload(wl, device=local)
    stream = torch.cuda.current_stream(dev)
    total_steps = args.warmup + args.steps
    # inputs resident in HBM before the timed region
    gen = torch.Generator(device=dev)
    gen.manual_seed(SEED + rank)
    actions = (torch.rand(total_steps, E, 2, device=dev, generator=gen) * 2 - 1).contiguous()
    obs = sim.new_obs()
    rew = torch.empty(E, device=dev)
    done = torch.empty(E, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    sim.reset(SEED + rank, obs)
    if args.launch:
        sim.set_launch(*[int(v) for v in args.launch.split(",")])
    else:
        sim.autotune(steps=12)
    launch = sim.get_launch()
    sim.reset(SEED + rank, obs)
    for t in range(args.warmup):
        sim.step(actions[t], obs, rew, done)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        for t in range(args.steps):
            flush.fill_(float(t))  # L2 flush between timed steps (untimed)
            starts[t].record(stream)
            sim.step(actions[args.warmup + t], obs, rew, done)
            ends[t].record(stream)
        barrier()
        wall = time.perf_counter() - w0
    sim.sync(60000)
    dur_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    step_ms = float(np.sum(dur_ms))
    step_ms = max_over_ranks(step_ms, world, dev)
    value = job_rate(world, E, args.steps, step_ms / 1e3)

    # work counted on an identical replay (same seed and actions): cell visits
    sim.reset(SEED + rank, obs)
    for t in range(args.warmup):
        sim.step(actions[t], obs, rew, done)
    sim.set_stats(True)
    for t in range(args.steps):
        sim.step(actions[args.warmup + t], obs, rew, done)
    visits, rays = sim.stats()
    sim.set_stats(False)

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e_steps = min(args.steps, 2000)
    h_act = torch.empty(e2e_steps, E, 2, dtype=torch.float32, pin_memory=True)
    h_act.copy_(actions[args.warmup:args.warmup + e2e_steps].cpu())
    h_obs = torch.empty(sim.obs_size, dtype=torch.float32, pin_memory=True)
    h_rew = torch.empty(E, dtype=torch.float32, pin_memory=True)
    h_done = torch.empty(E, dtype=torch.uint8, pin_memory=True)
    sim.reset(SEED + rank, obs)
    for t in range(args.warmup):
        sim.step(actions[t], obs, rew, done)
    barrier()
    e2e_s = 0.0
    for t in range(e2e_steps):
        flush.fill_(float(t))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step_host_ptrs(h_act[t].data_ptr(), h_obs.data_ptr(), h_rew.data_ptr(),
                           h_done.data_ptr())
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_value = job_rate(world, E, e2e_steps, e2e_s)

    if rank == 0:
        peaks, src = _peaks()
        sm_mhz = float(peaks.get("sm_max_mhz", SM_MAX_MHZ))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        traffic, ipv = _counters(launch)
        mean_launch_s = step_ms / 1e3 / args.steps
        visits_per_launch = visits / args.steps
        achieved = visits_per_launch / mean_launch_s / 1e9
        # one visit = one 32-bit shared-memory word gathered per lane; the SM
        # serves 32 such lanes per clock
        peak = n_sm * 32 * sm_mhz * 1e6 / 1e9
        issue = n_sm * 4 * sm_mhz * 1e6 / ipv / 1e9 if ipv else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "n_envs": E, "n_maps": len(wl.maps),
                       "map": "256x256", "beams": 360, "max_range_m": wl.max_range,
                       "robot": "disc r=0.18 m", "actions": "uniform [-1,1]^2",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"env shards x{world}",
                       "launch": {"tile_envs": launch[0], "block_threads": launch[1],
                                  "smem_map_bytes": launch[2], "max_regs": launch[3],
                                  "byte_cells": launch[4], "split": launch[5],
                                  "tile_order": sim.get_tile_order(),
                                  "chosen_by": "fixed" if args.launch else "autotuner"}},
            "beam_casts_per_s": world * rays / (step_ms / 1e3),
            "cell_visits_per_s": world * visits / (step_ms / 1e3),
            "visits_per_step": visits_per_launch,
            "timed_region_wall_s": wall,
            "gpu_launches": args.steps * (2 if launch[5] == 1 else 1),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "Gvisit/s", "frac": achieved / peak,
                         "traffic": traffic,
                         "peak_source": f"{n_sm} SMs x 32 shared-memory word gathers/clk x "
                                        f"{sm_mhz:.0f} MHz ({src} sm_max_mhz): the textbook "
                                        "walk's one lookup per visit; the kernel itself is "
                                        "bound by instruction issue (issue_bound)",
                         "kernel": "step kernel per launch.split (4: refilled lanes)",
                         # 4 warp instructions/clk/SM over the warp instructions
                         # per visit of this launch shape's ncu capture
                         "issue_bound": issue,
                         "frac_of_issue_bound": achieved / issue if issue else None},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": E * 2 * 4,
                    "d2h_bytes_per_step": sim.obs_size * 4 + E * 4 + E,
                    "steps": e2e_steps},
            "clocks": clk.summary(),
        }
        if world == 1 and args.extras:
            # measured random-gather ceilings beside the nominal one (the
            # 256x256 distance maps are staged in shared memory)
            g = gather_rates()
            line["roofline"]["measured_random_gather"] = g
            line["roofline"]["frac_of_measured_shared_gather"] = achieved / g["shared_64KiB"]
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl)
        if world == 1 and args.extras:
            ex = {"policy_rollout": policy_rollout()}
            ex["uneven_batch"] = ub = uneven_batch()
            # maps up to the staged size are read from shared memory
            ub["frac_of_measured_shared_gather"] = ub["cell_visits_per_s"] / 1e9 / g["shared_64KiB"]
            ex["paper_sensing"] = paper_sensing()
            ex["learner_update"] = learner_update()
            if args.train_seconds > 0:
                ex["training_paper_turtlebot2"] = training_paper(min(args.train_seconds, 25.0))
                for robot in ("disc", "rect"):
                    ex[f"training_config5_{robot}"] = training_run(min(args.train_seconds, 30.0),
                                                                   robot)
                ex["training_cycle_config5"] = training_cycle()
            print(json.dumps(ex), file=sys.stderr, flush=True)
            line["extras"] = compact(ex)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", type=int, default=1,
                    help="1: also time the policy-in-the-loop rollout and a training run")
    ap.add_argument("--train-seconds", type=float, default=45.0)
    ap.add_argument("--only", default="", choices=["", "policy_rollout", "policy_rollout_one_wave",
                             "policy_forward", "uneven_batch", "step_sizes",
                             "gather_rates", "mma_rates",
                             "paper_sensing", "training", "training_rect", "training_cycle",
                             "training_paper", "training_paper_go2", "training_paper_fastsac",
                             "learner_update", "table2"],
                    help="run one of the extra measurements alone")
    ap.add_argument("--seeds", type=int, default=5, help="table2: training seeds per setting")
    ap.add_argument("--eager", action="store_true",
                    help="learner_update, uneven_batch: eager launches instead of graph "
                         "replays (profiling)")
    ap.add_argument("--tile-order", type=int, default=-1,
                    help="uneven_batch with --launch: the tile queue order (0 or 1)")
    ap.add_argument("--launch", default="",
                    help="tile_envs,block_threads,smem_map_bytes,max_regs,byte_cells,split "
                         "(default: autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        fn = {"policy_rollout": policy_rollout,
              "policy_rollout_one_wave": lambda: policy_rollout(n_envs=18944, n_maps=4),
              "policy_forward": policy_forward,
              "step_sizes": step_sizes,
              "uneven_batch": lambda: uneven_batch(eager=args.eager, launch=args.launch,
                                                   tile_order=args.tile_order),
              "gather_rates": gather_rates,
              "mma_rates": mma_rates,
              "paper_sensing": lambda: paper_sensing(launch=args.launch),
              "learner_update": lambda: learner_update(graphs=not args.eager),
              "table2": lambda: table2(args.train_seconds, args.seeds),
              "training": lambda: training_run(args.train_seconds),
              "training_rect": lambda: training_run(args.train_seconds, "rect"),
              "training_cycle": training_cycle,
              "training_paper": lambda: training_paper(args.train_seconds),
              "training_paper_go2": lambda: training_paper(args.train_seconds, "go2"),
              "training_paper_fastsac": lambda: training_paper(args.train_seconds, "turtlebot2",
                                                               "fastsac")}[args.only]
        print(json.dumps({args.only: fn()}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
