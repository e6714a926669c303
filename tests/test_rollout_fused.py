"""The actor inside the step kernel (nav_rollout_fused: Sec. 2.3 collector,
Eq. 7 with the policy in the loop) against the CPU oracle simulator and the
FP64 actor.

Each launch steps a tile of envs, writes the new observations both to obs
and, scaled and rounded to BF16, into the actor's input tile in shared
memory, runs the 364-256-256-4 actor on the tensor cores and writes the next
actions.  The test steps one launch at a time, the actions of each launch
driving the next: the simulator outputs must match the oracle stepped with
the same actions (done flags bit-exact, ranges within 1e-4 m), and the
actions must match the FP64 actor on the observations the launch wrote, with
BF16 rounding at the GPU's points (inputs, hidden activations):
|a - a_ref| <= 3e-3 (the FP32 accumulation order differs).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav, torch, oracle


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).double().numpy()


def _unpack(w, sizes):
    params, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = w[off:off + a * b].reshape(b, a).astype(np.float64)
        off += a * b
        bb = w[off:off + b].astype(np.float64)
        off += b
        params.append([W, bb])
    return params


def _scale(K, max_range):
    s = np.ones(K + 4, np.float32)
    s[:K] = 1.0 / max_range
    s[K:] = [0.125, 1 / np.pi, 2.0, 1.0]
    return s


def _actor_bf16(params, obs, scale):
    """The FP64 actor with BF16 rounding at the GPU's points."""
    from oracle import mlp_oracle as M
    x = _bf16(obs * scale)
    for li, (W, b) in enumerate(params):
        z = x @ _bf16(W).T + b
        x = _bf16(M.leaky(z)) if li < len(params) - 1 else z
    return x


# hidden widths: 256 (the benchmark actor: two 128-row halves per K chunk),
# 200 (a partial second half) and 96 (one half)
@pytest.mark.parametrize("n_envs,n_maps,mode,hidden", [(2048, 4, 0, 256), (300, 3, 1, 256),
                                                       (18944, 16, 0, 256), (1024, 4, 0, 200),
                                                       (600, 3, 1, 96)])
def test_fused_rollout_lockstep_with_oracle_and_fp64_actor(env, n_envs, n_maps, mode, hidden):
    flashnav, torch, oracle = env
    lib = flashnav.load()
    wl = W.config_throughput(n_envs=n_envs, n_maps=n_maps)
    K = 360
    sim = flashnav.NavSim.from_workload(wl)
    ref = oracle.OracleSim.from_workload(wl, threads=16)
    h = C.c_void_p()
    assert lib.nav_policy_create(K + 4, hidden, n_envs, 13, C.byref(h)) == 0
    w = np.zeros(lib.nav_policy_num_params(h), np.float32)
    assert lib.nav_policy_get_weights(h, w.ctypes.data_as(C.c_void_p)) == 0
    params = _unpack(w, [K + 4, hidden, hidden, 4])
    scale = _scale(K, wl.max_range)
    assert lib.nav_policy_set_input_scale(h, scale.ctypes.data_as(C.c_void_p)) == 0
    sim.set_debug(True)
    obs = sim.reset(6)
    ref.reset(6)
    act = torch.empty(n_envs, 2, device="cuda")
    rew = torch.empty(n_envs, device="cuda")
    done = torch.empty(n_envs, dtype=torch.uint8, device="cuda")
    n_steps = 4 if n_envs > 4096 else 12
    for t in range(n_steps):
        sim._bind_stream()
        if t == 0:
            # the first action, from the inference path (nav_policy_act)
            assert lib.nav_policy_act(h, _p(obs), K + 4, n_envs, mode, 321, 0, _p(act), None,
                                      None, None) == 0
        a_t = act.cpu().numpy().copy()
        rc = lib.nav_rollout_fused(sim._h, h, 1, mode, 321, t, _p(obs), _p(act), _p(rew),
                                   _p(done), 1)
        assert rc == 0, lib.nav_last_error(sim._h)
        torch.cuda.synchronize()
        ro, rr, rd = ref.step(a_t)
        d = done.cpu().numpy()
        o = obs.cpu().numpy()
        assert np.array_equal(d, rd), f"step {t}: done flags"
        assert np.abs(rew.cpu().numpy() - rr).max() <= 1e-5
        _, hits, _ = sim.debug()
        _, rhits, _ = ref.debug()
        assert np.array_equal(hits, rhits), f"step {t}: hit cells"
        rows, rrows = o.reshape(n_envs, K + 4), ro.reshape(n_envs, K + 4)
        assert np.abs(rows[:, :K] - rrows[:, :K]).max() <= 1e-4, f"step {t}: ranges"
        # the in-kernel actor on the observations this launch wrote
        out = _actor_bf16(params, rows.astype(np.float64), scale.astype(np.float64))
        a = act.cpu().numpy().astype(np.float64)
        if mode == 0:
            err = np.abs(a - np.tanh(out[:, :2])).max()
            assert err <= 3e-3, f"step {t}: actions differ from the FP64 actor by {err}"
        else:
            # the same noise as the inference path for (seed, env, step t + 1)
            a2 = torch.empty(n_envs, 2, device="cuda")
            assert lib.nav_policy_act(h, _p(obs), K + 4, n_envs, 1, 321, t + 1, _p(a2), None,
                                      None, None) == 0
            torch.cuda.synchronize()
            err = np.abs(a - a2.cpu().numpy()).max()
            assert err <= 1e-2, f"step {t}: sampled actions differ by {err}"
    sim.sync(20000)
    lib.nav_policy_free(h)


def test_fused_rollout_rejects_what_it_does_not_cover(env):
    flashnav, torch, oracle = env
    lib = flashnav.load()
    h = C.c_void_p()
    assert lib.nav_policy_create(364, 256, 512, 3, C.byref(h)) == 0
    bad = [W.config_throughput(n_envs=512, n_maps=2) for _ in range(3)]
    bad[0].params = W.Params(n_sectors=12)
    bad[1].params = W.Params(n_dyn=2)
    bad[2].params = W.Params(sensor=1)
    act = torch.zeros(512, 2, device="cuda")
    rew = torch.empty(512, device="cuda")
    done = torch.empty(512, dtype=torch.uint8, device="cuda")
    for wl in bad:
        sim = flashnav.NavSim.from_workload(wl)
        obs = sim.reset(1)
        assert lib.nav_rollout_fused(sim._h, h, 1, 0, 1, 0, _p(obs), _p(act), _p(rew), _p(done),
                                     0) == -1
    wl = W.config_throughput(n_envs=512, n_maps=2)
    wl.env_beams[:] = 180  # obs_dim 184 != the policy's 364
    sim = flashnav.NavSim.from_workload(wl)
    obs = sim.reset(1)
    assert lib.nav_rollout_fused(sim._h, h, 1, 0, 1, 0, _p(obs), _p(act), _p(rew), _p(done), 0) == -1
    lib.nav_policy_free(h)
