"""GPU tests of the tensor-core MLP kernels against the FP64 reference.

The GEMM computes C = act(A B^T + bias) with BF16 inputs and FP32
accumulation; the reference is the binary64 product of the same BF16
values, so the only error is FP32 accumulation order (bounded by
K * 2^-23 * sum |a||b|) and, for BF16 outputs, one BF16 rounding.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav, torch


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


@pytest.mark.parametrize("m,n,k,lda,act", [
    (128, 256, 64, 64, 0), (4096, 256, 364, 368, 1), (200, 40, 100, 104, 0),
    (1, 4, 256, 256, 0), (333, 256, 256, 256, 1), (4096, 2, 256, 256, 0),
    (129, 17, 16, 16, 1), (4096, 256, 256, 264, 0),
    # several tiles per persistent CTA (626 tiles for 296 CTAs): accumulator
    # and stage-ring reuse across tiles
    (40000, 256, 256, 256, 1)])
def test_gemm_matches_fp64(env, m, n, k, lda, act):
    flashnav, torch = env
    lib = flashnav.load()
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n * 3 + k)
    A = torch.randn(m, lda, device="cuda", generator=g).to(torch.bfloat16)
    ldb = (k + 7) // 8 * 8
    B = torch.randn(n, ldb, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(n, device="cuda", generator=g)
    c32 = torch.full((m, n), float("nan"), device="cuda")
    c16 = torch.zeros(m, n, dtype=torch.bfloat16, device="cuda")
    c16t = torch.zeros(n, m, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.nav_gemm_bf16(_p(A), lda, _p(B), ldb, m, n, k, _p(bias), act, _p(c32), n, _p(c16), n,
                           _p(c16t), m, _p(status), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a64 = A[:, :k].double().cpu().numpy()
    b64 = B[:, :k].double().cpu().numpy()
    ref = a64 @ b64.T + bias.double().cpu().numpy()
    if act:
        ref = np.where(ref > 0, ref, 0.01 * ref)
    bound = (np.abs(a64) @ np.abs(b64).T) * (k * 2.0 ** -23) + 1e-6
    got = c32.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= bound + 1e-5).all(), np.abs(got - ref).max()
    g16 = c16.double().cpu().numpy()
    assert np.abs(g16 - got).max() <= np.abs(got).max() * 2.0 ** -8 + 1e-6
    assert torch.equal(c16t, c16.t())


# ---------------------------------------------------------------------------
# policy inference (Sec. 2.1 actor MLP, tanh-squashed Gaussian head)
# ---------------------------------------------------------------------------
def _bf16(x):
    import torch
    return torch.tensor(np.asarray(x, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def _unpack(w, sizes):
    params, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = w[off:off + a * b].reshape(b, a).astype(np.float64)
        off += a * b
        bb = w[off:off + b].astype(np.float64)
        off += b
        params.append([W, bb])
    return params


def _policy(lib, obs_dim, n, seed=5):
    h = C.c_void_p()
    assert lib.nav_policy_create(obs_dim, 256, n, seed, C.byref(h)) == 0
    npar = lib.nav_policy_num_params(h)
    w = np.zeros(npar, np.float32)
    assert lib.nav_policy_get_weights(h, w.ctypes.data_as(C.c_void_p)) == 0
    return h, w


def test_policy_forward_bf16_against_fp64(env):
    from oracle import mlp_oracle as M
    flashnav, torch = env
    lib = flashnav.load()
    obs_dim, n = 364, 4096
    h, w = _policy(lib, obs_dim, n)
    params = _unpack(w, [obs_dim, 256, 256, 4])
    rng = np.random.default_rng(0)
    obs = np.concatenate([rng.uniform(0, 6, (n, 360)), rng.uniform(0, 8, (n, 1)),
                          rng.uniform(-3, 3, (n, 1)), rng.uniform(0, 0.5, (n, 1)),
                          rng.uniform(-1, 1, (n, 1))], axis=1).astype(np.float32)
    obs_t = torch.from_numpy(obs).cuda()
    act = torch.empty(n, 2, device="cuda")
    out = torch.empty(n, 4, device="cuda")
    assert lib.nav_policy_act(h, _p(obs_t), obs_dim, n, 0, 0, 0, _p(act), None, _p(out), None) == 0
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    # (a) the same arithmetic with BF16 rounding at the same points, in FP64
    x = _bf16(obs)
    for li, (W, b) in enumerate(params):
        z = x @ _bf16(W).T + b
        x = _bf16(M.leaky(z)) if li < 2 else z
    assert np.abs(got - x).max() <= 2e-3 * max(1.0, np.abs(x).max())
    # (b) the precision error of the BF16 path against pure FP64, per layer
    ref, cache = M.mlp_forward(params, obs.astype(np.float64))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"actor output relative L2 error, BF16 tensor cores vs FP64: {rel:.2e}")
    assert rel < 3e-2
    a_ref = np.tanh(ref[:, :2])
    assert np.abs(act.cpu().numpy() - a_ref).max() < 5e-2
    lib.nav_policy_free(h)


def test_policy_fp32_path_against_fp64(env):
    from oracle import mlp_oracle as M
    flashnav, torch = env
    lib = flashnav.load()
    obs_dim, n = 364, 512
    h, w = _policy(lib, obs_dim, n, seed=9)
    params = _unpack(w, [obs_dim, 256, 256, 4])
    obs = np.random.default_rng(1).uniform(-1, 4, (n, obs_dim)).astype(np.float32)
    obs_t = torch.from_numpy(obs).cuda()
    act = torch.empty(n, 2, device="cuda")
    out = torch.empty(n, 4, device="cuda")
    assert lib.nav_policy_act_fp32(h, _p(obs_t), obs_dim, n, 0, 0, 0, _p(act), None, _p(out),
                                   None) == 0
    torch.cuda.synchronize()
    ref, _ = M.mlp_forward(params, obs.astype(np.float64))
    got = out.double().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    lib.nav_policy_free(h)


def test_sampled_actions_and_log_prob(env):
    from oracle import mlp_oracle as M
    flashnav, torch = env
    lib = flashnav.load()
    obs_dim, n = 364, 2048
    h, _ = _policy(lib, obs_dim, n, seed=3)
    obs_t = torch.rand(n, obs_dim, device="cuda") * 4
    act = torch.empty(n, 2, device="cuda")
    logp = torch.empty(n, device="cuda")
    out = torch.empty(n, 4, device="cuda")
    assert lib.nav_policy_act(h, _p(obs_t), obs_dim, n, 1, 77, 3, _p(act), _p(logp), _p(out),
                              None) == 0
    torch.cuda.synchronize()
    a = act.double().cpu().numpy()
    o = out.double().cpu().numpy()
    assert (np.abs(a) < 1).all()
    _, _, (u, r, ls, sig, _) = M.actor_head(o, np.zeros((n, 2)))
    eps = (np.arctanh(np.clip(a, -1 + 1e-7, 1 - 1e-7)) - u) / sig
    ok = (np.abs(a) < 0.999).all(axis=1)
    _, lp_ref, _ = M.actor_head(o[ok], eps[ok])
    assert np.abs(logp.double().cpu().numpy()[ok] - lp_ref).max() < 1e-2
    assert abs(eps[ok].mean()) < 0.1 and abs(eps[ok].std() - 1) < 0.1
    lib.nav_policy_free(h)


def test_rollout_with_policy_matches_oracle_sim(env, oracle):
    from paper_2606_15846_b300 import workloads as W
    flashnav, torch = env
    lib = flashnav.load()
    wl = W.config_throughput(n_envs=256, n_maps=2)
    sim = flashnav.NavSim.from_workload(wl)
    ref = oracle.OracleSim.from_workload(wl, threads=8)
    h, _ = _policy(lib, 364, wl.n_envs, seed=11)
    obs = sim.reset(4)
    ref.reset(4)
    act = torch.empty(wl.n_envs, 2, device="cuda")
    rew = torch.empty(wl.n_envs, device="cuda")
    done = torch.empty(wl.n_envs, dtype=torch.uint8, device="cuda")
    for t in range(10):
        sim._bind_stream()
        assert lib.nav_rollout(sim._h, h, 1, 1, 99, t, _p(obs), _p(act), _p(rew), _p(done), 0) == 0
        torch.cuda.synchronize()
        ro, rr, rd = ref.step(act.cpu().numpy())
        assert np.array_equal(done.cpu().numpy(), rd)
        assert np.abs(obs.cpu().numpy() - ro).max() <= 1e-4 * 10
    lib.nav_policy_free(h)


@pytest.mark.parametrize("fp32", [0, 1])
def test_paper_actor_with_ipap_against_fp64(env, fp32):
    """Table 3's actor, (100) x 4 hidden units (a width that is not a multiple
    of the 16-column MMA step), on 30 sector minima through Eq. 2 with
    beta = -0.3 and a scale on the goal / velocity features; both the BF16
    tensor-core path and the FP32 SIMT path against the FP64 oracle."""
    from oracle import mlp_oracle as M
    flashnav, torch = env
    lib = flashnav.load()
    od, n, ipap, beta = 34, 1000, 30, -0.3
    h = C.c_void_p()
    assert lib.nav_policy_create_ex(od, 100, 4, ipap, C.c_float(beta), n, 21, C.byref(h)) == 0
    npar = lib.nav_policy_num_params(h)
    sizes = [od, 100, 100, 100, 100, 4]
    assert npar == sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    w = np.zeros(npar, np.float32)
    assert lib.nav_policy_get_weights(h, w.ctypes.data_as(C.c_void_p)) == 0
    params = _unpack(w, sizes)
    scale = np.ones(od, np.float32)
    scale[ipap:] = [0.125, 1 / np.pi, 2.0, 4 / np.pi]
    assert lib.nav_policy_set_input_scale(h, scale.ctypes.data_as(C.c_void_p)) == 0
    rng = np.random.default_rng(5)
    obs = np.concatenate([rng.uniform(0, 20, (n, ipap)), rng.uniform(0, 8, (n, 1)),
                          rng.uniform(-3, 3, (n, 1)), rng.uniform(0, 0.5, (n, 1)),
                          rng.uniform(-0.8, 0.8, (n, 1))], axis=1).astype(np.float32)
    obs_t = torch.from_numpy(obs).cuda()
    act = torch.empty(n, 2, device="cuda")
    out = torch.empty(n, 4, device="cuda")
    fn = lib.nav_policy_act_fp32 if fp32 else lib.nav_policy_act
    assert fn(h, _p(obs_t), od, n, 0, 0, 0, _p(act), None, _p(out), None) == 0
    b_got = C.c_float()
    assert lib.nav_policy_get_beta(h, C.byref(b_got)) == 0 and b_got.value == np.float32(beta)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    ref, _ = M.mlp_forward(params, M.ipap_forward(obs.astype(np.float64), ipap, beta, scale))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"paper actor ({'FP32 SIMT' if fp32 else 'BF16 tensor cores'}) rel L2 vs FP64: {rel:.2e}")
    assert rel < (1e-5 if fp32 else 3e-2)
    lib.nav_policy_free(h)


def test_policy_forward_full_size_sampled_rows(env):
    """Config 4's policy at full size: 65536 rows, 364-256-256-4, BF16 tensor
    cores; 2000 sampled rows against FP64 (BF16 rounding points emulated)."""
    from oracle import mlp_oracle as M
    flashnav, torch = env
    lib = flashnav.load()
    obs_dim, n = 364, 65536
    h, w = _policy(lib, obs_dim, n, seed=7)
    params = _unpack(w, [obs_dim, 256, 256, 4])
    rng = np.random.default_rng(4)
    obs = np.concatenate([rng.uniform(0, 6, (n, 360)), rng.uniform(0, 8, (n, 1)),
                          rng.uniform(-3, 3, (n, 1)), rng.uniform(0, 0.5, (n, 1)),
                          rng.uniform(-1, 1, (n, 1))], axis=1).astype(np.float32)
    obs_t = torch.from_numpy(obs).cuda()
    act = torch.empty(n, 2, device="cuda")
    out = torch.empty(n, 4, device="cuda")
    assert lib.nav_policy_act(h, _p(obs_t), obs_dim, n, 0, 0, 0, _p(act), None, _p(out), None) == 0
    torch.cuda.synchronize()
    rows = rng.choice(n, 2000, replace=False)
    got = out.double().cpu().numpy()[rows]
    x = _bf16(obs[rows])
    for li, (W_, b) in enumerate(params):
        z = x @ _bf16(W_).T + b
        x = _bf16(M.leaky(z)) if li < 2 else z
    assert np.abs(got - x).max() <= 2e-3 * max(1.0, np.abs(x).max())
    lib.nav_policy_free(h)
