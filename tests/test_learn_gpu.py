"""GPU parity of the FastDSAC learner (Sec. 2.3; Table 4) with the FP64
oracle (oracle/mlp_oracle.py): one critic + actor update on a known replay,
with the batch indices and noise the GPU drew read back and replayed in FP64.
BF16 tensor-core operands make the gradients approximate; every layer's
relative L2 error against FP64 is printed and bounded."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OD = 364


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


def _bf16(x):
    import torch
    return torch.tensor(np.asarray(x, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def _unpack(w, sizes):
    params, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = w[off:off + a * b].reshape(b, a).astype(np.float64)
        off += a * b
        params.append([W, w[off:off + b].astype(np.float64)])
        off += b
    return params


def _io(lib, T, what, n, dtype=np.float32):
    buf = np.zeros(n, dtype)
    assert lib.nav_trainer_io(T, what, 0, buf.ctypes.data_as(C.c_void_p)) == 0
    return buf


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _rowwise(g, ref, floor=1e-3):
    """Largest element error scaled by its row's magnitude (plus a floor of
    the whole matrix's): a few wrong rows or columns (a mis-indexed bias, a
    bad accumulator lane group) show here although a norm could hide them."""
    g, ref = np.atleast_2d(np.asarray(g, np.float64)), np.atleast_2d(np.asarray(ref, np.float64))
    scale = np.abs(ref).max(axis=1, keepdims=True) + floor * np.abs(ref).max() + 1e-30
    return float((np.abs(g - ref) / scale).max())


def _emul_grads(M, params, x16, dout):
    """The GPU's arithmetic with its BF16 rounding points, in FP64: forward on
    BF16 weights with BF16 activations; backward with the upstream gradient
    rounded to BF16 for the GEMMs (weight gradient dZ^T h, input gradient
    dZ W) and kept unrounded for the bias sums."""
    hs, h = [x16], x16
    L = len(params)
    for li, (W, b) in enumerate(params):
        z = h @ _bf16(W).T + b
        if li < L - 1:
            h = _bf16(M.leaky(z))
            hs.append(h)
    grads = [None] * L
    g32 = dout
    for li in range(L - 1, -1, -1):
        g16 = _bf16(g32)
        grads[li] = [g16.T @ hs[li], g32.sum(axis=0)]
        if li > 0:
            dh = g16 @ _bf16(params[li][0])
            g32 = dh * np.where(hs[li] > 0, 1.0, M.SLOPE)
    return grads


CONFIGS = {
    # the benchmark's learner: 364-256-256-4 actor, Adam, raw ranges
    "bench": dict(od=OD, hidden=256, n_hidden=2, wd=0.0, ipap=0, scale=False),
    # Table 3 / Eq. 2: (100) x 4 nets, AdamW 1e-3, 30 sector minima through
    # 1 / (l - beta), goal / velocity features scaled
    "paper": dict(od=34, hidden=100, n_hidden=4, wd=1e-3, ipap=30, scale=True),
    # the same networks on the per-layer GEMM path instead of the fused passes
    "paper_per_layer": dict(od=34, hidden=100, n_hidden=4, wd=1e-3, ipap=30, scale=True,
                            fused=0),
    # FastSAC (Table 5): twin C51 critics, 101 atoms on [-20, 20]
    "fastsac": dict(od=34, hidden=100, n_hidden=4, wd=1e-3, ipap=30, scale=True, algo=1),
    # config 5 at full batch: 4096 rows, 364-256-256 networks
    "bench_full_batch": dict(od=OD, hidden=256, n_hidden=2, wd=0.0, ipap=0, scale=False,
                             batch=4096),
}


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_one_update_matches_fp64(env, name):
    flashnav, torch = env
    run_update(flashnav, torch, name, CONFIGS[name])


def run_update(flashnav, torch, name, P, strict=True):
    """One learner update on the GPU replayed in FP64; returns the relative
    errors (and asserts their bounds when strict)."""
    from oracle import mlp_oracle as M
    errs = {}

    def check(key, val, bound):
        errs[key] = val
        if strict:
            assert val < bound, (key, val, bound)

    od, H, NH, ipap = P["od"], P["hidden"], P["n_hidden"], P["ipap"]
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.obs_dim, cfg.hidden, cfg.n_hidden = od, H, NH
    cfg.batch, cfg.replay_capacity, cfg.policy_freq, cfg.seed = P.get("batch", 256), 8192, 1, 7
    cfg.weight_decay, cfg.ipap_features = P["wd"], ipap
    c51 = P.get("algo", 0) == 1
    if c51:
        cfg.algo, cfg.reward_scale = 1, 1.0
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
    if "fused" in P:
        assert lib.nav_trainer_set_fused(T, P["fused"]) == 0
    scale = None
    if P["scale"]:
        scale = np.ones(od, np.float32)
        scale[ipap:] = [0.125, 1 / np.pi, 2.0, 4 / np.pi]
        assert lib.nav_trainer_set_input_scale(T, scale.ctypes.data_as(C.c_void_p)) == 0
    sa = [od] + [H] * NH + [4]
    sc = [od + 2] + [H] * NH + [cfg.n_atoms if c51 else 2]
    n_a = sum(a * b + b for a, b in zip(sa[:-1], sa[1:]))
    n_c = sum(a * b + b for a, b in zip(sc[:-1], sc[1:]))
    actor0 = _unpack(_io(lib, T, 0, n_a), sa)
    q0 = [_unpack(_io(lib, T, 1 + i, n_c), sc) for i in range(2)]
    qt0 = [_unpack(_io(lib, T, 3 + i, n_c), sc) for i in range(2)]
    scal0 = _io(lib, T, 24, 16)
    rng = np.random.default_rng(3)
    N = max(700, cfg.batch + 500)
    obs = rng.uniform(0, 6, (N, od)).astype(np.float32)
    nxt = np.clip(obs + rng.normal(0, 0.05, (N, od)), 0, 6).astype(np.float32)
    act = rng.uniform(-0.99, 0.99, (N, 2)).astype(np.float32)
    rew = rng.normal(0, 1, N).astype(np.float32)
    done = rng.choice([0, 0, 0, 1, 2, 5, 9], N).astype(np.uint8)
    dev = [torch.from_numpy(a).cuda() for a in (obs, act, rew, done, nxt)]
    assert lib.nav_train_insert(T, *[_p(d) for d in dev], None, N, None) == 0
    assert lib.nav_train_update(T, 1, None) == 0
    torch.cuda.synchronize()
    B = cfg.batch
    idx = _io(lib, T, 20, B, np.int32)
    eps_new = _io(lib, T, 21, 2 * B).reshape(B, 2).astype(np.float64)
    eps_next = _io(lib, T, 22, 2 * B).reshape(B, 2).astype(np.float64)
    zn = _io(lib, T, 23, B).astype(np.float64)
    y_gpu, ym_gpu = _io(lib, T, 25, B), _io(lib, T, 26, B)
    scal1 = _io(lib, T, 24, 16)
    assert (idx >= 0).all() and (idx < N).all()
    beta0 = float(scal0[12])

    def net_in(x):
        """What the GPU feeds its networks: the replay's BF16 row (raw for the
        Eq. 2 features, scaled for the rest), Eq. 2 and the scale, BF16."""
        x = np.asarray(x, np.float64)
        stored = x * (scale if scale is not None and ipap == 0 else 1.0)
        if ipap:
            stored = x.copy()
            if scale is not None:
                stored[:, ipap:] = x[:, ipap:] * scale[ipap:]
        stored = _bf16(stored)
        if not ipap:
            return stored, stored
        y = stored.copy()
        y[:, :ipap] = 1.0 / (stored[:, :ipap] - beta0)
        if scale is not None:
            y[:, :ipap] *= scale[:ipap]
        return _bf16(y), stored

    ob, ob_raw = net_in(obs[idx])
    nb, _ = net_in(nxt[idx])
    ab = _bf16(act[idx])
    rb, tb = rew[idx].astype(np.float64), (done[idx] & 1).astype(np.float64)
    alpha = float(np.exp(scal0[0]))
    sbar = float(scal0[1])
    # critic targets
    out_n, _ = M.mlp_forward(actor0, nb)
    a_next, logp_next, _ = M.actor_head(out_n, eps_next)
    xnc = np.concatenate([nb, _bf16(a_next)], axis=1)
    tq = [M.mlp_forward(qt0[i], xnc)[0] for i in range(2)]
    if c51:
        m_ref = M.c51_targets(rb, tb, tq[0], tq[1], logp_next, alpha, cfg.gamma,
                              cfg.reward_scale, cfg.v_min, cfg.v_max)
        m_gpu = _io(lib, T, 32, B * cfg.n_atoms).reshape(B, cfg.n_atoms).astype(np.float64)
        print(f"[{name}] target distribution rel err {_rel(m_gpu, m_ref):.2e}")
        check("target_dist", _rel(m_gpu, m_ref), 2e-2)
        assert np.abs(m_gpu.sum(axis=1) - 1).max() < 1e-4
    else:
        y, ym = M.critic_targets(rb, tb, tq[0], tq[1], logp_next, alpha, zn, cfg.gamma,
                                 cfg.reward_scale)
        print(f"[{name}] targets rel err y {_rel(y_gpu, y):.2e}  y_mean {_rel(ym_gpu, ym):.2e}")
        check("y", _rel(y_gpu, y), 2e-2)
        check("y_mean", _rel(ym_gpu, ym), 2e-2)
        ey = float(np.abs(y_gpu - y).max() / (np.abs(y).max() + 1e-30))
        print(f"[{name}] targets element-wise max err / max |y| {ey:.2e}")
        check("y.elem", ey, 5e-2)
    # critic gradients: against the same arithmetic with the GPU's BF16
    # rounding points (tight: checks the kernels), and against pure FP64
    # (the precision cost of BF16 operands, which grows with depth)
    xc = np.concatenate([ob, ab], axis=1)
    fp64_bound = 6e-2 if NH <= 2 else 3e-1
    for i in range(2):
        q, cache = M.mlp_forward(q0[i], xc)
        if c51:
            _, dq = M.c51_critic_loss(q, m_ref)
            # the BF16-emulated reference takes the GPU's own target distribution
            emul = _emul_grads(M, q0[i], xc, M.c51_critic_loss(q, m_gpu)[1])
        else:
            _, dq = M.critic_loss(q, y, ym, sbar, cfg.huber_delta)
            emul = _emul_grads(M, q0[i], xc, dq)
        grads, _ = M.mlp_backward(q0[i], cache, dq)
        g_gpu = _unpack(_io(lib, T, 11 + i, n_c), sc)
        for li, ((dW, db), (mW, mb), (gW, gb)) in enumerate(zip(grads, emul, g_gpu)):
            eW, eb = _rel(gW, dW), _rel(gb, db)
            mW_, mb_ = _rel(gW, mW), _rel(gb, mb)
            print(f"[{name}] critic {i + 1} layer {li + 1} grad rel err vs FP64 W {eW:.2e} "
                  f"b {eb:.2e}; vs BF16-emulated W {mW_:.2e} b {mb_:.2e}")
            check(f"q{i + 1}.W{li + 1}", eW, fp64_bound)
            check(f"q{i + 1}.b{li + 1}", eb, fp64_bound)
            check(f"q{i + 1}.W{li + 1}.emul", mW_, 3e-2)
            check(f"q{i + 1}.b{li + 1}.emul", mb_, 3e-2)
            # element by element, each row against its own scale
            rW, rb = _rowwise(gW, mW), _rowwise(gb, mb)
            print(f"[{name}] critic {i + 1} layer {li + 1} element-wise vs BF16-emulated "
                  f"W {rW:.2e} b {rb:.2e}")
            check(f"q{i + 1}.W{li + 1}.elem", rW, 1e-1)
            check(f"q{i + 1}.b{li + 1}.elem", rb, 1e-1)
    # Adam / AdamW first step on the GPU's own gradients
    q1_post = _unpack(_io(lib, T, 1, n_c), sc)
    g1 = _unpack(_io(lib, T, 11, n_c), sc)
    for (W0, b0), (g, gb), (W1, b1) in zip(q0[0], g1, q1_post):
        Wr, _, _ = M.adamw_step(W0, g, 0 * g, 0 * g, 1, cfg.lr_critic, cfg.beta1, cfg.beta2,
                                wd=cfg.weight_decay)
        br, _, _ = M.adamw_step(b0, gb, 0 * gb, 0 * gb, 1, cfg.lr_critic, cfg.beta1, cfg.beta2,
                                wd=cfg.weight_decay)
        assert np.abs(W1 - Wr).max() < 1e-6 and np.abs(b1 - br).max() < 1e-6
    # actor gradients (critics after their Adam step, as the GPU uses them)
    q_post = [_unpack(_io(lib, T, 1 + i, n_c), sc) for i in range(2)]
    out_a, cache_a = M.mlp_forward(actor0, ob)
    a_new, logp, _ = M.actor_head(out_a, eps_new)
    xa = np.concatenate([ob, _bf16(a_new)], axis=1)
    qa, caches = [], []
    for i in range(2):
        o, c = M.mlp_forward(q_post[i], xa)
        qa.append(o)
        caches.append(c)
    if c51:
        _, dlogp, dl1, dl2 = M.c51_actor_grads(logp, qa[0], qa[1], alpha, cfg.v_min, cfg.v_max)
        douts = (dl1, dl2)
    else:
        _, dlogp, dq1, dq2 = M.actor_loss_grads(logp, qa[0][:, 0], qa[1][:, 0], alpha)
        douts = (np.stack([dq1, 0 * dq1], axis=1), np.stack([dq2, 0 * dq2], axis=1))
    da = np.zeros((B, 2))
    for i, dqi in enumerate(douts):
        _, dX = M.mlp_backward(q_post[i], caches[i], dqi)
        da += dX[:, od:od + 2]
    dout = M.actor_head_grad(out_a, eps_new, da, dlogp)
    grads_a, dxa = M.mlp_backward(actor0, cache_a, dout)
    g_gpu = _unpack(_io(lib, T, 10, n_a), sa)
    for li, ((dW, db), (gW, gb)) in enumerate(zip(grads_a, g_gpu)):
        eW, eb = _rel(gW, dW), _rel(gb, db)
        print(f"[{name}] actor layer {li + 1} grad rel err W {eW:.2e} b {eb:.2e}")
        check(f"a.W{li + 1}", eW, 1e-1)
        check(f"a.b{li + 1}", eb, 1e-1)
    if ipap:
        # Eq. 2's beta: gradient through the actor's input, then one Adam step
        gb_ref = M.ipap_beta_grad(dxa, ob_raw, ipap, beta0, scale)
        gb_gpu = float(scal1[11])
        print(f"[{name}] beta grad gpu {gb_gpu:.6e} fp64 {gb_ref:.6e}")
        check("beta_grad", abs(gb_gpu - gb_ref) / (abs(gb_ref) + 1e-6), 0.1)
        b1, _, _ = M.adam_step(np.array(beta0), np.array(gb_gpu), 0.0, 0.0, 1, cfg.lr_actor,
                               cfg.beta1, cfg.beta2)
        assert abs(float(scal1[12]) - min(float(b1), cfg.ipap_beta_max)) < 1e-6
    lib.nav_trainer_free(T)
    return errs


def test_eval_reduction_fp64(env):
    flashnav, torch = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.batch, cfg.replay_capacity = 128, 256
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
    E, S = 1000, 40
    rng = np.random.default_rng(5)
    rew = rng.normal(0, 3, (S, E)).astype(np.float32)
    done = rng.choice([0] * 30 + [1 | 4, 1 | 8, 2, 1 | 4 | 8], (S, E)).astype(np.uint8)
    assert lib.nav_eval_begin(T, E, None) == 0
    for t in range(S):
        r, d = torch.from_numpy(rew[t]).cuda(), torch.from_numpy(done[t]).cuda()
        assert lib.nav_eval_accumulate(T, _p(r), _p(d), E, None) == 0
    succ, ret = C.c_double(), C.c_double()
    assert lib.nav_eval_result(T, E, C.byref(succ), C.byref(ret), None) == 0
    want_s, want_r = 0.0, 0.0
    for e in range(E):
        for t in range(S):
            want_r += float(rew[t, e])
            if done[t, e] & 3:
                want_s += 1.0 if (done[t, e] & 4 and not done[t, e] & 8) else 0.0
                break
    assert succ.value == want_s
    assert abs(ret.value - want_r) <= 1e-9 * max(1.0, abs(want_r))
    lib.nav_trainer_free(T)


def test_graph_replayed_updates_match_eager(env):
    """The update reads its indices, replay size and Adam corrections from
    device counters, so a captured sequence replayed twice does what eight
    eager updates do (same draws; split-K atomics may reorder sums)."""
    flashnav, torch = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.obs_dim, cfg.hidden, cfg.n_hidden, cfg.ipap_features = 34, 100, 4, 30
    cfg.batch, cfg.replay_capacity, cfg.seed, cfg.weight_decay = 256, 4096, 5, 1e-3
    rng = np.random.default_rng(1)
    N = 1500
    data = [rng.uniform(0, 6, (N, 34)).astype(np.float32),
            rng.uniform(-1, 1, (N, 2)).astype(np.float32),
            rng.normal(0, 1, N).astype(np.float32),
            rng.choice([0, 0, 1, 2], N).astype(np.uint8),
            rng.uniform(0, 6, (N, 34)).astype(np.float32)]
    dev = [torch.from_numpy(a).cuda() for a in data]
    s = torch.cuda.Stream()
    S = C.c_void_p(s.cuda_stream)
    out = []
    for graphs in (0, 1):
        T = C.c_void_p()
        assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
        assert lib.nav_trainer_set_graphs(T, graphs) == 0
        with torch.cuda.stream(s):
            assert lib.nav_train_insert(T, *[_p(d) for d in dev], None, N, S) == 0
            for _ in range(2):
                assert lib.nav_train_update(T, 4, S) == 0
        s.synchronize()
        sizes = [34, 100, 100, 100, 100, 4]
        n_a = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
        out.append((_io(lib, T, 0, n_a), _io(lib, T, 24, 16), _io(lib, T, 20, 256, np.int32)))
        rs, cu, au = C.c_int64(), C.c_int64(), C.c_int64()
        assert lib.nav_trainer_counts(T, C.byref(rs), C.byref(cu), C.byref(au)) == 0
        assert (rs.value, cu.value, au.value) == (N, 8, 4)
        lib.nav_trainer_free(T)
    (wa, sa, ia), (wb, sb, ib) = out
    assert np.array_equal(ia, ib)  # the last batch drawn is the same
    assert _rel(wb, wa) < 1e-5
    assert abs(float(sa[12]) - float(sb[12])) < 1e-6  # beta


def test_fused_and_per_layer_paths_agree(env):
    """Four updates of the (100) x 4 networks on the fused passes and on the
    per-layer GEMM path from the same state and draws: the weights agree up
    to summation order (split-K atomics vs partial sums)."""
    flashnav, torch = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.obs_dim, cfg.hidden, cfg.n_hidden, cfg.ipap_features = 34, 100, 4, 30
    cfg.batch, cfg.replay_capacity, cfg.seed, cfg.weight_decay = 512, 4096, 9, 1e-3
    rng = np.random.default_rng(2)
    N = 2000
    data = [rng.uniform(0, 6, (N, 34)).astype(np.float32),
            rng.uniform(-1, 1, (N, 2)).astype(np.float32),
            rng.normal(0, 1, N).astype(np.float32),
            rng.choice([0, 0, 1, 2], N).astype(np.uint8),
            rng.uniform(0, 6, (N, 34)).astype(np.float32)]
    dev = [torch.from_numpy(a).cuda() for a in data]
    sa = [34, 100, 100, 100, 100, 4]
    sc = [36, 100, 100, 100, 100, 2]
    n_a = sum(a * b + b for a, b in zip(sa[:-1], sa[1:]))
    n_c = sum(a * b + b for a, b in zip(sc[:-1], sc[1:]))
    out = []
    for fused in (1, 0):
        T = C.c_void_p()
        assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
        assert lib.nav_trainer_set_fused(T, fused) == 0
        assert lib.nav_train_insert(T, *[_p(d) for d in dev], None, N, None) == 0
        assert lib.nav_train_update(T, 4, None) == 0
        torch.cuda.synchronize()
        out.append((_io(lib, T, 0, n_a), _io(lib, T, 1, n_c), _io(lib, T, 2, n_c),
                    _io(lib, T, 3, n_c), _io(lib, T, 24, 16), _io(lib, T, 11, n_c)))
        lib.nav_trainer_free(T)
    names = ["actor", "critic 1", "critic 2", "target 1", "scalars", "critic 1 grad"]
    for name, a, b in zip(names, *out):
        e = _rel(a, b)
        print(f"fused vs per-layer {name}: rel {e:.2e}")
        assert e < (2e-2 if name.endswith("grad") else 1e-3), (name, e)


def test_fused_path_is_refused_for_wide_networks(env):
    flashnav, _ = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.batch, cfg.replay_capacity = 256, 1024
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0  # 364 inputs, 256 wide
    assert lib.nav_trainer_set_fused(T, 1) != 0
    assert lib.nav_trainer_set_fused(T, 0) == 0
    lib.nav_trainer_free(T)


@pytest.mark.parametrize("size,pending,lo,hi", [(2000, 1000, 952, 2000), (2048, 512, 0, 2048)])
def test_overlapped_draws_skip_the_slots_being_written(env, size, pending, lo, hi):
    """Producer-consumer pipeline: with an insert of `pending` transitions in
    flight, the updates draw only slots that insert leaves alone (ring of
    2048; head at `size` mod 2048)."""
    flashnav, torch = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.obs_dim, cfg.hidden, cfg.n_hidden = 34, 100, 2
    cfg.batch, cfg.replay_capacity, cfg.seed = 1024, 2048, 3
    T = C.c_void_p()
    assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
    rng = np.random.default_rng(0)
    n_ins = size if size < 2048 else 2048 + 700  # full ring with the head at 700
    data = [rng.uniform(0, 6, (n_ins, 34)).astype(np.float32),
            rng.uniform(-1, 1, (n_ins, 2)).astype(np.float32),
            rng.normal(0, 1, n_ins).astype(np.float32),
            np.zeros(n_ins, np.uint8),
            rng.uniform(0, 6, (n_ins, 34)).astype(np.float32)]
    dev = [torch.from_numpy(a).cuda() for a in data]
    for s0 in range(0, n_ins, 1000):
        n = min(1000, n_ins - s0)
        part = [d[s0:s0 + n].contiguous() for d in dev]
        assert lib.nav_train_insert(T, *[_p(d) for d in part], None, n, None) == 0
    head = n_ins % 2048
    assert lib.nav_train_overlap(T, pending, None) == 0
    seen = []
    for _ in range(6):
        assert lib.nav_train_update(T, 1, None) == 0
        seen.append(_io(lib, T, 20, 1024, np.int32))
    assert lib.nav_train_overlap(T, 0, None) == 0
    idx = np.concatenate(seen)
    written = {(head + e) % 2048 for e in range(pending)}
    assert not (set(idx.tolist()) & written)
    if size < 2048:
        assert idx.min() >= lo and idx.max() < hi
    # the safe set is covered roughly uniformly
    assert len(set(idx.tolist())) > 0.9 * min(2048 - pending, len(idx)) * 0.6
    lib.nav_trainer_free(T)


def test_overlapped_schedule_matches_serial_schedule(env):
    """Producer-consumer pipeline (Sec. 3.3) against the serial schedule it
    replaces: four cycles of (insert 1000 transitions, 4 updates), once on
    one stream and once with every insert on a collector stream running
    beside the updates on the learner's stream.  The serial run takes the
    same replay snapshot before its insert (nav_train_overlap), so both runs
    draw the same batches from the same slots; the weights, the scalars and
    the counts must then agree, up to the summation order of the loss sums'
    atomics, which a race on the replay (an update reading a slot while the
    concurrent insert writes it, or reading the live replay size) would
    break."""
    flashnav, torch = env
    lib = flashnav.load()
    cfg = flashnav.nav_train_cfg()
    lib.nav_train_default_cfg(C.byref(cfg))
    cfg.obs_dim, cfg.hidden, cfg.n_hidden, cfg.ipap_features = 34, 100, 4, 30
    cfg.batch, cfg.replay_capacity, cfg.seed, cfg.weight_decay = 512, 8192, 7, 1e-3
    rng = np.random.default_rng(11)

    def chunk(n):
        return [torch.from_numpy(a).cuda() for a in (
            rng.uniform(0, 6, (n, 34)).astype(np.float32),
            rng.uniform(-1, 1, (n, 2)).astype(np.float32),
            rng.normal(0, 1, n).astype(np.float32),
            rng.choice([0, 0, 0, 1, 2], n).astype(np.uint8),
            rng.uniform(0, 6, (n, 34)).astype(np.float32))]

    N0, E, cycles, utd = 2000, 1000, 4, 4
    prefill = chunk(N0)
    data = [chunk(E) for _ in range(cycles)]
    sa = [34, 100, 100, 100, 100, 4]
    sc = [36, 100, 100, 100, 100, 2]
    n_a = sum(a * b + b for a, b in zip(sa[:-1], sa[1:]))
    n_c = sum(a * b + b for a, b in zip(sc[:-1], sc[1:]))
    learn, coll = torch.cuda.Stream(), torch.cuda.Stream()
    SL, SC = C.c_void_p(learn.cuda_stream), C.c_void_p(coll.cuda_stream)
    out = []
    for overlapped in (False, True):
        T = C.c_void_p()
        assert lib.nav_trainer_create(C.byref(cfg), C.byref(T)) == 0
        assert lib.nav_train_insert(T, *[_p(d) for d in prefill], None, N0, SL) == 0
        idx = []
        for c in range(cycles):
            assert lib.nav_train_overlap(T, E, SL) == 0
            if overlapped:
                fork, join = torch.cuda.Event(), torch.cuda.Event()
                fork.record(learn)
                coll.wait_event(fork)
                assert lib.nav_train_insert(T, *[_p(d) for d in data[c]], None, E, SC) == 0
                assert lib.nav_train_update(T, utd, SL) == 0
                join.record(coll)
                learn.wait_event(join)
            else:
                assert lib.nav_train_insert(T, *[_p(d) for d in data[c]], None, E, SL) == 0
                assert lib.nav_train_update(T, utd, SL) == 0
            assert lib.nav_train_overlap(T, 0, SL) == 0
            learn.synchronize()
            idx.append(_io(lib, T, 20, 512, np.int32))
        rs, cu, au = C.c_int64(), C.c_int64(), C.c_int64()
        assert lib.nav_trainer_counts(T, C.byref(rs), C.byref(cu), C.byref(au)) == 0
        out.append(dict(counts=(rs.value, cu.value, au.value), idx=np.stack(idx),
                        actor=_io(lib, T, 0, n_a), c1=_io(lib, T, 1, n_c), c2=_io(lib, T, 2, n_c),
                        t1=_io(lib, T, 3, n_c), t2=_io(lib, T, 4, n_c), scalars=_io(lib, T, 24, 16)))
        lib.nav_trainer_free(T)
    ser, ovl = out
    assert ser["counts"] == ovl["counts"] == (N0 + cycles * E, cycles * utd, cycles * utd // 2)
    # the same batches, and none of them touches the slots of its cycle's insert
    assert np.array_equal(ser["idx"], ovl["idx"])
    for c in range(cycles):
        head = N0 + c * E
        assert not (set(ovl["idx"][c].tolist()) & set(range(head, head + E)))
    for k in ("actor", "c1", "c2", "t1", "t2"):
        e = _rel(ovl[k], ser[k])
        print(f"overlapped vs serial {k}: rel {e:.2e}")
        assert e < 1e-5, (k, e)
    assert abs(float(ovl["scalars"][12]) - float(ser["scalars"][12])) < 1e-6  # beta
