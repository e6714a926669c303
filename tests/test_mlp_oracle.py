"""Pins of the FP64 MLP / FastDSAC oracle (oracle/mlp_oracle.py) against
facts fixed outside it: central finite differences, Adam's first step in
closed form (Kingma & Ba, Algorithm 1), normalisation of the squashed
Gaussian density, Huber's closed form, and the clipped-double-Q choice."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = x[i]
        x[i] = old + h
        fp = f()
        x[i] = old - h
        fm = f()
        x[i] = old
        g[i] = (fp - fm) / (2 * h)
    return g


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-12)


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = M.init_mlp(rng, [7, 6, 5, 3])
    x = rng.normal(size=(4, 7))
    R = rng.normal(size=(4, 3))
    loss = lambda: float((M.mlp_forward(params, x)[0] * R).sum())
    out, cache = M.mlp_forward(params, x)
    grads, dx = M.mlp_backward(params, cache, R)
    for (W, b), (dW, db) in zip(params, grads):
        assert _rel(dW, _fd(loss, W)) < 1e-6
        assert _rel(db, _fd(loss, b)) < 1e-6
    assert _rel(dx, _fd(loss, x)) < 1e-6


def test_leaky_relu_slope():
    z = np.array([-2.0, 0.0, 3.0])
    assert np.allclose(M.leaky(z), [-0.02, 0.0, 3.0])


def test_actor_head_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    out = rng.normal(size=(5, 4))
    eps = rng.normal(size=(5, 2))
    ca = rng.normal(size=(5, 2))
    cl = rng.normal(size=5)
    loss = lambda: float((M.actor_head(out, eps)[0] * ca).sum() + (M.actor_head(out, eps)[1] * cl).sum())
    g = M.actor_head_grad(out, eps, ca, cl)
    assert _rel(g, _fd(loss, out)) < 1e-6


def test_squashed_gaussian_density_integrates_to_one():
    quad = pytest.importorskip("scipy.integrate").quad
    for u, r in [(0.3, -0.5), (-1.2, 0.4), (0.0, 2.0)]:
        ls = M.LS_MIN + (M.LS_MAX - M.LS_MIN) * 0.5 * (math.tanh(r) + 1)
        sig = math.exp(ls)

        def dens(a):
            pre = math.atanh(a)
            eps = (pre - u) / sig
            out = np.array([[u, u, r, r]])
            _, logp, _ = M.actor_head(out, np.array([[eps, eps]]))
            return math.exp(float(logp[0]) / 2.0)  # one of two identical dims
        val = quad(dens, -1 + 1e-12, 1 - 1e-12, limit=400, points=[math.tanh(u)])[0]
        assert abs(val - 1.0) < 2e-3, (u, r, val)


def test_log_sigma_range():
    out = np.array([[0, 0, -50.0, 50.0]])
    _, _, (u, r, ls, sig, pre) = M.actor_head(out, np.zeros((1, 2)))
    assert ls[0, 0] == pytest.approx(M.LS_MIN) and ls[0, 1] == pytest.approx(M.LS_MAX)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    lr = 3e-4
    p1, m, v = M.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr, 0.9, 0.95, 1e-8)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.05 * g * g)


def test_huber_closed_form():
    d = 50.0
    assert M.huber(np.array([3.0]), d)[0] == 4.5
    assert M.huber(np.array([-60.0]), d)[0] == d * (60.0 - 25.0)
    assert M.huber(np.array([d]), d)[0] == 0.5 * d * d  # continuous at delta
    assert np.array_equal(M.huber_grad(np.array([-70.0, 2.0, 80.0]), d), [-50.0, 2.0, 50.0])


def test_critic_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    q = rng.normal(size=(6, 2))
    y = rng.normal(size=6)
    ym = rng.normal(size=6)
    for sbar in (1e-3, 1e3):  # the weight sits on a clip bound: constant in q
        m_sg = q[:, 0].copy()  # stop-gradient copy held fixed
        loss = lambda: M.critic_loss(q, y, ym, sbar, m_sg=m_sg)[0]
        _, dq = M.critic_loss(q, y, ym, sbar)
        assert _rel(dq, _fd(loss, q)) < 1e-6


def test_targets_use_the_smaller_mean_and_clip_the_sample():
    rew = np.array([1.0, 1.0])
    term = np.array([0.0, 1.0])
    tq1 = np.array([[2.0, 0.0], [2.0, 0.0]])
    tq2 = np.array([[3.0, 5.0], [1.0, 5.0]])
    y, ym = M.critic_targets(rew, term, tq1, tq2, np.zeros(2), 0.0, np.array([10.0, 0.0]),
                             0.99, 0.4)
    s1 = M.softplus(0.0) + M.SIG_FLOOR
    assert ym[0] == pytest.approx(0.4 + 0.99 * 2.0)
    assert y[0] == pytest.approx(0.4 + 0.99 * (2.0 + 3.0 * s1))  # clipped at 3 sigma
    assert ym[1] == pytest.approx(0.4) and y[1] == pytest.approx(0.4)  # terminal


def test_actor_loss_gradients():
    logp = np.array([0.5, -1.0])
    q1 = np.array([1.0, 3.0])
    q2 = np.array([2.0, 0.0])
    loss, dl, d1, d2 = M.actor_loss_grads(logp, q1, q2, 0.2)
    assert loss == pytest.approx(((0.2 * 0.5 - 1.0) + (0.2 * -1.0 - 0.0)) / 2)
    assert np.allclose(dl, [0.1, 0.1]) and np.allclose(d1, [-0.5, 0]) and np.allclose(d2, [0, -0.5])


def test_softplus_is_stable():
    assert M.softplus(np.array([800.0]))[0] == 800.0
    assert M.softplus(np.array([0.0]))[0] == pytest.approx(math.log(2.0))


def test_adamw_without_gradient_is_pure_decay():
    """AdamW's decay is decoupled: with a zero gradient (zero moments) the
    step is exactly p (1 - lr wd); with wd = 0 it is Adam's step."""
    rng = np.random.default_rng(4)
    p = rng.normal(size=(5, 3))
    z = np.zeros_like(p)
    out, _, _ = M.adamw_step(p, z, z, z, 1, 3e-4, wd=1e-3)
    np.testing.assert_allclose(out, p * (1 - 3e-7), rtol=0, atol=1e-15)
    g = rng.normal(size=p.shape)
    a, _, _ = M.adamw_step(p, g, z, z, 1, 3e-4, wd=0.0)
    b, _, _ = M.adam_step(p, g, z, z, 1, 3e-4)
    np.testing.assert_array_equal(a, b)
    # first step: p (1 - lr wd) - lr sign(g) (Kingma & Ba: |step| = lr at t = 1)
    c, _, _ = M.adamw_step(p, g, z, z, 1, 1e-2, wd=0.5)
    np.testing.assert_allclose(c, p * (1 - 5e-3) - 1e-2 * np.sign(g), rtol=0, atol=1e-6)


def test_ipap_transform_values():
    """Eq. 2: l_hat = 1 / (l - beta); l = 0 gives -1/beta, long ranges go to
    zero, other features pass through (then the scale applies)."""
    x = np.array([[0.0, 1.0, 19.0, 3.5, -2.0]])
    out = M.ipap_forward(x, 3, -0.25)
    np.testing.assert_allclose(out[0, :3], [4.0, 0.8, 1.0 / 19.25])
    np.testing.assert_array_equal(out[0, 3:], x[0, 3:])
    sc = np.array([1.0, 2.0, 1.0, 0.5, 1.0])
    np.testing.assert_allclose(M.ipap_forward(x, 3, -0.25, sc), out * sc)


def test_ipap_beta_gradient_matches_finite_differences():
    """dL/dbeta through Eq. 2 and a whole actor (MLP + squashed Gaussian
    head, eps fixed), against central differences in beta."""
    rng = np.random.default_rng(8)
    n, D = 6, 10
    x = np.concatenate([rng.uniform(0.1, 8.0, (5, n)), rng.normal(size=(5, D - n))], axis=1)
    params = M.init_mlp(rng, [D, 12, 12, 4])
    eps = rng.normal(size=(5, 2))
    R = rng.normal(size=(5, 2))
    sc = rng.uniform(0.5, 2.0, D)

    def loss(beta):
        out, _ = M.mlp_forward(params, M.ipap_forward(x, n, beta, sc))
        a, logp, _ = M.actor_head(out, eps)
        return float((a * R).sum() + 0.3 * logp.sum())

    beta = -0.3
    out, cache = M.mlp_forward(params, M.ipap_forward(x, n, beta, sc))
    a, logp, _ = M.actor_head(out, eps)
    dout = M.actor_head_grad(out, eps, R, np.full(5, 0.3))
    _, dx = M.mlp_backward(params, cache, dout)
    g = M.ipap_beta_grad(dx, x, n, beta, sc)
    h = 1e-6
    fd = (loss(beta + h) - loss(beta - h)) / (2 * h)
    assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# FastSAC C51 pieces (Table 5: 101 atoms, [-20, 20])
# --------------------------------------------------------------------------
def _dist(rng, B, n):
    return M.softmax(rng.normal(0, 2, (B, n)))


def test_c51_projection_keeps_mass_and_identity():
    rng = np.random.default_rng(0)
    p = _dist(rng, 6, 101)
    m = M.c51_project(p, rng.normal(0, 3, 6), rng.uniform(0, 1, 6), -20, 20)
    np.testing.assert_allclose(m.sum(axis=1), 1.0, atol=1e-12)
    assert (m >= -1e-15).all()
    # shift 0, scale 1: every atom lands on itself
    np.testing.assert_allclose(M.c51_project(p, np.zeros(6), np.ones(6), -20, 20), p, atol=1e-12)


def test_c51_projection_moves_mass_by_whole_atoms():
    """A shift of exactly k atoms moves the distribution by k, clamped at the
    ends of the support (Bellemare et al. 2017, Algorithm 1)."""
    rng = np.random.default_rng(1)
    p = _dist(rng, 3, 101)
    m = M.c51_project(p, np.full(3, 2 * 0.4), np.ones(3), -20, 20)
    np.testing.assert_allclose(m[:, 2:100], p[:, 0:98], atol=1e-12)
    np.testing.assert_allclose(m[:, 100], p[:, 98:].sum(axis=1), atol=1e-12)
    assert np.abs(m[:, :2]).max() < 1e-15


def test_c51_projection_preserves_the_mean_inside_the_support():
    """Linear interpolation keeps the expectation: E_m[z] = shift + scale E_p[z]
    when no atom is clipped."""
    rng = np.random.default_rng(2)
    z = M.c51_support(101, -20, 20)
    p = np.zeros((5, 101))
    p[:, 30:70] = _dist(rng, 5, 40)
    shift, scale = rng.uniform(-3, 3, 5), rng.uniform(0.5, 1.0, 5)
    m = M.c51_project(p, shift, scale, -20, 20)
    np.testing.assert_allclose(m @ z, shift + scale * (p @ z), atol=1e-10)


def test_c51_targets_pick_the_lower_critic():
    rng = np.random.default_rng(3)
    n = 101
    l1, l2 = rng.normal(0, 1, (4, n)), rng.normal(0, 1, (4, n))
    l2[:2] += np.linspace(-3, 3, n)  # critic 2 higher on samples 0, 1
    l1[2:] += np.linspace(-3, 3, n)  # critic 1 higher on samples 2, 3
    m = M.c51_targets(np.zeros(4), np.zeros(4), l1, l2, np.zeros(4), 0.0, 1.0, 1.0, -20, 20)
    np.testing.assert_allclose(m[:2], M.softmax(l1[:2]), atol=1e-12)
    np.testing.assert_allclose(m[2:], M.softmax(l2[2:]), atol=1e-12)


def test_c51_critic_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    logits = rng.normal(0, 1, (3, 11))
    m = _dist(rng, 3, 11)
    _, g = M.c51_critic_loss(logits, m)
    fd = _fd(lambda: M.c51_critic_loss(logits, m)[0], logits)
    assert _rel(g, fd) < 1e-6


def test_c51_actor_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    l1, l2 = rng.normal(0, 1, (4, 11)), rng.normal(0, 1, (4, 11))
    logp = rng.normal(0, 1, 4)
    _, dlogp, d1, d2 = M.c51_actor_grads(logp, l1, l2, 0.3, -20, 20)
    f = lambda: M.c51_actor_grads(logp, l1, l2, 0.3, -20, 20)[0]
    assert _rel(d1, _fd(f, l1)) < 1e-6 and _rel(d2, _fd(f, l2)) < 1e-6
    assert _rel(dlogp, _fd(f, logp)) < 1e-6


# --------------------------------------------------------------------------
# Pins of the FastDSAC target and critic loss and of the C51 target that do
# not go through the oracle's own formulas: single transitions worked by
# hand (the arithmetic is in each docstring), limits with a closed form, and
# library routines (scipy's Huber loss and normal log-density).
# --------------------------------------------------------------------------
LN2 = math.log(2.0)


def test_fastdsac_target_single_transition_by_hand():
    """r = 1, not terminal, gamma 0.9, reward scale 0.4, alpha 0.2,
    logpi(a'|s') = -1.5, noise 0.5.  Target critic 1: mean 2, raw scale 0
    (sigma = softplus(0) + 0.1 = ln 2 + 0.1); critic 2: mean 3.  The smaller
    mean is critic 1's, so z = 2 + 0.5 (ln 2 + 0.1) = 2.3965735902799725;
    the entropy bonus -alpha logpi = +0.3 is added:
    y = 0.4 + 0.9 (z + 0.3) = 2.826916231251975,
    y_mean = 0.4 + 0.9 (2 + 0.3) = 2.47."""
    y, ym = M.critic_targets(np.array([1.0]), np.array([0.0]), np.array([[2.0, 0.0]]),
                             np.array([[3.0, 0.0]]), np.array([-1.5]), 0.2, np.array([0.5]),
                             0.9, 0.4)
    z = 2.0 + 0.5 * (LN2 + 0.1)
    assert y[0] == pytest.approx(0.4 + 0.9 * (z + 0.3), abs=1e-14)
    assert y[0] == pytest.approx(2.826916231251975, abs=1e-12)
    assert ym[0] == pytest.approx(2.47, abs=1e-14)


def test_fastdsac_target_takes_sigma_from_the_smaller_mean_critic():
    """Critic 1: mean 5, raw scale 3; critic 2: mean 1, raw scale -2.  The
    smaller mean is critic 2's, so the draw uses its sigma,
    ln(1 + e^-2) + 0.1 = 0.22692801104297263 (critic 1's would be
    ln(1 + e^3) + 0.1 = 3.148587351...): with noise 1, r = 0, no entropy
    (alpha 0), gamma 1, y = 1 + 0.22692801104297263."""
    y, ym = M.critic_targets(np.array([0.0]), np.array([0.0]), np.array([[5.0, 3.0]]),
                             np.array([[1.0, -2.0]]), np.array([0.0]), 0.0, np.array([1.0]),
                             1.0, 1.0)
    assert y[0] == pytest.approx(1.0 + math.log1p(math.exp(-2.0)) + 0.1, abs=1e-14)
    assert ym[0] == pytest.approx(1.0, abs=1e-15)


def test_fastdsac_target_terminal_and_entropy_sign():
    """A terminal transition's target is the scaled reward alone, whatever
    the critics, the noise and the entropy (the (1 - term) mask); a less
    random next action (larger logpi) lowers the target by gamma alpha per
    unit of logpi."""
    tq1, tq2 = np.array([[7.0, 1.0]]), np.array([[-4.0, 2.0]])
    y, ym = M.critic_targets(np.array([2.5]), np.array([1.0]), tq1, tq2, np.array([9.0]), 0.7,
                             np.array([2.0]), 0.99, 0.4)
    assert y[0] == 1.0 and ym[0] == 1.0
    ya, _ = M.critic_targets(np.array([0.0]), np.array([0.0]), tq1, tq2, np.array([1.0]), 0.5,
                             np.array([0.0]), 0.8, 1.0)
    yb, _ = M.critic_targets(np.array([0.0]), np.array([0.0]), tq1, tq2, np.array([3.0]), 0.5,
                             np.array([0.0]), 0.8, 1.0)
    assert yb[0] - ya[0] == pytest.approx(-0.8 * 0.5 * 2.0, abs=1e-12)


def test_fastdsac_target_noise_is_clipped_at_three_sigma():
    """Noise -7 is clipped to -3: z = m - 3 sigma (critic 2, mean -1, raw
    scale 0: z = -1 - 3 (ln 2 + 0.1))."""
    y, _ = M.critic_targets(np.array([0.0]), np.array([0.0]), np.array([[4.0, 0.0]]),
                            np.array([[-1.0, 0.0]]), np.array([0.0]), 0.0, np.array([-7.0]),
                            1.0, 1.0)
    assert y[0] == pytest.approx(-1.0 - 3.0 * (LN2 + 0.1), abs=1e-14)


def test_fastdsac_target_without_noise_is_the_clipped_double_q_td_target():
    """Limit sigma' draw -> 0 (noise 0): the sampled target equals the
    deterministic soft TD target with clipped double Q (Fujimoto et al.
    2018; Haarnoja et al. 2018), r_s r + gamma (1 - d) (min(Q1', Q2') -
    alpha logpi'), for every transition of a random batch."""
    rng = np.random.default_rng(11)
    B = 64
    rew, term = rng.normal(size=B), (rng.random(B) < 0.3).astype(float)
    tq1, tq2 = rng.normal(size=(B, 2)), rng.normal(size=(B, 2))
    lp = rng.normal(size=B)
    y, ym = M.critic_targets(rew, term, tq1, tq2, lp, 0.3, np.zeros(B), 0.97, 0.4)
    td = 0.4 * rew + 0.97 * (1.0 - term) * (np.minimum(tq1[:, 0], tq2[:, 0]) - 0.3 * lp)
    np.testing.assert_allclose(y, td, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ym, td, rtol=0, atol=1e-13)


def test_fastdsac_critic_loss_with_unit_weight_is_huber_plus_gaussian_nll():
    """With every sigma equal and sbar^2 = sigma^2 + 1e-6 the weight is 1,
    and the loss is the batch mean of scipy's Huber loss (delta 50) of
    m - y_mean plus the Gaussian negative log-density of y under (m, sigma)
    less its constant (1/2) log(2 pi)."""
    from scipy import special, stats
    rng = np.random.default_rng(12)
    B = 16
    q = np.stack([rng.normal(0, 80, B), np.full(B, 0.7)], axis=1)  # errors on both Huber branches
    y, ym = rng.normal(0, 60, B), rng.normal(0, 60, B)
    s = math.log1p(math.exp(0.7)) + 0.1
    loss, _ = M.critic_loss(q, y, ym, math.sqrt(s * s + 1e-6), delta=50.0)
    ref = (special.huber(50.0, q[:, 0] - ym) - stats.norm.logpdf(y, q[:, 0], s)
           - 0.5 * math.log(2 * math.pi)).mean()
    assert loss == pytest.approx(ref, rel=1e-12)


def test_fastdsac_critic_loss_weight_is_clipped_to_half_and_two():
    """Table 4's scale range: a tiny sbar gives weight 0.5, a huge one 2
    (the mean term only; the NLL term is unweighted)."""
    from scipy import special
    q = np.array([[3.0, 0.2], [-40.0, -1.0]])
    y = q[:, 0].copy()  # NLL term at its minimum over m (y - m = 0)
    ym = np.array([1.0, 100.0])
    s = np.log1p(np.exp(q[:, 1])) + 0.1
    nll = np.log(s)
    for sbar, w in ((1e-6, 0.5), (1e6, 2.0)):
        loss, _ = M.critic_loss(q, y, ym, sbar, delta=50.0)
        assert loss == pytest.approx((w * special.huber(50.0, q[:, 0] - ym) + nll).mean(), rel=1e-12)


def test_fastdsac_nll_term_gives_the_mean_no_gradient():
    """The NLL term uses a stop-gradient copy of the mean: with m = y_mean
    (Huber term flat) the mean's gradient is exactly zero although y != m."""
    q = np.array([[1.0, 0.3], [-2.0, 1.5]])
    _, dq = M.critic_loss(q, np.array([4.0, 7.0]), q[:, 0].copy(), 1.0)
    assert np.all(dq[:, 0] == 0.0)


def test_fastdsac_sigma_gradient_vanishes_at_the_maximum_likelihood_sigma():
    """The Gaussian NLL of one sample y under (m, sigma) is smallest at
    sigma = |y - m|: choose the raw scale so that softplus(q) + 0.1 = |y - m|
    (and m = y_mean); the gradient in q is then zero, and positive / negative
    for sigma above / below it."""
    m, y = 0.5, 2.5  # |y - m| = 2
    qr = math.log(math.expm1(2.0 - 0.1))  # softplus(qr) = 1.9
    for dq_raw, sign in ((0.0, 0), (0.3, 1), (-0.3, -1)):
        q = np.array([[m, qr + dq_raw]])
        _, dq = M.critic_loss(q, np.array([y]), np.array([m]), 1.0)
        if sign == 0:
            assert abs(dq[0, 1]) < 1e-12
        else:
            assert np.sign(dq[0, 1]) == sign


def _logits(p):
    return np.log(np.asarray(p, np.float64))[None, :]


def test_c51_target_single_transition_by_hand():
    """Three atoms on [-1, 1] (spacing 1).  Target critic 1: p = (0.2, 0.5,
    0.3), mean 0.1; critic 2: p = (0.1, 0.2, 0.7), mean 0.6: critic 1 is the
    smaller.  r = 0.5, r_s = 1, gamma 0.5, alpha 0.2, logpi' = 0.5:
    shift = 0.5 - 0.5 * 0.2 * 0.5 = 0.45, scale = 0.5, so the atoms move to
    (-0.05, 0.45, 0.95), i.e. positions b = (0.95, 1.45, 1.95):
    atom 0: 0.2 * 0.05 = 0.01 to 0, 0.2 * 0.95 = 0.19 to 1;
    atom 1: 0.5 * 0.55 = 0.275 to 1, 0.5 * 0.45 = 0.225 to 2;
    atom 2: 0.3 * 0.05 = 0.015 to 1, 0.3 * 0.95 = 0.285 to 2;
    target (0.01, 0.48, 0.51), whose mean 0.5 = 0.45 + 0.5 * 0.1."""
    m = M.c51_targets(np.array([0.5]), np.array([0.0]), _logits([0.2, 0.5, 0.3]),
                      _logits([0.1, 0.2, 0.7]), np.array([0.5]), 0.2, 0.5, 1.0, -1.0, 1.0)
    np.testing.assert_allclose(m[0], [0.01, 0.48, 0.51], rtol=0, atol=1e-14)
    # swapped critics: the same choice (critic 2's distribution is now the smaller)
    m2 = M.c51_targets(np.array([0.5]), np.array([0.0]), _logits([0.1, 0.2, 0.7]),
                       _logits([0.2, 0.5, 0.3]), np.array([0.5]), 0.2, 0.5, 1.0, -1.0, 1.0)
    np.testing.assert_allclose(m2[0], [0.01, 0.48, 0.51], rtol=0, atol=1e-14)


def test_c51_target_terminal_and_entropy_sign():
    """Terminal: every atom collapses onto r_s r = 0.5, half-way between
    atoms 1 and 2: (0, 0.5, 0.5).  Not terminal, no reward, gamma 1: the
    mean moves by -alpha logpi' (0.1 for logpi' = -0.5, alpha 0.2)."""
    m = M.c51_targets(np.array([0.5]), np.array([1.0]), _logits([0.2, 0.5, 0.3]),
                      _logits([0.1, 0.2, 0.7]), np.array([3.0]), 0.9, 0.5, 1.0, -1.0, 1.0)
    np.testing.assert_allclose(m[0], [0.0, 0.5, 0.5], rtol=0, atol=1e-14)
    z = np.array([-1.0, 0.0, 1.0])
    # no mass (1e-12) on the top atom, so the 0.1 shift clips nothing
    p = np.array([0.5 - 5e-13, 0.5 - 5e-13, 1e-12])
    m = M.c51_targets(np.array([0.0]), np.array([0.0]), _logits(p), _logits([1e-3, 1e-3, 0.998]),
                      np.array([-0.5]), 0.2, 1.0, 1.0, -1.0, 1.0)
    assert float(m[0] @ z) - float(p @ z) == pytest.approx(0.1, abs=1e-12)
