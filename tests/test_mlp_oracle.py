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
