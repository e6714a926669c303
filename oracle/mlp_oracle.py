"""FP64 reference of the learned parts: the policy / critic MLPs (Sec. 2.1:
MLPs with LeakyReLU), the tanh-squashed Gaussian actor, Adam, and the
FastDSAC update (Sec. 2.3, FastDSAC paragraph; Table 4).

TEST INFRASTRUCTURE ONLY: used by tests/ and the CPU-baseline leg of the
benchmark; it never imports the CUDA package.  Plain numpy in binary64; the
matrix product is the only library primitive.

The FastDSAC target and critic loss (critic_targets, critic_loss) and the
C51 target (c51_targets) are readings of the paper's prose (Sec. 2.3 gives
no equations for them).  Outside this file they are pinned by single
transitions worked by hand (entropy sign, terminal mask, the smaller-mean
critic and its own sigma, the 3-sigma clip, a three-atom projection), by
limits with a closed form (zero noise gives the clipped-double-Q soft TD
target; the NLL's sigma gradient vanishes at the maximum-likelihood sigma;
the NLL term gives the mean no gradient), and by scipy's Huber loss and
normal log-density for the unit-weight loss; their gradients are pinned by
finite differences.

Readings (the paper states FastDSAC only in prose):
* Eq. 2 (IPAPRec): one trainable beta shared by the agent's networks, moved
  by the actor loss only (the critics see the transformed input with beta
  held fixed), kept below a negative bound so that l - beta > 0;
* AdamW (Table 3): decoupled decay on weights and biases alike;
* hidden activation LeakyReLU with slope 0.01;
* actor head: mean u (2) and raw log-std r (2); log sigma = LS_MIN +
  (LS_MAX - LS_MIN) (tanh(r) + 1) / 2 with [LS_MIN, LS_MAX] = [-5, 0]
  (Table 4 log sigma range); action a = tanh(u + sigma eps);
* critic head: mean m and raw scale q; sigma_Q = softplus(q) + SIG_FLOOR;
* target: z ~ N(m', sigma_Q') of the target critic with the smaller mean
  (clipped double Q), clipped to m' +- 3 sigma_Q'; y = rs r + gamma (1 - term)
  (z - alpha logpi'), y_mean the same with m' in place of z;
* critic loss per critic: w Huber_delta(m - y_mean) + NLL(y | sg(m), sigma_Q)
  with w = clip(sg(sbar^2 / (sigma_Q^2 + 1e-6)), 0.5, 2.0) (Table 4 scale
  range) and sbar a running mean of the batch-mean sigma_Q (rate tau_b);
* actor loss: mean(alpha logpi - min_i m_i(s, a~)); temperature: log alpha
  descends mean(-log alpha (logpi + target_entropy)).
"""
from __future__ import annotations

import math

import numpy as np

SLOPE = 0.01
LS_MIN, LS_MAX = -5.0, 0.0
SIG_FLOOR = 0.1
LOG_2PI = math.log(2.0 * math.pi)


# ---------------------------------------------------------------------------
# MLP: x -> [W1 x + b1 -> leaky] -> [W2 . + b2 -> leaky] -> W3 . + b3
# weights W_l have shape [out, in] (y = x W^T + b)
# ---------------------------------------------------------------------------
def init_mlp(rng, sizes):
    """Kaiming-uniform style init: U(-1/sqrt(in), 1/sqrt(in)) for W and b."""
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / math.sqrt(fan_in)
        params.append([rng.uniform(-lim, lim, (fan_out, fan_in)), rng.uniform(-lim, lim, fan_out)])
    return params


def leaky(z):
    return np.where(z > 0, z, SLOPE * z)


def mlp_forward(params, x):
    """Returns the output and the cache of layer inputs and pre-activations."""
    cache = []
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = leaky(z) if li < len(params) - 1 else z
    return h, cache


def mlp_backward(params, cache, dout):
    """Gradients [dW, db] per layer and the gradient w.r.t. the input."""
    grads = [None] * len(params)
    g = dout
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        h, z = cache[li]
        if li < len(params) - 1:
            g = g * np.where(z > 0, 1.0, SLOPE)
        grads[li] = [g.T @ h, g.sum(axis=0)]
        g = g @ W
    return grads, g


# ---------------------------------------------------------------------------
# Adam (Kingma & Ba 2015, Algorithm 1), bias-corrected, no weight decay
# ---------------------------------------------------------------------------
def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.95, eps=1e-8):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def adamw_step(p, g, m, v, t, lr, b1=0.9, b2=0.95, wd=0.0, eps=1e-8):
    """AdamW (Loshchilov & Hutter 2019, decoupled decay; Table 3's optimiser):
    p <- p (1 - lr wd), then the Adam step of adam_step."""
    return adam_step(p * (1.0 - lr * wd), g, m, v, t, lr, b1, b2, eps)


# ---------------------------------------------------------------------------
# IPAPRec input transform (Eq. 2): l_hat = 1 / (l - beta), beta trainable
# ---------------------------------------------------------------------------
def ipap_forward(x, n, beta, scale=None):
    """Network input from observation rows x [B, D]: the first n features
    become 1 / (l - beta); then every feature is multiplied by scale."""
    out = np.array(x, np.float64, copy=True)
    out[:, :n] = 1.0 / (out[:, :n] - beta)
    if scale is not None:
        out = out * scale
    return out


def ipap_beta_grad(dx, x, n, beta, scale=None):
    """dL/dbeta from dL/d(input) dx [B, D]: d/dbeta of s / (l - beta) is
    s / (l - beta)^2."""
    s = np.ones(n) if scale is None else np.asarray(scale, np.float64)[:n]
    return float((dx[:, :n] * s / (x[:, :n] - beta) ** 2).sum())


# ---------------------------------------------------------------------------
# tanh-squashed Gaussian policy
# ---------------------------------------------------------------------------
def actor_head(out, eps):
    """out [B, 4] = (u0, u1, r0, r1); eps [B, 2] standard normal.
    Returns action a, log pi(a|s) and the intermediates."""
    u, r = out[:, :2], out[:, 2:4]
    ls = LS_MIN + (LS_MAX - LS_MIN) * 0.5 * (np.tanh(r) + 1.0)
    sig = np.exp(ls)
    pre = u + sig * eps
    a = np.tanh(pre)
    logp = (-0.5 * eps ** 2 - ls - 0.5 * LOG_2PI - np.log(1.0 - a ** 2 + 1e-6)).sum(axis=1)
    return a, logp, (u, r, ls, sig, pre)


def actor_head_grad(out, eps, da, dlogp):
    """Backward of actor_head: d(out) from dL/da [B,2] and dL/dlogp [B]."""
    u, r, ls, sig, pre = actor_head(out, eps)[2]
    a = np.tanh(pre)
    dpre_a = 1.0 - a ** 2
    # logp = sum(-eps^2/2 - ls - c - log(1 - tanh(pre)^2 + 1e-6)), eps fixed
    dlog_dpre = 2.0 * a * (1.0 - a ** 2) / (1.0 - a ** 2 + 1e-6)
    dpre = da * dpre_a + dlogp[:, None] * dlog_dpre
    du = dpre
    dls = dpre * sig * eps - dlogp[:, None]
    dr = dls * (LS_MAX - LS_MIN) * 0.5 * (1.0 - np.tanh(r) ** 2)
    return np.concatenate([du, dr], axis=1)


def softplus(x):
    return np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def huber(x, delta):
    ax = np.abs(x)
    return np.where(ax <= delta, 0.5 * x * x, delta * (ax - 0.5 * delta))


def huber_grad(x, delta):
    return np.clip(x, -delta, delta)


# ---------------------------------------------------------------------------
# FastDSAC update pieces
# ---------------------------------------------------------------------------
def critic_targets(rew, term, tq1, tq2, logp_next, alpha, znoise, gamma, rscale):
    """tq_i [B, 2] target-critic heads (mean, raw scale); znoise [B] ~ N(0,1).
    Returns the sampled target y and the mean target y_mean."""
    m1, s1 = tq1[:, 0], softplus(tq1[:, 1]) + SIG_FLOOR
    m2, s2 = tq2[:, 0], softplus(tq2[:, 1]) + SIG_FLOOR
    pick1 = m1 <= m2
    m = np.where(pick1, m1, m2)
    s = np.where(pick1, s1, s2)
    z = m + s * np.clip(znoise, -3.0, 3.0)
    cont = gamma * (1.0 - term)
    y = rscale * rew + cont * (z - alpha * logp_next)
    y_mean = rscale * rew + cont * (m - alpha * logp_next)
    return y, y_mean


def critic_loss(q, y, y_mean, sbar, delta=50.0, m_sg=None):
    """q [B, 2] (mean, raw scale).  Returns the batch-mean loss and dL/dq.
    m_sg: the stop-gradient copy of the mean used by the NLL term (defaults
    to the value of q[:, 0]; pass a fixed copy to differentiate numerically)."""
    B = q.shape[0]
    m, qr = q[:, 0], q[:, 1]
    m_sg = m.copy() if m_sg is None else m_sg
    s = softplus(qr) + SIG_FLOOR
    w = np.clip(sbar ** 2 / (s ** 2 + 1e-6), 0.5, 2.0)  # treated as a constant
    e = m - y_mean
    loss_mean = w * huber(e, delta)
    # Gaussian NLL of y under (sg(m), s): log s + (y - m)^2 / (2 s^2)
    d2 = (y - m_sg) ** 2
    loss_std = np.log(s) + d2 / (2.0 * s * s)
    loss = (loss_mean + loss_std).mean()
    dm = w * huber_grad(e, delta) / B
    ds = (1.0 / s - d2 / s ** 3) / B
    dq = np.stack([dm, ds * sigmoid(qr)], axis=1)
    return loss, dq


def actor_loss_grads(logp, q1_mean, q2_mean, alpha):
    """L = mean(alpha logp - min(q1, q2)); returns L, dL/dlogp, dL/dq1, dL/dq2."""
    B = logp.shape[0]
    pick1 = q1_mean <= q2_mean
    qmin = np.where(pick1, q1_mean, q2_mean)
    loss = (alpha * logp - qmin).mean()
    dlogp = np.full(B, alpha / B)
    dq1 = np.where(pick1, -1.0 / B, 0.0)
    dq2 = np.where(pick1, 0.0, -1.0 / B)
    return loss, dlogp, dq1, dq2


def alpha_grad(log_alpha, logp, target_entropy):
    """d/dlog_alpha of mean(-log_alpha (logp + target_entropy))."""
    return -(logp + target_entropy).mean()


def soft_update(target, online, tau):
    return (1.0 - tau) * target + tau * online


# ---------------------------------------------------------------------------
# FastSAC with categorical (C51) critics (Sec. 2.3 FastSAC paragraph; Table 5:
# 101 atoms on [-20, 20]).  Readings: each critic outputs one logit per atom;
# the target takes, per sample, the target critic whose expected value is
# smaller (clipped double Q); soft target atoms rs r + gamma (1 - term)
# (z_j - alpha logpi') are clipped to [v_min, v_max] and projected onto the
# fixed support by linear interpolation (Bellemare et al. 2017, Algorithm 1);
# both critics minimise the cross-entropy to that target; the actor minimises
# mean(alpha logpi - min_j E[Q_j]).
# ---------------------------------------------------------------------------
def c51_support(n_atoms, v_min, v_max):
    return np.linspace(v_min, v_max, n_atoms)


def softmax(x):
    e = np.exp(x - x.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def c51_project(p, shift, scale, v_min, v_max):
    """Projection of the distribution p [B, n] on the support z, moved to
    shift + scale z (per sample), onto the same support."""
    B, n = p.shape
    z = c51_support(n, v_min, v_max)
    dz = (v_max - v_min) / (n - 1)
    tz = np.clip(shift[:, None] + scale[:, None] * z[None, :], v_min, v_max)
    b = (tz - v_min) / dz
    lo = np.floor(b).astype(np.int64)
    hi = np.ceil(b).astype(np.int64)
    m = np.zeros_like(p)
    for i in range(B):
        for j in range(n):
            if lo[i, j] == hi[i, j]:
                m[i, lo[i, j]] += p[i, j]
            else:
                m[i, lo[i, j]] += p[i, j] * (hi[i, j] - b[i, j])
                m[i, hi[i, j]] += p[i, j] * (b[i, j] - lo[i, j])
    return m


def c51_targets(rew, term, tl1, tl2, logp_next, alpha, gamma, rscale, v_min, v_max):
    """Target distribution from the two target critics' logits [B, n]."""
    n = tl1.shape[1]
    z = c51_support(n, v_min, v_max)
    p1, p2 = softmax(tl1), softmax(tl2)
    pick1 = (p1 @ z) <= (p2 @ z)
    p = np.where(pick1[:, None], p1, p2)
    cont = gamma * (1.0 - term)
    shift = rscale * rew - cont * alpha * logp_next
    return c51_project(p, shift, cont, v_min, v_max)


def c51_critic_loss(logits, m):
    """Mean cross-entropy -sum_i m_i log softmax(logits)_i and its gradient."""
    B = logits.shape[0]
    lse = np.log(np.exp(logits - logits.max(axis=1, keepdims=True)).sum(axis=1)) + logits.max(axis=1)
    logp = logits - lse[:, None]
    loss = -(m * logp).sum(axis=1).mean()
    return loss, (softmax(logits) - m) / B


def c51_actor_grads(logp, l1, l2, alpha, v_min, v_max):
    """L = mean(alpha logp - min_j E[Q_j]) with E[Q_j] = softmax(l_j) . z:
    returns L, dL/dlogp and dL/dl_j (the logits of both critics)."""
    B, n = l1.shape
    z = c51_support(n, v_min, v_max)
    p1, p2 = softmax(l1), softmax(l2)
    q1, q2 = p1 @ z, p2 @ z
    pick1 = q1 <= q2
    loss = (alpha * logp - np.where(pick1, q1, q2)).mean()
    dq1 = -(p1 * (z[None, :] - q1[:, None])) / B
    dq2 = -(p2 * (z[None, :] - q2[:, None])) / B
    dl1 = np.where(pick1[:, None], dq1, 0.0)
    dl2 = np.where(pick1[:, None], 0.0, dq2)
    return loss, np.full(B, alpha / B), dl1, dl2
