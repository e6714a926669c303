// FastDSAC learner on the GPU (Sec. 2.3, FastDSAC paragraph; Table 4) and the
// evaluation reductions.  Readings of the update (the paper states it in prose):
//  critic i outputs (mean m_i, raw scale q_i), sigma_i = softplus(q_i) + 0.1;
//  target: z ~ N(m', sigma') of the target critic with the smaller mean
//  (clipped double Q), the normal draw clipped to +-3;
//  y = rs r + gamma (1 - term) (z - alpha logpi(a'|s')), y_mean with m';
//  critic loss w Huber_delta(m - y_mean) + log sigma + (y - sg(m))^2/(2 sigma^2),
//  w = clip(sbar^2 / (sigma^2 + 1e-6), 0.5, 2) constant, sbar a running mean
//  (rate tau_b) of the batch-mean sigma;
//  actor loss mean(alpha logpi(a~|s) - min_i m_i(s, a~)), every policy_freq
//  critic updates; log alpha by Adam on mean(-log alpha (logpi + H_target));
//  target critics by Polyak averaging with rate tau.
// All GEMMs run on the tcgen05 kernel (BF16 operands, FP32 accumulation);
// master weights, Adam moments and every reduction are FP32, the evaluation
// success count and return sums FP64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "nav_internal.h"
#include "pdl.cuh"
#include "nav_policy.h"

namespace flashnav {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ unsigned long long hmix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float softplusf(float x) {
    return log1pf(expf(-fabsf(x))) + fmaxf(x, 0.0f);
}

// ---------------------------------------------------------------- replay ---
// Device counters of a trainer (read by the kernels, so that a captured
// update graph replays correctly): [0] critic updates, [1] actor updates,
// [2] replay head, [3] replay size.  corr holds Adam's bias corrections
// (1 - b1^t, 1 - b2^t) of the current critic [0..1] and actor [2..3] step.
enum { kCtrCritic = 0, kCtrActor = 1, kCtrHead = 2, kCtrSize = 3, kCtrSnapHead = 4,
       kCtrSnapSize = 5, kCtrPending = 6 };

// Starts critic (which 0) or actor (which 1) step t = ++ctr[which]; the
// step's kernels use t - 1 as their update index.
__global__ void k_count(unsigned long long *ctr, int which, float b1, float b2, float *corr) {
    pdl_enter();
    const unsigned long long t = ++ctr[which];
    corr[2 * which] = 1.0f - powf(b1, (float)t);
    corr[2 * which + 1] = 1.0f - powf(b2, (float)t);
}

// k_count for the critic step and, in an actor step, for the actor step
// too, whose loss accumulators acc[0..1] it also clears: the first launch of
// a fused update
__global__ void k_count_start(unsigned long long *ctr, int actor, float b1, float b2, float *corr,
                              float *acc) {
    pdl_enter();
    const unsigned long long t = ++ctr[kCtrCritic];
    corr[0] = 1.0f - powf(b1, (float)t);
    corr[1] = 1.0f - powf(b2, (float)t);
    if (actor) {
        const unsigned long long ta = ++ctr[kCtrActor];
        corr[2] = 1.0f - powf(b1, (float)ta);
        corr[3] = 1.0f - powf(b2, (float)ta);
        acc[0] = 0.0f;
        acc[1] = 0.0f;
    }
}

__global__ void k_insert_done(unsigned long long *ctr, int n, long long cap) {
    ctr[kCtrHead] = (ctr[kCtrHead] + (unsigned long long)n) % (unsigned long long)cap;
    const unsigned long long s = ctr[kCtrSize] + (unsigned long long)n;
    ctr[kCtrSize] = s < (unsigned long long)cap ? s : (unsigned long long)cap;
}

__global__ void k_replay_insert(const float *__restrict__ obs, const float *__restrict__ act,
                                const float *__restrict__ rew, const unsigned char *__restrict__ done,
                                const float *__restrict__ obs_next,
                                const float *__restrict__ final_obs, int E, int od, int ld,
                                const unsigned long long *__restrict__ ctr, long long cap,
                                const float *__restrict__ scale, int ipap, bf16 *r_obs,
                                bf16 *r_next, float *r_act, float *r_rew, float *r_term) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)E * ld) return;
    const int e = (int)(i / ld), c = (int)(i - (long long)e * ld);
    const long long slot = (long long)((ctr[kCtrHead] + (unsigned long long)e) % (unsigned long long)cap);
    const bool ended = (done[e] & 3) != 0;
    const float *nxt = (ended && final_obs) ? final_obs : obs_next;
    // features under Eq. 2 are stored raw (beta changes while they sit in the
    // replay); the transform and their scale are applied when a batch is drawn
    const float sc = (scale && c < od && c >= ipap) ? scale[c] : 1.0f;
    r_obs[slot * ld + c] = __float2bfloat16_rn(c < od ? obs[(long long)e * od + c] * sc : 0.0f);
    r_next[slot * ld + c] = __float2bfloat16_rn(c < od ? nxt[(long long)e * od + c] * sc : 0.0f);
    if (c == 0) {
        r_act[slot * 2] = act[2 * e];
        r_act[slot * 2 + 1] = act[2 * e + 1];
        r_rew[slot] = rew[e];
        r_term[slot] = (done[e] & 1) ? 1.0f : 0.0f; // truncation still bootstraps
    }
}

// Uniform replay indices.  While a collector inserts E = ctr[pending]
// transitions concurrently (overlapped pipeline), the draw uses the (head,
// size) snapshot taken before the insert began and skips the E slots it
// writes: with s + E <= cap those lie beyond the s valid ones; otherwise the
// n = cap - E safe slots start right after them.
__device__ __forceinline__ int sample_index(int b, const unsigned long long *__restrict__ ctr,
                                            unsigned long long seed, long long cap) {
    const unsigned long long update = ctr[kCtrCritic] - 1, E = ctr[kCtrPending];
    const unsigned long long s = E ? ctr[kCtrSnapSize] : ctr[kCtrSize];
    const unsigned long long hd = E ? ctr[kCtrSnapHead] : ctr[kCtrHead];
    const unsigned long long C = (unsigned long long)cap;
    const bool wrap = s + E > C;
    const unsigned long long n = wrap ? C - E : s;
    const unsigned long long h = hmix(seed ^ (update * 0xD6E8FEB86659FD93ull) ^ ((unsigned long long)b << 1));
    const unsigned long long r = ((h >> 32) * n) >> 32;
    return (int)(wrap ? (hd + E + r) % C : r);
}

__global__ void k_sample(int *idx, int B, const unsigned long long *__restrict__ ctr,
                         unsigned long long seed, long long cap) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    idx[b] = sample_index(b, ctr, seed, cap);
}

// overlapped pipeline: snapshot (head, size) and the pending insert count
__global__ void k_overlap(unsigned long long *ctr, unsigned long long pending) {
    ctr[kCtrSnapHead] = ctr[kCtrHead];
    ctr[kCtrSnapSize] = ctr[kCtrSize];
    ctr[kCtrPending] = pending;
}

// Eq. 2 on a stored raw range: s / (l - beta), rounded to BF16
__device__ __forceinline__ bf16 ipap_in(bf16 l, float beta, const float *scale, int c) {
    const float x = 1.0f / (__bfloat162float(l) - beta);
    return __float2bfloat16_rn(scale ? x * scale[c] : x);
}

// batch rows: Xo = obs, Xn = next obs (BF16 [B][ld]); Xc = [obs, act] ([B][ldc]);
// the first ipap features go through Eq. 2 with the current beta, and their
// raw ranges of obs are kept in Lraw [B][ipap] for the gradient of beta
__global__ void k_gather(const int *__restrict__ idx, const bf16 *__restrict__ r_obs,
                         const bf16 *__restrict__ r_next, const float *__restrict__ r_act,
                         const float *__restrict__ r_rew, const float *__restrict__ r_term, int B,
                         int od, int ld, int ldc, int ipap, const float *__restrict__ beta_dev,
                         const float *__restrict__ scale, bf16 *Xo, bf16 *Xn, bf16 *Xc,
                         float *Lraw, float *rew, float *term) {
    pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * ldc) return;
    const int b = (int)(i / ldc), c = (int)(i - (long long)b * ldc);
    const long long s = idx[b];
    const float beta = ipap > 0 ? *beta_dev : 0.0f;
    bf16 xo = __float2bfloat16_rn(0.0f);
    if (c < ld) {
        xo = r_obs[s * ld + c];
        bf16 xn = r_next[s * ld + c];
        if (c < ipap) {
            Lraw[(long long)b * ipap + c] = __bfloat162float(xo);
            xo = ipap_in(xo, beta, scale, c);
            xn = ipap_in(xn, beta, scale, c);
        }
        Xo[(long long)b * ld + c] = xo;
        Xn[(long long)b * ld + c] = xn;
    }
    bf16 v = __float2bfloat16_rn(0.0f);
    if (c < od) v = xo;
    else if (c < od + 2) v = __float2bfloat16_rn(r_act[s * 2 + (c - od)]);
    Xc[(long long)b * ldc + c] = v;
    if (c == 0) {
        rew[b] = r_rew[s];
        term[b] = r_term[s];
    }
}

// One launch for the fused update: the replay index of each row (as
// k_sample, also stored in idx), the rows of k_gather, and the layouts the update reads later:
// Xc transposed (XcT [od + 2][B]), Xo's first od columns transposed (XoT
// [od][B]), and the observation columns (with the zero padding) of Xnc =
// [Xn, a'] and Xa = [Xo, a], whose action columns the actor head writes.
__global__ void k_gather_all(const bf16 *__restrict__ r_obs, const bf16 *__restrict__ r_next,
                             const float *__restrict__ r_act, const float *__restrict__ r_rew,
                             const float *__restrict__ r_term, int B, int od, int ld, int ldc,
                             int ipap, const float *__restrict__ beta_dev,
                             const float *__restrict__ scale, const unsigned long long *ctr,
                             unsigned long long seed, long long cap, int *idx, bf16 *Xo, bf16 *Xn,
                             bf16 *Xc, bf16 *XcT, bf16 *XoT, bf16 *Xnc, bf16 *Xa, float *Lraw,
                             float *rew, float *term) {
    pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * ldc) return;
    const int b = (int)(i / ldc), c = (int)(i - (long long)b * ldc);
    const long long s = sample_index(b, ctr, seed, cap);
    const float beta = ipap > 0 ? *beta_dev : 0.0f;
    const bf16 zero = __float2bfloat16_rn(0.0f);
    bf16 xo = zero, xn = zero;
    if (c < ld) {
        xo = r_obs[s * ld + c];
        xn = r_next[s * ld + c];
        if (c < ipap) {
            Lraw[(long long)b * ipap + c] = __bfloat162float(xo);
            xo = ipap_in(xo, beta, scale, c);
            xn = ipap_in(xn, beta, scale, c);
        }
        Xo[(long long)b * ld + c] = xo;
        Xn[(long long)b * ld + c] = xn;
    }
    bf16 v = zero;
    if (c < od) v = xo;
    else if (c < od + 2) v = __float2bfloat16_rn(r_act[s * 2 + (c - od)]);
    Xc[(long long)b * ldc + c] = v;
    if (c < od + 2) XcT[(long long)c * B + b] = v;
    if (c < od) XoT[(long long)c * B + b] = xo;
    if (c < od || c >= od + 2) {
        Xnc[(long long)b * ldc + c] = c < od ? xn : zero;
        Xa[(long long)b * ldc + c] = c < od ? xo : zero;
    }
    if (c == 0) {
        idx[b] = (int)s;
        rew[b] = r_rew[s];
        term[b] = r_term[s];
    }
}

// Xc = [Xo[:, :od], a] for the actor's own action
__global__ void k_concat(const bf16 *__restrict__ Xo, int ld, const float *__restrict__ a, int B,
                         int od, int ldc, bf16 *Xc) {
    pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * ldc) return;
    const int b = (int)(i / ldc), c = (int)(i - (long long)b * ldc);
    bf16 v = __float2bfloat16_rn(0.0f);
    if (c < od) v = Xo[(long long)b * ld + c];
    else if (c < od + 2) v = __float2bfloat16_rn(a[2 * b + (c - od)]);
    Xc[(long long)b * ldc + c] = v;
}

// out[c][r] = in[r][c] for r < rows, c < cols (32 x 32 tiles through smem)
__global__ void k_transpose(const bf16 *__restrict__ in, int ld_in, int rows, int cols, bf16 *out,
                            int ld_out) {
    pdl_enter();
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[j][threadIdx.x] = in[(long long)r * ld_in + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(long long)c * ld_out + r] = t[threadIdx.x][j];
    }
}

// ----------------------------------------------------------------- heads ---
// Distributional target of sample b (Sec. 2.3 FastDSAC): the smaller-mean
// target critic's Gaussian, sampled with clipped counter-hash noise, minus
// the entropy term; ym uses the mean instead of the sample.
__device__ __forceinline__ void target_row(const float *__restrict__ rew,
                                           const float *__restrict__ term,
                                           const float *__restrict__ tq1,
                                           const float *__restrict__ tq2,
                                           const float *__restrict__ logp_next, float alpha, int b,
                                           float gamma, float rs, unsigned long long seed,
                                           unsigned long long update, float &y, float &ym,
                                           float &zn) {
    const float m1 = tq1[2 * b], s1 = softplusf(tq1[2 * b + 1]) + 0.1f;
    const float m2 = tq2[2 * b], s2 = softplusf(tq2[2 * b + 1]) + 0.1f;
    const bool p1 = m1 <= m2;
    const float m = p1 ? m1 : m2, s = p1 ? s1 : s2;
    const unsigned long long h = hmix(seed ^ (update * 0x8CB92BA72F3D8DD7ull) ^ ((unsigned long long)b << 20) ^ 0xA11CEull);
    const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (float)((h >> 8) & 0xFFFFFFull) * (1.0f / 16777216.0f);
    zn = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    const float z = m + s * fminf(fmaxf(zn, -3.0f), 3.0f);
    const float cont = gamma * (1.0f - term[b]);
    y = rs * rew[b] + cont * (z - alpha * logp_next[b]);
    ym = rs * rew[b] + cont * (m - alpha * logp_next[b]);
}

__global__ void k_targets(const float *__restrict__ rew, const float *__restrict__ term,
                          const float *__restrict__ tq1, const float *__restrict__ tq2,
                          const float *__restrict__ logp_next, const float *__restrict__ log_alpha,
                          int B, float gamma, float rs, unsigned long long seed,
                          const unsigned long long *__restrict__ ctr, float *y, float *ym,
                          float *znoise) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float yb, ymb, zn;
    target_row(rew, term, tq1, tq2, logp_next, expf(*log_alpha), b, gamma, rs, seed,
               ctr[kCtrCritic] - 1, yb, ymb, zn);
    y[b] = yb;
    ym[b] = ymb;
    if (znoise) znoise[b] = zn;
}

// dL/dq of one critic for sample b (written to dq); returns sigma and the
// sample's loss
__device__ __forceinline__ float2 critic_row(const float *__restrict__ q, float yb, float ymb,
                                             float sb, int B, float delta, int b, float *dq) {
    const float m = q[2 * b], qr = q[2 * b + 1];
    const float s = softplusf(qr) + 0.1f;
    const float w = fminf(fmaxf(sb * sb / (s * s + 1e-6f), 0.5f), 2.0f);
    const float e = m - ymb;
    const float ae = fabsf(e);
    const float hub = ae <= delta ? 0.5f * e * e : delta * (ae - 0.5f * delta);
    const float d2 = (yb - m) * (yb - m);
    const float ll = w * hub + logf(s) + d2 / (2.0f * s * s);
    const float inv = 1.0f / (float)B;
    dq[2 * b] = w * fminf(fmaxf(e, -delta), delta) * inv;
    const float sig = 1.0f / (1.0f + expf(-qr));
    dq[2 * b + 1] = (1.0f / s - d2 / (s * s * s)) * inv * sig;
    return make_float2(s, ll);
}

__device__ __forceinline__ void add_sigma_loss(float ss, float ll, float *acc) {
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        ll += __shfl_xor_sync(0xffffffffu, ll, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], ss);
        atomicAdd(&acc[1], ll);
    }
}

// dL/dq for one critic; accumulates the batch sum of sigma and the loss
__device__ __forceinline__ void critic_grad(const float *__restrict__ q, const float *__restrict__ y,
                                            const float *__restrict__ ym,
                                            const float *__restrict__ sbar, int B, float delta,
                                            float *dq, float *acc) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float2 r = make_float2(0.0f, 0.0f);
    if (b < B) r = critic_row(q, y[b], ym[b], *sbar, B, delta, b, dq);
    add_sigma_loss(r.x, r.y, acc);
}

__global__ void k_critic_grad(const float *__restrict__ q, const float *__restrict__ y,
                              const float *__restrict__ ym, const float *__restrict__ sbar, int B,
                              float delta, float *dq, float *acc /*[0] sum sigma, [1] loss*/) {
    pdl_enter();
    critic_grad(q, y, ym, sbar, B, delta, dq, acc);
}

__global__ void k_sbar_update(float *sbar, float *acc, int n, float tau_b) {
    pdl_enter();
    *sbar = (1.0f - tau_b) * (*sbar) + tau_b * (acc[0] / (float)n);
    acc[2] = acc[1];
    acc[0] = 0.0f;
    acc[1] = 0.0f;
}

// The targets, both critics' dL/dq and the running sigma of one update in
// one launch: each thread takes one sample through k_targets' and
// critic_grad's arithmetic (same values), and the last block to finish (a
// ticket counter, reset by that block) folds the batch sums into sbar as
// k_sbar_update does.
__global__ void k_targets_grad2(const float *__restrict__ rew, const float *__restrict__ term,
                                const float *__restrict__ tq1, const float *__restrict__ tq2,
                                const float *__restrict__ logp_next,
                                const float *__restrict__ log_alpha, int B, float gamma, float rs,
                                unsigned long long seed, const unsigned long long *__restrict__ ctr,
                                float *y, float *ym, float *znoise, const float *__restrict__ q0,
                                const float *__restrict__ q1, float *sbar, float delta, float *dq0,
                                float *dq1, float *acc, float tau_b, unsigned *ticket) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float ss = 0.0f, ll = 0.0f;
    if (b < B) {
        float yb, ymb, zn;
        target_row(rew, term, tq1, tq2, logp_next, expf(*log_alpha), b, gamma, rs, seed,
                   ctr[kCtrCritic] - 1, yb, ymb, zn);
        y[b] = yb;
        ym[b] = ymb;
        if (znoise) znoise[b] = zn;
        const float sb = *sbar;
        const float2 r0 = critic_row(q0, yb, ymb, sb, B, delta, b, dq0);
        const float2 r1 = critic_row(q1, yb, ymb, sb, B, delta, b, dq1);
        ss = r0.x + r1.x;
        ll = r0.y + r1.y;
    }
    add_sigma_loss(ss, ll, acc);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
            __threadfence();
            const float a0 = __ldcg(&acc[0]), a1 = __ldcg(&acc[1]);
            *sbar = (1.0f - tau_b) * (*sbar) + tau_b * (a0 / (float)(2 * B));
            acc[2] = a1;
            acc[0] = 0.0f;
            acc[1] = 0.0f;
            *ticket = 0u;
        }
    }
}

// actor loss mean(alpha logp - min(q1, q2)) -> dL/dlogp and dL/dq_i (mean column)
__global__ void k_actor_loss(const float *__restrict__ logp, const float *__restrict__ q1,
                             const float *__restrict__ q2, const float *__restrict__ log_alpha,
                             int B, float *dlogp, float *dq1, float *dq2, float *acc) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float ll = 0.0f, lp = 0.0f;
    if (b < B) {
        const float alpha = expf(*log_alpha);
        const bool p1 = q1[2 * b] <= q2[2 * b];
        const float inv = 1.0f / (float)B;
        dlogp[b] = alpha * inv;
        dq1[2 * b] = p1 ? -inv : 0.0f;
        dq2[2 * b] = p1 ? 0.0f : -inv;
        dq1[2 * b + 1] = 0.0f;
        dq2[2 * b + 1] = 0.0f;
        ll = alpha * logp[b] - (p1 ? q1[2 * b] : q2[2 * b]);
        lp = logp[b];
    }
    for (int o = 16; o > 0; o >>= 1) {
        ll += __shfl_xor_sync(0xffffffffu, ll, o);
        lp += __shfl_xor_sync(0xffffffffu, lp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], ll);
        atomicAdd(&acc[1], lp);
    }
}

// backward of the squashed-Gaussian head: d out4 from dL/da and dL/dlogp
__global__ void k_actor_head_bwd(const float *__restrict__ out4, const float *__restrict__ eps,
                                 const float *__restrict__ dX1, const float *__restrict__ dX2,
                                 int ldx, int od, const float *__restrict__ dlogp, int B,
                                 float *dout) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const float u = out4[4 * b + d], r = out4[4 * b + 2 + d];
        const float tr = tanhf(r);
        const float ls = kLogStdMin + (kLogStdMax - kLogStdMin) * 0.5f * (tr + 1.0f);
        const float sg = expf(ls);
        const float e = eps[2 * b + d];
        const float a = tanhf(u + sg * e);
        const float da = dX1[(long long)b * ldx + od + d] + dX2[(long long)b * ldx + od + d];
        const float om = 1.0f - a * a;
        const float dpre = da * om + dlogp[b] * (2.0f * a * om / (om + 1e-6f));
        const float dls = dpre * sg * e - dlogp[b];
        dout[4 * b + d] = dpre;
        dout[4 * b + 2 + d] = dls * (kLogStdMax - kLogStdMin) * 0.5f * (1.0f - tr * tr);
    }
}

// ------------------------------------------------------------- backward ---
// FP32 [B][n] -> BF16 [B][ldp] (zero pad) and its transpose [n][B]
__global__ void k_grad_to_bf16(const float *__restrict__ g, int B, int n, int ldp, bf16 *g16,
                               bf16 *gT16) {
    pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * ldp) return;
    const int b = (int)(i / ldp), c = (int)(i - (long long)b * ldp);
    const bf16 v = __float2bfloat16_rn(c < n ? g[(long long)b * n + c] : 0.0f);
    g16[i] = v;
    if (c < n) gT16[(long long)c * B + b] = v;
}

// dZ = dH * leaky'(z) with the sign of z read from the activation h = leaky(z);
// writes dZ in place (FP32 [B][H]), as BF16 [B][ldh] and as BF16 [H][B]
// (32 x 32 tiles); h is BF16 [B][ldh]
__global__ void k_leaky_bwd(float *dH, const bf16 *__restrict__ h, int B, int H, int ldh,
                            bf16 *dZ16, bf16 *dZT16) {
    pdl_enter();
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < B && c < H) {
            const long long o = (long long)r * H + c, oh = (long long)r * ldh + c;
            const float d = dH[o] * (__bfloat162float(h[oh]) > 0.0f ? 1.0f : 0.01f);
            dH[o] = d;
            const bf16 v = __float2bfloat16_rn(d);
            dZ16[oh] = v;
            t[j][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (r < B && c < H) dZT16[(long long)c * B + r] = t[threadIdx.x][j];
    }
}

// column sums of FP32 [B][n] (bias gradients)
__global__ void k_colsum(const float *__restrict__ g, int B, int n, float *out) {
    pdl_enter();
    __shared__ float part[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (c < n)
        for (int r = threadIdx.y; r < B; r += 8) s += g[(long long)r * n + c];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < n) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
        out[c] = t;
    }
}

// ----------------------------------------------------------- optimiser ---
// log alpha <- Adam step on mean(-log alpha (logp + H_target)); acc[1] = sum logp
__global__ void k_alpha(float *log_alpha, float *am, float *av, const float *acc, int B,
                        float target_entropy, float lr, float b1, float b2,
                        const float *__restrict__ corr) {
    pdl_enter();
    const float c1 = corr[0], c2 = corr[1];
    const float g = -(acc[1] / (float)B + target_entropy);
    const float mi = b1 * (*am) + (1.0f - b1) * g;
    const float vi = b2 * (*av) + (1.0f - b2) * g * g;
    *am = mi;
    *av = vi;
    *log_alpha -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// The actor step's last launch: Eq. 2's beta Adam step (when beta_s is not
// null, as k_beta_adam) and the alpha Adam step (as k_alpha), one thread.
__global__ void k_alpha_beta(float *log_alpha, float *am, float *av, const float *acc, int B,
                             float target_entropy, float lr, float b1, float b2,
                             const float *__restrict__ corr, float *beta_s, float beta_lr,
                             float beta_max) {
    pdl_enter();
    const float c1 = corr[0], c2 = corr[1];
    if (beta_s) {
        const float g = beta_s[3];
        beta_s[-1] = g;
        const float mi = b1 * beta_s[1] + (1.0f - b1) * g;
        const float vi = b2 * beta_s[2] + (1.0f - b2) * g * g;
        beta_s[1] = mi;
        beta_s[2] = vi;
        beta_s[0] = fminf(beta_s[0] - beta_lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f), beta_max);
        beta_s[3] = 0.0f;
    }
    const float g = -(acc[1] / (float)B + target_entropy);
    const float mi = b1 * (*am) + (1.0f - b1) * g;
    const float vi = b2 * (*av) + (1.0f - b2) * g * g;
    *am = mi;
    *av = vi;
    *log_alpha -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// ------------------------------------------------------- FastSAC (C51) ---
// One warp per sample (8 per 256-thread block); lane i holds atoms i, i + 32,
// ...; atoms z_i = v_min + i dz.
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// softmax statistics of one logit row: max, sum of exp, expected atom value
__device__ __forceinline__ void c51_stats(const float *l, int n, float v_min, float dz, int lane,
                                          float &mx, float &sum, float &mean) {
    float m = -INFINITY;
    for (int i = lane; i < n; i += 32) m = fmaxf(m, l[i]);
    mx = warp_max(m);
    float s = 0.0f, zs = 0.0f;
    for (int i = lane; i < n; i += 32) {
        const float e = expf(l[i] - mx);
        s += e;
        zs += e * (v_min + (float)i * dz);
    }
    sum = warp_sum(s);
    mean = warp_sum(zs) / sum;
}

// Cross-entropy of sample b's logits to the target row mr (one warp):
// dL/dlogits = (softmax - m) / B; acc[1] += loss
__device__ __forceinline__ void c51_ce_row(const float *__restrict__ q, const float *mr, int b,
                                           int B, int n, float *dq, float *acc) {
    const int lane = threadIdx.x & 31;
    const float *l = q + (size_t)b * n;
    float mv = -INFINITY;
    for (int i = lane; i < n; i += 32) mv = fmaxf(mv, l[i]);
    const float mx = warp_max(mv);
    float s = 0.0f;
    for (int i = lane; i < n; i += 32) s += expf(l[i] - mx);
    const float sum = warp_sum(s);
    const float lse = mx + logf(sum), inv = 1.0f / sum, ib = 1.0f / (float)B;
    float ll = 0.0f;
    for (int i = lane; i < n; i += 32) {
        ll -= mr[i] * (l[i] - lse);
        dq[(size_t)b * n + i] = (expf(l[i] - mx) * inv - mr[i]) * ib;
    }
    ll = warp_sum(ll);
    if (lane == 0) atomicAdd(&acc[1], ll);
}

// Target distribution m [B][n]: the target critic with the smaller expected
// value, atoms moved to rs r + gamma (1 - term) (z - alpha logpi') and
// clipped, projected back by linear interpolation (shared-memory bins).
// With qc0 (and qc1, dq0, dq1, acc), the same warp then forms both
// critics' cross-entropy gradients from the row it holds.
__global__ void __launch_bounds__(256) k_c51_targets(
    const float *__restrict__ rew, const float *__restrict__ term, const float *__restrict__ tl1,
    const float *__restrict__ tl2, const float *__restrict__ logp_next,
    const float *__restrict__ log_alpha, int B, int n, float gamma, float rs, float v_min,
    float v_max, float *m, const float *__restrict__ qc0, const float *__restrict__ qc1,
    float *dq0, float *dq1, float *acc) {
    pdl_enter();
    __shared__ float bins[8][kFusedMaxWidth];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + w;
    if (b >= B) return; // whole warp
    const float dz = (v_max - v_min) / (float)(n - 1);
    const float *l1 = tl1 + (size_t)b * n, *l2 = tl2 + (size_t)b * n;
    float mx1, s1, q1, mx2, s2, q2;
    c51_stats(l1, n, v_min, dz, lane, mx1, s1, q1);
    c51_stats(l2, n, v_min, dz, lane, mx2, s2, q2);
    const bool p1 = q1 <= q2;
    const float *l = p1 ? l1 : l2;
    const float mx = p1 ? mx1 : mx2, inv = 1.0f / (p1 ? s1 : s2);
    const float cont = gamma * (1.0f - term[b]);
    const float shift = rs * rew[b] - cont * expf(*log_alpha) * logp_next[b];
    for (int i = lane; i < n; i += 32) bins[w][i] = 0.0f;
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
        const float pj = expf(l[j] - mx) * inv;
        const float tz = fminf(fmaxf(shift + cont * (v_min + (float)j * dz), v_min), v_max);
        const float bj = (tz - v_min) / dz;
        const int lo = (int)floorf(bj), hi = (int)ceilf(bj);
        if (lo == hi) {
            atomicAdd(&bins[w][lo], pj);
        } else {
            atomicAdd(&bins[w][lo], pj * ((float)hi - bj));
            atomicAdd(&bins[w][hi], pj * (bj - (float)lo));
        }
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) m[(size_t)b * n + i] = bins[w][i];
    // both critics' cross-entropy gradients against this target row
    if (qc0) {
        c51_ce_row(qc0, bins[w], b, B, n, dq0, acc);
        c51_ce_row(qc1, bins[w], b, B, n, dq1, acc);
    }
}

// Actor loss mean(alpha logp - min_j E[Q_j]): dL/dlogp, and dL/dlogits of the
// smaller critic, -p_i (z_i - E[Q]) / B (zero for the other)
__global__ void __launch_bounds__(256) k_c51_actor_loss(
    const float *__restrict__ logp, const float *__restrict__ l1, const float *__restrict__ l2,
    const float *__restrict__ log_alpha, int B, int n, float v_min, float v_max, float *dlogp,
    float *dq1, float *dq2, float *acc) {
    pdl_enter();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + w;
    if (b >= B) return;
    const float dz = (v_max - v_min) / (float)(n - 1), ib = 1.0f / (float)B;
    const float *a = l1 + (size_t)b * n, *c = l2 + (size_t)b * n;
    float mx1, s1, q1, mx2, s2, q2;
    c51_stats(a, n, v_min, dz, lane, mx1, s1, q1);
    c51_stats(c, n, v_min, dz, lane, mx2, s2, q2);
    const bool p1 = q1 <= q2;
    const float alpha = expf(*log_alpha);
    const float *l = p1 ? a : c;
    const float mx = p1 ? mx1 : mx2, inv = 1.0f / (p1 ? s1 : s2), qm = p1 ? q1 : q2;
    float *dsel = (p1 ? dq1 : dq2) + (size_t)b * n, *doth = (p1 ? dq2 : dq1) + (size_t)b * n;
    for (int i = lane; i < n; i += 32) {
        const float pi = expf(l[i] - mx) * inv;
        dsel[i] = -pi * ((v_min + (float)i * dz) - qm) * ib;
        doth[i] = 0.0f;
    }
    if (lane == 0) {
        dlogp[b] = alpha * ib;
        atomicAdd(&acc[0], alpha * logp[b] - qm);
        atomicAdd(&acc[1], logp[b]);
    }
}

// dL/dbeta of Eq. 2 through the actor's input: x = s / (l - beta) gives
// dx/dbeta = s / (l - beta)^2; summed over the batch into *acc
__global__ void k_beta_grad(const float *__restrict__ dX, int ldx, const float *__restrict__ Lraw,
                            int B, int ipap, const float *__restrict__ beta_dev,
                            const float *__restrict__ scale, float *acc) {
    pdl_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float g = 0.0f;
    if (i < (long long)B * ipap) {
        const int b = (int)(i / ipap), c = (int)(i - (long long)b * ipap);
        const float d = Lraw[i] - *beta_dev;
        g = dX[(long long)b * ldx + c] * (scale ? scale[c] : 1.0f) / (d * d);
    }
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, g);
}

// Adam step on beta (s[0] beta, s[1..2] moments, s[3] gradient, cleared and
// kept in s[-1]), then beta <- min(beta, beta_max) so that l - beta > 0 for
// every range l >= 0
__global__ void k_beta_adam(float *s, float lr, float b1, float b2, const float *__restrict__ corr,
                            float beta_max) {
    pdl_enter();
    const float c1 = corr[0], c2 = corr[1];
    const float g = s[3];
    s[-1] = g;
    const float mi = b1 * s[1] + (1.0f - b1) * g;
    const float vi = b2 * s[2] + (1.0f - b2) * g * g;
    s[1] = mi;
    s[2] = vi;
    s[0] = fminf(s[0] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f), beta_max);
    s[3] = 0.0f;
}

__global__ void k_zero(float *p, int n) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.0f;
}

// ----------------------------------------------------------- evaluation ---
// first episode of each env: FP64 return, success = goal before collision or
// timeout
__global__ void k_eval_acc(const float *__restrict__ rew, const unsigned char *__restrict__ done,
                           int E, unsigned char *finished, unsigned char *success, double *ret) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E || finished[e]) return;
    ret[e] += (double)rew[e];
    if (done[e] & 3) {
        finished[e] = 1;
        success[e] = (done[e] & 4) && !(done[e] & 8) ? 1 : 0;
    }
}

// FP64 block reduction of success count and return sum into out[0..1]
__global__ void k_eval_reduce(const unsigned char *__restrict__ success,
                              const double *__restrict__ ret, int E, double *out) {
    __shared__ double s0[256], s1[256];
    double a = 0.0, b = 0.0;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        a += (double)success[e];
        b += ret[e];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0];
        out[1] = s1[0];
    }
}

unsigned blocks(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

} // namespace
} // namespace flashnav

using namespace flashnav;

struct nav_trainer {
    nav_train_cfg cfg{};
    int od = 0, ld = 0, ldc = 0, H = 0, Hp = 0, NH = 0, B = 0, ipap = 0;
    int qout = 2;            // critic outputs: (mean, scale), or n_atoms logits (FastSAC)
    float *tdist = nullptr;  // FastSAC target distributions [B][n_atoms]
    long long cap = 0, size = 0, head = 0;
    unsigned long long n_critic = 0, n_actor = 0, n_alpha = 0;
    Mlp actor, q[2], qt[2];
    std::string err;
    std::vector<void *> mem;
    // replay
    bf16 *r_obs = nullptr, *r_next = nullptr;
    float *r_act = nullptr, *r_rew = nullptr, *r_term = nullptr;
    // batch
    int *idx = nullptr;
    bf16 *Xo = nullptr, *Xn = nullptr, *Xc = nullptr, *Xnc = nullptr, *Xa = nullptr;
    bf16 *XoT = nullptr, *XcT = nullptr;
    float *rew = nullptr, *term = nullptr;
    // activations per hidden layer: [0] actor, [1] q0, [2] q1, [3] scratch,
    // [4] [5] the target critics (per-layer path: their forward runs beside
    // the online critics')
    bf16 *h16[6][kMaxLayers - 1] = {}, *ht16[6][kMaxLayers - 1] = {};
    float *Lraw = nullptr, *dXa = nullptr; // raw Eq. 2 ranges of obs; actor input gradient
    unsigned *mask[4][kMaxLayers - 1] = {}; // fused passes: LeakyReLU' sign bits per slot
    float *out_a = nullptr, *out_an = nullptr, *qo[2] = {}, *tq[2] = {}, *qa[2] = {};
    float *a_next = nullptr, *logp_next = nullptr, *a_new = nullptr, *logp_new = nullptr,
          *eps_new = nullptr, *eps_next = nullptr;
    float *y = nullptr, *ym = nullptr, *znoise = nullptr, *dq[2] = {}, *dlogp = nullptr,
          *dout = nullptr;
    // backward scratch per chain: the twin critics' backward passes run
    // concurrently on two streams (chain 0 also serves the actor)
    float *dH[2] = {}, *dX[2] = {};
    bf16 *g16[2] = {}, *gT16[2] = {}, *dZ16[2] = {}, *dZT16[2] = {};
    cudaStream_t st2 = nullptr;          // second stream of the per-layer twin-critic chains
    cudaStream_t st3 = nullptr, st4 = nullptr; // online critic 0, target critic 1
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join3 = nullptr, ev_join4 = nullptr;
    float *scal = nullptr; // [0] log_alpha [1] sbar [2..3] alpha Adam [4..7] critic acc
                           // [8..9] actor acc [11] last beta gradient [12] beta
                           // [13..14] its Adam moments [15] its gradient accumulator
    int *status = nullptr;
    // evaluation
    unsigned char *ev_fin = nullptr, *ev_succ = nullptr;
    double *ev_ret = nullptr, *ev_out = nullptr;
    int ev_cap = 0;
    float *scale = nullptr; // per-feature input scale applied when storing obs
    // fused small-network passes (every width <= 128): per-CTA partial
    // gradients [n_cta][params] of the actor and the two critics
    bool fused = false;
    int n_cta = 0;
    float *part_a = nullptr, *part_q[2] = {};
    unsigned long long *ctr = nullptr; // device counters (kCtr*)
    unsigned *ticket = nullptr;        // last-block ticket of k_targets_grad2 (0 between launches)
    float *corr = nullptr;             // device Adam bias corrections
    // captured update sequences, keyed by (updates per call, policy phase)
    bool use_graphs = false;
    struct Graph {
        int n, phase;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
};

namespace {

template <class T> cudaError_t talloc(nav_trainer *t, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e == cudaSuccess) {
        cudaMemset(q, 0, std::max<size_t>(count * sizeof(T), 16));
        t->mem.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

int tfail(nav_trainer *t, int code, const std::string &m) {
    if (t) t->err = m;
    return code;
}

// Backward through an MLP from dL/dout (FP32 [B][n_out], n_out <= 8).  `s`
// holds the saved hidden activations (BF16 [B][Hp] and transposed [H][B]),
// XT the transposed input [in][B].  wgrad: fill the layer gradients; dX:
// input gradient FP32 [B][ldx] (may be null).  Per layer, top down: weight
// gradient dZ^T x_in (split-K GEMM over the batch), bias gradient (column
// sums), then the gradient of the layer's input dZ W, gated by LeakyReLU'
// into the next dZ.
int mlp_backward(nav_trainer *T, Mlp &net, const float *dout, int s, const bf16 *XT, bool wgrad,
                 float *dX, int ldx, cudaStream_t st, int ch = 0) {
    const int B = T->B, H = T->H, Hp = T->Hp;
    const int last = net.n_layers - 1;
    const int n_out = net.layer[last].out;
    int rc = 0;
    bf16 *g16 = T->g16[ch], *gT16 = T->gT16[ch], *dZ16 = T->dZ16[ch], *dZT16 = T->dZT16[ch];
    float *dH = T->dH[ch];
    launch_pdl(k_grad_to_bf16, blocks((long long)B * 8), 256, 0, st, dout, B, n_out, 8, g16, gT16);
    const dim3 tb(32, 8), tg((H + 31) / 32, (B + 31) / 32);
    for (int l = last; l >= 0; --l) {
        Layer &L = net.layer[l];
        const bool top = l == last;
        const bf16 *G = top ? g16 : dZ16;
        const int ldg = top ? 8 : Hp;
        const bf16 *GT = top ? gT16 : dZT16;
        const float *G32 = top ? dout : dH;
        const bf16 *inT = l == 0 ? XT : T->ht16[s][l - 1];
        if (wgrad) {
            rc |= launch_gemm_bf16_splitk(GT, B, inT, B, L.out, L.in, B, L.gW, L.in, T->status,
                                          st);
            launch_pdl(k_colsum, blocks(L.out, 32), dim3(32, 8), 0, st, G32, B, L.out, L.gb);
        }
        if (l > 0) {
            rc |= launch_gemm_bf16(G, ldg, L.WT16, L.ld_out, B, H, L.out, nullptr, 0, dH, H,
                                   nullptr, 0, nullptr, 0, T->status, st);
            launch_pdl(k_leaky_bwd, tg, tb, 0, st, dH, T->h16[s][l - 1], B, H, Hp, dZ16, dZT16);
        } else if (dX) {
            rc |= launch_gemm_bf16(G, ldg, L.WT16, L.ld_out, B, L.in, L.out, nullptr, 0, dX, ldx,
                                   nullptr, 0, nullptr, 0, T->status, st);
        }
    }
    rc |= (int)cudaGetLastError();
    return rc;
}

int copy_net(Mlp &dst, const Mlp &src) {
    for (int l = 0; l < dst.n_layers; ++l) {
        const size_t nw = (size_t)dst.layer[l].in * dst.layer[l].out;
        cudaMemcpy(dst.layer[l].W, src.layer[l].W, nw * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(dst.layer[l].b, src.layer[l].b, dst.layer[l].out * 4, cudaMemcpyDeviceToDevice);
    }
    return dst.refresh(nullptr);
}

// forward with saved activations (slot s) of a network on BF16 input x
int fwd(nav_trainer *T, const Mlp &net, const bf16 *x, int s, bool save_t, float *out,
        cudaStream_t st) {
    void *h[kMaxLayers - 1], *ht[kMaxLayers - 1];
    for (int l = 0; l < kMaxLayers - 1; ++l) {
        h[l] = T->h16[s][l];
        ht[l] = T->ht16[s][l];
    }
    return net.forward_tc(x, T->B, h, save_t ? ht : nullptr, out, T->status, st);
}

} // namespace

extern "C" {

void nav_train_default_cfg(nav_train_cfg *c) {
    if (!c) return;
    c->obs_dim = 364;
    c->hidden = 256;
    c->batch = 4096;
    c->replay_capacity = 4 << 20;
    c->lr_actor = 3e-4f;
    c->lr_critic = 3e-4f;
    c->lr_alpha = 3e-4f;
    c->beta1 = 0.9f;
    c->beta2 = 0.95f;
    c->gamma = 0.99f;
    c->tau = 0.1f;
    c->tau_b = 0.005f;
    c->reward_scale = 0.4f;
    c->huber_delta = 50.0f;
    c->alpha_init = 0.001f;
    c->target_entropy = -1.0f;
    c->policy_freq = 2;
    c->seed = 1;
    c->n_hidden = 2;
    c->weight_decay = 0.0f;
    c->ipap_features = 0;
    c->ipap_beta_init = -0.2f;
    c->ipap_beta_max = -0.01f;
    c->algo = 0;
    c->n_atoms = 101;
    c->v_min = -20.0f;
    c->v_max = 20.0f;
}

void nav_trainer_free(nav_trainer *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    for (auto &g : t->graphs) cudaGraphExecDestroy(g.exec);
    t->actor.release();
    for (int i = 0; i < 2; ++i) {
        t->q[i].release();
        t->qt[i].release();
    }
    for (void *p : t->mem) cudaFree(p);
    for (cudaEvent_t ev : {t->ev_fork, t->ev_join, t->ev_join3, t->ev_join4})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t s : {t->st2, t->st3, t->st4})
        if (s) cudaStreamDestroy(s);
    delete t;
}

int nav_trainer_create(const nav_train_cfg *cfg, nav_trainer **out) {
    if (!out) return NAV_E_INVAL;
    *out = nullptr;
    nav_train_cfg c;
    if (cfg) c = *cfg;
    else nav_train_default_cfg(&c);
    if (c.obs_dim <= 0 || c.hidden <= 0 || c.batch < 128 || c.batch % 128 ||
        c.replay_capacity < c.batch || c.replay_capacity > ((long long)1 << 31) ||
        c.policy_freq < 1 || c.n_hidden < 1 || c.n_hidden > kMaxLayers - 1 ||
        !(c.weight_decay >= 0.0f) || c.ipap_features < 0 || c.ipap_features > c.obs_dim ||
        (c.ipap_features > 0 &&
         !(c.ipap_beta_max < 0.0f && c.ipap_beta_init <= c.ipap_beta_max)) ||
        (c.algo != 0 && c.algo != 1) ||
        (c.algo == 1 && (c.n_atoms < 2 || c.n_atoms > kFusedMaxWidth || !(c.v_min < c.v_max))))
        return NAV_E_INVAL;
    nav_trainer *T = new (std::nothrow) nav_trainer();
    if (!T) return NAV_E_NOMEM;
    T->cfg = c;
    T->od = c.obs_dim;
    T->ld = (c.obs_dim + 7) / 8 * 8;
    T->ldc = (c.obs_dim + 2 + 7) / 8 * 8;
    T->H = c.hidden;
    T->Hp = act_ld(c.hidden);
    T->NH = c.n_hidden;
    T->ipap = c.ipap_features;
    T->B = c.batch;
    T->cap = c.replay_capacity;
    T->qout = c.algo == 1 ? c.n_atoms : 2;
    std::vector<int> sa(1, T->od), sq(1, T->od + 2);
    for (int l = 0; l < T->NH; ++l) {
        sa.push_back(T->H);
        sq.push_back(T->H);
    }
    sa.push_back(4);
    sq.push_back(T->qout);
    int rc = T->actor.init(sa, c.seed * 4 + 1, T->err);
    for (int i = 0; i < 2 && rc == NAV_OK; ++i) {
        rc = T->q[i].init(sq, c.seed * 4 + 2 + i, T->err);
        if (rc == NAV_OK) rc = T->qt[i].init(sq, c.seed * 4 + 2 + i, T->err);
    }
    cudaError_t e = rc == NAV_OK ? cudaSuccess : cudaErrorUnknown;
    const long long B = T->B, H = T->H;
#define TA(p, n) if (e == cudaSuccess) e = talloc(T, &(p), (size_t)(n))
    TA(T->r_obs, T->cap * T->ld);
    TA(T->r_next, T->cap * T->ld);
    TA(T->r_act, T->cap * 2);
    TA(T->r_rew, T->cap);
    TA(T->r_term, T->cap);
    TA(T->idx, B);
    TA(T->Xo, B * T->ld);
    TA(T->Xn, B * T->ld);
    TA(T->Xc, B * T->ldc);
    TA(T->Xnc, B * T->ldc);
    TA(T->Xa, B * T->ldc);
    TA(T->XoT, (long long)T->od * B);
    TA(T->XcT, (long long)(T->od + 2) * B);
    TA(T->rew, B);
    TA(T->term, B);
    for (int s = 0; s < 6; ++s)
        for (int l = 0; l < T->NH; ++l) {
            TA(T->h16[s][l], B * T->Hp);
            TA(T->ht16[s][l], B * H);
        }
    TA(T->Lraw, B * std::max(T->ipap, 1));
    TA(T->dXa, B * T->ld);
    TA(T->out_a, B * 4);
    TA(T->out_an, B * 4);
    for (int i = 0; i < 2; ++i) {
        TA(T->qo[i], B * T->qout);
        TA(T->tq[i], B * T->qout);
        TA(T->qa[i], B * T->qout);
        TA(T->dq[i], B * T->qout);
        TA(T->dX[i], B * T->ldc);
    }
    TA(T->a_next, B * 2);
    TA(T->logp_next, B);
    TA(T->a_new, B * 2);
    TA(T->logp_new, B);
    TA(T->eps_new, B * 2);
    TA(T->eps_next, B * 2);
    TA(T->y, B);
    TA(T->ym, B);
    TA(T->znoise, B);
    TA(T->dlogp, B);
    TA(T->dout, B * 4);
    for (int ch = 0; ch < 2; ++ch) {
        TA(T->g16[ch], B * 8);
        TA(T->gT16[ch], 8 * B);
        TA(T->dH[ch], B * H);
        TA(T->dZ16[ch], B * T->Hp);
        TA(T->dZT16[ch], B * H);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&T->st2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&T->st3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&T->st4, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&T->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&T->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&T->ev_join3, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&T->ev_join4, cudaEventDisableTiming);
    TA(T->scal, 16);
    TA(T->status, 1);
    TA(T->ctr, 8);
    TA(T->corr, 4);
    TA(T->ticket, 1);
    T->fused = rc == NAV_OK && fused_ok(T->actor, T->B) && fused_ok(T->q[0], T->B);
    if (c.algo == 1) TA(T->tdist, B * T->qout);
    if (e == cudaSuccess && rc == NAV_OK && c.algo == 1 && !T->fused) {
        T->err = "FastSAC needs networks on the fused passes (every width <= 128)";
        rc = NAV_E_INVAL;
        e = cudaErrorInvalidValue;
    }
    if (T->fused) {
        T->n_cta = T->B / 128;
        for (int sl = 0; sl < 4; ++sl)
            for (int l = 0; l < T->NH; ++l) TA(T->mask[sl][l], B * 4);
        TA(T->part_a, (long long)T->n_cta * T->actor.num_params());
        for (int i = 0; i < 2; ++i) TA(T->part_q[i], (long long)T->n_cta * T->q[i].num_params());
    }
#undef TA
    if (e != cudaSuccess) {
        nav_trainer_free(T);
        return rc != NAV_OK ? rc : NAV_E_NOMEM;
    }
    copy_net(T->qt[0], T->q[0]);
    copy_net(T->qt[1], T->q[1]);
    float init[2] = {std::log(c.alpha_init), 1.0f};
    cudaMemcpy(T->scal, init, sizeof(init), cudaMemcpyHostToDevice);
    cudaMemcpy(T->scal + 12, &c.ipap_beta_init, 4, cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        nav_trainer_free(T);
        return NAV_E_CUDA;
    }
    *out = T;
    return NAV_OK;
}

const char *nav_trainer_last_error(const nav_trainer *t) { return t ? t->err.c_str() : "null"; }

int nav_train_insert(nav_trainer *T, const float *obs_dev, const float *act_dev,
                     const float *rew_dev, const uint8_t *done_dev, const float *next_obs_dev,
                     const float *final_obs_dev, int n_envs, void *stream) {
    if (!T || !obs_dev || !act_dev || !rew_dev || !done_dev || !next_obs_dev || n_envs <= 0 ||
        n_envs > T->cap)
        return tfail(T, NAV_E_INVAL, "nav_train_insert: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_replay_insert<<<blocks((long long)n_envs * T->ld), 256, 0, st>>>(
        obs_dev, act_dev, rew_dev, done_dev, next_obs_dev, final_obs_dev, n_envs, T->od, T->ld,
        T->ctr, T->cap, T->scale, T->ipap, T->r_obs, T->r_next, T->r_act, T->r_rew, T->r_term);
    k_insert_done<<<1, 1, 0, st>>>(T->ctr, n_envs, T->cap);
    T->head = (T->head + n_envs) % T->cap;
    T->size = std::min(T->cap, T->size + n_envs);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

} // extern "C"

namespace {

// forward of up to four networks through one fused launch, network k on
// input X[k] (leading dimension ldx[k]); slot[k] >= 0 saves its hidden
// activations' LeakyReLU' bits (and, with save_t[k], their transposes) there
int ffwd_n(nav_trainer *T, Mlp *const *nets, int n, const bf16 *const *X, const int *ldx,
           float *const *out, const int *slot, const bool *save_t, cudaStream_t st) {
    FGroup g{};
    g.n_nets = n;
    g.B = T->B;
    g.status = T->status;
    for (int k = 0; k < n; ++k) {
        FNet &f = g.net[k];
        fused_layers(*nets[k], f);
        f.X = X[k];
        f.ldx = ldx[k];
        f.out32 = out[k];
        f.ldh = T->Hp;
        for (int l = 0; l + 1 < nets[k]->n_layers; ++l) {
            f.M[l] = slot[k] >= 0 ? T->mask[slot[k]][l] : nullptr;
            f.HT16[l] = (slot[k] >= 0 && save_t[k]) ? T->ht16[slot[k]][l] : nullptr;
        }
    }
    return launch_mlp_fwd_fused(g, st);
}

// up to two networks on one input
int ffwd(nav_trainer *T, Mlp *const *nets, int n, const bf16 *X, int ldx, float *const *out,
         const int *slot, bool save_t, cudaStream_t st) {
    const bf16 *Xs[2] = {X, X};
    const int lds[2] = {ldx, ldx};
    const bool sv[2] = {save_t, save_t};
    return ffwd_n(T, nets, n, Xs, lds, out, slot, sv, st);
}

// backward of up to two networks: part[k] receives the per-CTA partial
// gradients (null: no weight gradients), dX[k] the input gradient (or null)
int fbwd(nav_trainer *T, Mlp *const *nets, int n, float *const *dout, const int *slot,
         const bf16 *XT, float *const *part, float *const *dX, int lddx, cudaStream_t st) {
    FGroup g{};
    g.n_nets = n;
    g.B = T->B;
    g.status = T->status;
    for (int k = 0; k < n; ++k) {
        const Mlp &m = *nets[k];
        FNet &f = g.net[k];
        fused_layers(m, f);
        f.dout = dout[k];
        f.XT = XT;
        f.ldh = T->Hp;
        f.cta_stride = m.num_params();
        f.dX = dX ? dX[k] : nullptr;
        f.lddx = lddx;
        long long off = 0;
        for (int l = 0; l < m.n_layers; ++l) {
            const Layer &L = m.layer[l];
            if (l + 1 < m.n_layers) {
                f.M[l] = T->mask[slot[k]][l];
                f.HT16[l] = T->ht16[slot[k]][l];
            }
            f.gWp[l] = part ? part[k] + off : nullptr;
            f.gbp[l] = part ? part[k] + off + (long long)L.in * L.out : nullptr;
            off += (long long)L.in * L.out + L.out;
        }
    }
    return launch_mlp_bwd_fused(g, st);
}

// One critic update (and the actor update that falls on it) on the fused
// passes: the same arithmetic as the per-layer path in 8 launches (FastDSAC
// critic step; 16-17 with an actor step), each launched with programmatic
// dependent launch.
int fused_update(nav_trainer *T, bool actor_step, cudaStream_t st) {
    const nav_train_cfg &c = T->cfg;
    const int B = T->B;
    int rc = 0;
    Mlp *qs[2] = {&T->q[0], &T->q[1]}, *qts[2] = {&T->qt[0], &T->qt[1]}, *act[1] = {&T->actor};
    const int qslot[2] = {1, 2}, aslot[1] = {0};
    const bool c51 = c.algo == 1;
    launch_pdl(k_count_start, 1, 1, 0, st, T->ctr, actor_step ? 1 : 0, c.beta1, c.beta2, T->corr,
               T->scal + 8);
    launch_pdl(k_gather_all, blocks((long long)B * T->ldc), 256, 0, st, T->r_obs, T->r_next,
               T->r_act, T->r_rew, T->r_term, B, T->od, T->ld, T->ldc, T->ipap, T->scal + 12,
               T->scale, T->ctr, c.seed, T->cap, T->idx, T->Xo, T->Xn, T->Xc, T->XcT, T->XoT,
               T->Xnc, T->Xa, T->Lraw, T->rew, T->term);
    // the actor on the next observations (targets) and, in an actor step, on
    // the observations (activations saved for its backward) in one launch:
    // the actor's weights do not change before its own update
    {
        Mlp *aa[2] = {&T->actor, &T->actor};
        const bf16 *Xs[2] = {T->Xn, T->Xo};
        const int lds[2] = {T->ld, T->ld};
        float *outs[2] = {T->out_an, T->out_a};
        const int sl[2] = {-1, 0};
        const bool sv[2] = {false, true};
        rc |= ffwd_n(T, aa, actor_step ? 2 : 1, Xs, lds, outs, sl, sv, st);
    }
    // a' (written into Xnc's action columns too)
    rc |= launch_actor_head_ctr(T->out_an, B, 1, c.seed ^ 0x5A5Aull, T->ctr, kCtrCritic, 2u, 1u,
                                T->a_next, T->logp_next, T->eps_next, st, T->Xnc, T->ldc, T->od);
    // the target critics on [s', a'] and the critics on [s, a] in one launch
    {
        Mlp *four[4] = {&T->qt[0], &T->qt[1], &T->q[0], &T->q[1]};
        const bf16 *Xs[4] = {T->Xnc, T->Xnc, T->Xc, T->Xc};
        const int lds[4] = {T->ldc, T->ldc, T->ldc, T->ldc};
        float *outs[4] = {T->tq[0], T->tq[1], T->qo[0], T->qo[1]};
        const int sl[4] = {-1, -1, 1, 2};
        const bool sv[4] = {false, false, true, true};
        rc |= ffwd_n(T, four, 4, Xs, lds, outs, sl, sv, st);
    }
    // targets and dL/dq of both critics (with the running sigma for FastDSAC)
    if (c51) {
        launch_pdl(k_c51_targets, blocks(B, 8), 256, 0, st, T->rew, T->term, T->tq[0], T->tq[1],
                   T->logp_next, T->scal + 0, B, T->qout, c.gamma, c.reward_scale, c.v_min,
                   c.v_max, T->tdist, T->qo[0], T->qo[1], T->dq[0], T->dq[1], T->scal + 4);
    } else {
        launch_pdl(k_targets_grad2, blocks(B), 256, 0, st, T->rew, T->term, T->tq[0], T->tq[1],
                   T->logp_next, T->scal + 0, B, c.gamma, c.reward_scale, c.seed, T->ctr, T->y,
                   T->ym, T->znoise, T->qo[0], T->qo[1], T->scal + 1, c.huber_delta, T->dq[0],
                   T->dq[1], T->scal + 4, c.tau_b, T->ticket);
    }
    rc |= fbwd(T, qs, 2, T->dq, qslot, T->XcT, T->part_q, nullptr, 0, st);
    // the critics' Adam step and the target critics' Polyak step in one pass
    // (nothing after it in the update reads the targets)
    rc |= launch_adam_fused(qs, T->part_q, 2, T->n_cta, c.lr_critic, c.beta1, c.beta2, T->corr,
                            c.weight_decay, st, qts, c.tau);
    if (actor_step) {
        // the actor's own action a, written into Xa's action columns too
        rc |= launch_actor_head_ctr(T->out_a, B, 1, c.seed ^ 0xA5A5ull, T->ctr, kCtrActor, 2u, 0u,
                                    T->a_new, T->logp_new, T->eps_new, st, T->Xa, T->ldc, T->od);
        rc |= ffwd(T, qs, 2, T->Xa, T->ldc, T->qa, qslot, false, st);
        if (c51)
            launch_pdl(k_c51_actor_loss, blocks(B, 8), 256, 0, st, T->logp_new, T->qa[0], T->qa[1],
                       T->scal + 0, B, T->qout, c.v_min, c.v_max, T->dlogp, T->dq[0], T->dq[1],
                       T->scal + 8);
        else
            launch_pdl(k_actor_loss, blocks(B), 256, 0, st, T->logp_new, T->qa[0], T->qa[1],
                       T->scal + 0, B, T->dlogp, T->dq[0], T->dq[1], T->scal + 8);
        rc |= fbwd(T, qs, 2, T->dq, qslot, nullptr, nullptr, T->dX, T->ldc, st);
        launch_pdl(k_actor_head_bwd, blocks(B), 256, 0, st, T->out_a, T->eps_new, T->dX[0],
                   T->dX[1], T->ldc, T->od, T->dlogp, B, T->dout);
        float *douts[1] = {T->dout}, *pa[1] = {T->part_a}, *dxa[1] = {T->dXa};
        rc |= fbwd(T, act, 1, douts, aslot, T->XoT, pa, T->ipap > 0 ? dxa : nullptr, T->ld, st);
        rc |= launch_adam_fused(act, pa, 1, T->n_cta, c.lr_actor, c.beta1, c.beta2, T->corr + 2,
                                c.weight_decay, st);
        if (T->ipap > 0)
            launch_pdl(k_beta_grad, blocks((long long)B * T->ipap), 256, 0, st, T->dXa, T->ld,
                       T->Lraw, B, T->ipap, T->scal + 12, T->scale, T->scal + 15);
        launch_pdl(k_alpha_beta, 1, 1, 0, st, T->scal + 0, T->scal + 2, T->scal + 3, T->scal + 8,
                   B, c.target_entropy, c.lr_alpha, c.beta1, c.beta2, T->corr + 2,
                   T->ipap > 0 ? T->scal + 12 : nullptr, c.lr_actor, c.ipap_beta_max);
    }
    rc |= (int)cudaGetLastError();
    return rc;
}

// The launches of n critic updates (and the actor updates that fall among
// them) on `st`; every value that changes from update to update is read from
// the device counters, so the sequence can be captured once and replayed.
// The twin critics' per-layer chains run side by side: fork2 makes the
// second stream wait for the work `st` has queued, join2 makes `st` wait for
// the second stream's (events, so a graph capture records both branches).
int fork_to(nav_trainer *T, cudaStream_t st, cudaStream_t to) {
    cudaError_t e = cudaEventRecord(T->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, T->ev_fork, 0);
    return (int)e;
}
int join_from(cudaEvent_t ev, cudaStream_t from, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    return (int)e;
}
int fork2(nav_trainer *T, cudaStream_t st) { return fork_to(T, st, T->st2); }
int join2(nav_trainer *T, cudaStream_t st) { return join_from(T->ev_join, T->st2, st); }

int update_body(nav_trainer *T, int n_updates, unsigned long long n_critic, cudaStream_t st) {
    const nav_train_cfg &c = T->cfg;
    const int B = T->B;
    int rc = 0;
    if (T->fused) {
        for (int u = 0; u < n_updates; ++u) {
            ++n_critic;
            rc |= fused_update(T, n_critic % (unsigned long long)c.policy_freq == 0, st);
            if (rc) return rc;
        }
        return 0;
    }
    for (int u = 0; u < n_updates; ++u) {
        // ---- critic update (index ctr[critic] - 1 after k_count)
        launch_pdl(k_count, 1, 1, 0, st, T->ctr, kCtrCritic, c.beta1, c.beta2, T->corr);
        launch_pdl(k_sample, blocks(B), 256, 0, st, T->idx, B, T->ctr, c.seed, T->cap);
        launch_pdl(k_gather, blocks((long long)B * T->ldc), 256, 0, st, 
            T->idx, T->r_obs, T->r_next, T->r_act, T->r_rew, T->r_term, B, T->od, T->ld, T->ldc,
            T->ipap, T->scal + 12, T->scale, T->Xo, T->Xn, T->Xc, T->Lraw, T->rew, T->term);
        const dim3 tb(32, 8);
        launch_pdl(k_transpose, dim3((T->od + 2 + 31) / 32, (B + 31) / 32), tb, 0, st, 
            T->Xc, T->ldc, B, T->od + 2, T->XcT, B);
        // three branches: the online critics' forwards (slots 1, 2, on st3 and
        // st2) beside the target path on st (next action, the target critics
        // in slots 4, 5 side by side, the targets)
        rc |= fork_to(T, st, T->st3);
        rc |= fork_to(T, st, T->st2);
        rc |= fwd(T, T->q[0], T->Xc, 1, true, T->qo[0], T->st3);
        rc |= fwd(T, T->q[1], T->Xc, 2, true, T->qo[1], T->st2);
        // next action from the current actor (noise step 2 index + 1)
        rc |= fwd(T, T->actor, T->Xn, 3, false, T->out_a, st);
        rc |= launch_actor_head_ctr(T->out_a, B, 1, c.seed ^ 0x5A5Aull, T->ctr, kCtrCritic, 2u,
                                    1u, T->a_next, T->logp_next, T->eps_next, st);
        launch_pdl(k_concat, blocks((long long)B * T->ldc), 256, 0, st, T->Xn, T->ld, T->a_next, B, T->od,
                                                                T->ldc, T->Xnc);
        rc |= fork_to(T, st, T->st4);
        rc |= fwd(T, T->qt[1], T->Xnc, 5, false, T->tq[1], T->st4);
        rc |= fwd(T, T->qt[0], T->Xnc, 4, false, T->tq[0], st);
        rc |= join_from(T->ev_join4, T->st4, st);
        launch_pdl(k_targets, blocks(B), 256, 0, st, T->rew, T->term, T->tq[0], T->tq[1], T->logp_next,
                                             T->scal + 0, B, c.gamma, c.reward_scale, c.seed,
                                             T->ctr, T->y, T->ym, T->znoise);
        // each online critic: loss gradient (needs the targets) and backward
        rc |= fork_to(T, st, T->st3);
        rc |= fork_to(T, st, T->st2);
        for (int i = 1; i >= 0; --i) {
            cudaStream_t si = i ? T->st2 : T->st3;
            launch_pdl(k_critic_grad, blocks(B), 256, 0, si, T->qo[i], T->y, T->ym, T->scal + 1, B,
                                                     c.huber_delta, T->dq[i], T->scal + 4);
            rc |= mlp_backward(T, T->q[i], T->dq[i], 1 + i, T->XcT, true, nullptr, 0, si, i);
        }
        rc |= join_from(T->ev_join3, T->st3, st);
        rc |= join2(T, st);
        launch_pdl(k_sbar_update, 1, 1, 0, st, T->scal + 1, T->scal + 4, 2 * B, c.tau_b);
        {
            Mlp *qs[2] = {&T->q[0], &T->q[1]};
            rc |= launch_adam_fused(qs, nullptr, 2, 1, c.lr_critic, c.beta1, c.beta2, T->corr,
                                    c.weight_decay, st);
        }
        ++n_critic;
        // ---- actor and temperature update every policy_freq critic updates
        if (n_critic % (unsigned long long)c.policy_freq == 0) {
            launch_pdl(k_count, 1, 1, 0, st, T->ctr, kCtrActor, c.beta1, c.beta2, T->corr);
            launch_pdl(k_transpose, dim3((T->od + 31) / 32, (B + 31) / 32), tb, 0, st, T->Xo, T->ld, B,
                                                                              T->od, T->XoT, B);
            rc |= fwd(T, T->actor, T->Xo, 0, true, T->out_a, st);
            rc |= launch_actor_head_ctr(T->out_a, B, 1, c.seed ^ 0xA5A5ull, T->ctr, kCtrActor, 2u,
                                        0u, T->a_new, T->logp_new, T->eps_new, st);
            launch_pdl(k_concat, blocks((long long)B * T->ldc), 256, 0, st, T->Xo, T->ld, T->a_new, B,
                                                                    T->od, T->ldc, T->Xa);
            rc |= fork2(T, st);
            rc |= fwd(T, T->q[1], T->Xa, 2, false, T->qa[1], T->st2);
            rc |= fwd(T, T->q[0], T->Xa, 1, false, T->qa[0], st);
            rc |= join2(T, st);
            launch_pdl(k_zero, 1, 32, 0, st, T->scal + 8, 2);
            launch_pdl(k_actor_loss, blocks(B), 256, 0, st, T->logp_new, T->qa[0], T->qa[1], T->scal + 0,
                                                    B, T->dlogp, T->dq[0], T->dq[1], T->scal + 8);
            rc |= fork2(T, st);
            rc |= mlp_backward(T, T->q[1], T->dq[1], 2, nullptr, false, T->dX[1], T->ldc, T->st2, 1);
            rc |= mlp_backward(T, T->q[0], T->dq[0], 1, nullptr, false, T->dX[0], T->ldc, st, 0);
            rc |= join2(T, st);
            launch_pdl(k_actor_head_bwd, blocks(B), 256, 0, st, T->out_a, T->eps_new, T->dX[0], T->dX[1],
                                                        T->ldc, T->od, T->dlogp, B, T->dout);
            rc |= mlp_backward(T, T->actor, T->dout, 0, T->XoT, true,
                               T->ipap > 0 ? T->dXa : nullptr, T->ld, st);
            {
                Mlp *act[1] = {&T->actor};
                rc |= launch_adam_fused(act, nullptr, 1, 1, c.lr_actor, c.beta1, c.beta2,
                                        T->corr + 2, c.weight_decay, st);
            }
            if (T->ipap > 0) {
                // Eq. 2's beta trained with the actor (same Adam settings)
                launch_pdl(k_beta_grad, blocks((long long)B * T->ipap), 256, 0, st, 
                    T->dXa, T->ld, T->Lraw, B, T->ipap, T->scal + 12, T->scale, T->scal + 15);
                launch_pdl(k_beta_adam, 1, 1, 0, st, T->scal + 12, c.lr_actor, c.beta1, c.beta2,
                                             T->corr + 2, c.ipap_beta_max);
            }
            launch_pdl(k_alpha, 1, 1, 0, st, T->scal + 0, T->scal + 2, T->scal + 3, T->scal + 8, B,
                                     c.target_entropy, c.lr_alpha, c.beta1, c.beta2, T->corr + 2);
        }
        {
            Mlp *qts[2] = {&T->qt[0], &T->qt[1]}, *qs[2] = {&T->q[0], &T->q[1]};
            rc |= launch_polyak_fused(qts, qs, 2, c.tau, st);
        }
        rc |= (int)cudaGetLastError();
        if (rc) return rc;
    }
    return 0;
}

} // namespace

extern "C" {

int nav_train_update(nav_trainer *T, int n_updates, void *stream) {
    if (!T || n_updates <= 0) return tfail(T, NAV_E_INVAL, "nav_train_update: bad argument");
    if (T->size < T->B) return tfail(T, NAV_E_INVAL, "nav_train_update: replay smaller than a batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int pf = T->cfg.policy_freq;
    const int phase = (int)(T->n_critic % (unsigned long long)pf);
    const unsigned long long n_act =
        (T->n_critic + (unsigned long long)n_updates) / (unsigned long long)pf -
        T->n_critic / (unsigned long long)pf;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st) cudaStreamIsCapturing(st, &cap);
    int rc = 0;
    if (T->use_graphs && st && cap == cudaStreamCaptureStatusNone) {
        cudaGraphExec_t exec = nullptr;
        for (auto &g : T->graphs)
            if (g.n == n_updates && g.phase == phase) exec = g.exec;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = update_body(T, n_updates, T->n_critic, st);
                e = cudaStreamEndCapture(st, &graph);
            }
            if (e == cudaSuccess && rc == 0) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess || rc != 0)
                return tfail(T, NAV_E_CUDA, "nav_train_update: graph capture failed");
            T->graphs.push_back({n_updates, phase, exec});
        }
        if (cudaGraphLaunch(exec, st) != cudaSuccess)
            return tfail(T, NAV_E_CUDA, "nav_train_update: graph launch failed");
    } else {
        rc = update_body(T, n_updates, T->n_critic, st);
        if (rc) return tfail(T, NAV_E_CUDA, "nav_train_update: launch failed");
    }
    T->n_critic += (unsigned long long)n_updates;
    T->n_actor += n_act;
    return NAV_OK;
}

int nav_train_overlap(nav_trainer *T, int n_pending, void *stream) {
    if (!T || n_pending < 0 || (long long)n_pending >= T->cap)
        return tfail(T, NAV_E_INVAL, "nav_train_overlap: bad argument");
    k_overlap<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(T->ctr,
                                                             (unsigned long long)n_pending);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_trainer_set_fused(nav_trainer *T, int on) {
    if (!T) return NAV_E_INVAL;
    if (on && !T->part_a) return tfail(T, NAV_E_INVAL, "networks too wide for the fused passes");
    if (!on && T->cfg.algo == 1)
        return tfail(T, NAV_E_INVAL, "FastSAC runs on the fused passes only");
    T->fused = on != 0;
    for (auto &g : T->graphs) cudaGraphExecDestroy(g.exec);
    T->graphs.clear();
    return NAV_OK;
}

int nav_trainer_set_graphs(nav_trainer *T, int on) {
    if (!T) return NAV_E_INVAL;
    T->use_graphs = on != 0;
    return NAV_OK;
}

int nav_trainer_io(nav_trainer *T, int what, int set, void *host) {
    if (!T || !host) return NAV_E_INVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return NAV_E_CUDA;
    Mlp *nets[5] = {&T->actor, &T->q[0], &T->q[1], &T->qt[0], &T->qt[1]};
    float *fh = static_cast<float *>(host);
    if (what >= 0 && what < 5) return nets[what]->copy_params(fh, !set) == 0 ? NAV_OK : NAV_E_CUDA;
    if (what >= 10 && what < 13 && !set) {
        Mlp &n = *nets[what - 10];
        long long off = 0;
        for (int l = 0; l < n.n_layers; ++l) {
            const size_t nw = (size_t)n.layer[l].in * n.layer[l].out;
            cudaMemcpy(fh + off, n.layer[l].gW, nw * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(fh + off + nw, n.layer[l].gb, n.layer[l].out * 4, cudaMemcpyDeviceToHost);
            off += (long long)nw + n.layer[l].out;
        }
        return NAV_OK;
    }
    const size_t B = (size_t)T->B;
    struct { int id; void *p; size_t bytes; } bufs[] = {
        {20, T->idx, B * 4},        {21, T->eps_new, B * 8},  {22, T->eps_next, B * 8},
        {23, T->znoise, B * 4},     {24, T->scal, 16 * 4},    {25, T->y, B * 4},
        {26, T->ym, B * 4},         {27, T->qo[0], B * 4 * T->qout}, {28, T->logp_new, B * 4},
        {29, T->a_new, B * 8},      {30, T->out_a, B * 16},   {31, T->logp_next, B * 4},
        {32, T->tdist, T->tdist ? B * 4 * T->qout : 0}};
    for (auto &b : bufs)
        if (b.id == what) {
            const cudaError_t e = set ? cudaMemcpy(b.p, host, b.bytes, cudaMemcpyHostToDevice)
                                      : cudaMemcpy(host, b.p, b.bytes, cudaMemcpyDeviceToHost);
            return e == cudaSuccess ? NAV_OK : NAV_E_CUDA;
        }
    return NAV_E_INVAL;
}

int nav_trainer_set_input_scale(nav_trainer *T, const float *scale_host) {
    if (!T || !scale_host) return NAV_E_INVAL;
    cudaError_t e = cudaSuccess;
    if (!T->scale) e = talloc(T, &T->scale, T->od);
    if (e == cudaSuccess) e = cudaMemcpy(T->scale, scale_host, (size_t)T->od * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_trainer_sync_policy(nav_trainer *T, nav_policy *p, void *stream) {
    Mlp *dst = p ? policy_actor(p) : nullptr;
    if (!T || !dst || dst->n_layers != T->actor.n_layers || policy_ipap(p) != T->ipap)
        return NAV_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T->ipap > 0)
        cudaMemcpyAsync(policy_beta(p), T->scal + 12, 4, cudaMemcpyDeviceToDevice, st);
    for (int l = 0; l < dst->n_layers; ++l) {
        const Layer &S = T->actor.layer[l];
        Layer &D = dst->layer[l];
        if (D.in != S.in || D.out != S.out) return NAV_E_INVAL;
        cudaMemcpyAsync(D.W, S.W, (size_t)S.in * S.out * 4, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(D.b, S.b, (size_t)S.out * 4, cudaMemcpyDeviceToDevice, st);
    }
    return dst->refresh(stream) == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_trainer_counts(const nav_trainer *T, int64_t *replay_size, int64_t *critic_updates,
                       int64_t *actor_updates) {
    if (!T) return NAV_E_INVAL;
    unsigned long long c[4];
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(c, T->ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return NAV_E_CUDA;
    if (replay_size) *replay_size = (int64_t)c[kCtrSize];
    if (critic_updates) *critic_updates = (int64_t)c[kCtrCritic];
    if (actor_updates) *actor_updates = (int64_t)c[kCtrActor];
    return NAV_OK;
}

int nav_eval_begin(nav_trainer *T, int n_envs, void *stream) {
    if (!T || n_envs <= 0) return NAV_E_INVAL;
    if (n_envs > T->ev_cap) {
        cudaError_t e = talloc(T, &T->ev_fin, n_envs);
        if (e == cudaSuccess) e = talloc(T, &T->ev_succ, n_envs);
        if (e == cudaSuccess) e = talloc(T, &T->ev_ret, n_envs);
        if (e == cudaSuccess && !T->ev_out) e = talloc(T, &T->ev_out, 2);
        if (e != cudaSuccess) return NAV_E_NOMEM;
        T->ev_cap = n_envs;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(T->ev_fin, 0, n_envs, st);
    cudaMemsetAsync(T->ev_succ, 0, n_envs, st);
    cudaMemsetAsync(T->ev_ret, 0, n_envs * sizeof(double), st);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_eval_accumulate(nav_trainer *T, const float *reward_dev, const uint8_t *done_dev,
                        int n_envs, void *stream) {
    if (!T || !reward_dev || !done_dev || n_envs <= 0 || n_envs > T->ev_cap) return NAV_E_INVAL;
    k_eval_acc<<<blocks(n_envs), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reward_dev, done_dev, n_envs, T->ev_fin, T->ev_succ, T->ev_ret);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_eval_result(nav_trainer *T, int n_envs, double *successes, double *return_sum,
                    void *stream) {
    if (!T || n_envs <= 0 || n_envs > T->ev_cap) return NAV_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_eval_reduce<<<1, 256, 0, st>>>(T->ev_succ, T->ev_ret, n_envs, T->ev_out);
    double out[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(out, T->ev_out, sizeof(out), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return NAV_E_CUDA;
    if (successes) *successes = out[0];
    if (return_sum) *return_sum = out[1];
    return NAV_OK;
}

} // extern "C"
