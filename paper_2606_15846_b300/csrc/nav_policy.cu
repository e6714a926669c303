// Policy network and its in-loop inference (Sec. 2.1 policy MLP; the FastDSAC
// actor of Sec. 2.3, a tanh-squashed Gaussian).  The actor is
// obs -> 256 -> 256 -> (mean 2, raw log-std 2) with LeakyReLU (slope 0.01);
// weights are kept in FP32 (master) with BF16 copies for the tensor cores:
// W [out][ld_in] (forward, K-major) and W^T [in][ld_out] (backward data).
//
// Inference: observations (FP32 rows) are converted to BF16 rows padded to a
// multiple of 8, run through three tcgen05 GEMMs (bias and LeakyReLU fused in
// the epilogues) and the squashed-Gaussian head:
//   log sigma = -5 + 5 (tanh(r) + 1) / 2,  a = tanh(u + sigma eps)
// with eps standard normal from the counter hash keyed by (seed, row, step)
// (Box-Muller), or a = tanh(u) when deterministic.  A plain FP32 SIMT path
// (register-blocked shared-memory GEMM on the CUDA cores, no tensor cores) is
// kept as the unfused baseline.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nav_internal.h"
#include "pdl.cuh"
#include "nav_policy.h"

namespace flashnav {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Network input feature c of an observation row: Eq. 2's 1 / (l - beta) for
// the first ipap features, then the per-feature scale.
__device__ __forceinline__ float in_feature(const float *src, int c, const float *scale, int ipap,
                                            float beta) {
    float x = src[c];
    if (c < ipap) x = 1.0f / (x - beta);
    return scale ? x * scale[c] : x;
}

// one thread per 4 columns of a row: FP32 -> BF16, zero beyond dim
__global__ void obs_to_bf16(const float *__restrict__ obs, int n, int dim, long long stride,
                            const float *__restrict__ scale, int ipap,
                            const float *__restrict__ beta_dev, __nv_bfloat16 *out, int ld) {
    const int groups = ld >> 2;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || g >= groups) return;
    const float *src = obs + (long long)r * stride;
    const float beta = ipap > 0 ? *beta_dev : 0.0f;
    const int c = 4 * g;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = c + k < dim ? in_feature(src, c + k, scale, ipap, beta) : 0.0f;
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 pk;
    pk.x = *reinterpret_cast<const unsigned *>(&a);
    pk.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(out + (long long)r * ld + c) = pk;
}

__global__ void obs_to_fp32(const float *__restrict__ obs, int n, int dim, long long stride,
                            const float *__restrict__ scale, int ipap,
                            const float *__restrict__ beta_dev, float *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * dim) return;
    const int r = (int)(i / dim), c = (int)(i - (long long)r * dim);
    out[i] = in_feature(obs + (long long)r * stride, c, scale, ipap, ipap > 0 ? *beta_dev : 0.0f);
}

// a = tanh(u + sigma eps) (or tanh(u)), logp per row.
// With ctr set, the noise step is mul * (ctr[which] - sub) + add, read on the
// device (so that a captured launch draws fresh noise on every replay).
__global__ void actor_head_fwd(const float *__restrict__ out4, int n, int mode,
                               unsigned long long seed, unsigned step,
                               const unsigned long long *__restrict__ ctr, int which,
                               unsigned long long sub, unsigned mul, unsigned add, float *act,
                               float *logp, float *eps_out, __nv_bfloat16 *xc, int ldc, int col0) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (ctr) step = mul * (unsigned)(ctr[which] - sub) + add;
    const float *o = out4 + (size_t)r * 4;
    float lp = 0.0f;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const float u = o[d];
        const float ls = kLogStdMin + (kLogStdMax - kLogStdMin) * 0.5f * (tanhf(o[2 + d]) + 1.0f);
        float e = 0.0f;
        if (mode == 1) {
            const unsigned long long h = mix64(seed ^ ((unsigned long long)r * 0xD1B54A32D192ED03ull) ^
                                               ((unsigned long long)step << 32) ^ (unsigned)d);
            const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
            const float u2 = (float)((h >> 8) & 0xFFFFFFull) * (1.0f / 16777216.0f);
            e = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
        }
        const float a = tanhf(u + expf(ls) * e);
        lp += -0.5f * e * e - ls - 0.91893853320467274f - logf(1.0f - a * a + 1e-6f);
        act[(size_t)r * 2 + d] = a;
        if (eps_out) eps_out[(size_t)r * 2 + d] = e;
        if (xc) xc[(size_t)r * ldc + col0 + d] = __float2bfloat16_rn(a);
    }
    if (logp) logp[r] = lp;
}

__global__ void k_bump(unsigned long long *c) { *c += 1; }

// Plain FP32 layer on the CUDA cores (the unfused baseline; no tensor
// cores): y[r][o] = act(sum_k x[r][k] W[o][k] + b[o]).  A register-blocked
// SIMT GEMM: each 256-thread CTA computes a 128-row x 64-output tile from
// 16-wide K tiles of x and W staged in shared memory (stored K-major, so a
// thread reads its 8 rows and 4 outputs as vectors), each thread 8 x 4
// results with FP32 FMAs.
constexpr int kSgBM = 128, kSgBN = 64, kSgBK = 16;

__global__ void __launch_bounds__(256) dense_fp32(const float *__restrict__ x, long long ldx, int n,
                                                  int in, const float *__restrict__ W,
                                                  const float *__restrict__ b, int out, int leaky,
                                                  float *y) {
    __shared__ __align__(16) float As[kSgBK][kSgBM + 4];
    __shared__ __align__(16) float Bs[kSgBK][kSgBN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long r0 = (long long)blockIdx.x * kSgBM;
    const int o0 = blockIdx.y * kSgBN;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < in; k0 += kSgBK) {
        // x tile: row tid / 2, 8 consecutive k; W tile: output tid / 4, 4 k
        {
            const int r = tid >> 1, kk = (tid & 1) * 8;
            const long long gr = r0 + r;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + kk + q;
                As[kk + q][r] = (gr < n && k < in) ? x[gr * ldx + k] : 0.0f;
            }
            const int o = tid >> 2, kb = (tid & 3) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + kb + q;
                Bs[kb + q][o] = (o0 + o < out && k < in) ? W[(size_t)(o0 + o) * in + k] : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSgBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][ty * 8 + 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bw[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long r = r0 + ty * 8 + i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = o0 + tx * 4 + j;
            if (o >= out) continue;
            float v = acc[i][j] + b[o];
            if (leaky) v = v > 0.0f ? v : 0.01f * v;
            y[r * out + o] = v;
        }
    }
}

// FP32 master -> BF16 W [out][ld_in] and W^T [in][ld_out] (pads zero)
__global__ void refresh_bf16(const float *__restrict__ W, int out, int in, __nv_bfloat16 *W16,
                             int ld_in, __nv_bfloat16 *WT16, int ld_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out * in) return;
    const int o = i / in, k = i - o * in;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
    W16[(size_t)o * ld_in + k] = v;
    WT16[(size_t)k * ld_out + o] = v;
}

// Reactive goal-seeking controller (the fallback policy without learning):
// among beams whose range and both neighbours' ranges exceed `clear` metres,
// head for the one closest in angle to the goal bearing; turn rate
// proportional to that heading error, speed reduced while turning or when
// the beam straight ahead is short.  Outputs normalised actions.
__global__ void reactive_kernel(const float *__restrict__ obs, long long stride, int n, int K,
                                float fov, float v_max, float w_max, float clear, float *act) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float *o = obs + (long long)r * stride;
    const float dgoal = o[K], phi = o[K + 1];
    const float step = fov / (float)K;
    float best = -2.0f, target = 0.0f;
    for (int k = 0; k < K; ++k) {
        const int km = k == 0 ? K - 1 : k - 1, kp = k == K - 1 ? 0 : k + 1;
        const float need = fminf(clear, dgoal + 0.1f);
        if (o[k] < need || o[km] < need || o[kp] < need) continue;
        const float a = -0.5f * fov + ((float)k + 0.5f) * step;
        const float sc = cosf(a - phi);
        if (sc > best) { best = sc; target = a; }
    }
    float w = 2.0f * target, v;
    if (best < -1.5f) { // boxed in: rotate in place
        w = w_max;
        v = 0.0f;
    } else {
        const int kf = (int)(0.5f * (float)K - 0.5f); // beam nearest straight ahead (360 deg fan)
        const float front = o[kf < 0 ? 0 : kf];
        v = v_max * fmaxf(0.0f, cosf(target)) * fminf(1.0f, front / 1.0f);
    }
    act[2 * r] = fminf(fmaxf(2.0f * v / v_max - 1.0f, -1.0f), 1.0f);
    act[2 * r + 1] = fminf(fmaxf(w / w_max, -1.0f), 1.0f);
}

} // namespace

int Mlp::init(const std::vector<int> &sizes, unsigned long long seed, std::string &err) {
    n_layers = (int)sizes.size() - 1;
    if (n_layers < 1 || n_layers > kMaxLayers) {
        err = "bad layer count";
        return NAV_E_INVAL;
    }
    // U(-1/sqrt(in), 1/sqrt(in)) for weights and biases, from the counter hash
    std::vector<float> host;
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = layer[l];
        L.in = sizes[l];
        L.out = sizes[l + 1];
        L.ld_in = (L.in + 7) / 8 * 8;
        L.ld_out = (L.out + 7) / 8 * 8;
        const size_t nw = (size_t)L.in * L.out;
        const float lim = 1.0f / std::sqrt((float)L.in);
        host.resize(nw + L.out);
        for (size_t i = 0; i < host.size(); ++i) {
            unsigned long long z = seed ^ ((unsigned long long)(l + 1) << 56) ^ (i * 0x9E3779B97F4A7C15ull);
            z += 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            host[i] = lim * (2.0f * ((float)(z >> 40) * (1.0f / 16777216.0f)) - 1.0f);
        }
        cudaError_t e = cudaSuccess;
        auto A = [&](void **p, size_t bytes) {
            if (e == cudaSuccess) e = cudaMalloc(p, bytes);
            if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
        };
        A((void **)&L.W, nw * 4);
        A((void **)&L.b, L.out * 4);
        A((void **)&L.W16, (size_t)L.out * L.ld_in * 2);
        A((void **)&L.WT16, (size_t)L.in * L.ld_out * 2);
        A((void **)&L.mW, nw * 4);
        A((void **)&L.vW, nw * 4);
        A((void **)&L.mb, L.out * 4);
        A((void **)&L.vb, L.out * 4);
        A((void **)&L.gW, nw * 4);
        A((void **)&L.gb, L.out * 4);
        if (e == cudaSuccess) e = cudaMemcpy(L.W, host.data(), nw * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(L.b, host.data() + nw, L.out * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            err = cudaGetErrorString(e);
            return NAV_E_CUDA;
        }
    }
    return refresh(nullptr) == 0 ? NAV_OK : NAV_E_CUDA;
}

void Mlp::release() {
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = layer[l];
        void *ps[] = {L.W, L.b, L.W16, L.WT16, L.mW, L.vW, L.mb, L.vb, L.gW, L.gb};
        for (void *p : ps)
            if (p) cudaFree(p);
        L = Layer{};
    }
    n_layers = 0;
}

int Mlp::refresh(void *stream) {
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = layer[l];
        const int n = L.in * L.out;
        refresh_bf16<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
            L.W, L.out, L.in, static_cast<__nv_bfloat16 *>(L.W16), L.ld_in,
            static_cast<__nv_bfloat16 *>(L.WT16), L.ld_out);
    }
    return (int)cudaGetLastError();
}

long long Mlp::num_params() const {
    long long n = 0;
    for (int l = 0; l < n_layers; ++l) n += (long long)layer[l].in * layer[l].out + layer[l].out;
    return n;
}

int Mlp::copy_params(float *host, bool to_host) {
    long long off = 0;
    for (int l = 0; l < n_layers; ++l) {
        Layer &L = layer[l];
        const size_t nw = (size_t)L.in * L.out;
        cudaError_t e;
        if (to_host) {
            e = cudaMemcpy(host + off, L.W, nw * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(host + off + nw, L.b, L.out * 4, cudaMemcpyDeviceToHost);
        } else {
            e = cudaMemcpy(L.W, host + off, nw * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(L.b, host + off + nw, L.out * 4, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return (int)e;
        off += (long long)nw + L.out;
    }
    return to_host ? 0 : refresh(nullptr);
}

// Forward through the tensor cores: x16 [n][layer0.ld_in] BF16 -> out32 [n][out]
// FP32; hidden activations h16[l] [n][act_ld(out_l)] and (if ht16) their
// transposes [out_l][n].
int Mlp::forward_tc(const void *x16, int n, void *const *h16, void *const *ht16, float *out32,
                    int *status, void *stream) const {
    const void *in = x16;
    int ld = layer[0].ld_in;
    for (int l = 0; l < n_layers; ++l) {
        const Layer &L = layer[l];
        const bool last = l == n_layers - 1;
        const int rc = launch_gemm_bf16(in, ld, L.W16, L.ld_in, n, L.out, L.in, L.b, last ? 0 : 1,
                                        last ? out32 : nullptr, L.out, last ? nullptr : h16[l],
                                        act_ld(L.out), (!last && ht16) ? ht16[l] : nullptr, n,
                                        status, stream);
        if (rc != 0) return rc;
        in = h16[l];
        ld = act_ld(L.out);
    }
    return 0;
}

int Mlp::forward_fp32(const float *x, long long ldx, int n, float *const *h32, float *out32,
                      void *stream) const {
    const float *in = x;
    long long ld = ldx;
    for (int l = 0; l < n_layers; ++l) {
        const Layer &L = layer[l];
        const bool last = l == n_layers - 1;
        float *y = last ? out32 : h32[l];
        const dim3 grid((unsigned)((n + kSgBM - 1) / kSgBM), (unsigned)((L.out + kSgBN - 1) / kSgBN));
        dense_fp32<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, ld, n, L.in, L.W, L.b,
                                                                        L.out, last ? 0 : 1, y);
        in = y;
        ld = L.out;
    }
    return (int)cudaGetLastError();
}

int launch_obs_to_bf16(const float *obs, int n, int dim, long long stride, const float *scale,
                       int ipap, const float *beta_dev, void *out, int ld, void *stream) {
    const dim3 tb(32, 8), grid((ld / 4 + 31) / 32, (n + 7) / 8);
    obs_to_bf16<<<grid, tb, 0, static_cast<cudaStream_t>(stream)>>>(
        obs, n, dim, stride, scale, ipap, beta_dev, static_cast<__nv_bfloat16 *>(out), ld);
    return (int)cudaGetLastError();
}

int launch_obs_to_fp32(const float *obs, int n, int dim, long long stride, const float *scale,
                       int ipap, const float *beta_dev, float *out, void *stream) {
    const long long tot = (long long)n * dim;
    obs_to_fp32<<<(unsigned)((tot + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        obs, n, dim, stride, scale, ipap, beta_dev, out);
    return (int)cudaGetLastError();
}

int launch_actor_head(const float *out4, int n, int mode, unsigned long long seed, unsigned step,
                      float *act, float *logp, float *eps, void *stream) {
    actor_head_fwd<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        out4, n, mode, seed, step, nullptr, 0, 0, 0, 0, act, logp, eps, nullptr, 0, 0);
    return (int)cudaGetLastError();
}

int launch_actor_head_ctr(const float *out4, int n, int mode, unsigned long long seed,
                          const unsigned long long *ctr, int which, unsigned mul, unsigned add,
                          float *act, float *logp, float *eps, void *stream, void *xc, int ldc,
                          int col0) {
    launch_pdl(actor_head_fwd, (n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream), out4, n,
               mode, seed, 0u, ctr, which, 1ull, mul, add, act, logp, eps,
               static_cast<__nv_bfloat16 *>(xc), ldc, col0);
    return (int)cudaGetLastError();
}

} // namespace flashnav

using namespace flashnav;

struct nav_policy {
    Mlp actor;
    int obs_dim = 0, max_batch = 0, n_hidden = 0, ipap = 0;
    std::string err;
    // inference scratch, sized for max_batch rows at create
    void *x16 = nullptr, *h16[kMaxLayers - 1] = {};
    float *x32 = nullptr, *out32 = nullptr, *h32[kMaxLayers - 1] = {};
    int *status = nullptr;
    float *scale = nullptr; // per-feature input scale (null: none)
    float *beta = nullptr;  // Eq. 2's beta (device float), used when ipap > 0
};

namespace flashnav {
Mlp *policy_actor(nav_policy *p) { return p ? &p->actor : nullptr; }
int policy_ipap(const nav_policy *p) { return p ? p->ipap : 0; }
int policy_obs_dim(const nav_policy *p) { return p ? p->obs_dim : 0; }
int policy_max_batch(const nav_policy *p) { return p ? p->max_batch : 0; }
const float *policy_scale(const nav_policy *p) { return p ? p->scale : nullptr; }
float *policy_beta(nav_policy *p) { return p ? p->beta : nullptr; }
} // namespace flashnav

extern "C" {

int nav_policy_create_ex(int obs_dim, int hidden, int n_hidden, int ipap_features,
                         float ipap_beta, int max_batch, uint64_t seed, nav_policy **out) {
    if (!out || obs_dim <= 0 || hidden <= 0 || n_hidden < 1 || n_hidden > kMaxLayers - 1 ||
        max_batch <= 0 || ipap_features < 0 || ipap_features > obs_dim ||
        (ipap_features > 0 && !(ipap_beta < 0.0f)))
        return NAV_E_INVAL;
    *out = nullptr;
    nav_policy *p = new (std::nothrow) nav_policy();
    if (!p) return NAV_E_NOMEM;
    p->obs_dim = obs_dim;
    p->max_batch = max_batch;
    p->n_hidden = n_hidden;
    p->ipap = ipap_features;
    std::vector<int> sizes(1, obs_dim);
    for (int l = 0; l < n_hidden; ++l) sizes.push_back(hidden);
    sizes.push_back(4);
    int rc = p->actor.init(sizes, seed, p->err);
    cudaError_t e = cudaSuccess;
    if (rc == NAV_OK) {
        const size_t mb = (size_t)max_batch;
        e = cudaMalloc(&p->x16, mb * act_ld(obs_dim) * 2);
        if (e == cudaSuccess) e = cudaMemset(p->x16, 0, mb * act_ld(obs_dim) * 2);
        if (e == cudaSuccess) e = cudaMalloc(&p->x32, mb * obs_dim * 4);
        for (int i = 0; i < n_hidden && e == cudaSuccess; ++i) {
            e = cudaMalloc(&p->h16[i], mb * act_ld(hidden) * 2);
            if (e == cudaSuccess) e = cudaMemset(p->h16[i], 0, mb * act_ld(hidden) * 2);
            if (e == cudaSuccess) e = cudaMalloc(&p->h32[i], mb * hidden * 4);
        }
        if (e == cudaSuccess) e = cudaMalloc(&p->out32, mb * 4 * 4);
        if (e == cudaSuccess) e = cudaMalloc(&p->status, 4);
        if (e == cudaSuccess) e = cudaMemset(p->status, 0, 4);
        if (e == cudaSuccess) e = cudaMalloc(&p->beta, 4);
        if (e == cudaSuccess) e = cudaMemcpy(p->beta, &ipap_beta, 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = NAV_E_CUDA;
    }
    if (rc != NAV_OK) {
        nav_policy_free(p);
        return rc;
    }
    *out = p;
    return NAV_OK;
}

int nav_policy_create(int obs_dim, int hidden, int max_batch, uint64_t seed, nav_policy **out) {
    return nav_policy_create_ex(obs_dim, hidden, 2, 0, -1.0f, max_batch, seed, out);
}

void nav_policy_free(nav_policy *p) {
    if (!p) return;
    p->actor.release();
    for (int i = 0; i < kMaxLayers - 1; ++i) {
        if (p->h16[i]) cudaFree(p->h16[i]);
        if (p->h32[i]) cudaFree(p->h32[i]);
    }
    void *ps[] = {p->x16, p->x32, p->out32, p->status, p->scale, p->beta};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete p;
}

int nav_policy_get_beta(const nav_policy *p, float *beta_host) {
    if (!p || !beta_host) return NAV_E_INVAL;
    return cudaMemcpy(beta_host, p->beta, 4, cudaMemcpyDeviceToHost) == cudaSuccess ? NAV_OK
                                                                                    : NAV_E_CUDA;
}

int64_t nav_policy_num_params(const nav_policy *p) { return p ? p->actor.num_params() : NAV_E_INVAL; }

int nav_policy_get_weights(nav_policy *p, float *host) {
    if (!p || !host) return NAV_E_INVAL;
    return p->actor.copy_params(host, true) == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_policy_set_weights(nav_policy *p, const float *host) {
    if (!p || !host) return NAV_E_INVAL;
    int rc = p->actor.copy_params(const_cast<float *>(host), false);
    if (rc == 0) rc = (int)cudaDeviceSynchronize();
    return rc == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_policy_act(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n, int mode,
                   uint64_t seed, uint32_t step, float *actions_dev, float *logp_dev,
                   float *out_dev, void *stream) {
    if (!p || !obs_dev || !actions_dev || n <= 0 || n > p->max_batch || obs_stride < p->obs_dim ||
        (mode != 0 && mode != 1))
        return NAV_E_INVAL;
    const int ld0 = p->actor.layer[0].ld_in;
    int rc = launch_obs_to_bf16(obs_dev, n, p->obs_dim, obs_stride, p->scale, p->ipap, p->beta,
                                p->x16, ld0, stream);
    if (rc == 0) rc = p->actor.forward_tc(p->x16, n, p->h16, nullptr, p->out32, p->status, stream);
    if (rc == 0) rc = launch_actor_head(p->out32, n, mode, seed, step, actions_dev, logp_dev, nullptr, stream);
    if (rc == 0 && out_dev)
        rc = (int)cudaMemcpyAsync(out_dev, p->out32, (size_t)n * 16, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
    return rc == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_policy_act_counted(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n,
                           int mode, uint64_t seed, uint64_t *step_dev, float *actions_dev,
                           float *logp_dev, float *out_dev, void *stream) {
    if (!p || !obs_dev || !actions_dev || !step_dev || n <= 0 || n > p->max_batch ||
        obs_stride < p->obs_dim || (mode != 0 && mode != 1))
        return NAV_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ld0 = p->actor.layer[0].ld_in;
    int rc = launch_obs_to_bf16(obs_dev, n, p->obs_dim, obs_stride, p->scale, p->ipap, p->beta,
                                p->x16, ld0, stream);
    if (rc == 0) rc = p->actor.forward_tc(p->x16, n, p->h16, nullptr, p->out32, p->status, stream);
    if (rc == 0) {
        unsigned long long *c = reinterpret_cast<unsigned long long *>(step_dev);
        k_bump<<<1, 1, 0, st>>>(c);
        rc = launch_actor_head_ctr(p->out32, n, mode, seed, c, 0, 1u, 0u, actions_dev, logp_dev,
                                   nullptr, stream);
    }
    if (rc == 0 && out_dev)
        rc = (int)cudaMemcpyAsync(out_dev, p->out32, (size_t)n * 16, cudaMemcpyDeviceToDevice, st);
    return rc == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_policy_act_fp32(nav_policy *p, const float *obs_dev, int64_t obs_stride, int n, int mode,
                        uint64_t seed, uint32_t step, float *actions_dev, float *logp_dev,
                        float *out_dev, void *stream) {
    if (!p || !obs_dev || !actions_dev || n <= 0 || n > p->max_batch || obs_stride < p->obs_dim ||
        (mode != 0 && mode != 1))
        return NAV_E_INVAL;
    const bool prep = p->scale || p->ipap > 0;
    int rc = prep ? launch_obs_to_fp32(obs_dev, n, p->obs_dim, obs_stride, p->scale, p->ipap,
                                       p->beta, p->x32, stream)
                  : 0;
    if (rc == 0)
        rc = p->actor.forward_fp32(prep ? p->x32 : obs_dev, prep ? p->obs_dim : obs_stride, n,
                                   p->h32, p->out32, stream);
    if (rc == 0) rc = launch_actor_head(p->out32, n, mode, seed, step, actions_dev, logp_dev, nullptr, stream);
    if (rc == 0 && out_dev)
        rc = (int)cudaMemcpyAsync(out_dev, p->out32, (size_t)n * 16, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
    return rc == 0 ? NAV_OK : NAV_E_CUDA;
}

int nav_policy_set_input_scale(nav_policy *p, const float *scale_host) {
    if (!p) return NAV_E_INVAL;
    if (!scale_host) {
        if (p->scale) cudaFree(p->scale);
        p->scale = nullptr;
        return NAV_OK;
    }
    cudaError_t e = cudaSuccess;
    if (!p->scale) e = cudaMalloc(&p->scale, (size_t)p->obs_dim * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->scale, scale_host, (size_t)p->obs_dim * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_reactive_act(const float *obs_dev, int64_t obs_stride, int n, int n_beams, float fov_deg,
                     float v_max, float w_max, float *actions_dev, void *stream) {
    if (!obs_dev || !actions_dev || n <= 0 || n_beams <= 0 || obs_stride < n_beams + 4 ||
        !(v_max > 0.0f) || !(w_max > 0.0f))
        return NAV_E_INVAL;
    reactive_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        obs_dev, obs_stride, n, n_beams, fov_deg * 0.017453292519943295f, v_max, w_max, 0.6f,
        actions_dev);
    return cudaGetLastError() == cudaSuccess ? NAV_OK : NAV_E_CUDA;
}

int nav_rollout(nav_handle *h, nav_policy *p, int n_steps, int mode, uint64_t seed,
                uint32_t step0, float *obs_dev, float *actions_dev, float *reward_dev,
                uint8_t *done_dev, int fp32_path) {
    HandleView hv;
    if (!h || !p || handle_view(h, &hv) != NAV_OK) return NAV_E_INVAL;
    if (!obs_dev || !actions_dev || !reward_dev || !done_dev || n_steps <= 0)
        return handle_fail(h, NAV_E_INVAL, "nav_rollout: bad argument");
    if (hv.uniform_d < 0 || hv.uniform_d + 4 != p->obs_dim || hv.n_envs > p->max_batch)
        return handle_fail(h, NAV_E_INVAL,
                           "nav_rollout: policy obs_dim / max_batch do not match the handle");
    for (int t = 0; t < n_steps; ++t) {
        int rc = fp32_path
                     ? nav_policy_act_fp32(p, obs_dev, p->obs_dim, hv.n_envs, mode, seed,
                                           step0 + (uint32_t)t, actions_dev, nullptr, nullptr,
                                           hv.stream)
                     : nav_policy_act(p, obs_dev, p->obs_dim, hv.n_envs, mode, seed,
                                      step0 + (uint32_t)t, actions_dev, nullptr, nullptr,
                                      hv.stream);
        if (rc != NAV_OK) return handle_fail(h, rc, "nav_rollout: policy launch failed");
        rc = nav_step(h, actions_dev, obs_dev, reward_dev, done_dev, nullptr);
        if (rc != NAV_OK) return rc;
    }
    return NAV_OK;
}

} // extern "C"
