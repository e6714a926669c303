// Private declarations of the MLP pieces shared by nav_policy.cu and
// nav_learn.cu.  Not part of the public ABI.
#pragma once
#include <string>
#include <vector>

namespace flashnav {

constexpr float kLogStdMin = -5.0f; // actor log-std range (Table 4)
constexpr float kLogStdMax = 0.0f;
constexpr int kMaxLayers = 5; // up to four hidden layers and the output layer

// Leading dimension (elements) of a BF16 activation row of n features: the
// tensor-core GEMM reads K-major rows that start on 16-byte boundaries, and
// the fused passes read whole 16-column groups.
inline int act_ld(int n) { return (n + 15) / 16 * 16; }

// One dense layer: FP32 master weights W [out][in] and bias, BF16 copies for
// the tensor cores (W16 [out][ld_in], WT16 [in][ld_out]), Adam moments and
// gradient buffers.
struct Layer {
    int in = 0, out = 0, ld_in = 0, ld_out = 0;
    float *W = nullptr, *b = nullptr;
    void *W16 = nullptr, *WT16 = nullptr;
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    float *gW = nullptr, *gb = nullptr;
};

struct Mlp {
    Layer layer[kMaxLayers];
    int n_layers = 0;
    int init(const std::vector<int> &sizes, unsigned long long seed, std::string &err);
    void release();
    int refresh(void *stream); // FP32 master -> BF16 copies
    long long num_params() const;
    int copy_params(float *host, bool to_host); // [W0, b0, W1, b1, ...]
    int forward_tc(const void *x16, int n, void *const *h16, void *const *ht16, float *out32,
                   int *status, void *stream) const;
    int forward_fp32(const float *x, long long ldx, int n, float *const *h32, float *out32,
                     void *stream) const;
};

// Observation rows -> network input: features c < ipap become
// 1 / (l - beta) (Eq. 2, beta read from beta_dev), then every feature is
// multiplied by scale[c] (if scale is set).  BF16 [n][ld] (zero pad) for the
// tensor cores, or FP32 [n][dim] for the SIMT path.
int launch_obs_to_bf16(const float *obs, int n, int dim, long long stride, const float *scale,
                       int ipap, const float *beta_dev, void *out, int ld, void *stream);
int launch_obs_to_fp32(const float *obs, int n, int dim, long long stride, const float *scale,
                       int ipap, const float *beta_dev, float *out, void *stream);
int launch_actor_head(const float *out4, int n, int mode, unsigned long long seed, unsigned step,
                      float *act, float *logp, float *eps, void *stream);
// The same with the noise step mul * (ctr[which] - 1) + add read on the device;
// with xc set, the actions are also stored as BF16 in columns col0, col0 + 1
// of the rows of xc (leading dimension ldc).
int launch_actor_head_ctr(const float *out4, int n, int mode, unsigned long long seed,
                          const unsigned long long *ctr, int which, unsigned mul, unsigned add,
                          float *act, float *logp, float *eps, void *stream, void *xc = nullptr,
                          int ldc = 0, int col0 = 0);

// ---------------------------------------------------------------------------
// Fused passes for small networks (every layer's in and out <= 128, batch a
// multiple of 128): one CTA per 128 batch rows runs every
// layer of a network with its operands in shared memory and accumulators in
// TMEM; grid.y selects one of up to four networks (e.g. the twin critics and
// their targets, each on its own input).
// ---------------------------------------------------------------------------
constexpr int kFusedMaxWidth = 128;

struct FLayer {
    const void *W16, *WT16; // BF16 [out][ld_in] and [in][ld_out]
    const float *b;
    int ld_in, ld_out, in, out;
};

struct FNet {
    FLayer L[kMaxLayers];
    int n_layers;
    // forward: X [B][ldx] (K = L[0].in) -> out32 [B][n_out]; optional saves of
    // every hidden activation, H16 [B][ldh] and HT16 [H][B]
    const void *X;
    int ldx;
    float *out32;
    void *H16[kMaxLayers - 1], *HT16[kMaxLayers - 1];
    int ldh;
    // LeakyReLU' of every hidden activation as sign bits, [B][4] words per
    // layer (bit c of word w: activation 32 w + c > 0); written by the
    // forward when set, read by the backward
    unsigned *M[kMaxLayers - 1];
    // backward: dout [B][n_out] -> per-CTA partial gradients, CTA c's at
    // gWp[l] + c cta_stride ([out][in]) and gbp[l] + c cta_stride ([out])
    // (gWp[l] null: that layer's gradients are not formed),
    // input gradient dX [B][lddx] (null: none); XT [in0][B] for layer 0's dW
    const float *dout;
    const void *XT;
    float *gWp[kMaxLayers], *gbp[kMaxLayers];
    long long cta_stride; // floats between two CTAs' partials
    float *dX;
    int lddx;
};

constexpr int kFusedMaxNets = 4; // networks one fused launch walks (grid.y)
struct FGroup {
    FNet net[kFusedMaxNets];
    int n_nets, B;
    int *status;
};

// True when the net fits the fused passes.
bool fused_ok(const Mlp &m, int B);
// Fills the layer table of an FNet from an Mlp (io fields untouched).
void fused_layers(const Mlp &m, FNet &f);
int launch_mlp_fwd_fused(const FGroup &g, void *stream);
int launch_mlp_bwd_fused(const FGroup &g, void *stream);

// One Adam / AdamW step on every parameter of up to two networks, whose
// gradients are the sums of n_cta partials (written back to gW / gb for
// inspection), or, with gWp_base null, the layers' gW / gb themselves; BF16
// copies refreshed.  corr: device bias corrections.
// With `targets` (networks of the same shapes), each target parameter also
// takes its Polyak step target <- (1 - tau) target + tau new in the same
// pass, its BF16 copies refreshed.
int launch_adam_fused(Mlp *const *nets, float *const *gWp_base, int n_nets, int n_cta, float lr,
                      float b1, float b2, const float *corr, float wd, void *stream,
                      Mlp *const *targets = nullptr, float tau = 0.0f);
// Polyak averaging tgt <- (1 - tau) tgt + tau src of up to two networks, with
// the targets' BF16 copies refreshed.
int launch_polyak_fused(Mlp *const *tgt, Mlp *const *src, int n_nets, float tau, void *stream);

} // namespace flashnav

struct nav_policy;
namespace flashnav {
// The actor network inside a policy handle (weights shared with a trainer
// through nav_trainer_sync_policy), its IPAPRec feature count and the device
// float holding its beta.
Mlp *policy_actor(nav_policy *p);
int policy_ipap(const nav_policy *p);
int policy_obs_dim(const nav_policy *p);
int policy_max_batch(const nav_policy *p);
const float *policy_scale(const nav_policy *p); // per-feature input scale (null: none)
float *policy_beta(nav_policy *p);
} // namespace flashnav
