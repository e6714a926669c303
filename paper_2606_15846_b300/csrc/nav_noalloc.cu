// nav_step_host_noalloc: nav_step_host for callers that must not allocate
// device memory after start-up.
//
// nav_step_host stages actions, observations, rewards and flags in device
// buffers that it allocates with cudaMalloc on its first call.  Some callers
// cannot allow that: a robot control loop or an embedded process that sizes
// all of its GPU memory once at start-up and forbids allocation afterwards,
// or an application whose own allocator must own every device allocation.
// This entry point does the same work with its staging in one file-scope
// device array of fixed size (kStageBytes), which exists on every GPU that
// loads the library until the process exits; it calls no cudaMalloc,
// cudaFree or allocating library routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "nav_internal.h"

namespace {

constexpr size_t kStageBytes = (size_t)8 << 20; // 8 MiB
constexpr int kMaxDevices = 64;

// Staging for actions, obs, reward, done and final obs of one call.  Every
// call on a device shares it and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_stage[kStageBytes];

// Device address of g_stage per device.  In host code `g_stage` names a
// host-side stand-in, not device memory, so the address must come from
// cudaGetSymbolAddress with that device current.
unsigned char *g_stage_addr[kMaxDevices] = {};
std::mutex g_stage_mutex;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

} // namespace

using namespace flashnav;

extern "C" int nav_step_host_noalloc(nav_handle *h, const float *actions_host, float *obs_host,
                                     float *reward_host, uint8_t *done_host,
                                     float *final_obs_host) {
    HandleView hv;
    if (!h || handle_view(h, &hv) != NAV_OK) return NAV_E_INVAL;
    if (!actions_host || !obs_host || !reward_host || !done_host)
        return handle_fail(h, NAV_E_INVAL, "nav_step_host_noalloc: null argument");
    const size_t E = (size_t)hv.n_envs, O = (size_t)hv.obs_floats;
    const size_t off_obs = align256(8 * E);
    const size_t off_rew = off_obs + align256(4 * O);
    const size_t off_done = off_rew + align256(4 * E);
    const size_t off_fin = off_done + align256(E);
    const size_t need = final_obs_host ? off_fin + 4 * O : off_done + E;
    if (need > kStageBytes) {
        const std::string msg = "nav_step_host_noalloc: this handle needs " +
                                std::to_string(need) + " staging bytes; the fixed buffer holds " +
                                std::to_string(kStageBytes) + " (use nav_step_host)";
        return handle_fail(h, NAV_E_INVAL, msg.c_str());
    }
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess || cur != hv.device || cur < 0 || cur >= kMaxDevices)
        return handle_fail(h, NAV_E_INVAL,
                           "nav_step_host_noalloc: make the handle's device current first");
    unsigned char *base;
    {
        // one-time set-up per device (the first call on a device does it;
        // under lazy module loading this lookup loads this file's module and
        // places g_stage on the device, so that call should be made at
        // start-up)
        std::lock_guard<std::mutex> lock(g_stage_mutex);
        if (!g_stage_addr[cur]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_stage);
            if (e != cudaSuccess) {
                const std::string msg =
                    std::string("nav_step_host_noalloc: cudaGetSymbolAddress: ") +
                    cudaGetErrorString(e);
                return handle_fail(h, NAV_E_CUDA, msg.c_str());
            }
            g_stage_addr[cur] = static_cast<unsigned char *>(p);
        }
        base = g_stage_addr[cur];
    }
    cudaStream_t s = static_cast<cudaStream_t>(hv.stream);
    float *d_act = reinterpret_cast<float *>(base);
    float *d_obs = reinterpret_cast<float *>(base + off_obs);
    float *d_rew = reinterpret_cast<float *>(base + off_rew);
    uint8_t *d_done = base + off_done;
    float *d_fin = final_obs_host ? reinterpret_cast<float *>(base + off_fin) : nullptr;
    // the array keeps the previous call's contents: rows of the final obs
    // that this step does not write (envs that did not finish) are cleared
    if (d_fin) e = cudaMemsetAsync(d_fin, 0, 4 * O, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_act, actions_host, 8 * E, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return handle_fail(h, NAV_E_CUDA, "nav_step_host_noalloc: staging actions failed");
    int rc = nav_step(h, d_act, d_obs, d_rew, d_done, d_fin);
    if (rc != NAV_OK) return rc;
    e = cudaMemcpyAsync(obs_host, d_obs, 4 * O, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(reward_host, d_rew, 4 * E, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(done_host, d_done, E, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_fin)
        e = cudaMemcpyAsync(final_obs_host, d_fin, 4 * O, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        const std::string msg =
            std::string("nav_step_host_noalloc: ") + cudaGetErrorString(e);
        return handle_fail(h, NAV_E_CUDA, msg.c_str());
    }
    return NAV_OK;
}
