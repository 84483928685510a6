// vans_static.cu -- vans_step_static: one step with no workspace and no device
// allocation, for callers that cannot hand the library any memory of its own
// (see include/vans.h).  The only scratch the step needs beyond the caller's
// buffers -- the padded copy of eps that the kernel reads -- lives in the
// file-scope array below, which the CUDA runtime places in device memory when
// the library is loaded on a device and keeps until the process exits.
#include <stdint.h>

#include <mutex>

#include "vans.h"
#include "vans_internal.h"

namespace {

// 4 Mi floats = 16 MiB per device: rows (ny*nz) x padded pitch must fit.  The
// last 64 floats hold the word the eps-padding kernel flags out-of-range values
// in (written, never read, in this path).
constexpr long long kStaticEpsFloats = 4LL * 1024 * 1024;
static __device__ __align__(256) float g_static_eps[kStaticEpsFloats + 64];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float *g_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_eps on the current device; looked up once per
// device (the host-side name is only a stand-in, never a device address).
float *static_eps_ptr(int dev) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_eps) != cudaSuccess) return nullptr;
        g_ptr[dev] = (float *)p;
    }
    return g_ptr[dev];
}

}  // namespace

extern "C" int vans_step_static(const vans_params *p, const float *eps_dev, const float *state_in,
                                float *state_out, void *cuda_stream) {
    if (!p || !eps_dev || !state_in || !state_out) return VANS_ERR_ARG;
    // the same parameter rules as vans_create, through its size query
    const long long n = vans_state_floats(p);
    if (n < 0) return VANS_ERR_ARG;
    if (p->wall_mask & 1) return VANS_ERR_UNSUPPORTED;
    // the pull reads state_in around every cell it writes in state_out, so the
    // two ranges must not overlap at all
    const uintptr_t a = (uintptr_t)state_in, b = (uintptr_t)state_out;
    const uintptr_t bytes = (uintptr_t)n * sizeof(float);
    if (a < b + bytes && b < a + bytes) return VANS_ERR_ARG;
    vans::VDom d;
    vans::fill_dom(p, d);
    if ((long long)d.rows * d.pitch > kStaticEpsFloats) return VANS_ERR_ARG;  // beyond the scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VANS_ERR_CUDA;
    float *eps_pad = static_eps_ptr(dev);
    if (!eps_pad) return VANS_ERR_CUDA;
    d.eps = eps_pad;

    cudaStream_t s = (cudaStream_t)cuda_stream;
    // every entry of the padded rows is rewritten, so the previous call's
    // contents never leak into this one; the range flag is not read here
    int *flag = (int *)(eps_pad + kStaticEpsFloats);
    if (vans::launch_pad_eps(d, eps_dev, eps_pad, flag, s) != cudaSuccess) return VANS_ERR_CUDA;
    const vans::Launch L = (p->q == 9) ? vans::Launch{4, 4, 1, 0} : vans::Launch{2, 4, 1, 0};
    if (vans::launch_step(p->q, d, state_in, state_out, L, s) != cudaSuccess) return VANS_ERR_CUDA;
    return VANS_OK;
}
