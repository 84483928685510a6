// vans_static.cu -- vans_step_static: one step with no workspace and no device
// allocation, for callers that cannot hand the library any memory of its own
// (see include/vans.h).  The only scratch the step needs beyond the caller's
// buffers -- the padded copy of eps that the kernel reads -- lives in the
// file-scope array below, which the CUDA runtime places in device memory when
// the library is loaded on a device and keeps until the process exits.
#include <math.h>

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

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace

extern "C" int vans_step_static(const vans_params *p, const float *eps_dev, const float *state_in,
                                float *state_out, void *cuda_stream) {
    if (!p || !eps_dev || !state_in || !state_out || state_in == state_out) return VANS_ERR_ARG;
    // the same parameter rules as vans_create, through its size query
    if (vans_state_floats(p) < 0) return VANS_ERR_ARG;
    if (p->wall_mask & 1) return VANS_ERR_UNSUPPORTED;
    const int pitch = (int)round_up(VANS_OFF + round_up(p->nx, 128) + 1, 32);
    const long long rows = (long long)p->ny * p->nz;
    if (rows * pitch > kStaticEpsFloats) return VANS_ERR_ARG;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VANS_ERR_CUDA;
    float *eps_pad = static_eps_ptr(dev);
    if (!eps_pad) return VANS_ERR_CUDA;

    vans::VDom d{};
    d.q = p->q;
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.rows = (int)rows;
    d.pitch = pitch;
    d.plane = rows * pitch;
    d.wall_y = (p->wall_mask >> 1) & 1;
    d.wall_z = (p->wall_mask >> 2) & 1;
    const double tau = p->tau;
    d.omega = (float)(1.0 / tau);
    d.ctau = (float)(1.0 - 0.5 / tau);
    d.g[0] = p->g[0];
    d.g[1] = p->g[1];
    d.g[2] = (p->q == 19) ? p->g[2] : 0.f;
    d.drag_mode = p->drag_mode;
    d.k_mode = p->k_mode;
    const double nu = (tau - 0.5) / 3.0;
    if (p->k_mode == 0) {
        d.ca = (float)(150.0 * nu / ((double)p->d_p * p->d_p));
        d.cb = (float)(1.75 / p->d_p);
    } else if (p->k_mode == 1) {
        d.ca = (float)(nu / p->K);
        d.cb = (float)(p->F_eps / sqrt((double)p->K));
    } else {
        d.ca = (float)(nu / p->K);
        d.cb = (float)(1.75 / sqrt(150.0 * p->K));
    }
    d.cells = (long long)p->nx * p->ny * p->nz;
    d.uw[0] = p->u_wall[0];
    d.uw[1] = p->u_wall[1];
    d.uw[2] = (p->q == 19) ? p->u_wall[2] : 0.f;
    d.nee = (p->wall_kind == 1) ? 1 : 0;
    // the bounce-back gain of a moving wall; plates on nodes impose u_wall directly
    d.moving = (!d.nee && (d.uw[0] != 0.f || d.uw[1] != 0.f || d.uw[2] != 0.f)) ? 1 : 0;
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
