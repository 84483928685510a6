// vans_api.cu -- host runtime behind the C ABI of include/vans.h: parameter
// validation, workspace layout, the ping-pong state, CUDA-graph replay of long
// step sequences, the launch-configuration autotuner and the batched tile list.
// The library allocates no device memory: everything lives in the caller's
// workspace.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <iterator>
#include <vector>

#include "vans.h"
#include "vans_internal.h"

using vans::Launch;
using vans::Tile;
using vans::VDom;

namespace {

// Step sequences are replayed from captured CUDA graphs of 64, 32, ..., 2
// steps (even lengths restore the buffer parity): a run of n steps is the
// binary decomposition of n, so even short runs leave the per-launch overhead
// of single launches behind (about 3 us of a 200 us step on GB300).
constexpr int kGraphSizes = 6;
constexpr int kGraphSteps = 64;   // the longest graph; size k holds kGraphSteps >> k steps

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// floats of one state buffer (Q planes of rows*pitch), rounded to 256 bytes
using vans::pitch_for;

long long state_floats_of(int q, int nx, int ny, int nz) {
    const long long plane = (long long)ny * nz * pitch_for(q, nx);
    return round_up((long long)q * plane, 64);
}

long long eps_floats_of(int q, int nx, int ny, int nz) {
    return round_up((long long)ny * nz * pitch_for(q, nx), 64);
}

constexpr long long kFlagFloats = 64;   // 256 bytes of status words
constexpr long long kMonFloats = 3 * vans::kMonSlots;   // partial maxima of vans_step_monitored

int validate(const vans_params *p, bool batched) {
    if (!p) return VANS_ERR_ARG;
    if (p->q != 9 && p->q != 19) return VANS_ERR_ARG;
    if (batched && p->q != 9) return VANS_ERR_UNSUPPORTED;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return VANS_ERR_ARG;
    if (p->q == 9 && p->nz != 1) return VANS_ERR_ARG;
    if (p->wall_mask & ~7) return VANS_ERR_ARG;
    if (p->wall_mask & 1) return VANS_ERR_UNSUPPORTED;
    if (p->q == 9 && (p->wall_mask & 4)) return VANS_ERR_ARG;
    if (!(p->tau > 0.5f) || !isfinite(p->tau)) return VANS_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(p->g[k]) || !isfinite(p->u_wall[k])) return VANS_ERR_ARG;
    const bool moving = p->u_wall[0] != 0.f || p->u_wall[1] != 0.f || p->u_wall[2] != 0.f;
    if (moving && !(p->wall_mask & 2)) return VANS_ERR_ARG;     // the plate is a y wall
    if (p->wall_kind != 0 && p->wall_kind != 1) return VANS_ERR_ARG;
    if (p->wall_kind == 1) {
        // plates on nodes: y walls only, at least one fluid row between them
        if (!(p->wall_mask & 2) || p->ny < 3) return VANS_ERR_ARG;
        if ((p->wall_mask & 4) || batched) return VANS_ERR_UNSUPPORTED;
    }
    if (p->drag_mode < 0 || p->drag_mode > 2) return VANS_ERR_ARG;
    if (p->k_mode < 0 || p->k_mode > 2) return VANS_ERR_ARG;
    if (p->drag_mode != 0) {
        if (p->k_mode == 0 && !(p->d_p > 0.f && isfinite(p->d_p))) return VANS_ERR_ARG;
        if (p->k_mode != 0 && !(p->K > 0.f && isfinite(p->K))) return VANS_ERR_ARG;
        if (p->k_mode == 1 && !(p->F_eps >= 0.f && isfinite(p->F_eps))) return VANS_ERR_ARG;
    }
    // index arithmetic limits: rows and columns are int, offsets 64-bit
    const long long rows = (long long)p->ny * p->nz;
    if (rows > (1LL << 30) || p->nx > (1 << 28)) return VANS_ERR_ARG;
    return VANS_OK;
}

bool launch_ok(const vans_launch *c, int q, bool batched) {
    if (!c) return false;
    if (c->cpt != 1 && c->cpt != 2 && c->cpt != 4) return false;
    if (c->ctas < 0 || c->ctas > 4) return false;
    if (c->kind == 0) {
        if (c->ctas != 0) return false;
        if (c->warps < 1 || c->warps > 8 || c->rows < 1 || c->rows > 8) return false;
        return c->warps * c->rows <= 8;
    }
    if (c->kind == 8)       // cluster-resident steps: cluster of up to `rows` CTAs
        return !batched && c->cpt == 1 && c->ctas == 0 && (c->warps == 8 || c->warps == 16) &&
               c->rows >= 2 && c->rows <= 16;
    // kinds 1 and 3 are not built (never the fastest at any measured size)
    if (c->kind < 2 || c->kind > 7 || c->kind == 3) return false;
    if (c->rows < 2 || c->rows > 6) return false;
    // the instantiated pipeline shapes
    const int nt = 32 * c->warps;
    if (c->kind == 7 && q == 19 && (nt == 96 || nt == 160 || nt == 192))
        // 192-, 320-, 384-cell D3Q19 tiles
        return c->cpt == 2 && !batched;
    if (c->kind == 5 || c->kind == 7)
        return (nt == 64 || nt == 128) && c->cpt == (q == 9 ? 4 : 2) && (q == 9 || !batched);
    if (c->kind == 6)
        return q == 9 ? (c->cpt == 2 && (nt == 128 || nt == 256))
                      : (c->cpt == 1 && (nt == 128 || nt == 256) && !batched);
    if (q == 9)
        return (nt == 128 && (c->cpt == 2 || c->cpt == 4)) || (nt == 256 && c->cpt <= 2);
    return (nt == 128 && c->cpt <= 2) || (nt == 256 && c->cpt == 1);
}

}  // namespace

namespace vans {

int pitch_for(int q, int nx) {
    return (int)((col0_for(q) + ((long long)nx + 127) / 128 * 128 + 1 + 31) / 32 * 32);
}

// Host-side constants of the drag law: alpha = ca * a(eps), beta = cb * b(eps).
void fill_dom(const vans_params *p, VDom &d) {
    memset(&d, 0, sizeof(d));
    d.q = p->q;
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.rows = p->ny * p->nz;
    d.pitch = pitch_for(p->q, p->nx);
    d.off = col0_for(p->q);
    d.xwrap = 1;
    d.plane = (long long)d.rows * d.pitch;
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
    const double nu = (tau - 0.5) / 3.0;        // nu = cs^2 (tau - 1/2)
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
}

}  // namespace vans

struct vans_s {
    bool batched = false;
    int q = 9;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;                 // private stream for graph capture
    int device = 0;
    long long launches = 0;
    Launch L{4, 4, 1, 0};
    cudaGraphExec_t gexec[kGraphSizes] = {};   // 64, 32, ..., 2 steps
    int *flag = nullptr;                        // device status words (workspace)
    float *mon_part = nullptr;                  // monitoring partial maxima (workspace)
    int adj_fp64 = 0;                           // reverse-step arithmetic in FP64
    Launch adjL{1, 4, 4, 1};                    // reverse-step launch shape
    // single domain
    vans_params p{};
    VDom dom{};
    float *st[2] = {nullptr, nullptr};
    int cur = 0;
    float *eps_pad = nullptr;
    bool eps_set = false;
    bool slab = false;                          // x halos come from neighbouring slabs
    long long sfloats = 0;
    // batched
    int n = 0;
    std::vector<vans_params> bp;
    std::vector<VDom> doms;                     // host copy of the device table
    VDom *doms_d = nullptr;
    Tile *tiles_d = nullptr;
    long long tile_cap = 0;
    std::vector<Tile> tiles;
    int grid = 0;
    int parity = 0;
    std::vector<char> dom_ready;
    // captured reverse-pass segments (adjoint), keyed by their buffers and length
    struct SegGraph {
        const float *seg;
        int len;
        const float *lam, *tmp, *grad;
        cudaGraphExec_t exec;
    };
    std::vector<SegGraph> seg_graphs;
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? VANS_OK : VANS_ERR_CUDA; }

void drop_graph(vans_t h) {
    for (auto &g : h->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    for (auto &g : h->seg_graphs) cudaGraphExecDestroy(g.exec);
    h->seg_graphs.clear();
}

// one batched step with the handle's launch (strip kernels for kinds 2, 4, 5)
cudaError_t batched_step(vans_t h, cudaStream_t s, int par) {
    if (h->L.kind != 0)
        return vans::launch_ring_batched(h->doms_d, h->tiles_d, (int)h->tiles.size(), par, h->L,
                                         h->flag + 1, s);
    return vans::launch_step_batched(h->doms_d, h->tiles_d, (int)h->tiles.size(), par, h->L,
                                     h->grid, s);
}

cudaError_t one_step(vans_t h, cudaStream_t s, int par) {
    ++h->launches;
    if (h->batched) return batched_step(h, s, par);
    return vans::launch_step(h->q, h->dom, h->st[par], h->st[par ^ 1], h->L, s);
}

// capture the graph of n steps starting at parity 0
int capture_steps(vans_t h, int n, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return VANS_ERR_CUDA;
    const long long before = h->launches;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < n && le == cudaSuccess; ++s) le = one_step(h, h->cap, s & 1);
    h->launches = before;                       // capture does not run anything
    e = cudaStreamEndCapture(h->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return VANS_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return VANS_ERR_CUDA;
    }
    return VANS_OK;
}

// all graph sizes at once, so the first run that needs any of them pays the
// capture for every later run length
int ensure_graph(vans_t h) {
    if (h->gexec[0]) return VANS_OK;
    for (int k = 0; k < kGraphSizes; ++k) {
        const int rc = capture_steps(h, kGraphSteps >> k, &h->gexec[k]);
        if (rc) {
            drop_graph(h);
            return rc;
        }
    }
    return VANS_OK;
}

// nsteps steps; the parity lives in h->cur (single) or h->parity (batched)
int run_steps(vans_t h, int nsteps) {
    int &par = h->batched ? h->parity : h->cur;
    if (!h->batched && h->L.kind == 8 && nsteps > 0) {
        // all the steps in one launch; the result lands where the step-by-step
        // run would leave it
        ++h->launches;
        if (vans::launch_step_cluster(h->q, h->dom, h->st[par], h->st[par ^ (nsteps & 1)], nsteps,
                                      h->L, h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
        par ^= nsteps & 1;
        return VANS_OK;
    }
    int left = nsteps;
    if (left >= 2) {
        if (par != 0) {
            if (one_step(h, h->stream, par) != cudaSuccess) return VANS_ERR_CUDA;
            par ^= 1;
            --left;
        }
        if (left >= 2) {
            int rc = ensure_graph(h);
            if (rc) return rc;
            for (int k = 0; k < kGraphSizes; ++k) {
                const int n = kGraphSteps >> k;
                while (left >= n) {
                    if (cudaGraphLaunch(h->gexec[k], h->stream) != cudaSuccess) return VANS_ERR_CUDA;
                    h->launches += n;
                    left -= n;
                }
            }
        }
    }
    while (left > 0) {
        if (one_step(h, h->stream, par) != cudaSuccess) return VANS_ERR_CUDA;
        par ^= 1;
        --left;
    }
    return VANS_OK;
}

int make_streams(vans_t h, void *stream) {
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) return VANS_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) return VANS_ERR_CUDA;
    return VANS_OK;
}

// read the status words (flag[0]: range / divergence, flag[1]: a bounded
// wait in a kernel timed out, flag[2]: the porosity of the last
// vans_set_eps_async was out of range); synchronises the stream
int read_flag(vans_t h, int *value, int *timeout = nullptr, int *eps_bad = nullptr) {
    int v[3] = {0, 0, 0};
    if (cudaMemcpyAsync(v, h->flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    *value = v[0];
    if (timeout) *timeout = v[1];
    if (eps_bad) *eps_bad = v[2];
    return VANS_OK;
}

// The rest state after a new porosity: the current buffer all zeros (the
// deviations of f = w eps), plus the moving wall's gain.  The other buffer is
// written whole (every cell and halo column) by the next step before anything
// reads it, and its row padding is never read into a stored value.
int reset_to_rest(vans_t h) {
    if (cudaMemsetAsync(h->st[0], 0, h->sfloats * sizeof(float), h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    if (h->dom.moving) {
        ++h->launches;
        if (vans::launch_init_moving(h->q, h->dom, h->st[0], h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
    }
    h->cur = 0;
    h->eps_set = true;
    if (h->slab) drop_graph(h);
    h->slab = false;
    h->dom.xwrap = 1;
    return VANS_OK;
}

constexpr int kStripRows = 32;   // rows per strip of the batched pipeline kernel

void build_tiles(vans_t h, const Launch &L, std::vector<Tile> &out) {
    out.clear();
    const int bx = 32 * L.cpt * L.warps;
    if (L.kind == 6 || L.kind == 7) {
        // every row of every domain in column blocks, domain after domain: the
        // persistent CTAs take tiles b, b + G, ... of this order
        for (int d = 0; d < h->n; ++d) {
            const VDom &D = h->doms[d];
            for (int r = 0; r < D.rows; ++r)
                for (int x = 0; x < D.nx; x += bx) out.push_back(Tile{d, r, x, 0});
        }
        return;
    }
    if (L.kind != 0) {
        // strips of up to kStripRows rows per column block.  The column blocks
        // of one band of rows stay next to each other in the table, so their
        // CTAs run at the same time and the 128-byte line two neighbouring
        // blocks both stage (the halo column of each) comes from DRAM once;
        // bands go largest first (rows x the domain's width), so the last wave
        // of CTAs holds the short ones
        for (int d = 0; d < h->n; ++d) {
            const VDom &D = h->doms[d];
            const int per_y = (D.ny + kStripRows - 1) / kStripRows;
            for (int yc = 0; yc < per_y; ++yc) {
                const int y0 = (int)((long long)yc * D.ny / per_y);
                const int y1 = (int)((long long)(yc + 1) * D.ny / per_y);
                for (int x = 0; x < D.nx; x += bx) out.push_back(Tile{d, y0, x, y1});
            }
        }
        std::stable_sort(out.begin(), out.end(), [&](const Tile &a, const Tile &b) {
            const long long wa = (long long)(a.pad - a.row) * h->doms[a.dom].nx;
            const long long wb = (long long)(b.pad - b.row) * h->doms[b.dom].nx;
            return wa > wb;
        });
        return;
    }
    for (int d = 0; d < h->n; ++d) {
        const VDom &D = h->doms[d];
        for (int r = 0; r < D.rows; r += L.rows)
            for (int x = 0; x < D.nx; x += bx) out.push_back(Tile{d, r, x, 0});
    }
}

int set_batch_launch(vans_t h, const Launch &L) {
    std::vector<Tile> t;
    build_tiles(h, L, t);
    if ((long long)t.size() > h->tile_cap) return VANS_ERR_ARG;
    if (cudaMemcpyAsync(h->tiles_d, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    h->tiles.swap(t);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (sms <= 0) sms = 1;
    h->grid = sms * vans::batched_blocks_per_sm(L);
    h->L = L;
    drop_graph(h);
    return VANS_OK;
}

// Fastest of three timed trials (after two untimed) of `reps` launches
// replayed as one CUDA graph, as run_steps issues them: one noisy trial does
// not decide the pick, and small domains are not judged by a launch overhead
// that the graph replay does not pay.  fn(stream) issues one launch; a shape
// that fails to launch or capture scores 1e30.
template <class F>
float time_launches(vans_t h, F &&fn, int reps) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return 1e30f;
    }
    bool ok = true;
    for (int i = 0; i < reps && ok; ++i) ok = fn(h->cap) == cudaSuccess;
    const cudaError_t ec = cudaStreamEndCapture(h->cap, &g);
    if (!ok || ec != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return 1e30f;
    }
    cudaGraphDestroy(g);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int i = 0; i < 2; ++i) cudaGraphLaunch(ge, h->stream);
    float best = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
        cudaEventRecord(a, h->stream);
        cudaGraphLaunch(ge, h->stream);
        cudaEventRecord(b, h->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess) ms = 1e30f;
        else cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGraphExecDestroy(ge);
    return best;
}

std::vector<Launch> candidates(int q, bool batched) {
    std::vector<Launch> c;
    const int cpts[3] = {1, 2, 4};
    for (int cpt : cpts)
        for (int warps = 1; warps <= 8; warps *= 2)
            for (int rows = 1; rows <= 4; rows *= 2) {
                if (warps * rows > 8 || warps * rows < 2) continue;
                if (q == 19 && cpt == 4 && warps * rows > 4) continue;
                c.push_back(Launch{cpt, warps, rows, 0});
            }
    if (batched) {
        const Launch t[] = {{2, 4, 3, 2}, {4, 4, 2, 2}, {4, 4, 3, 2}, {2, 8, 2, 2}, {2, 8, 3, 2},
                            {1, 8, 3, 2}, {2, 8, 2, 4}, {2, 4, 2, 4}, {4, 2, 2, 5}, {4, 2, 3, 5},
                            {4, 4, 2, 5}, {4, 4, 3, 5}, {4, 4, 4, 5}, {2, 4, 2, 6}, {2, 8, 2, 6},
                            {4, 2, 4, 7}, {4, 2, 3, 7}, {4, 4, 2, 7}, {4, 4, 4, 7},
                            {4, 4, 2, 5, 2}, {4, 4, 2, 7, 2}, {4, 4, 3, 7, 2},
                            {2, 4, 2, 2}, {2, 4, 4, 2}, {2, 4, 3, 4}};
        c.insert(c.end(), std::begin(t), std::end(t));
        return c;
    }
    // bulk-copy pipeline shapes {cpt, warps, stages, kind}
    if (q == 9) {
        const Launch t[] = {{2, 4, 3, 2}, {2, 4, 4, 2}, {4, 4, 3, 2}, {1, 8, 3, 2},
                            {1, 8, 4, 2}, {2, 8, 3, 2}, {2, 8, 2, 4}, {4, 4, 2, 4},
                            {4, 2, 2, 5}, {4, 4, 2, 5}, {4, 4, 4, 5}, {4, 4, 5, 5},
                            {4, 4, 6, 5}, {2, 8, 2, 6}, {2, 4, 2, 6}, {4, 4, 4, 7},
                            {4, 2, 4, 7}, {4, 4, 2, 7}, {4, 4, 2, 5, 2}, {4, 4, 3, 5, 2},
                            {4, 4, 2, 7, 2}, {4, 4, 3, 7, 2}, {4, 4, 2, 7, 3}};
        c.insert(c.end(), std::begin(t), std::end(t));
    } else {
        const Launch t[] = {{1, 4, 3, 2}, {2, 4, 2, 2}, {2, 4, 3, 2}, {1, 8, 2, 2},
                            {1, 8, 3, 2}, {1, 4, 3, 4}, {1, 8, 2, 4}, {2, 4, 2, 5},
                            {2, 4, 3, 5}, {2, 4, 4, 5}, {2, 2, 3, 5}, {1, 4, 3, 6},
                            {1, 8, 3, 6}, {2, 4, 3, 7}, {2, 2, 3, 7}, {2, 4, 2, 7},
                            {2, 4, 2, 7, 2}, {2, 4, 2, 7, 1}, {2, 4, 3, 7, 1}, {2, 4, 3, 7, 2},
                            {2, 4, 2, 5, 2}, {2, 2, 2, 7}, {2, 2, 4, 7}, {2, 6, 2, 7},
                            {2, 3, 2, 7}, {2, 3, 3, 7}, {2, 5, 2, 7}};
        c.insert(c.end(), std::begin(t), std::end(t));
    }
    // cluster-resident multi-step shapes {1, warps, largest cluster, 8}; the
    // autotuner skips those whose cluster cannot hold the domain
    const Launch k8[] = {{1, 8, 16, 8}, {1, 16, 16, 8}, {1, 8, 8, 8}, {1, 16, 8, 8}};
    c.insert(c.end(), std::begin(k8), std::end(k8));
    return c;
}

}  // namespace

// ===================================================================== ABI ==
extern "C" {

long long vans_state_floats(const vans_params *p) {
    if (validate(p, false) != VANS_OK) return -1;
    return state_floats_of(p->q, p->nx, p->ny, p->nz);
}

size_t vans_workspace_bytes(const vans_params *p) {
    if (validate(p, false) != VANS_OK) return 0;
    const long long f = 2 * state_floats_of(p->q, p->nx, p->ny, p->nz) +
                        eps_floats_of(p->q, p->nx, p->ny, p->nz) + kFlagFloats + kMonFloats;
    return (size_t)f * sizeof(float);
}

int vans_create(const vans_params *p, void *workspace, size_t workspace_bytes, void *cuda_stream,
                vans_t *out) {
    if (!out) return VANS_ERR_ARG;
    *out = nullptr;
    const int v = validate(p, false);
    if (v) return v;
    if (!workspace || ((uintptr_t)workspace & 255)) return VANS_ERR_ARG;
    if (workspace_bytes < vans_workspace_bytes(p)) return VANS_ERR_ARG;
    vans_t h = new (std::nothrow) vans_s();
    if (!h) return VANS_ERR_ARG;
    h->q = p->q;
    h->p = *p;
    vans::fill_dom(p, h->dom);
    h->sfloats = state_floats_of(p->q, p->nx, p->ny, p->nz);
    float *w = (float *)workspace;
    h->st[0] = w;
    h->st[1] = w + h->sfloats;
    h->eps_pad = w + 2 * h->sfloats;
    h->flag = (int *)(h->eps_pad + eps_floats_of(p->q, p->nx, p->ny, p->nz));
    h->dom.eps = h->eps_pad;
    h->dom.status = h->flag + 1;
    h->mon_part = (float *)(h->flag + kFlagFloats);
    h->L = (p->q == 9) ? Launch{4, 4, 1, 0} : Launch{2, 4, 1, 0};
    // the pipelined reverse step, one cell per thread, 4 stages: fastest on GB300 at 512^2
    // (backward pass 17.4 us per step against 20.8 with the register-load kernel)
    h->adjL = (p->q == 19) ? Launch{1, 4, 2, 1} : Launch{1, 4, 4, 1};   // D3Q19: 0.78 vs 0.61 of HBM
    int rc = make_streams(h, cuda_stream);
    if (rc) {
        vans_destroy(h);
        return rc;
    }
    // a defined padding (1.0 porosity, zero deviations) for lanes past nx
    if (cudaMemsetAsync(workspace, 0, vans_workspace_bytes(p), h->stream) != cudaSuccess) {
        vans_destroy(h);
        return VANS_ERR_CUDA;
    }
    *out = h;
    return VANS_OK;
}

void vans_destroy(vans_t h) {
    if (!h) return;
    drop_graph(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

int vans_set_eps(vans_t h, const float *eps_dev) {
    if (!h || h->batched || !eps_dev) return VANS_ERR_ARG;
    if (cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_pad_eps(h->dom, eps_dev, nullptr, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    int bad = 0;
    int rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return VANS_ERR_ARG;
    ++h->launches;
    if (cudaMemsetAsync(h->flag + 2, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    if (vans::launch_pad_eps(h->dom, eps_dev, h->eps_pad, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    return reset_to_rest(h);
}

int vans_set_eps_async(vans_t h, const float *eps_dev) {
    if (!h || h->batched || !eps_dev) return VANS_ERR_ARG;
    // one pass pads eps and flags any value outside (0, 1] in flag[2]
    if (cudaMemsetAsync(h->flag + 2, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_pad_eps(h->dom, eps_dev, h->eps_pad, h->flag + 2, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    return reset_to_rest(h);
}

int vans_update_eps(vans_t h, const float *eps_dev) {
    if (!h || h->batched || !eps_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    if (h->slab) return VANS_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_pad_eps(h->dom, eps_dev, nullptr, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    int bad = 0;
    int rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return VANS_ERR_ARG;
    h->launches += 2;
    if (vans::launch_rebase_eps(h->q, h->dom, eps_dev, h->st[h->cur], h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    if (vans::launch_pad_eps(h->dom, eps_dev, h->eps_pad, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    return VANS_OK;
}

int vans_step(vans_t h, int nsteps) {
    if (!h || h->batched || nsteps < 0) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    if (h->slab && nsteps > 1) return VANS_ERR_UNSUPPORTED;   // a halo exchange after each step
    return run_steps(h, nsteps);
}

int vans_step_monitored(vans_t h, int nsteps, int every, float *rho_dev, float *u_dev,
                        float *stats_dev) {
    if (!h || h->batched || nsteps < 0 || every < 1 || !rho_dev || !u_dev || !stats_dev)
        return VANS_ERR_ARG;
    if (h->dom.nee || h->slab) return VANS_ERR_UNSUPPORTED;    // plates on nodes: use vans_moments
    if (!h->eps_set) return VANS_ERR_STATE;
    if (cudaMemsetAsync(stats_dev, 0, 4 * sizeof(float), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->mon_part, 0, kMonFloats * sizeof(float), h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    int done = 0;
    while (done < nsteps) {
        // every-1 plain steps (graph-replayed when long), then one monitoring step
        const int plain = std::min(every - 1, nsteps - done - 1);
        if (plain > 0) {
            const int rc = run_steps(h, plain);
            if (rc) return rc;
            done += plain;
        }
        ++h->launches;
        if (vans::launch_step_monitor(h->q, h->dom, h->st[h->cur], h->st[h->cur ^ 1], rho_dev, u_dev,
                                      stats_dev, h->mon_part, h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
        h->cur ^= 1;
        ++done;
    }
    if (nsteps > 0) {
        ++h->launches;
        if (vans::launch_monitor_finalize(h->mon_part, stats_dev, h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
    }
    return VANS_OK;
}

int vans_step_raw(vans_t h, const float *in, float *out) {
    if (!h || h->batched || !in || !out || in == out) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(vans::launch_step(h->q, h->dom, in, out, h->L, h->stream));
}

int vans_moments(vans_t h, float *rho_dev, float *u_dev) {
    if (!h || h->batched) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    if (!rho_dev && !u_dev) return VANS_OK;
    ++h->launches;
    return cuda_status(vans::launch_moments(h->q, h->dom, h->st[h->cur], rho_dev, u_dev, h->stream));
}

int vans_get_populations(vans_t h, float *f_dev) {
    if (!h || h->batched || !f_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(vans::launch_export(h->q, h->dom, h->st[h->cur], f_dev, h->stream));
}

int vans_set_populations(vans_t h, const float *f_dev) {
    if (!h || h->batched || !f_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(vans::launch_import(h->q, h->dom, f_dev, h->st[h->cur], h->stream));
}

int vans_get_state(vans_t h, float *state_dev) {
    if (!h || h->batched || !state_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    return cuda_status(cudaMemcpyAsync(state_dev, h->st[h->cur], h->sfloats * sizeof(float),
                                       cudaMemcpyDeviceToDevice, h->stream));
}

int vans_set_state(vans_t h, const float *state_dev) {
    if (!h || h->batched || !state_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    return cuda_status(cudaMemcpyAsync(h->st[h->cur], state_dev, h->sfloats * sizeof(float),
                                       cudaMemcpyDeviceToDevice, h->stream));
}

int vans_get_launch(vans_t h, vans_launch *cfg) {
    if (!h || !cfg) return VANS_ERR_ARG;
    cfg->cpt = h->L.cpt;
    cfg->warps = h->L.warps;
    cfg->rows = h->L.rows;
    cfg->kind = h->L.kind;
    cfg->ctas = h->L.ctas;
    return VANS_OK;
}

int vans_set_launch(vans_t h, const vans_launch *cfg) {
    if (!h || !launch_ok(cfg, h->q, h->batched)) return VANS_ERR_ARG;
    const Launch L{cfg->cpt, cfg->warps, cfg->rows, cfg->kind, cfg->ctas};
    if (!h->batched && h->dom.nee && !vans::launch_has_plates(h->q, L)) return VANS_ERR_UNSUPPORTED;
    if (L.kind == 8 && !vans::cluster_fits(h->q, h->dom, L.rows, L.warps)) return VANS_ERR_UNSUPPORTED;
    if (h->batched) return set_batch_launch(h, L);
    h->L = L;
    drop_graph(h);
    return VANS_OK;
}

int vans_autotune(vans_t h, vans_launch *chosen) {
    if (!h || h->batched) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    // time each candidate on the current state; the output goes to the other
    // buffer, which holds nothing live, so the state is unchanged
    const std::vector<Launch> cs = candidates(h->q, false);
    Launch best = h->L;
    float best_ms = 1e30f;
    const float *in = h->st[h->cur];
    float *outb = h->st[h->cur ^ 1];
    const int reps = h->dom.cells > (1 << 22) ? 5 : 21;
    for (const Launch &L : cs) {
        if (h->dom.nee && !vans::launch_has_plates(h->q, L)) continue;   // no plate instance
        if (L.kind == 8 && !vans::cluster_fits(h->q, h->dom, L.rows, L.warps)) continue;
        // kind 8 runs the reps steps in one launch (odd reps: the result
        // lands in the spare buffer, as one step of the other kinds does)
        const float ms =
            L.kind == 8
                ? time_launches(h, [&](cudaStream_t st) {
                      return vans::launch_step_cluster(h->q, h->dom, in, outb, reps, L, st);
                  }, 1)
                : time_launches(h, [&](cudaStream_t st) {
                      return vans::launch_step(h->q, h->dom, in, outb, L, st);
                  }, reps);
        h->launches += L.kind == 8 ? 5 : 5 * reps;
        if (ms < best_ms) {
            best_ms = ms;
            best = L;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return VANS_ERR_CUDA;
    h->L = best;
    drop_graph(h);
    if (chosen) {
        chosen->cpt = best.cpt;
        chosen->warps = best.warps;
        chosen->rows = best.rows;
        chosen->kind = best.kind;
        chosen->ctas = best.ctas;
    }
    return VANS_OK;
}

int vans_flux(vans_t h, const float *state, int x_out, float *J_dev) {
    if (!h || h->batched || !J_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    if (x_out < 0 || x_out >= h->dom.nx) return VANS_ERR_ARG;
    ++h->launches;
    return cuda_status(
        vans::launch_flux(h->q, h->dom, state ? state : h->st[h->cur], x_out, J_dev, h->stream));
}

int vans_flux_seed(vans_t h, const float *state, int x_out, float *lam_dev, float *grad_acc) {
    if (!h || h->batched || !lam_dev || !grad_acc) return VANS_ERR_ARG;
    if (h->dom.nee || h->slab) return VANS_ERR_UNSUPPORTED;    // the adjoint covers bounce-back walls
    if (!h->eps_set) return VANS_ERR_STATE;
    if (x_out < 0 || x_out >= h->dom.nx) return VANS_ERR_ARG;
    const int D = h->q == 9 ? 2 : 3;
    if (cudaMemsetAsync(lam_dev, 0, h->sfloats * sizeof(float), h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    if (cudaMemsetAsync(grad_acc, 0, 2 * (1 + D) * h->dom.cells * sizeof(float), h->stream) !=
        cudaSuccess)
        return VANS_ERR_CUDA;
    ++h->launches;
    return cuda_status(vans::launch_flux_seed(h->q, h->dom, state ? state : h->st[h->cur], x_out,
                                              lam_dev, grad_acc, h->adj_fp64, h->stream));
}

int vans_step_adjoint(vans_t h, const float *state_t, const float *lam_in, float *lam_out,
                      float *grad_acc) {
    if (!h || h->batched || !state_t || !lam_in || !lam_out || !grad_acc) return VANS_ERR_ARG;
    if (lam_in == lam_out || (const float *)lam_out == state_t) return VANS_ERR_ARG;
    if (h->dom.nee || h->slab) return VANS_ERR_UNSUPPORTED;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(vans::launch_step_adjoint(h->q, h->dom, state_t, lam_in, lam_out, grad_acc,
                                                 h->adj_fp64, h->adjL, h->stream));
}

int vans_adjoint_segment(vans_t h, const float *ckpt, float *seg, int len, float *lam, float *tmp,
                         float *grad_acc) {
    if (!h || h->batched || !ckpt || !seg || !lam || !tmp || !grad_acc || len < 1) return VANS_ERR_ARG;
    if (h->dom.nee || h->slab) return VANS_ERR_UNSUPPORTED;
    if (lam == tmp) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    const long long sf = h->sfloats;
    if (cudaMemcpyAsync(seg, ckpt, sf * sizeof(float), cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess)
        return VANS_ERR_CUDA;
    vans_s::SegGraph *g = nullptr;
    for (auto &e : h->seg_graphs)
        if (e.seg == seg && e.len == len && e.lam == lam && e.tmp == tmp && e.grad == grad_acc) g = &e;
    if (!g) {
        if (h->seg_graphs.size() >= 4) {
            cudaGraphExecDestroy(h->seg_graphs.front().exec);
            h->seg_graphs.erase(h->seg_graphs.begin());
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return VANS_ERR_CUDA;
        cudaError_t le = cudaSuccess;
        // recompute the segment's states with the forward step kernel
        for (int k = 0; k < len && le == cudaSuccess; ++k)
            le = vans::launch_step(h->q, h->dom, seg + k * sf, seg + (k + 1) * sf, h->L, h->cap);
        // then walk back through them
        float *a = lam, *b = tmp;
        for (int k = len - 1; k >= 0 && le == cudaSuccess; --k) {
            le = vans::launch_step_adjoint(h->q, h->dom, seg + k * sf, a, b, grad_acc, h->adj_fp64,
                                           h->adjL, h->cap);
            float *t = a;
            a = b;
            b = t;
        }
        if (le == cudaSuccess && a != lam)
            le = cudaMemcpyAsync(lam, a, sf * sizeof(float), cudaMemcpyDeviceToDevice, h->cap);
        cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return VANS_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return VANS_ERR_CUDA;
        h->seg_graphs.push_back(vans_s::SegGraph{seg, len, lam, tmp, grad_acc, exec});
        g = &h->seg_graphs.back();
    }
    if (cudaGraphLaunch(g->exec, h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    h->launches += 2LL * len;
    return VANS_OK;
}

int vans_set_adjoint_launch(vans_t h, const vans_launch *cfg) {
    if (!h || h->batched || !cfg || cfg->ctas != 0) return VANS_ERR_ARG;
    if (cfg->kind == 0) {
        if (cfg->warps < 1 || cfg->rows < 1 || cfg->warps * cfg->rows > 8) return VANS_ERR_ARG;
        if (!(cfg->cpt == 1 || (cfg->cpt == 2 && h->q == 9))) return VANS_ERR_ARG;
    } else if (cfg->kind == 1) {
        // pipeline: 2 or 4 compute warps, 2..8 stages; shapes with an instance
        const int nt = 32 * cfg->warps;
        const bool ok = h->q == 9 ? ((nt == 64 && cfg->cpt == 1) || (nt == 128 && cfg->cpt <= 2))
                                  : (nt == 128 && cfg->cpt == 1);
        if (!ok || cfg->rows < 2 || cfg->rows > 8) return VANS_ERR_ARG;
    } else {
        return VANS_ERR_ARG;
    }
    h->adjL = Launch{cfg->cpt, cfg->warps, cfg->rows, cfg->kind};
    drop_graph(h);
    return VANS_OK;
}

int vans_set_adjoint_precision(vans_t h, int bits) {
    if (!h || (bits != 32 && bits != 64)) return VANS_ERR_ARG;
    const int v = (bits == 64);
    if (v != h->adj_fp64) {
        h->adj_fp64 = v;
        drop_graph(h);
    }
    return VANS_OK;
}

int vans_grad_finalize(vans_t h, const float *lam0, const float *grad_acc, float *dJdeps_dev) {
    if (!h || h->batched || !lam0 || !grad_acc || !dJdeps_dev) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(
        vans::launch_grad_finalize(h->q, h->dom, lam0, grad_acc, dJdeps_dev, h->stream));
}

int vans_check(vans_t h) {
    if (!h) return VANS_ERR_ARG;
    if (cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    if (h->batched) {
        for (int d = 0; d < h->n; ++d) {
            if (!h->dom_ready[d]) continue;
            ++h->launches;
            if (vans::launch_check(9, h->doms[d], h->doms[d].f[h->parity], h->flag, h->stream) !=
                cudaSuccess)
                return VANS_ERR_CUDA;
        }
    } else {
        if (!h->eps_set) return VANS_ERR_STATE;
        ++h->launches;
        if (vans::launch_check(h->q, h->dom, h->st[h->cur], h->flag, h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
    }
    int bad = 0, tmo = 0, eps_bad = 0;
    int rc = read_flag(h, &bad, &tmo, &eps_bad);
    if (rc) return rc;
    if (tmo) return VANS_ERR_TIMEOUT;
    if (eps_bad) return VANS_ERR_ARG;
    return bad ? VANS_ERR_DIVERGED : VANS_OK;
}

long long vans_halo_floats(vans_t h) {
    if (!h || h->batched) return -1;
    return vans::halo_floats(h->q, h->dom);
}

int vans_set_eps_slab(vans_t h, const float *eps_dev, const float *eps_left,
                      const float *eps_right) {
    if (!h || h->batched || !eps_dev || !eps_left || !eps_right) return VANS_ERR_ARG;
    // the halo columns first (check only), then the slab's own field
    if (cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_eps_halo(h->dom, eps_left, eps_right, nullptr, h->flag, h->stream) !=
        cudaSuccess)
        return VANS_ERR_CUDA;
    int bad = 0;
    int rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return VANS_ERR_ARG;
    rc = vans_set_eps(h, eps_dev);
    if (rc) return rc;
    ++h->launches;
    if (vans::launch_eps_halo(h->dom, eps_left, eps_right, h->eps_pad, h->flag, h->stream) !=
        cudaSuccess)
        return VANS_ERR_CUDA;
    h->slab = true;
    h->dom.xwrap = 0;            // the halo columns are the neighbours', not the row's own ends
    drop_graph(h);
    return VANS_OK;
}

int vans_halo_pack(vans_t h, float *to_left, float *to_right) {
    if (!h || h->batched || !to_left || !to_right || to_left == to_right) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(
        vans::launch_halo_pack(h->q, h->dom, h->st[h->cur], to_left, to_right, h->stream));
}

int vans_halo_unpack(vans_t h, const float *from_left, const float *from_right) {
    if (!h || h->batched || !from_left || !from_right) return VANS_ERR_ARG;
    if (!h->eps_set) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(
        vans::launch_halo_unpack(h->q, h->dom, h->st[h->cur], from_left, from_right, h->stream));
}

long long vans_cells(vans_t h) {
    if (!h) return -1;
    if (h->batched) return vans_batch_cells(h);
    return h->dom.cells;
}

long long vans_launch_count(vans_t h) { return h ? h->launches : -1; }

// ------------------------------------------------------------- batched ----

static long long batch_tile_cap(const vans_params *p, int n) {
    long long t = 0;   // the smallest tile the autotuner may pick: 32 cells x 1 row
    for (int d = 0; d < n; ++d) t += (long long)p[d].ny * ((p[d].nx + 31) / 32);
    return t;
}

size_t vans_batch_workspace_bytes(const vans_params *p, int n) {
    if (!p || n < 1) return 0;
    long long bytes = round_up((long long)n * sizeof(VDom), 256) +
                      round_up(batch_tile_cap(p, n) * (long long)sizeof(Tile), 256);
    for (int d = 0; d < n; ++d) {
        if (validate(&p[d], true) != VANS_OK) return 0;
        bytes += (2 * state_floats_of(9, p[d].nx, p[d].ny, 1) + eps_floats_of(9, p[d].nx, p[d].ny, 1)) *
                 (long long)sizeof(float);
    }
    bytes += kFlagFloats * sizeof(float);
    return (size_t)bytes;
}

int vans_batch_create(const vans_params *p, int n, void *workspace, size_t workspace_bytes,
                      void *cuda_stream, vans_t *out) {
    if (!out) return VANS_ERR_ARG;
    *out = nullptr;
    if (!p || n < 1) return VANS_ERR_ARG;
    for (int d = 0; d < n; ++d) {
        const int v = validate(&p[d], true);
        if (v) return v;
    }
    if (!workspace || ((uintptr_t)workspace & 255)) return VANS_ERR_ARG;
    const size_t need = vans_batch_workspace_bytes(p, n);
    if (need == 0 || workspace_bytes < need) return VANS_ERR_ARG;
    vans_t h = new (std::nothrow) vans_s();
    if (!h) return VANS_ERR_ARG;
    h->batched = true;
    h->q = 9;
    h->n = n;
    h->bp.assign(p, p + n);
    char *w = (char *)workspace;
    h->doms_d = (VDom *)w;
    w += round_up((long long)n * sizeof(VDom), 256);
    h->tiles_d = (Tile *)w;
    h->tile_cap = batch_tile_cap(p, n);
    w += round_up(h->tile_cap * (long long)sizeof(Tile), 256);
    h->doms.resize(n);
    long long dense = 0;
    for (int d = 0; d < n; ++d) {
        VDom &D = h->doms[d];
        vans::fill_dom(&p[d], D);
        const long long sf = state_floats_of(9, p[d].nx, p[d].ny, 1);
        D.f[0] = (float *)w;
        D.f[1] = (float *)w + sf;
        D.eps = (float *)w + 2 * sf;
        D.dense_off = dense;
        dense += D.cells;
        w += (2 * sf + eps_floats_of(9, p[d].nx, p[d].ny, 1)) * sizeof(float);
    }
    h->flag = (int *)w;
    for (VDom &D : h->doms) D.status = h->flag + 1;
    h->dom_ready.assign(n, 0);
    int rc = make_streams(h, cuda_stream);
    if (rc) {
        vans_destroy(h);
        return rc;
    }
    if (cudaMemsetAsync(workspace, 0, need, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->doms_d, h->doms.data(), n * sizeof(VDom), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess) {
        vans_destroy(h);
        return VANS_ERR_CUDA;
    }
    rc = set_batch_launch(h, Launch{4, 4, 1, 0});
    if (rc) {
        vans_destroy(h);
        return rc;
    }
    *out = h;
    return VANS_OK;
}

int vans_batch_set_eps(vans_t h, int d, const float *eps_dev) {
    if (!h || !h->batched || d < 0 || d >= h->n || !eps_dev) return VANS_ERR_ARG;
    const VDom &D = h->doms[d];
    if (cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_pad_eps(D, eps_dev, nullptr, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    int bad = 0;
    int rc = read_flag(h, &bad);
    if (rc) return rc;
    if (bad) return VANS_ERR_ARG;
    ++h->launches;
    if (vans::launch_pad_eps(D, eps_dev, (float *)D.eps, h->flag, h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    const long long sf = state_floats_of(9, D.nx, D.ny, 1);
    if (cudaMemsetAsync(D.f[0], 0, 2 * sf * sizeof(float), h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    if (D.moving) {
        ++h->launches;
        if (vans::launch_init_moving(9, D, D.f[h->parity], h->stream) != cudaSuccess)
            return VANS_ERR_CUDA;
    }
    h->dom_ready[d] = 1;
    return VANS_OK;
}

int vans_batch_step(vans_t h, int nsteps) {
    if (!h || !h->batched || nsteps < 0) return VANS_ERR_ARG;
    for (int d = 0; d < h->n; ++d)
        if (!h->dom_ready[d]) return VANS_ERR_STATE;
    return run_steps(h, nsteps);
}

int vans_batch_moments(vans_t h, int d, float *rho_dev, float *u_dev) {
    if (!h || !h->batched || d < 0 || d >= h->n) return VANS_ERR_ARG;
    if (!h->dom_ready[d]) return VANS_ERR_STATE;
    if (!rho_dev && !u_dev) return VANS_OK;
    ++h->launches;
    return cuda_status(vans::launch_moments(9, h->doms[d], h->doms[d].f[h->parity], rho_dev, u_dev,
                                            h->stream));
}

int vans_batch_get_populations(vans_t h, int d, float *f_dev) {
    if (!h || !h->batched || d < 0 || d >= h->n || !f_dev) return VANS_ERR_ARG;
    if (!h->dom_ready[d]) return VANS_ERR_STATE;
    ++h->launches;
    return cuda_status(vans::launch_export(9, h->doms[d], h->doms[d].f[h->parity], f_dev, h->stream));
}

int vans_batch_autotune(vans_t h, vans_launch *chosen) {
    if (!h || !h->batched) return VANS_ERR_ARG;
    for (int d = 0; d < h->n; ++d)
        if (!h->dom_ready[d]) return VANS_ERR_STATE;
    const Launch keep = h->L;
    Launch best = keep;
    float best_ms = 1e30f;
    const int par = h->parity;
    for (const Launch &L : candidates(9, true)) {
        if (set_batch_launch(h, L) != VANS_OK) continue;
        // reads the current parity and writes the other buffer of every domain
        const float ms =
            time_launches(h, [&](cudaStream_t st) { return batched_step(h, st, par); }, 5);
        h->launches += 25;
        if (ms < best_ms) {
            best_ms = ms;
            best = L;
        }
    }
    int rc = set_batch_launch(h, best);
    if (rc) return rc;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return VANS_ERR_CUDA;
    if (chosen) {
        chosen->cpt = best.cpt;
        chosen->warps = best.warps;
        chosen->rows = best.rows;
        chosen->kind = best.kind;
        chosen->ctas = best.ctas;
    }
    return VANS_OK;
}

int vans_batch_profile_step(vans_t h, unsigned long long *records_dev, long long capacity,
                            long long *n_records) {
    if (!h || !h->batched || !n_records) return VANS_ERR_ARG;
    const long long n = (long long)h->tiles.size();    // CTAs of a step, at most
    *n_records = n;
    if (!records_dev) return VANS_OK;
    if (capacity < 3 * n) return VANS_ERR_ARG;
    for (int d = 0; d < h->n; ++d)
        if (!h->dom_ready[d]) return VANS_ERR_STATE;
    if (h->L.kind == 0) return VANS_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(records_dev, 0, 3 * n * sizeof(unsigned long long), h->stream) != cudaSuccess)
        return VANS_ERR_CUDA;
    ++h->launches;
    if (vans::launch_ring_batched(h->doms_d, h->tiles_d, (int)n, h->parity, h->L, h->flag + 1,
                                  h->stream, records_dev) != cudaSuccess)
        return VANS_ERR_CUDA;
    h->parity ^= 1;
    return VANS_OK;
}

long long vans_batch_cells(vans_t h) {
    if (!h || !h->batched) return -1;
    long long c = 0;
    for (const VDom &D : h->doms) c += D.cells;
    return c;
}

const char *vans_status_string(int status) {
    switch (status) {
        case VANS_OK: return "ok";
        case VANS_ERR_ARG: return "invalid argument";
        case VANS_ERR_CUDA: return "CUDA error";
        case VANS_ERR_DIVERGED: return "state diverged (non-finite or |u| >= 0.5)";
        case VANS_ERR_TIMEOUT: return "device wait timed out";
        case VANS_ERR_UNSUPPORTED: return "unsupported configuration";
        case VANS_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char *vans_version(void) { return "vans-gb300 0.1 (sm_103a)"; }

}  // extern "C"
