// vans_internal.h -- types shared by the host runtime and the kernels (not part
// of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vans.h"

// Column 0 of a padded row sits VDom::off floats into the row: 8 (one 32-byte
// sector) for D2Q9, 32 (one 128-byte line) for D3Q19, whose rows of a few
// hundred cells are staged whole, cells only, so that they cover whole lines.

namespace vans {

// Everything a kernel needs to know about one domain.  Plain data, passed by
// value to the single-domain kernels and stored in a device table for the
// batched kernel.
struct VDom {
    int q, nx, ny, nz;
    int rows;             // ny * nz padded rows per direction plane
    int pitch;            // floats per padded row (multiple of 32)
    int off;              // floats from a row's start to its column 0 (8 or 32)
    int xwrap;            // 1: the x halo columns mirror the row's own ends (periodic
                          // x); 0: a slab, whose halos come from its neighbours
    long long plane;      // rows * pitch floats per direction
    int wall_y, wall_z;   // 1: bounce-back walls on both faces of that axis
    float omega;          // 1 / tau
    float ctau;           // 1 - 1/(2 tau), the prefactor of Eqs. pi and Fi
    float g[3];           // body force per unit mass
    int drag_mode, k_mode;
    float ca, cb;         // drag constants: alpha = ca * a(eps), beta = cb * b(eps)
    const float *eps;     // padded porosity rows (same row layout, one plane)
    float *f[2];          // the two state buffers (batched kernel only)
    long long cells;      // nx * ny * nz
    long long dense_off;  // offset of this domain in packed dense outputs (batched)
    int *status;          // device status word: bit 1 = a bounded wait timed out
    int moving;           // 1: the upper y wall moves with velocity uw (bounce-back walls)
    float uw[3];          // velocity of the upper y wall / plate
    int nee;              // 1: rows 0 and ny-1 are plate nodes (non-equilibrium extrapolation)
};

// One tile of the batched register-load kernel: a block-sized piece of one
// domain.  The batched pipeline kernel reuses the record as a strip:
// {dom, y0, x0, y1} = rows y0..y1-1 of the column block at x0.
struct Tile {
    int dom;   // domain index
    int row;   // first row of the tile (strip: first row)
    int x0;    // first column of the tile
    int pad;   // strip: one past the last row
};

// kind 0: register-load kernel k_step (cpt cells per lane, warps x rows per block)
// kinds 2-7: bulk-copy pipelines (32*warps compute threads, cpt cells per
//         thread per tile, rows = pipeline stages)
// kind 8: cluster-resident multi-step kernel (32*warps threads per CTA, rows =
//         the largest cluster)
// ctas: at most that many CTAs per SM for the pipelined kinds (0: as many as fit)
struct Launch {
    int cpt, warps, rows, kind;
    int ctas;
};

// ------------------------------------------------------- host helpers ----
// Floats from a row's start to its column 0 for lattice q (VDom::off).
inline int col0_for(int q) { return q == 19 ? 32 : 8; }
// Floats per padded row for a row of nx cells: column 0 at col0_for(q),
// columns -1 and nx as halo copies, rounded up to whole 128-byte lines.
int pitch_for(int q, int nx);
// The kernel descriptor of one domain from validated parameters: sizes, row
// layout, relaxation and drag constants, walls.  Buffers (eps, f, status) are
// left null for the caller to set.
void fill_dom(const vans_params *p, VDom &d);

// ------------------------------------------------------ kernel launchers ----
// Each returns cudaSuccess or the launch error.  `stream` is where they enqueue.

cudaError_t launch_step(int q, const VDom &d, const float *fin, float *fout, Launch L,
                        cudaStream_t stream);
// partial maxima of the monitoring reductions: kMonSlots per statistic
constexpr int kMonSlots = 256;
cudaError_t launch_step_monitor(int q, const VDom &d, const float *fin, float *fout, float *rho,
                                float *u, float *stats, float *part, cudaStream_t stream);
// stats[0..2] = maxima of the partials (after the monitoring steps of a call)
cudaError_t launch_monitor_finalize(const float *part, float *stats, cudaStream_t stream);
cudaError_t launch_step_tma(int q, const VDom &d, const float *fin, float *fout, Launch L,
                            cudaStream_t stream);
// kind 8: nsteps steps in one launch of one thread-block cluster that holds the
// whole state in its shared memory; reads fin, writes fout (which may be fin)
cudaError_t launch_step_cluster(int q, const VDom &d, const float *fin, float *fout, int nsteps,
                                Launch L, cudaStream_t stream);
// whether a cluster of at most cmax CTAs of `warps` warps holds the domain
// (never plates on nodes)
bool cluster_fits(int q, const VDom &d, int cmax, int warps);
// the reverse step with a bulk-copy pipeline (adjoint launch kind 1)
cudaError_t launch_adjoint_tma(int q, const VDom &d, const float *state, const float *lam_in,
                               float *lam_out, float *grad, int fp64, Launch L, cudaStream_t s);
// whether launch L has an instance for plates on nodes (wall_kind 1)
bool launch_has_plates(int q, Launch L);
// kinds 2, 4, 5: strip table (one CTA per strip); 6, 7: interleaved tile table
// prof (nullptr: none): 3 words per CTA, {SM id, start ns, end ns}, zeroed by the caller
cudaError_t launch_ring_batched(const VDom *doms, const Tile *strips, int nstrips, int parity,
                                Launch L, int *status, cudaStream_t stream,
                                unsigned long long *prof = nullptr);
cudaError_t launch_step_batched(const VDom *doms_dev, const Tile *tiles_dev, int ntiles, int parity,
                                Launch L, int grid, cudaStream_t stream);
int batched_blocks_per_sm(Launch L);
cudaError_t launch_moments(int q, const VDom &d, const float *state, float *rho, float *u,
                           cudaStream_t stream);
cudaError_t launch_export(int q, const VDom &d, const float *state, float *f, cudaStream_t stream);
cudaError_t launch_import(int q, const VDom &d, const float *f, float *state, cudaStream_t stream);
cudaError_t launch_pad_eps(const VDom &d, const float *eps_dense, float *eps_pad, int *flag,
                           cudaStream_t stream);
cudaError_t launch_rebase_eps(int q, const VDom &d, const float *eps_new, float *state,
                              cudaStream_t stream);
cudaError_t launch_init_moving(int q, const VDom &d, float *state, cudaStream_t stream);
cudaError_t launch_check(int q, const VDom &d, const float *state, int *flag, cudaStream_t stream);
cudaError_t launch_flux(int q, const VDom &d, const float *state, int x_out, float *J,
                        cudaStream_t stream);
cudaError_t launch_flux_seed(int q, const VDom &d, const float *state, int x_out, float *lam,
                             float *grad, int fp64, cudaStream_t stream);
cudaError_t launch_step_adjoint(int q, const VDom &d, const float *state, const float *lam_in,
                                float *lam_out, float *grad, int fp64, Launch L,
                                cudaStream_t stream);
cudaError_t launch_grad_finalize(int q, const VDom &d, const float *lam0, const float *grad,
                                 float *dJ, cudaStream_t stream);
// slabs along x: floats of one halo message, pack / unpack of the edge
// columns' crossing populations, the porosity halo columns
int halo_floats(int q, const VDom &d);
cudaError_t launch_halo_pack(int q, const VDom &d, const float *state, float *to_left,
                             float *to_right, cudaStream_t stream);
cudaError_t launch_halo_unpack(int q, const VDom &d, float *state, const float *from_left,
                               const float *from_right, cudaStream_t stream);
cudaError_t launch_eps_halo(const VDom &d, const float *left, const float *right, float *eps_pad,
                            int *flag, cudaStream_t stream);

}  // namespace vans
