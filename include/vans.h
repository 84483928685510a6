/*
 * vans.h -- C ABI of the GB300 (sm_103a) porous lattice Boltzmann library.
 *
 * The library advances the lattice Boltzmann model for the volume-averaged
 * Navier-Stokes equations of Zhang, Wang & Ouyang ("Lattice Boltzmann Model for
 * the Volume-Averaged Navier-Stokes Equations"):
 *
 *   f_i(x + e_i, t + 1) - f_i(x, t) = -(f_i - f_i^eq)/tau + P_i + F_i
 *
 * with the porosity-weighted equilibrium (Eq. d2q9eq), the pressure correction
 * P_i (Eq. pi), the Guo forcing term F_i (Eq. Fi) carrying the body force and the
 * Darcy/Forchheimer drag (drag law and the Ergun K, F_eps of the "Examples and
 * discussions" section), and the moments eps*rho, eps*rho*u of Eqs. 0moment and
 * 1moment.  Walls are half-way bounce-back; x is always periodic.
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers (CUDA global memory) unless stated.
 *     The caller allocates and owns every buffer, including the workspace; the
 *     library owns only the handle (host memory) and never frees caller memory.
 *   - Work is enqueued asynchronously on the stream given to vans_create; a call
 *     returns before the GPU has finished.  Launch errors are reported; errors
 *     that happen later on the device surface at the next call or sync.
 *   - Every int-returning call returns VANS_OK (0) or a negative VANS_ERR_*.
 *     No exception crosses the ABI.  A NULL handle gives VANS_ERR_ARG.
 *   - Dense field layout ("dense"): x fastest, then y, then z; a vector field
 *     stores its components one after the other (component-major).  For D2Q9,
 *     nz = 1 and vectors have 2 components; for D3Q19 they have 3.
 *   - Direction order.  D2Q9: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
 *     5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).  D3Q19: 0 (0,0,0), 1 (1,0,0),
 *     2 (-1,0,0), 3 (0,1,0), 4 (0,-1,0), 5 (0,0,1), 6 (0,0,-1), 7 (1,1,0),
 *     8 (-1,-1,0), 9 (1,-1,0), 10 (-1,1,0), 11 (1,0,1), 12 (-1,0,-1),
 *     13 (1,0,-1), 14 (-1,0,1), 15 (0,1,1), 16 (0,-1,-1), 17 (0,1,-1), 18 (0,-1,1).
 *   - "state" buffers hold the populations in the library's own padded layout
 *     (vans_state_floats() floats each, 16-byte aligned).  Their content is the
 *     post-collision populations of the previous step stored as deviations from
 *     w_i * eps; use vans_get_populations() for the physical f_i(x, t).
 */
#ifndef VANS_H
#define VANS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    VANS_OK = 0,
    VANS_ERR_ARG = -1,          /* bad argument, size, pointer or parameter          */
    VANS_ERR_CUDA = -2,         /* a CUDA call or kernel launch failed                */
    VANS_ERR_DIVERGED = -3,     /* non-finite or supersonic state detected            */
    VANS_ERR_TIMEOUT = -4,      /* a bounded device wait gave up                      */
    VANS_ERR_UNSUPPORTED = -5,  /* valid request this build does not implement        */
    VANS_ERR_STATE = -6         /* call out of order (e.g. step before set_eps)       */
};

typedef struct vans_s *vans_t; /* opaque handle, owned by the library */

/* Model and domain parameters of one domain. */
typedef struct {
    int q;          /* 9 (D2Q9) or 19 (D3Q19)                                        */
    int nx, ny, nz; /* lattice size; nz must be 1 for D2Q9; each >= 1                */
    int wall_mask;  /* bit1: bounce-back walls on both y faces; bit2: on both z faces;
                       a cleared bit means periodic.  bit0 (x walls) is unsupported. */
    float tau;      /* relaxation time, > 0.5; nu = (tau - 1/2)/3 (after Eq. VNS2)   */
    float g[3];     /* body force per unit mass; the force density is eps*rho*g      */
    int drag_mode;  /* 0 none, 1 Darcy only, 2 Darcy + Forchheimer (drag law)        */
    int k_mode;     /* 0: Ergun K(eps) = eps^3 d_p^2 / (150 (1-eps)^2) and
                          F_eps(eps) = 1.75 / sqrt(150 eps^3);
                       1: K and F_eps fixed (fields K, F_eps);
                       2: K fixed, F_eps(eps) = 1.75 / sqrt(150 eps^3)                 */
    float d_p;      /* particle diameter (k_mode 0)                                  */
    float K;        /* permeability (k_mode 1, 2)                                    */
    float F_eps;    /* geometric function (k_mode 1)                                 */
    float u_wall[3];/* velocity of the upper y wall (y = ny side), the plate that drives
                       the Couette flow of the validation case; needs y walls.  A
                       population that bounces off it gains 2 w_i eps rho_w (e_i.u_w)/cs^2
                       with rho_w = 1 (moving-wall bounce-back with the eps-weighted
                       equilibrium of Eq. d2q9eq).  All zero: resting walls.         */
    int wall_kind;  /* the y walls (bit1 of wall_mask): 0 half-way bounce-back, the
                       walls half a cell outside rows 0 and ny-1 (H = ny); 1 the
                       non-equilibrium extrapolation scheme the paper's validation
                       runs use (Sec. "Examples and discussions"): rows 0 and ny-1
                       are nodes on the plates (H = ny - 1); each takes
                       f^eq(eps, rho, u_plate) plus the non-equilibrium part of its
                       fluid neighbour and relaxes with no source term; u_plate = 0
                       below and u_wall above.  Needs ny >= 3, no z walls; the
                       single-domain solver only (vans_batch_* and the adjoint
                       answer VANS_ERR_UNSUPPORTED).                                 */
} vans_params;

/* Launch configuration of the step kernels (chosen by vans_autotune).
 * kind 0: register-load kernel: cpt cells per lane (1, 2, 4), `warps` warps
 *         along x times `rows` rows per block (warps*rows <= 8).
 * kind 2: bulk-copy pipeline (rows staged in shared memory by cp.async.bulk),
 *         32*warps threads (warps 4 or 8), cpt cells per thread per tile
 *         (1, 2, 4), `rows` = pipeline stages (2..6); each CTA walks a strip
 *         of consecutive rows (one column block, one z plane) and keeps the
 *         porosity rows in a shared-memory ring, so each eps row is read from
 *         HBM once per strip.
 * kind 4, 5: kind 2 with one extra producer warp per CTA (warps counts the
 *         compute warps only): stages are released per warp through "empty"
 *         mbarriers instead of a block-wide barrier per tile; kind 5 puts each
 *         thread on consecutive cells (D2Q9: cpt 4, D3Q19: cpt 2; warps 2 or 4)
 *         with 16- or 8-byte shared loads and global stores.
 * kind 6, 7: persistent CTAs that take tiles b, b+G, b+2G, ... of the row-major
 *         tile order (the whole grid sweeps one band of rows), porosity rows
 *         staged per tile, producer warp as in kinds 4, 5; 6 strided cells
 *         (D2Q9 cpt 2, D3Q19 cpt 1; warps 4 or 8), 7 consecutive cells as in
 *         kind 5 (single D3Q19 domains also warps 3, 5 or 6: 192-, 320- or
 *         384-cell tiles).
 * kind 8: every step of a vans_step call in ONE launch of one thread-block
 *         cluster (up to `rows` CTAs, 2..16; `warps` 8 or 16 per CTA; cpt 1)
 *         that keeps the whole state in its distributed shared memory for the
 *         run, one cluster barrier per step: for domains of a few hundred KB,
 *         whose single-step launches cost more than their work.  Accepted
 *         only if the cluster holds the domain (D2Q9: at most 2 cells per
 *         thread, D3Q19: 1; two copies of each CTA's rows within 227 KB):
 *         VANS_ERR_UNSUPPORTED otherwise.  Plates on nodes included.
 * Kinds 1 and 3 are not built (VANS_ERR_ARG).
 *         The batched path takes kinds 0, 2, 4 and 5 (one CTA per strip of
 *         up to 32 rows of one domain) and 6, 7 (one table of every domain's
 *         row tiles); the batch is D2Q9 only. */
typedef struct {
    int cpt;
    int warps;
    int rows;
    int kind;
    int ctas;   /* kinds 2-7: at most this many CTAs per SM (1..4; the
                   dynamic shared memory request is raised until no more
                   fit), 0 = as many as fit; kinds 0 and 8: must be 0 */
} vans_launch;

/* ---------------------------------------------------------------- sizes -- */

/* Floats in one state buffer for these parameters, or -1 if they are invalid. */
long long vans_state_floats(const vans_params *p);

/* Bytes of workspace vans_create needs (two state buffers, a padded copy of eps,
 * a few status words and the partial maxima of vans_step_monitored), or 0 if
 * the parameters are invalid. */
size_t vans_workspace_bytes(const vans_params *p);

/* ------------------------------------------------------------ lifecycle -- */

/* Validate p and build a handle that uses `workspace` (device memory of at
 * least vans_workspace_bytes(p) bytes, 256-byte aligned; owned by the caller and
 * it must outlive the handle) and enqueues on `cuda_stream` (a cudaStream_t;
 * NULL is the legacy default stream).  Allocates no device memory.
 * Errors: VANS_ERR_ARG (invalid p, small or misaligned workspace, NULL out),
 * VANS_ERR_UNSUPPORTED (x walls). */
int vans_create(const vans_params *p, void *workspace, size_t workspace_bytes,
                void *cuda_stream, vans_t *out);

/* Release the handle and its CUDA graphs.  Never frees caller memory. */
void vans_destroy(vans_t h);

/* Copy the porosity field eps (dense, nx*ny*nz floats, device) into the
 * workspace and reset the populations to rest, rho = 1 and u = 0, i.e.
 * f_i = w_i eps (the initial state of the validation case), also next to a
 * moving upper wall.  Every eps must
 * satisfy 0 < eps <= 1; otherwise VANS_ERR_ARG and the handle keeps its
 * previous state.  (Synchronises the stream once to check the range.) */
int vans_set_eps(vans_t h, const float *eps_dev);

/* vans_set_eps without the stream synchronisation, for pipelines that run
 * one job per porosity field back to back: the range check runs on the device
 * in the same pass that pads eps, and does not stop the reset.  If a value is
 * outside (0, 1] the state is undefined and the next vans_check (which
 * synchronises) returns VANS_ERR_ARG; the next vans_set_eps or
 * vans_set_eps_async with a valid field clears that.  Otherwise identical to
 * vans_set_eps. */
int vans_set_eps_async(vans_t h, const float *eps_dev);

/* Replace the porosity field by eps_dev (dense, 0 < eps <= 1 else
 * VANS_ERR_ARG and nothing changes) while keeping the physical populations
 * f_i(x, t) of the current state: a porosity that varies in time, the
 * direction the paper names for two-fluid models (its concluding section).
 * The stored deviations are re-expressed for the new eps in place.
 * Synchronises once to check the range.  VANS_ERR_STATE before vans_set_eps. */
int vans_update_eps(vans_t h, const float *eps_dev);

/* ----------------------------------------------------------- time step -- */

/* Advance the current state by nsteps >= 0 steps of the final LBE with P_i and
 * F_i.  Long runs replay a captured CUDA graph.  Errors: VANS_ERR_STATE before
 * vans_set_eps, VANS_ERR_ARG for nsteps < 0, VANS_ERR_CUDA. */
int vans_step(vans_t h, int nsteps);

/* nsteps steps that watch themselves (no extra pass over the populations):
 * the last step of every block of `every` steps (every >= 1; also the last of
 * the call) writes rho (dense N floats) and u (dense D*N floats) of the state
 * it reads -- the moments of Eqs. 0moment and 1moment, as vans_moments gives --
 * and reduces, over all cells, into stats_dev (device float[4], cleared at the
 * call): [0] max |u - u_prev| with u_prev what u_dev held before that step
 * (convergence; the first comparison is against u_dev's contents on entry),
 * [1] max |u|, [2] 1.0 if a non-finite state or |u| >= 0.5 was met, [3] the
 * number of monitoring steps.  Stats [0] and [1] are the maxima over all
 * monitoring steps of the call. */
int vans_step_monitored(vans_t h, int nsteps, int every, float *rho_dev, float *u_dev,
                        float *stats_dev);

/* One step from the caller's state buffer `in` to the caller's state buffer
 * `out` (both vans_state_floats() floats; they must not overlap).  Uses the
 * handle's eps and parameters; the handle's own state is untouched. */
int vans_step_raw(vans_t h, const float *in, float *out);

/* rho (dense, N floats) and u (dense, D*N floats) of the current state: the
 * moments of Eqs. 0moment and 1moment, with the drag solved in closed form.
 * Either pointer may be NULL to skip it. */
int vans_moments(vans_t h, float *rho_dev, float *u_dev);

/* Physical populations f_i(x, t) of the current state, dense [q][nz][ny][nx]. */
int vans_get_populations(vans_t h, float *f_dev);

/* Replace the current state by the physical populations f (dense [q][nz][ny][nx]). */
int vans_set_populations(vans_t h, const float *f_dev);

/* Raw copies of the current state (checkpoints; vans_state_floats() floats). */
int vans_get_state(vans_t h, float *state_dev);
int vans_set_state(vans_t h, const float *state_dev);

/* Pick the fastest launch configuration for this domain by timing candidates
 * on the handle's own buffers (the state is not changed), each as a CUDA graph
 * of its launches replayed the way vans_step issues them.  Synchronises.
 * `chosen` may be NULL. */
int vans_autotune(vans_t h, vans_launch *chosen);

/* Read or force the launch configuration (invalid values give VANS_ERR_ARG). */
int vans_get_launch(vans_t h, vans_launch *cfg);
int vans_set_launch(vans_t h, const vans_launch *cfg);

/* -------------------------------------------------------------- adjoint -- */
/* Reverse mode for J = sum over the plane x = x_out of eps*rho*u_x (Eq. 1moment)
 * at the final step.  A "lambda" buffer has the state layout and holds dJ/df*
 * of the populations a state buffer stores.  grad_acc is dense, 2 * (1 + D) * N
 * floats: the running sums of dJ/deps(x) and of dJ/d(grad eps)(x) per
 * component ((1 + D) * N floats), then their FP32 compensation words (same
 * layout): the accumulation is compensated (Neumaier), because dJ/deps is a
 * small residual of large grad-eps sensitivities that cancel in the
 * transposed stencil. */

/* J of a state buffer (NULL = the current state) written to J_dev[0] (FP32,
 * fixed-order reduction).  Errors: VANS_ERR_ARG for x_out outside [0, nx). */
int vans_flux(vans_t h, const float *state, int x_out, float *J_dev);

/* Start the reverse pass: lam (lambda of `state`, NULL = current state) is set
 * to dJ/df*; grad_acc is overwritten with the direct partials of J. */
int vans_flux_seed(vans_t h, const float *state, int x_out, float *lam_dev, float *grad_acc);

/* One reverse step through the forward step that read `state_t`: lam_out =
 * (d step / d state)^T lam_in, and the eps partials of that step are added
 * into grad_acc.  state_t, lam_in and lam_out must be distinct buffers. */
int vans_step_adjoint(vans_t h, const float *state_t, const float *lam_in, float *lam_out,
                      float *grad_acc);

/* The reverse pass over one checkpointed segment in one call: copies the
 * checkpoint `ckpt` (a state) into seg[0], recomputes len >= 1 forward steps
 * seg[k] -> seg[k+1] with the step kernel (so the states equal the forward
 * run's), then applies len reverse steps from seg[len-1] down to seg[0].  On
 * entry lam holds the lambda of seg[len]; on return the lambda of seg[0].  seg
 * is (len+1) state buffers back to back; tmp is a second lambda buffer; the
 * eps partials are added into grad_acc.  The work is captured once per
 * (buffers, len) into a CUDA graph and replayed on later calls. */
int vans_adjoint_segment(vans_t h, const float *ckpt, float *seg, int len, float *lam, float *tmp,
                         float *grad_acc);

/* Launch shape of the reverse step.  kind 0: register-load kernel, cpt cells
 * per lane (1, or 2 for D2Q9), `warps` x `rows` threads per block (at most 8
 * warps).  kind 1 (the default: cpt 1, 4 warps, 4 stages for D2Q9, 2 for
 * D3Q19): bulk-copy pipeline
 * with a producer warp, persistent CTAs over the row tiles; `warps` compute
 * warps (D2Q9: 2 with cpt 1, or 4 with cpt 1 or 2; D3Q19: 4 with cpt 1),
 * `rows` = pipeline stages (2..8); ctas must be 0.  VANS_ERR_ARG otherwise. */
int vans_set_adjoint_launch(vans_t h, const vans_launch *cfg);

/* Arithmetic of the per-cell reverse step: 32 (FP32, the default) or 64 (FP64;
 * loads, stores and the compensated accumulation stay FP32).  The eps gradient
 * is a small residual of large grad-eps sensitivities, so FP32 per-cell
 * rounding limits its relative accuracy on long rollouts.  VANS_ERR_ARG for
 * other values. */
int vans_set_adjoint_precision(vans_t h, int bits);

/* dJ/deps (dense, N floats) from the lambda of the initial state and grad_acc:
 * adds the initial condition f = w eps and the transposed grad-eps stencil. */
int vans_grad_finalize(vans_t h, const float *lam0, const float *grad_acc, float *dJdeps_dev);

/* -------------------------------------------------------------- batched -- */
/* n independent D2Q9 domains (each its own size, eps, tau and parameters)
 * advanced by one persistent kernel per step over a flattened tile list.  The
 * domain index d selects a domain in the calls that take it. */

size_t vans_batch_workspace_bytes(const vans_params *p, int n);
int vans_batch_create(const vans_params *p, int n, void *workspace, size_t workspace_bytes,
                      void *cuda_stream, vans_t *out);
/* eps of domain d (dense ny*nx floats); resets that domain to rest. */
int vans_batch_set_eps(vans_t h, int d, const float *eps_dev);
int vans_batch_step(vans_t h, int nsteps);
int vans_batch_moments(vans_t h, int d, float *rho_dev, float *u_dev);
int vans_batch_get_populations(vans_t h, int d, float *f_dev);
/* vans_autotune for the batch: the candidates are timed the same way, and the
 * step tables rebuilt for the pick. */
int vans_batch_autotune(vans_t h, vans_launch *chosen);

/* One batched step (the same update as vans_batch_step(h, 1)) that also
 * records, per CTA, {SM id, start, end} in nanoseconds of the GPU's global
 * timer: 3 words per CTA into records_dev (device memory of `capacity` words,
 * owned by the caller; unused slots stay 0).  With records_dev NULL only
 * *n_records, the number of CTA slots a step can use, is set (the capacity
 * must be 3 * *n_records).  The caller derives the load balance, e.g. the
 * mean over SMs of their busy span over the step's makespan.  The pipelined
 * kinds only (2, 4-7): VANS_ERR_UNSUPPORTED for kind 0. */
int vans_batch_profile_step(vans_t h, unsigned long long *records_dev, long long capacity,
                            long long *n_records);
/* Cells summed over all domains. */
long long vans_batch_cells(vans_t h);

/* ------------------------------------------------- no-allocation step --- */

/* One step from state_in to state_out (vans_state_floats(p) floats each;
 * the two ranges must not overlap, else VANS_ERR_ARG; without a moving wall
 * an all-zero buffer is the rest state f = w eps) for a
 * caller that cannot allocate device memory or hand the library a workspace:
 * code that runs inside another framework's memory pool or allocator, code that
 * may not call cudaMalloc while a CUDA graph is being captured, or an embedded
 * host whose device memory budget is fixed in advance.  It needs no handle and
 * allocates nothing: the only scratch the step uses besides the caller's
 * buffers, the padded copy of eps (dense nx*ny*nz floats, 0 < eps <= 1; not
 * range-checked here), is a 16 MiB array that the library holds in device
 * memory on every GPU where it is loaded, until the process exits.
 * Limit: ny*nz rows times the padded row length (nx rounded up to 128, plus 9
 * for D2Q9 or 33 for D3Q19, rounded up to 32 floats) must not exceed 4 Mi
 * floats, e.g. a D2Q9 domain of 2048 x 2016
 * cells, or a D3Q19 cube of up to 128^3 (from 129 cells on the padded row
 * jumps to 320 floats); larger domains get VANS_ERR_ARG.
 * Parameter errors as in vans_create.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * All calls share the array, so calls whose GPU work overlaps (on different
 * streams or threads) race and must be serialised by the caller.  The paper has
 * no counterpart to this entry point. */
int vans_step_static(const vans_params *p, const float *eps_dev, const float *state_in,
                     float *state_out, void *cuda_stream);

/* -------------------------------------------------- slabs along x --- */
/* A domain too large for one GPU is cut along x, its periodic axis, into
 * slabs of whole columns, one handle per slab (each created with its own nx).
 * The paper credits the scheme's explicit update with its parallelism
 * (abstract and introduction): in the final LBE a cell's next populations
 * come from its neighbours' post-collision ones only, so across a cut only
 * the populations that stream over it have to move, once per step: those
 * with e_x = +1 (D2Q9: 3, D3Q19: 5) of a slab's last column go right, those
 * with e_x = -1 of its first column go left.  The cycle per step, for every
 * slab: vans_step(h, 1), vans_halo_pack, the exchange of the packed messages
 * (a device copy on one GPU, a send/recv between GPUs; the caller's), then
 * vans_halo_unpack.  A message holds vans_halo_floats(h) floats, laid out
 * [k][row] with k the k-th direction (index order) of that x sign and row =
 * z * ny + y.  The y and z walls are those of the whole domain. */

/* Floats of one halo message of this handle, or -1 for a batch or NULL. */
long long vans_halo_floats(vans_t h);

/* vans_set_eps for a slab: eps_dev is the slab's own field (dense, its nx
 * columns), eps_left and eps_right the porosity of the column just left of
 * the slab and just right of it (the neighbouring slabs' edge columns; dense,
 * ny * nz floats each, row = z * ny + y), which the slab's edge cells read
 * for grad eps (Eq. pi) and for the populations they send across.  All
 * values must lie in (0, 1], else VANS_ERR_ARG and nothing changes.  The
 * handle then steps one step per vans_step call (VANS_ERR_UNSUPPORTED for
 * nsteps > 1, for vans_step_monitored, vans_update_eps and the reverse
 * pass) until the next vans_set_eps.  Synchronises. */
int vans_set_eps_slab(vans_t h, const float *eps_dev, const float *eps_left,
                      const float *eps_right);

/* The messages of the current state: to_left gets the first column's
 * populations with e_x = -1, to_right the last column's with e_x = +1
 * (vans_halo_floats(h) floats each, distinct device buffers). */
int vans_halo_pack(vans_t h, float *to_left, float *to_right);

/* Write the neighbours' messages into the current state: from_left is the
 * left neighbour's to_right, from_right the right neighbour's to_left.  A
 * single slab that is its own neighbour (from_left = its to_right) gets the
 * same state as the periodic wrap of vans_step. */
int vans_halo_unpack(vans_t h, const float *from_left, const float *from_right);

/* ---------------------------------------------------------------- misc --- */

/* Total cells of the handle (single domain: nx*ny*nz). */
long long vans_cells(vans_t h);

/* Number of kernel launches this handle has enqueued so far (graph replays
 * count every kernel node they contain). */
long long vans_launch_count(vans_t h);

/* Check the current state for non-finite values or |u| >= 0.5 (Mach ~0.9);
 * returns VANS_OK or VANS_ERR_DIVERGED, VANS_ERR_TIMEOUT if a bounded device
 * wait of a step kernel gave up, VANS_ERR_ARG if the field of the last
 * vans_set_eps_async was out of range.  Synchronises. */
int vans_check(vans_t h);

const char *vans_status_string(int status);
const char *vans_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VANS_H */
