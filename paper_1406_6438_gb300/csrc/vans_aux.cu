// vans_aux.cu -- everything around the step: porosity set-up, moments, state
// import/export, divergence check, outlet flux, and the register-load form of
// the reverse-mode adjoint step (the pipelined one is in vans_adjoint_tma.cu).
#include "vans_adjoint.cuh"
#include "vans_device.cuh"

namespace vans {

// ------------------------------------------------------- scalar helpers ----
template <int Q>
__device__ __forceinline__ void nb_yz(const VDom &d, int y, int z, Nb3 &Y, Nb3 &Z) {
    Y = nb3<true>(y, d.ny, d.wall_y);
    if (Q == 19) {
        Z = nb3<true>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }
}

// Index, within a state buffer, of the stored value that the pull of cell
// (x,y,z) reads for direction i (periodic x through the halo, bounce-back at
// walls).  This map is a bijection onto the live entries of the buffer.
template <int Q>
__device__ __forceinline__ long long pull_index(const VDom &d, int i, int x, int y, int z,
                                                const Nb3 &Y, const Nb3 &Z) {
    using L = Lat<Q>;
    const int ey = L::ey(i), ez = L::ez(i);
    const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
    if (bb) return L::opp(i) * d.plane + row_offset(d, y, z) + x;
    return i * d.plane + row_offset(d, Y.r[1 - ey], Z.r[1 - ez]) + x - L::ex(i);
}

template <int Q>
__device__ __forceinline__ void eps_cell(const VDom &d, int x, int y, int z, const Nb3 &Y,
                                         const Nb3 &Z, float &e0, float et[Q]) {
    using L = Lat<Q>;
    e0 = d.eps[row_offset(d, y, z) + x];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool wall = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
        et[i] = (i == 0 || wall)
                    ? e0
                    : d.eps[row_offset(d, Y.r[1 + L::ey(i)], Z.r[1 + L::ez(i)]) + x + L::ex(i)];
    }
}

template <int Q>
__device__ __forceinline__ void pull_cell(const VDom &d, const float *__restrict__ st, int x, int y,
                                          int z, const Nb3 &Y, const Nb3 &Z, float h[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = st[pull_index<Q>(d, i, x, y, z, Y, Z)];
}

__device__ __forceinline__ void cell_xyz(const VDom &d, long long n, int &x, int &y, int &z) {
    if (d.cells <= 0xffffffffLL) {                // 32-bit divisions where they suffice
        const unsigned m = (unsigned)n, nx = (unsigned)d.nx, ny = (unsigned)d.ny;
        const unsigned r = m / nx;
        x = (int)(m - r * nx);
        y = (int)(r % ny);
        z = (int)(r / ny);
        return;
    }
    x = (int)(n % d.nx);
    const long long r = n / d.nx;
    y = (int)(r % d.ny);
    z = (int)(r / d.ny);
}

// Populations (as deviations from w_i eps(x)) that cell (x,y,z) holds before
// its collision: pulled from the state, or, for a plate node (wall_kind 1),
// f^eq(eps_b, rho_f, u_b) plus its fluid neighbour's non-equilibrium part.
template <int Q>
__device__ __forceinline__ void cell_state(const VDom &d, const float *__restrict__ st, int x, int y,
                                           int z, const Nb3 &Y, const Nb3 &Z, float h[Q]) {
    if (d.nee && (y == 0 || y == d.ny - 1)) {
        const int yf = (y == 0) ? 1 : d.ny - 2;
        Nb3 Yf, Zf;
        nb_yz<Q>(d, yf, z, Yf, Zf);
        float hf[Q], ef, etf[Q];
        pull_cell<Q>(d, st, x, yf, z, Yf, Zf, hf);
        eps_cell<Q>(d, x, yf, z, Yf, Zf, ef, etf);
        Macro<Q> M;
        macro<Q>(d, hf, ef, etf, M);
        const float eb = d.eps[row_offset(d, y, z) + x];
        const float zero[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < Q; ++i)
            h[i] = plate_value<Q>(d, i, hf[i], M, eb, eb, y == 0 ? zero : d.uw, 1.f);
        return;
    }
    pull_cell<Q>(d, st, x, y, z, Y, Z, h);
    apply_moving_wall<Q>(d, Y.wall[2], Z, d.eps[row_offset(d, y, z) + x], h);
}

// --------------------------------------------------------------- S8 -----
// rho and u of the current state (Eqs. 0moment and 1moment, drag in closed form)
template <int Q>
__global__ void k_moments(const VDom d, const float *__restrict__ st, float *__restrict__ rho,
                          float *__restrict__ u) {
    constexpr int D = Lat<Q>::D;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        float h[Q], e0, et[Q];
        cell_state<Q>(d, st, x, y, z, Y, Z, h);
        eps_cell<Q>(d, x, y, z, Y, Z, e0, et);
        Macro<Q> M;
        macro<Q>(d, h, e0, et, M);
        if (rho) rho[n] = M.rho;
        if (u) {
#pragma unroll
            for (int c = 0; c < D; ++c) u[c * d.cells + n] = M.u[c];
        }
    }
}

// physical populations f_i = h_i + w_i eps(x), dense [q][N]
template <int Q>
__global__ void k_export(const VDom d, const float *__restrict__ st, float *__restrict__ f) {
    using L = Lat<Q>;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        const float e0 = d.eps[row_offset(d, y, z) + x];
        float h[Q];
        cell_state<Q>(d, st, x, y, z, Y, Z, h);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i * d.cells + n] = h[i] + L::w(i) * e0;
    }
}

// Write v into the entry the pull of cell (x,y,z) reads for direction i; a halo
// entry (column -1 or nx) also goes to its mirror at the row's other end
// (column nx-1 or 0), so that the two copies the step kernels leave agree after
// any write: kernels that stage rows without their halo columns read the mirror.
template <int Q>
__device__ __forceinline__ void store_pulled(const VDom &d, float *__restrict__ st, int i, int x,
                                             int y, int z, const Nb3 &Y, const Nb3 &Z, float v) {
    using L = Lat<Q>;
    const long long k = pull_index<Q>(d, i, x, y, z, Y, Z);
    st[k] = v;
    const bool bb = Y.wall[1 - L::ey(i)] || Z.wall[1 - L::ez(i)];
    if (!bb && L::ex(i) > 0 && x == 0) st[k + d.nx] = v;            // column -1 -> nx-1
    if (!bb && L::ex(i) < 0 && x == d.nx - 1) st[k - d.nx] = v;     // column nx -> 0
}

// inverse of k_export: writes every live entry of the state
template <int Q>
__global__ void k_import(const VDom d, const float *__restrict__ f, float *__restrict__ st) {
    using L = Lat<Q>;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        const float e0 = d.eps[row_offset(d, y, z) + x];
        const bool top = d.moving && Y.wall[2];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float v = f[i * d.cells + n] - L::w(i) * e0;
            if (top && L::ey(i) < 0 && !Z.wall[1 - L::ez(i)]) v -= wall_gain<Q>(d, i, e0);
            store_pulled<Q>(d, st, i, x, y, z, Y, Z, v);
        }
    }
}

// Rest state f = w eps with a moving upper wall: the all-zero deviation buffer
// would pull w eps plus the wall gain in the top rows, so store minus the gain
// in the entries those rows pull through the moving wall.
template <int Q>
__global__ void k_init_moving(const VDom d, float *__restrict__ st) {
    using L = Lat<Q>;
    const long long n_top = (long long)d.nx * d.nz;        // cells of the rows y = ny-1
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_top;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % d.nx);
        const int z = (int)(t / d.nx);
        const int y = d.ny - 1;
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        const float e0 = d.eps[row_offset(d, y, z) + x];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::ey(i) < 0 && !Z.wall[1 - L::ez(i)])
                st[pull_index<Q>(d, i, x, y, z, Y, Z)] = -wall_gain<Q>(d, i, e0);
    }
}

// A new porosity field under an unchanged physical state f: every live entry
// stores f - w eps~ (minus the moving-wall gain where one applies), so it is
// re-expressed from the old eps (the padded rows still in d.eps) to the new
// one (dense eps_new).  Each entry belongs to exactly one cell (pull_index is
// a bijection), so the update runs in place.
template <int Q>
__global__ void k_rebase_eps(const VDom d, const float *__restrict__ eps_new, float *__restrict__ st) {
    using L = Lat<Q>;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        const float e_old = d.eps[row_offset(d, y, z) + x];
        const float e_new = eps_new[n];
        const bool top = d.moving && Y.wall[2];
        // every entry read before any is written: interleaved, each load had to
        // wait for the store before it (the same pointer)
        float v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = st[pull_index<Q>(d, i, x, y, z, Y, Z)];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            v[i] += L::w(i) * (e_old - e_new);
            if (top && L::ey(i) < 0 && !Z.wall[1 - L::ez(i)])
                v[i] += wall_gain<Q>(d, i, e_old) - wall_gain<Q>(d, i, e_new);
            store_pulled<Q>(d, st, i, x, y, z, Y, Z, v[i]);
        }
    }
}

// eps into padded rows with periodic halo columns; padding gets 1.0.  Flags any
// value outside (0, 1] (NaN included).
__global__ void k_pad_eps(const VDom d, const float *__restrict__ eps, float *__restrict__ pad,
                          int *flag) {
    const long long total = (long long)d.rows * d.pitch;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long r;
        int c;
        if (total <= 0xffffffffLL) {            // 32-bit division where it suffices
            const unsigned tt = (unsigned)t, rr = tt / (unsigned)d.pitch;
            r = rr;
            c = (int)(tt - rr * (unsigned)d.pitch) - d.off;
        } else {
            r = t / d.pitch;
            c = (int)(t % d.pitch) - d.off;
        }
        float v = 1.0f;
        if (c >= 0 && c < d.nx) {
            v = eps[r * d.nx + c];
            if (!(v > 0.0f && v <= 1.0f)) atomicOr(flag, 1);
            if (pad == nullptr) continue;       // range check only
        } else if (pad == nullptr) {
            continue;
        } else if (c == -1) {
            v = eps[r * d.nx + d.nx - 1];
        } else if (c == d.nx) {
            v = eps[r * d.nx];
        }
        pad[t] = v;
    }
}

template <int Q>
__global__ void k_check(const VDom d, const float *__restrict__ st, int *flag) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        float h[Q], e0, et[Q];
        cell_state<Q>(d, st, x, y, z, Y, Z, h);
        eps_cell<Q>(d, x, y, z, Y, Z, e0, et);
        Macro<Q> M;
        macro<Q>(d, h, e0, et, M);
        if (!isfinite(M.R) || !isfinite(M.un) || !(M.un < 0.5f)) atomicOr(flag, 1);
    }
}

// ------------------------------------------------------ reverse mode -----

// J = sum over the plane x = x_out of eps rho u_x; one block, fixed-order sum.
template <int Q>
__global__ void __launch_bounds__(256) k_flux(const VDom d, const float *__restrict__ st, int x_out, float *J) {
    __shared__ float red[256];
    float acc = 0.f;
    for (int r = threadIdx.x; r < d.rows; r += blockDim.x) {
        const int y = r % d.ny, z = r / d.ny;
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        float h[Q], e0, et[Q];
        cell_state<Q>(d, st, x_out, y, z, Y, Z, h);
        eps_cell<Q>(d, x_out, y, z, Y, Z, e0, et);
        Macro<Q> M;
        macro<Q>(d, h, e0, et, M);
        acc += M.R * M.u[0];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) J[0] = red[0];
}

// Seed of the reverse pass: lambda at the entries the outlet cells pull, and
// the direct eps / grad-eps partials of J.  lam and grad are zeroed beforehand.
template <int Q, typename T>
__global__ void k_flux_seed(const VDom d, const float *__restrict__ st, int x_out,
                            float *__restrict__ lam, float *__restrict__ grad) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < d.rows; r += gridDim.x * blockDim.x) {
        const int y = r % d.ny, z = r / d.ny;
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        float h[Q], e0, et[Q];
        pull_cell<Q>(d, st, x_out, y, z, Y, Z, h);
        eps_cell<Q>(d, x_out, y, z, Y, Z, e0, et);
        apply_moving_wall<Q>(d, Y.wall[2], Z, e0, h);
        MacroT<Q, T> M;
        macro_t<Q, T>(d, h, e0, et, M);
        // J_cell = R u_x
        T ubar[3] = {M.R, T(0), T(0)}, Vbar[3] = {T(0), T(0), T(0)};
        T lam0, jbar[3], ebar, gbar[3];
        macro_vjp_t<Q, T>(d, M, M.u[0], ubar, Vbar, lam0, jbar, ebar, gbar);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T l = lam0;
            if (L::ex(i)) l += L::ex(i) * jbar[0];
            if (L::ey(i)) l += L::ey(i) * jbar[1];
            if (D == 3 && L::ez(i)) l += L::ez(i) * jbar[2];
            lam[pull_index<Q>(d, i, x_out, y, z, Y, Z)] = (float)l;
        }
        const long long n = (long long)r * d.nx + x_out;
        const long long nc = (1 + D) * d.cells;   // sums and compensations were zeroed
        acc2_term(&grad[n], &grad[nc + n], ebar);
#pragma unroll
        for (int c = 0; c < D; ++c)
            acc2_term(&grad[(1 + c) * d.cells + n], &grad[nc + (1 + c) * d.cells + n], gbar[c]);
    }
}

// One reverse step (S9): the transposed Jacobian of one forward step applied to
// lambda.  The forward state is pulled exactly as the step pulls it; lambda of
// the step's outputs is read where the step wrote the copy that is streamed on
// (the halo column at the periodic seam); the result is scattered to the very
// entries the pull read, so the scatter is a permutation and needs no atomics.
template <int Q, int CPT, bool EDGE, typename T>
__device__ __forceinline__ void adj_row(const VDom &d, const float *__restrict__ st,
                                        const float *__restrict__ lin, float *__restrict__ lout,
                                        float *__restrict__ grad, int y, int z, int x0, int lane) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    const Nb3 Y = nb3<EDGE>(y, d.ny, d.wall_y);
    Nb3 Z;
    if (Q == 19) {
        Z = nb3<EDGE>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }
    float h[Q][CPT];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long ro = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        ld_shift<CPT>(st + si * d.plane + ro, x0, bb ? 0 : -ex, lane, h[i]);
    }
    float E[3][3][CPT + 2];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if (Q == 9 && dz != 0) continue;
            const float *row = d.eps + row_offset(d, Y.r[1 + dy], Z.r[1 + dz]);
            if (dy != 0 && dz != 0) {
                float t[CPT];
                ld_vec<CPT>(row + x0, t);
#pragma unroll
                for (int k = 0; k < CPT; ++k) E[1 + dy][1 + dz][k + 1] = t[k];
            } else {
                ld_ext<CPT>(row, x0, lane, E[1 + dy][1 + dz]);
            }
        }
    }
    const long long ro = row_offset(d, y, z);
    float mu[Q][CPT];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *row = lin + i * d.plane + ro;
        ld_vec<CPT>(row + x0, mu[i]);
        const bool wall_out = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
        if (!wall_out && L::ex(i) > 0) {
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                if (x0 + k == d.nx - 1) mu[i][k] = row[-1];
        }
        if (!wall_out && L::ex(i) < 0 && x0 == 0) mu[i][0] = row[d.nx];
    }
    float lam[Q][CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        float hh[Q], et[Q], mm[Q], ll[Q];
        const float e0 = E[1][1][k + 1];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            hh[i] = h[i][k];
            mm[i] = mu[i][k];
            const bool wall = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
            et[i] = (i == 0 || wall) ? e0 : E[1 + L::ey(i)][1 + L::ez(i)][k + 1 + L::ex(i)];
        }
        if (EDGE) apply_moving_wall<Q>(d, Y.wall[2], Z, e0, hh);
        T ebar, gbar[3];
        collide_vjp_t<Q, T>(d, hh, e0, et, mm, ll, ebar, gbar);
        if (EDGE && d.moving && Y.wall[2]) {
            // the populations this cell sends into the moving wall come back
            // as their opposites with a gain that is linear in eps(x)
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ey(i) > 0 && !Z.wall[1 + L::ez(i)])
                    ebar += (T)wall_gain<Q>(d, L::opp(i), 1.f) * (T)mm[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[i][k] = ll[i];
        if (x0 + k < d.nx) {
            const long long n = ((long long)z * d.ny + y) * d.nx + x0 + k;
            const long long nc = (1 + D) * d.cells;   // compensation words follow the sums
            acc2_term(&grad[n], &grad[nc + n], ebar);
#pragma unroll
            for (int c = 0; c < D; ++c)
                acc2_term(&grad[(1 + c) * d.cells + n], &grad[nc + (1 + c) * d.cells + n], gbar[c]);
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long rs = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        st_shift<CPT>(lout + si * d.plane + rs, x0, bb ? 0 : -ex, lane, lam[i]);
    }
}

template <int Q, int CPT, typename T>
__global__ void __launch_bounds__(256) k_step_adjoint(const VDom d, const float *__restrict__ st,
                                                      const float *__restrict__ lin,
                                                      float *__restrict__ lout,
                                                      float *__restrict__ grad, int nxb) {
    const int lane = threadIdx.x & 31;
    const int wx = threadIdx.x >> 5;
    const int bx = blockIdx.x % nxb;
    const int by = blockIdx.x / nxb;
    const int r = by * blockDim.y + threadIdx.y;
    if (r >= d.rows) return;
    const int xw = (bx * (blockDim.x >> 5) + wx) * 32 * CPT;
    if (xw >= d.nx) return;
    const int x0 = xw + lane * CPT;
    const int y = r % d.ny, z = r / d.ny;
    const bool edge = (y == 0) || (y == d.ny - 1) || (Q == 19 && (z == 0 || z == d.nz - 1));
    if (edge)
        adj_row<Q, CPT, true, T>(d, st, lin, lout, grad, y, z, x0, lane);
    else
        adj_row<Q, CPT, false, T>(d, st, lin, lout, grad, y, z, x0, lane);
}

// dJ/deps = G_eps + sum_i w_i lambda_i(0) (from f(0) = w eps) + the transposed
// grad-eps stencil applied to G_grad.  Runs once per reverse pass; it combines
// each compensated accumulator (sum + compensation) and evaluates the stencil,
// whose terms cancel to a much smaller result, in FP64.
template <int Q>
__global__ void k_grad_finalize(const VDom d, const float *__restrict__ lam0,
                                const float *__restrict__ grad, float *__restrict__ out) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    const long long nc = (1 + D) * d.cells;
    auto G = [&](int comp, long long m) -> double {
        return (double)grad[comp * d.cells + m] + (double)grad[nc + comp * d.cells + m];
    };
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        double v = G(0, n);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            v += (double)L::w(i) * (double)lam0[pull_index<Q>(d, i, x, y, z, Y, Z)];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
            // cell x - e_i, whose stencil reads eps(x) through direction i
            if (!(Y.wall[1 - e[1]] || Z.wall[1 - e[2]])) {
                int xs = x - e[0];
                xs = xs < 0 ? xs + d.nx : (xs >= d.nx ? xs - d.nx : xs);
                const long long m = ((long long)Z.r[1 - e[2]] * d.ny + Y.r[1 - e[1]]) * d.nx + xs;
                double s = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) s += e[c] * G(1 + c, m);
                v += 3.0 * (double)L::w(i) * s;
            }
            // x itself, whose neighbour x + e_i lies past a wall
            if (Y.wall[1 + e[1]] || Z.wall[1 + e[2]]) {
                double s = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) s += e[c] * G(1 + c, n);
                v += 3.0 * (double)L::w(i) * s;
            }
        }
        out[n] = (float)v;
    }
}

// --------------------------------------------------------------- launch ---
// ------------------------------------------------------ slabs along x ----
// A domain cut along x into slabs: the pull of a slab's column 0 reads the
// halo column -1 for the directions with e_x = +1, and that of its last column
// reads column nx for e_x = -1.  These entries belong to the neighbouring
// slabs' edge cells, so after every step each slab sends its last column's
// e_x = +1 entries to the right and its first column's e_x = -1 entries to
// the left.  A message is [k][row], k the k-th direction with e_x = +1 (resp.
// -1) in index order, row = z * ny + y.

// the k-th direction (index order) whose x component is sx
template <int Q>
__host__ __device__ constexpr int xdir(int sx, int k) {
    for (int i = 0, n = 0; i < Q; ++i)
        if (Lat<Q>::ex(i) == sx && n++ == k) return i;
    return -1;
}

template <int Q>
__host__ __device__ constexpr int n_xdirs() {
    int n = 0;
    for (int i = 0; i < Q; ++i) n += Lat<Q>::ex(i) == 1;
    return n;
}

template <int Q>
__global__ void k_halo_pack(const VDom d, const float *__restrict__ st, float *__restrict__ to_left,
                            float *__restrict__ to_right) {
    constexpr int NX = n_xdirs<Q>();
    const long long total = (long long)d.rows * NX;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / d.rows);
        const long long r = t - (long long)k * d.rows;
        const long long ro = r * d.pitch + d.off;
        int ip = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NX; ++j)
            if (j == k) { ip = xdir<Q>(1, j); im = xdir<Q>(-1, j); }
        to_right[t] = st[ip * d.plane + ro + d.nx - 1];
        to_left[t] = st[im * d.plane + ro];
    }
}

template <int Q>
__global__ void k_halo_unpack(const VDom d, float *__restrict__ st, const float *__restrict__ from_left,
                              const float *__restrict__ from_right) {
    constexpr int NX = n_xdirs<Q>();
    const long long total = (long long)d.rows * NX;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / d.rows);
        const long long r = t - (long long)k * d.rows;
        const long long ro = r * d.pitch + d.off;
        int ip = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NX; ++j)
            if (j == k) { ip = xdir<Q>(1, j); im = xdir<Q>(-1, j); }
        st[ip * d.plane + ro - 1] = from_left[t];
        st[im * d.plane + ro + d.nx] = from_right[t];
    }
}

// The porosity halo columns of a slab: column -1 from the left neighbour's
// last column, column nx from the right neighbour's first (dense, one value
// per row).  Values outside (0, 1] set *flag; pad == nullptr checks only.
__global__ void k_eps_halo(const VDom d, const float *__restrict__ left,
                           const float *__restrict__ right, float *__restrict__ pad, int *flag) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < d.rows;
         r += (long long)gridDim.x * blockDim.x) {
        const float a = left[r], b = right[r];
        if (!(a > 0.0f && a <= 1.0f) || !(b > 0.0f && b <= 1.0f)) atomicOr(flag, 1);
        if (pad) {
            pad[r * d.pitch + d.off - 1] = a;
            pad[r * d.pitch + d.off + d.nx] = b;
        }
    }
}

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

#define VANS_DISPATCH_Q(q, CALL9, CALL19) \
    do {                                  \
        if ((q) == 9) { CALL9; }          \
        else if ((q) == 19) { CALL19; }   \
        else return cudaErrorInvalidValue; \
    } while (0)

cudaError_t launch_moments(int q, const VDom &d, const float *state, float *rho, float *u,
                           cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_moments<9><<<g, 256, 0, s>>>(d, state, rho, u)),
                    (k_moments<19><<<g, 256, 0, s>>>(d, state, rho, u)));
    return cudaGetLastError();
}

cudaError_t launch_export(int q, const VDom &d, const float *state, float *f, cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_export<9><<<g, 256, 0, s>>>(d, state, f)),
                    (k_export<19><<<g, 256, 0, s>>>(d, state, f)));
    return cudaGetLastError();
}

cudaError_t launch_import(int q, const VDom &d, const float *f, float *state, cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_import<9><<<g, 256, 0, s>>>(d, f, state)),
                    (k_import<19><<<g, 256, 0, s>>>(d, f, state)));
    return cudaGetLastError();
}

cudaError_t launch_pad_eps(const VDom &d, const float *eps_dense, float *eps_pad, int *flag,
                           cudaStream_t s) {
    const int g = grid_for((long long)d.rows * d.pitch, 256);
    k_pad_eps<<<g, 256, 0, s>>>(d, eps_dense, eps_pad, flag);
    return cudaGetLastError();
}

cudaError_t launch_rebase_eps(int q, const VDom &d, const float *eps_new, float *state,
                              cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_rebase_eps<9><<<g, 256, 0, s>>>(d, eps_new, state)),
                    (k_rebase_eps<19><<<g, 256, 0, s>>>(d, eps_new, state)));
    return cudaGetLastError();
}

cudaError_t launch_init_moving(int q, const VDom &d, float *state, cudaStream_t s) {
    if (!d.moving || !d.wall_y) return cudaSuccess;
    const int g = grid_for((long long)d.nx * d.nz, 256);
    VANS_DISPATCH_Q(q, (k_init_moving<9><<<g, 256, 0, s>>>(d, state)),
                    (k_init_moving<19><<<g, 256, 0, s>>>(d, state)));
    return cudaGetLastError();
}

cudaError_t launch_check(int q, const VDom &d, const float *state, int *flag, cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_check<9><<<g, 256, 0, s>>>(d, state, flag)),
                    (k_check<19><<<g, 256, 0, s>>>(d, state, flag)));
    return cudaGetLastError();
}

cudaError_t launch_flux(int q, const VDom &d, const float *state, int x_out, float *J,
                        cudaStream_t s) {
    VANS_DISPATCH_Q(q, (k_flux<9><<<1, 256, 0, s>>>(d, state, x_out, J)),
                    (k_flux<19><<<1, 256, 0, s>>>(d, state, x_out, J)));
    return cudaGetLastError();
}

cudaError_t launch_flux_seed(int q, const VDom &d, const float *state, int x_out, float *lam,
                             float *grad, int fp64, cudaStream_t s) {
    const int g = grid_for(d.rows, 256);
    if (fp64)
        VANS_DISPATCH_Q(q, (k_flux_seed<9, double><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)),
                        (k_flux_seed<19, double><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)));
    else
        VANS_DISPATCH_Q(q, (k_flux_seed<9, float><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)),
                        (k_flux_seed<19, float><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)));
    return cudaGetLastError();
}

template <int Q, int CPT, typename T>
static cudaError_t launch_adj_t(const VDom &d, const float *state, const float *lam_in,
                                float *lam_out, float *grad, Launch L, cudaStream_t s) {
    const int nxb = (d.nx + 32 * CPT * L.warps - 1) / (32 * CPT * L.warps);
    const int nrb = (d.rows + L.rows - 1) / L.rows;
    const long long nb = (long long)nxb * nrb;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 block(32 * L.warps, L.rows);
    k_step_adjoint<Q, CPT, T><<<(unsigned)nb, block, 0, s>>>(d, state, lam_in, lam_out, grad, nxb);
    return cudaGetLastError();
}

// kind 0: the register-load kernel, L.cpt cells per lane (1 or 2; D3Q19 takes 1),
// L.warps x L.rows threads per block; kind 1: the bulk-copy pipeline kernel
cudaError_t launch_step_adjoint(int q, const VDom &d, const float *state, const float *lam_in,
                                float *lam_out, float *grad, int fp64, Launch L, cudaStream_t s) {
    if (L.kind == 1) return launch_adjoint_tma(q, d, state, lam_in, lam_out, grad, fp64, L, s);
    if (L.kind != 0) return cudaErrorInvalidValue;
    if (L.warps < 1 || L.rows < 1 || L.warps * L.rows > 8) return cudaErrorInvalidValue;
    if (q == 9 && L.cpt == 2)
        return fp64 ? launch_adj_t<9, 2, double>(d, state, lam_in, lam_out, grad, L, s)
                    : launch_adj_t<9, 2, float>(d, state, lam_in, lam_out, grad, L, s);
    if (q == 9 && L.cpt == 1)
        return fp64 ? launch_adj_t<9, 1, double>(d, state, lam_in, lam_out, grad, L, s)
                    : launch_adj_t<9, 1, float>(d, state, lam_in, lam_out, grad, L, s);
    if (q == 19 && L.cpt == 1)
        return fp64 ? launch_adj_t<19, 1, double>(d, state, lam_in, lam_out, grad, L, s)
                    : launch_adj_t<19, 1, float>(d, state, lam_in, lam_out, grad, L, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_grad_finalize(int q, const VDom &d, const float *lam0, const float *grad,
                                 float *dJ, cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_grad_finalize<9><<<g, 256, 0, s>>>(d, lam0, grad, dJ)),
                    (k_grad_finalize<19><<<g, 256, 0, s>>>(d, lam0, grad, dJ)));
    return cudaGetLastError();
}

int halo_floats(int q, const VDom &d) {
    return (int)((q == 9 ? n_xdirs<9>() : n_xdirs<19>()) * (long long)d.rows);
}

cudaError_t launch_halo_pack(int q, const VDom &d, const float *state, float *to_left,
                             float *to_right, cudaStream_t s) {
    const int g = grid_for(halo_floats(q, d), 256);
    VANS_DISPATCH_Q(q, (k_halo_pack<9><<<g, 256, 0, s>>>(d, state, to_left, to_right)),
                    (k_halo_pack<19><<<g, 256, 0, s>>>(d, state, to_left, to_right)));
    return cudaGetLastError();
}

cudaError_t launch_halo_unpack(int q, const VDom &d, float *state, const float *from_left,
                               const float *from_right, cudaStream_t s) {
    const int g = grid_for(halo_floats(q, d), 256);
    VANS_DISPATCH_Q(q, (k_halo_unpack<9><<<g, 256, 0, s>>>(d, state, from_left, from_right)),
                    (k_halo_unpack<19><<<g, 256, 0, s>>>(d, state, from_left, from_right)));
    return cudaGetLastError();
}

cudaError_t launch_eps_halo(const VDom &d, const float *left, const float *right, float *eps_pad,
                            int *flag, cudaStream_t s) {
    k_eps_halo<<<grid_for(d.rows, 256), 256, 0, s>>>(d, left, right, eps_pad, flag);
    return cudaGetLastError();
}

}  // namespace vans
