// vans_aux.cu -- everything around the step: porosity set-up, moments, state
// import/export, divergence check, outlet flux, and the reverse-mode adjoint.
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
    x = (int)(n % d.nx);
    const long long r = n / d.nx;
    y = (int)(r % d.ny);
    z = (int)(r / d.ny);
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
        pull_cell<Q>(d, st, x, y, z, Y, Z, h);
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
#pragma unroll
        for (int i = 0; i < Q; ++i)
            f[i * d.cells + n] = st[pull_index<Q>(d, i, x, y, z, Y, Z)] + L::w(i) * e0;
    }
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
#pragma unroll
        for (int i = 0; i < Q; ++i)
            st[pull_index<Q>(d, i, x, y, z, Y, Z)] = f[i * d.cells + n] - L::w(i) * e0;
    }
}

// eps into padded rows with periodic halo columns; padding gets 1.0.  Flags any
// value outside (0, 1] (NaN included).
__global__ void k_pad_eps(const VDom d, const float *__restrict__ eps, float *__restrict__ pad,
                          int *flag) {
    const long long total = (long long)d.rows * d.pitch;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / d.pitch;
        const int c = (int)(t % d.pitch) - VANS_OFF;
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
        pull_cell<Q>(d, st, x, y, z, Y, Z, h);
        eps_cell<Q>(d, x, y, z, Y, Z, e0, et);
        Macro<Q> M;
        macro<Q>(d, h, e0, et, M);
        if (!isfinite(M.R) || !isfinite(M.un) || !(M.un < 0.5f)) atomicOr(flag, 1);
    }
}

// ------------------------------------------------------ reverse mode -----
// Reverse of macro(): given dJ/dR, dJ/du and dJ/dV, returns the part of dJ/dh_i
// common to all i (lam0) plus e_i . jbar, and the partial derivatives of J with
// respect to eps(x) (at fixed f) and grad eps(x).
template <int Q>
__device__ __forceinline__ void macro_vjp(const VDom &d, const Macro<Q> &M, float Rbar,
                                          float ubar[3], const float Vbar[3], float &lam0,
                                          float jbar[3], float &ebar, float gbar[3]) {
    constexpr int D = Lat<Q>::D;
    float Pcbar[3], Fbar[3], mbar[3];
    float Fu = 0.f;
    // V = Pc + F,  F = R g - alpha u - beta |u| u
#pragma unroll
    for (int c = 0; c < D; ++c) {
        Pcbar[c] = Vbar[c];
        Fbar[c] = Vbar[c];
        Rbar += Fbar[c] * d.g[c];
        Fu += Fbar[c] * M.u[c];
    }
    float alphabar = -Fu;
    float betabar = -M.un * Fu;
    const float kd = M.alpha + M.beta * M.un;
    const float ib = (M.un > 0.f) ? M.beta * Fu / M.un : 0.f;
    float ubu = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        ubar[c] += -kd * Fbar[c] - ib * M.u[c];
        ubu += ubar[c] * M.u[c];
    }
    // u = m * 2/D,  D = a + sqrt(a^2 + 4 b |m|)
    const float Dbar = -ubu / M.D;
    const float abar = Dbar * (1.f + M.a / M.sq);
    const float bbar = Dbar * 2.f * M.mm / M.sq;
    const float mmbar = Dbar * 2.f * M.b / M.sq;
    const float im = (M.mm > 0.f) ? mmbar / M.mm : 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) mbar[c] = ubar[c] * M.s + im * M.m[c];
    // a = R + alpha/2, b = beta/2
    Rbar += abar;
    alphabar += 0.5f * abar;
    betabar += 0.5f * bbar;
    // m = j + Pc/2 + R g/2
    float rhobar = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        jbar[c] = mbar[c];
        Pcbar[c] += 0.5f * mbar[c];
        Rbar += 0.5f * mbar[c] * d.g[c];
        // Pc = rho grad eps / 3
        rhobar += (1.f / 3.f) * Pcbar[c] * M.ge[c];
        gbar[c] = (1.f / 3.f) * M.rho * Pcbar[c];
    }
    // rho = R / eps
    Rbar += rhobar * M.inv_e;
    ebar = -rhobar * M.R * M.inv_e * M.inv_e;
    float al, be, da, db;
    drag<true>(d, M.e0, M.inv_e, al, be, &da, &db);
    ebar += alphabar * da + betabar * db;
    lam0 = Rbar;
}

// Reverse of the collision of one cell.  mu_i = dJ/df*_i; returns lam_i =
// dJ/df_i, the eps partial and the grad-eps partial.  With M_i = mu_i w_i,
// SM = sum M_i, SMe = sum M_i e_i and T = sum M_i e_i e_i^T, the adjoints of
// f^eq (Eq. d2q9eq) and of P_i + F_i (Eqs. pi, Fi) reduce to
//   Rbar = omega (SM + 3 SMe.u + 4.5 u.T.u - 1.5 u.u SM)
//   ubar = omega R (3 SMe + 9 T u - 3 u SM) + ct (9 T V - 3 V SM)
//   Vbar = ct (3 SMe - 3 u SM + 9 T u).
template <int Q>
__device__ __forceinline__ void collide_vjp(const VDom &d, const float h[Q], float e0,
                                            const float et[Q], const float mu[Q], float lam[Q],
                                            float &ebar, float gbar[3]) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    Macro<Q> M;
    macro<Q>(d, h, e0, et, M);
    float SM = 0.f, SMe[3] = {0.f, 0.f, 0.f}, T[3][3] = {{0.f}};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float Mi = mu[i] * L::w(i);
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        SM += Mi;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (e[a] == 0) continue;
            SMe[a] += e[a] * Mi;
#pragma unroll
            for (int b = a; b < D; ++b)
                if (e[b] != 0) T[a][b] += (e[a] * e[b]) * Mi;
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < a; ++b) T[a][b] = T[b][a];
    float Tu[3], TV[3], uu = 0.f, SMeu = 0.f, uTu = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Tu[a] = 0.f;
        TV[a] = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            Tu[a] += T[a][b] * M.u[b];
            TV[a] += T[a][b] * M.V[b];
        }
        uu += M.u[a] * M.u[a];
        SMeu += SMe[a] * M.u[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) uTu += M.u[a] * Tu[a];
    const float om = d.omega, ct = d.ctau;
    const float Rbar = om * (SM + 3.f * SMeu + 4.5f * uTu - 1.5f * uu * SM);
    float ubar[3], Vbar[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        ubar[a] = om * M.R * (3.f * SMe[a] + 9.f * Tu[a] - 3.f * M.u[a] * SM) +
                  ct * (9.f * TV[a] - 3.f * M.V[a] * SM);
        Vbar[a] = ct * (3.f * SMe[a] - 3.f * M.u[a] * SM + 9.f * Tu[a]);
    }
    float lam0, jbar[3];
    macro_vjp<Q>(d, M, Rbar, ubar, Vbar, lam0, jbar, ebar, gbar);
    const float om1 = 1.f - om;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float l = om1 * mu[i] + lam0;
        if (L::ex(i)) l += L::ex(i) * jbar[0];
        if (L::ey(i)) l += L::ey(i) * jbar[1];
        if (D == 3 && L::ez(i)) l += L::ez(i) * jbar[2];
        lam[i] = l;
    }
}

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
        pull_cell<Q>(d, st, x_out, y, z, Y, Z, h);
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
template <int Q>
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
        Macro<Q> M;
        macro<Q>(d, h, e0, et, M);
        // J_cell = R u_x
        float ubar[3] = {M.R, 0.f, 0.f}, Vbar[3] = {0.f, 0.f, 0.f};
        float lam0, jbar[3], ebar, gbar[3];
        macro_vjp<Q>(d, M, M.u[0], ubar, Vbar, lam0, jbar, ebar, gbar);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float l = lam0;
            if (L::ex(i)) l += L::ex(i) * jbar[0];
            if (L::ey(i)) l += L::ey(i) * jbar[1];
            if (D == 3 && L::ez(i)) l += L::ez(i) * jbar[2];
            lam[pull_index<Q>(d, i, x_out, y, z, Y, Z)] = l;
        }
        const long long n = (long long)r * d.nx + x_out;
        grad[n] = ebar;
#pragma unroll
        for (int c = 0; c < D; ++c) grad[(1 + c) * d.cells + n] = gbar[c];
    }
}

// One reverse step (S9): the transposed Jacobian of one forward step applied to
// lambda.  The forward state is pulled exactly as the step pulls it; lambda of
// the step's outputs is read where the step wrote the copy that is streamed on
// (the halo column at the periodic seam); the result is scattered to the very
// entries the pull read, so the scatter is a permutation and needs no atomics.
template <int Q, int CPT, bool EDGE>
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
        float ebar, gbar[3];
        collide_vjp<Q>(d, hh, e0, et, mm, ll, ebar, gbar);
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[i][k] = ll[i];
        if (x0 + k < d.nx) {
            const long long n = ((long long)z * d.ny + y) * d.nx + x0 + k;
            grad[n] += ebar;
#pragma unroll
            for (int c = 0; c < D; ++c) grad[(1 + c) * d.cells + n] += gbar[c];
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

template <int Q, int CPT>
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
        adj_row<Q, CPT, true>(d, st, lin, lout, grad, y, z, x0, lane);
    else
        adj_row<Q, CPT, false>(d, st, lin, lout, grad, y, z, x0, lane);
}

// dJ/deps = G_eps + sum_i w_i lambda_i(0) (from f(0) = w eps) + the transposed
// grad-eps stencil applied to G_grad.
template <int Q>
__global__ void k_grad_finalize(const VDom d, const float *__restrict__ lam0,
                                const float *__restrict__ grad, float *__restrict__ out) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < d.cells;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, n, x, y, z);
        Nb3 Y, Z;
        nb_yz<Q>(d, y, z, Y, Z);
        float v = grad[n];
#pragma unroll
        for (int i = 0; i < Q; ++i) v += L::w(i) * lam0[pull_index<Q>(d, i, x, y, z, Y, Z)];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
            // cell x - e_i, whose stencil reads eps(x) through direction i
            if (!(Y.wall[1 - e[1]] || Z.wall[1 - e[2]])) {
                int xs = x - e[0];
                xs = xs < 0 ? xs + d.nx : (xs >= d.nx ? xs - d.nx : xs);
                const long long m = ((long long)Z.r[1 - e[2]] * d.ny + Y.r[1 - e[1]]) * d.nx + xs;
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < D; ++c) s += e[c] * grad[(1 + c) * d.cells + m];
                v += 3.f * L::w(i) * s;
            }
            // x itself, whose neighbour x + e_i lies past a wall
            if (Y.wall[1 + e[1]] || Z.wall[1 + e[2]]) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < D; ++c) s += e[c] * grad[(1 + c) * d.cells + n];
                v += 3.f * L::w(i) * s;
            }
        }
        out[n] = v;
    }
}

// --------------------------------------------------------------- launch ---
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
                             float *grad, cudaStream_t s) {
    const int g = grid_for(d.rows, 256);
    VANS_DISPATCH_Q(q, (k_flux_seed<9><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)),
                    (k_flux_seed<19><<<g, 256, 0, s>>>(d, state, x_out, lam, grad)));
    return cudaGetLastError();
}

cudaError_t launch_step_adjoint(int q, const VDom &d, const float *state, const float *lam_in,
                                float *lam_out, float *grad, cudaStream_t s) {
    // two cells per lane for D2Q9, one for D3Q19 (register pressure); 4 warps x 2 rows
    const int warps = 4, rows = 2;
    const int cpt = (q == 9) ? 2 : 1;
    const int nxb = (d.nx + 32 * cpt * warps - 1) / (32 * cpt * warps);
    const int nrb = (d.rows + rows - 1) / rows;
    dim3 block(32 * warps, rows);
    const unsigned nb = (unsigned)((long long)nxb * nrb);
    VANS_DISPATCH_Q(q, (k_step_adjoint<9, 2><<<nb, block, 0, s>>>(d, state, lam_in, lam_out, grad, nxb)),
                    (k_step_adjoint<19, 1><<<nb, block, 0, s>>>(d, state, lam_in, lam_out, grad, nxb)));
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(int q, const VDom &d, const float *lam0, const float *grad,
                                 float *dJ, cudaStream_t s) {
    const int g = grid_for(d.cells, 256);
    VANS_DISPATCH_Q(q, (k_grad_finalize<9><<<g, 256, 0, s>>>(d, lam0, grad, dJ)),
                    (k_grad_finalize<19><<<g, 256, 0, s>>>(d, lam0, grad, dJ)));
    return cudaGetLastError();
}

}  // namespace vans
