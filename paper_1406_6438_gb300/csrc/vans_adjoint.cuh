// vans_adjoint.cuh -- per-cell reverse mode of the step, in a chosen scalar
// type T (float or double).  The forward quantities of one cell are rebuilt
// from the pulled populations in T with correctly rounded square roots and
// divisions; the adjoints of f^eq (Eq. d2q9eq), of P_i + F_i (Eqs. pi, Fi), of
// the implicit velocity (Eq. 1moment with the drag law) and of eps rho (Eq.
// 0moment) are then taken in reverse order.  dJ/deps is a small residual of
// large grad-eps sensitivities that cancel in the transposed stencil, so the
// systematic error of these per-cell terms is what limits its accuracy; the
// double instance removes it at the cost of FP64 arithmetic.
#pragma once

#include "vans_device.cuh"

namespace vans {

// Compensated (Neumaier) FP32 accumulation: *s holds the running sum and *c the
// rounding error lost so far; s + c is the sum to about one FP32 ulp however
// many steps are added.  The eps gradient is a small residual of large
// grad-eps sensitivities (they cancel through the transposed stencil), so the
// plain FP32 running sum would lose most of it over thousands of steps.
__device__ __forceinline__ void acc2(float *s, float *c, float x) {
    const float a = *s;
    const float t = a + x;
    const float e = (fabsf(a) >= fabsf(x)) ? (a - t) + x : (x - t) + a;
    *s = t;
    *c += e;
}

// the same on values held in registers
__device__ __forceinline__ void acc2_reg(float &s, float &c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// Add a term formed in type T: an FP64 term goes in as its FP32 leading part
// plus the FP32 rounding of the remainder, so the accumulation keeps about 48
// of its bits instead of 24 (the terms are large sensitivities whose sum over
// the steps cancels to the small eps gradient).
__device__ __forceinline__ void acc2_term(float *s, float *c, float x) { acc2(s, c, x); }
__device__ __forceinline__ void acc2_term(float *s, float *c, double x) {
    const float hi = (float)x;
    acc2(s, c, hi);
    *c += (float)(x - (double)hi);
}
__device__ __forceinline__ void acc2_reg_term(float &s, float &c, float x) { acc2_reg(s, c, x); }
__device__ __forceinline__ void acc2_reg_term(float &s, float &c, double x) {
    const float hi = (float)x;
    acc2_reg(s, c, hi);
    c += (float)(x - (double)hi);
}

// Square root and reciprocal of the reverse arithmetic: FP64 correctly
// rounded; FP32 the hardware estimates refined by one Newton step (rcp_nr,
// sqrt_nr: within about an ulp, without the division's slow-path branch).
template <typename T> __device__ __forceinline__ T vsqrt(T x);
template <> __device__ __forceinline__ float vsqrt<float>(float x) { return x > 0.f ? sqrt_nr(x) : 0.f; }
template <> __device__ __forceinline__ double vsqrt<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T vrcp(T x);
template <> __device__ __forceinline__ float vrcp<float>(float x) { return rcp_nr(x); }
template <> __device__ __forceinline__ double vrcp<double>(double x) { return 1.0 / x; }

template <int Q, typename T>
struct MacroT {
    T dl, e0, R, inv_e, rho, rho3;
    T ge[3], j[3], Pc[3], m[3];
    T alpha, beta, dalpha, dbeta;
    T a, b, mm, sq, D, inv_D;
    T u[3], un, V[3];
};

template <int Q, typename T>
__device__ __forceinline__ void macro_t(const VDom &d, const float h[Q], float e0f, const float et[Q],
                                        MacroT<Q, T> &M) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    T dl = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) dl += (T)h[i];
    const T e0 = (T)e0f;
    M.dl = dl;
    M.e0 = e0;
    M.R = e0 + dl;
    M.inv_e = vrcp<T>(e0);
    M.rho = M.R * M.inv_e;
#pragma unroll
    for (int c = 0; c < D; ++c) { M.ge[c] = 0; M.j[c] = 0; }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int k = L::opp(i);
        const T de = T(3) * (T)L::w(i) * ((T)et[i] - (T)et[k]);
        const T dh = (T)h[i] - (T)h[k];
        if (L::ex(i)) { M.ge[0] += L::ex(i) * de; M.j[0] += L::ex(i) * dh; }
        if (L::ey(i)) { M.ge[1] += L::ey(i) * de; M.j[1] += L::ey(i) * dh; }
        if (D == 3 && L::ez(i)) { M.ge[2] += L::ez(i) * de; M.j[2] += L::ez(i) * dh; }
    }
    // drag coefficients and their eps-derivatives (host constants ca, cb)
    T a = 0, b = 0, da = 0, db = 0;
    const T ca = (T)d.ca, cb = (T)d.cb;
    if (d.k_mode == 0) {
        const T om = T(1) - e0;
        a = ca * om * om * M.inv_e;
        b = cb * om;
        da = -ca * om * (T(1) + e0) * (M.inv_e * M.inv_e);
        db = -cb;
    } else if (d.k_mode == 1) {
        a = ca * e0 * e0;
        b = cb * e0 * e0 * e0;
        da = T(2) * ca * e0;
        db = T(3) * cb * e0 * e0;
    } else {
        const T se = vsqrt<T>(e0);
        a = ca * e0 * e0;
        b = cb * e0 * se;
        da = T(2) * ca * e0;
        db = T(1.5) * cb * se;
    }
    if (d.drag_mode == 0) { a = b = da = db = 0; }
    if (d.drag_mode == 1) { b = db = 0; }
    M.alpha = a; M.beta = b; M.dalpha = da; M.dbeta = db;
    const T pc = M.rho * (T(1) / T(3));
    M.rho3 = pc;
    T mm2 = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        M.Pc[c] = pc * M.ge[c];
        M.m[c] = M.j[c] + T(0.5) * (M.Pc[c] + M.R * (T)d.g[c]);
        mm2 += M.m[c] * M.m[c];
    }
    M.a = M.R + T(0.5) * M.alpha;
    M.b = T(0.5) * M.beta;
    M.mm = vsqrt<T>(mm2);
    M.sq = vsqrt<T>(M.a * M.a + T(4) * M.b * M.mm);
    M.D = M.a + M.sq;
    M.inv_D = vrcp<T>(M.D);
    const T s = T(2) * M.inv_D;
    M.un = M.mm * s;
    const T kd = M.alpha + M.beta * M.un;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        M.u[c] = M.m[c] * s;
        M.V[c] = M.Pc[c] + M.R * (T)d.g[c] - kd * M.u[c];
    }
}

// Reverse of macro_t: from dJ/dR, dJ/du and dJ/dV, the part of dJ/dh_i common
// to all i (lam0), the momentum adjoint jbar (dJ/dh_i gets e_i . jbar), and the
// partials of J with respect to eps(x) (at fixed f) and grad eps(x).
template <int Q, typename T>
__device__ __forceinline__ void macro_vjp_t(const VDom &d, const MacroT<Q, T> &M, T Rbar, T ubar[3],
                                            const T Vbar[3], T &lam0, T jbar[3], T &ebar, T gbar[3]) {
    constexpr int D = Lat<Q>::D;
    T Pcbar[3], Fbar[3], mbar[3];
    T Fu = 0;
    // V = Pc + F,  F = R g - alpha u - beta |u| u
#pragma unroll
    for (int c = 0; c < D; ++c) {
        Pcbar[c] = Vbar[c];
        Fbar[c] = Vbar[c];
        Rbar += Fbar[c] * (T)d.g[c];
        Fu += Fbar[c] * M.u[c];
    }
    T alphabar = -Fu;
    T betabar = -M.un * Fu;
    const T kd = M.alpha + M.beta * M.un;
    const T ib = (M.un > T(0)) ? M.beta * Fu * vrcp<T>(M.un) : T(0);
    // reciprocals formed once (each a correctly rounded division); the
    // quotients below are products with them
    T ubu = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        ubar[c] += -kd * Fbar[c] - ib * M.u[c];
        ubu += ubar[c] * M.u[c];
    }
    // u = 2 m / D,  D = a + sqrt(a^2 + 4 b |m|)
    const T inv_sq = vrcp<T>(M.sq);
    const T Dbar = -ubu * M.inv_D;
    const T abar = Dbar * (T(1) + M.a * inv_sq);
    const T bbar = Dbar * T(2) * M.mm * inv_sq;
    const T mmbar = Dbar * T(2) * M.b * inv_sq;
    const T im = (M.mm > T(0)) ? mmbar * vrcp<T>(M.mm) : T(0);
    const T s2 = T(2) * M.inv_D;
#pragma unroll
    for (int c = 0; c < D; ++c) mbar[c] = ubar[c] * s2 + im * M.m[c];
    // a = R + alpha/2, b = beta/2
    Rbar += abar;
    alphabar += T(0.5) * abar;
    betabar += T(0.5) * bbar;
    // m = j + Pc/2 + R g/2;  Pc = rho grad eps / 3
    T pg = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        jbar[c] = mbar[c];
        Pcbar[c] += T(0.5) * mbar[c];
        Rbar += T(0.5) * mbar[c] * (T)d.g[c];
        pg += Pcbar[c] * M.ge[c];
        gbar[c] = M.rho3 * Pcbar[c];
    }
    const T rhobar = pg * (T(1) / T(3));
    // rho = R / eps
    Rbar += rhobar * M.inv_e;
    ebar = -rhobar * M.rho * M.inv_e;
    ebar += alphabar * M.dalpha + betabar * M.dbeta;
    lam0 = Rbar;
}

// Reverse of the collision of one cell.  mu_i = dJ/df*_i; returns lam_i =
// dJ/df_i, the eps partial and the grad-eps partial.  With M_i = mu_i w_i,
// SM = sum M_i, SMe = sum M_i e_i and T = sum M_i e_i e_i^T, the adjoints of
// f^eq and of P_i + F_i reduce to
//   Rbar = omega (SM + 3 SMe.u + 4.5 u.T.u - 1.5 u.u SM)
//   ubar = omega R (3 SMe + 9 T u - 3 u SM) + ct (9 T V - 3 V SM)
//   Vbar = ct (3 SMe - 3 u SM + 9 T u).
template <int Q, typename T>
__device__ __forceinline__ void collide_vjp_t(const VDom &d, const float h[Q], float e0,
                                              const float et[Q], const float mu[Q], float lam[Q],
                                              T &ebar, T gbar[3]) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    MacroT<Q, T> M;
    macro_t<Q, T>(d, h, e0, et, M);
    T SM = 0, SMe[3] = {0, 0, 0}, Tm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T Mi = (T)mu[i] * (T)L::w(i);
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        SM += Mi;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (e[a] == 0) continue;
            SMe[a] += e[a] * Mi;
#pragma unroll
            for (int b = a; b < D; ++b)
                if (e[b] != 0) Tm[a][b] += (e[a] * e[b]) * Mi;
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < a; ++b) Tm[a][b] = Tm[b][a];
    T Tu[3], TV[3], uu = 0, SMeu = 0, uTu = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Tu[a] = 0;
        TV[a] = 0;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            Tu[a] += Tm[a][b] * M.u[b];
            TV[a] += Tm[a][b] * M.V[b];
        }
        uu += M.u[a] * M.u[a];
        SMeu += SMe[a] * M.u[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) uTu += M.u[a] * Tu[a];
    const T om = (T)d.omega, ct = (T)d.ctau;
    const T Rbar = om * (SM + T(3) * SMeu + T(4.5) * uTu - T(1.5) * uu * SM);
    T ubar[3], Vbar[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        ubar[a] = om * M.R * (T(3) * SMe[a] + T(9) * Tu[a] - T(3) * M.u[a] * SM) +
                  ct * (T(9) * TV[a] - T(3) * M.V[a] * SM);
        Vbar[a] = ct * (T(3) * SMe[a] - T(3) * M.u[a] * SM + T(9) * Tu[a]);
    }
    T lam0, jbar[3];
    macro_vjp_t<Q, T>(d, M, Rbar, ubar, Vbar, lam0, jbar, ebar, gbar);
    const T om1 = T(1) - om;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T l = om1 * (T)mu[i] + lam0;
        if (L::ex(i)) l += L::ex(i) * jbar[0];
        if (L::ey(i)) l += L::ey(i) * jbar[1];
        if (D == 3 && L::ez(i)) l += L::ez(i) * jbar[2];
        lam[i] = (float)l;
    }
}

}  // namespace vans
