// vans_device.cuh -- device-side building blocks of the porous LBM step.
//
// State layout.  One state buffer holds Q planes, one per direction i; a plane
// holds rows = ny*nz padded rows of `pitch` floats (pitch is a multiple of 32
// floats, so every row starts on a 128-byte boundary).  Column c of a row lives
// at row + d.off + c for c in [-1, nx]: columns -1 and nx are halo copies
// that make the periodic x wrap free for the pull.  What a plane stores for cell
// x is the post-collision population of direction i of the previous step, as a
// deviation from w_i * eps~(x + e_i), the porosity of the cell it streams to
// (eps~ = eps(x) when that cell lies past a wall).  The pull then reads exactly
// the deviation h_i = f_i - w_i eps(x) of the receiving cell, and the rest
// state f = w eps is stored as all zeros.  Deviations are O(1e-3) of f, so FP32
// keeps about 3 more decimal digits of the flow than it would on raw f.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vans_internal.h"

#define VANS_FULL 0xffffffffu

namespace vans {

// ------------------------------------------- programmatic dependent launch ----
// A step kernel launched with the programmatic-serialization attribute may
// start while the previous kernel of its stream is still finishing: each of its
// CTAs first lets the NEXT kernel launch (pdl_trigger: that kernel is scheduled
// once every CTA of this one has triggered or exited, so its CTAs only take SM
// slots this grid no longer needs), then waits until the previous kernel has
// completed and its writes are visible (pdl_wait), before touching memory.  A
// launch without the attribute, or one after a non-kernel operation, waits as
// usual and both instructions return at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with the programmatic-serialization attribute (the kernel calls
// pdl_trigger and pdl_wait before its first global memory access).  Only the
// register-load step uses it: on the pipelined kinds it measured between -9 %
// (kind 7 at 1024^2) and +1 % (kind 6 at 2048^2).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// ------------------------------------------------------------ lattices ----
// D2Q9 and D3Q19 velocity sets and weights (Qian, d'Humieres & Lallemand 1992,
// the lattice family of Eq. d2q9eq), in the direction order of vans.h.
template <int Q> struct Lat;

template <> struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
};

template <> struct Lat<19> {
    static constexpr int D = 3;
    // 0 rest; 1..6 faces (+x,-x,+y,-y,+z,-z); 7..18 edges in opposite pairs
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
};

// ------------------------------------------------------- vector memory ----
template <int CPT> struct Vec;
template <> struct Vec<1> { using T = float; };
template <> struct Vec<2> { using T = float2; };
template <> struct Vec<4> { using T = float4; };

template <int CPT>
__device__ __forceinline__ void ld_vec(const float *p, float v[CPT]) {
    if constexpr (CPT == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (CPT == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = __ldg(p);
    }
}

template <int CPT>
__device__ __forceinline__ void st_vec(float *p, const float v[CPT]) {
    if constexpr (CPT == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (CPT == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

// Values at columns x0+s .. x0+s+CPT-1 of a row (row points at column 0),
// s in {-1, 0, +1} and the same for the whole warp.  One aligned vector load per
// lane; the value that crosses into the neighbouring lane comes by shuffle and
// the warp's edge lanes fetch theirs with one scalar load.  All 32 lanes must
// take part.
template <int CPT>
__device__ __forceinline__ void ld_shift(const float *__restrict__ row, int x0, int s, int lane,
                                         float v[CPT]) {
    float a[CPT];
    ld_vec<CPT>(row + x0, a);
    if (s == 0) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) v[k] = a[k];
    } else if (s < 0) {
        float left = __shfl_up_sync(VANS_FULL, a[CPT - 1], 1);
        if (lane == 0) left = __ldg(row + x0 - 1);
        v[0] = left;
#pragma unroll
        for (int k = 1; k < CPT; ++k) v[k] = a[k - 1];
    } else {
        float right = __shfl_down_sync(VANS_FULL, a[0], 1);
        if (lane == 31) right = __ldg(row + x0 + CPT);
#pragma unroll
        for (int k = 0; k < CPT - 1; ++k) v[k] = a[k + 1];
        v[CPT - 1] = right;
    }
}

// Columns x0-1 .. x0+CPT of a row (the cells plus one neighbour on each side).
template <int CPT>
__device__ __forceinline__ void ld_ext(const float *__restrict__ row, int x0, int lane,
                                       float v[CPT + 2]) {
    float a[CPT];
    ld_vec<CPT>(row + x0, a);
    float left = __shfl_up_sync(VANS_FULL, a[CPT - 1], 1);
    float right = __shfl_down_sync(VANS_FULL, a[0], 1);
    if (lane == 0) left = __ldg(row + x0 - 1);
    if (lane == 31) right = __ldg(row + x0 + CPT);
    v[0] = left;
#pragma unroll
    for (int k = 0; k < CPT; ++k) v[k + 1] = a[k];
    v[CPT + 1] = right;
}

// Store cells x0..x0+CPT-1 of a row, skipping columns >= nx.
template <int CPT>
__device__ __forceinline__ void st_masked(float *row, int x0, int nx, const float v[CPT]) {
    if (x0 + CPT <= nx) {
        st_vec<CPT>(row + x0, v);
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k)
            if (x0 + k < nx) row[x0 + k] = v[k];
    }
}

// Halo copies of one direction's row (row points at column 0): column -1
// mirrors column nx-1 (read by the pull of directions moving +x), column nx
// mirrors column 0 (directions moving -x).  Column 0 starts a 32-byte sector,
// so column -1 is the last float of a sector that otherwise holds row padding,
// and so is column nx when nx is a multiple of 8.  A sector that L2 holds
// partly written at write-back costs a DRAM read of the sector; on D3Q19's
// short rows (256 cells: 10 such sectors per 19 KB of row data, 20 MB of reads
// per 256^3 step) the copy is therefore stored with its whole sector, the
// padding as zeros (0.85 -> 0.92 of the copy bandwidth).  The D2Q9 kernels
// keep the 4-byte store: with the two vector stores compiled in, even where
// they do not run, they measured 4 % slower on 4096-cell rows and 5 % on the
// batch's 64-1024-cell rows.
template <int Q>
__device__ __forceinline__ void store_halo_lo(float *row, float v) {
    if constexpr (Q == 19) {
        float4 *s = reinterpret_cast<float4 *>(row - 8);
        s[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        s[1] = make_float4(0.f, 0.f, 0.f, v);
    } else {
        row[-1] = v;
    }
}

template <int Q>
__device__ __forceinline__ void store_halo_hi(float *row, int nx, float v) {
    if (Q == 19 && (nx & 7) == 0) {
        float4 *s = reinterpret_cast<float4 *>(row + nx);
        s[0] = make_float4(v, 0.f, 0.f, 0.f);
        s[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        row[nx] = v;
    }
}



// Inverse of ld_shift: value v[k] of cell x0+k goes to column x0+k+s.  Lanes
// compose aligned vectors with a shuffle; the value that crosses into the next
// warp is written by a scalar store.  Cells past nx write into columns that no
// pull reads, so no mask is needed.
template <int CPT>
__device__ __forceinline__ void st_shift(float *row, int x0, int s, int lane, const float v[CPT]) {
    if (s == 0) {
        st_vec<CPT>(row + x0, v);
    } else if (s < 0) {
        const float nxt = __shfl_down_sync(VANS_FULL, v[0], 1);
        if (lane != 31) {
            float a[CPT];
#pragma unroll
            for (int k = 0; k < CPT - 1; ++k) a[k] = v[k + 1];
            a[CPT - 1] = nxt;
            st_vec<CPT>(row + x0, a);
        } else {
#pragma unroll
            for (int k = 0; k < CPT - 1; ++k) row[x0 + k] = v[k + 1];
        }
        if (lane == 0) row[x0 - 1] = v[0];
    } else {
        const float prv = __shfl_up_sync(VANS_FULL, v[CPT - 1], 1);
        if (lane != 0) {
            float a[CPT];
            a[0] = prv;
#pragma unroll
            for (int k = 1; k < CPT; ++k) a[k] = v[k - 1];
            st_vec<CPT>(row + x0, a);
        } else {
#pragma unroll
            for (int k = 0; k < CPT - 1; ++k) row[x0 + 1 + k] = v[k];
        }
        if (lane == 31) row[x0 + CPT] = v[CPT - 1];
    }
}

// ------------------------------------------------------- row neighbours ----
// Neighbour row indices along y (or z) at offsets -1, 0, +1 and whether that
// neighbour lies past a bounce-back wall.  Periodic axes wrap.
struct Nb3 {
    int r[3];
    bool wall[3];
};

template <bool EDGE>
__device__ __forceinline__ Nb3 nb3(int c, int n, int walls) {
    Nb3 o;
    o.r[1] = c;
    o.wall[1] = false;
    if (EDGE) {
        o.r[0] = (c == 0) ? n - 1 : c - 1;
        o.r[2] = (c == n - 1) ? 0 : c + 1;
        o.wall[0] = walls && c == 0;
        o.wall[2] = walls && c == n - 1;
    } else {
        o.r[0] = c - 1;
        o.r[2] = c + 1;
        o.wall[0] = false;
        o.wall[2] = false;
    }
    return o;
}

__device__ __forceinline__ long long row_offset(const VDom &d, int y, int z) {
    return ((long long)z * d.ny + y) * d.pitch + d.off;
}

// Moving upper wall: a population pulled through the upper y wall (direction
// i with e_iy < 0 in a top row) left the cell as its opposite and bounced off
// the moving plate, gaining 2 w_i eps (e_i . u_w)/cs^2 (rho_w = 1).  top is
// true in the rows whose +y neighbour lies past that wall.  A population that
// crossed a z wall at the same time (a D3Q19 edge direction in a corner row)
// takes a plain bounce-back.
template <int Q>
__device__ __forceinline__ float wall_gain(const VDom &d, int i, float e0) {
    using L = Lat<Q>;
    float eu = 0.f;
    if (L::ex(i)) eu += L::ex(i) * d.uw[0];
    if (L::ey(i)) eu += L::ey(i) * d.uw[1];
    if (Q == 19 && L::ez(i)) eu += L::ez(i) * d.uw[2];
    return 6.f * L::w(i) * e0 * eu;
}

template <int Q>
__device__ __forceinline__ void apply_moving_wall(const VDom &d, bool top, const Nb3 &Z, float e0,
                                                  float h[Q]) {
    using L = Lat<Q>;
    if (!(d.moving && top)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (L::ey(i) < 0 && !Z.wall[1 - L::ez(i)]) h[i] += wall_gain<Q>(d, i, e0);
}

// ----------------------------------------------------------- the drag ----
// alpha = eps^2 nu / K and beta = eps^3 F_eps / sqrt(K) (drag law) with K and
// F_eps per k_mode; ca, cb are the host-side constants of vans_internal.h.
// inv_e = 1/eps.  Also returns d alpha/d eps and d beta/d eps when asked.
template <bool DERIV>
__device__ __forceinline__ void drag(const VDom &d, float e, float inv_e, float &alpha, float &beta,
                                     float *dalpha = nullptr, float *dbeta = nullptr) {
    float a = 0.f, b = 0.f, da = 0.f, db = 0.f;
    if (d.k_mode == 0) {          // Ergun: 150 nu (1-eps)^2/(eps d_p^2), 1.75 (1-eps)/d_p
        const float om = 1.f - e;
        a = d.ca * om * om * inv_e;
        b = d.cb * om;
        if (DERIV) {
            da = -d.ca * om * (1.f + e) * inv_e * inv_e;
            db = -d.cb;
        }
    } else if (d.k_mode == 1) {   // fixed K, F_eps
        a = d.ca * e * e;
        b = d.cb * e * e * e;
        if (DERIV) {
            da = 2.f * d.ca * e;
            db = 3.f * d.cb * e * e;
        }
    } else {                      // fixed K, F_eps(eps) = 1.75/sqrt(150 eps^3)
        const float se = sqrtf(e);
        a = d.ca * e * e;
        b = d.cb * e * se;
        if (DERIV) {
            da = 2.f * d.ca * e;
            db = 1.5f * d.cb * se;
        }
    }
    if (d.drag_mode == 0) { a = b = da = db = 0.f; }
    if (d.drag_mode == 1) { b = db = 0.f; }
    alpha = a;
    beta = b;
    if (DERIV) { *dalpha = da; *dbeta = db; }
}

// --------------------------------------------------- reciprocal and root ----
// The hardware estimates (MUFU rcp / rsqrt) carry a small input-dependent bias;
// on a near-steady flow it acts the same way every step and accumulates.  One
// Newton-Raphson step on each estimate (the textbook iteration r <- r (2 - x r)
// for 1/x, s <- s + (x - s^2)/(2 s) for sqrt x) removes it for a few FMAs,
// far cheaper than the correctly rounded library routines.
__device__ __forceinline__ float rcp_nr(float x) {
    const float r = __fdividef(1.f, x);
    const float e = fmaf(-x, r, 1.f);
    return fmaf(r, e, r);
}

__device__ __forceinline__ float sqrt_nr(float x) {     // x > 0
    const float y = rsqrtf(x);
    const float s = x * y;
    const float e = fmaf(-s, s, x);
    return fmaf(0.5f * y, e, s);
}

// ----------------------------------------------------- cell macroscopics ----
// Moments of one cell (Eqs. 0moment and 1moment) from its pulled deviations
// h_i = f_i - w_i eps(x) and the porosities eps~_i = eps(x + e_i).
template <int Q>
struct Macro {
    float dl;            // sum_i h_i = eps rho - eps
    float e0;            // eps(x)
    float R, inv_e, rho; // eps rho, 1/eps, rho
    float ge[3];         // grad eps (lattice stencil)
    float j[3];          // sum_i e_i f_i
    float Pc[3];         // p grad eps = cs^2 rho grad eps
    float m[3];          // j + Pc/2 + R g/2
    float alpha, beta;
    float a, b, mm, sq, D, s; // velocity solve: D = a + sq, s = 2/D
    float u[3], un;
    float V[3];          // p grad eps + F, the vector P_i + F_i act on
};

template <int Q>
__device__ __forceinline__ void macro(const VDom &d, const float h[Q], float e0, const float et[Q],
                                      Macro<Q> &M) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    // Eq. 0moment: eps rho = sum f_i = eps(x) + sum h_i
    float dl = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) dl += h[i];
    M.dl = dl;
    M.e0 = e0;
    M.R = e0 + dl;
#if defined(VANS_IEEE_MATH)
    M.inv_e = __frcp_rn(e0);
#elif defined(VANS_RAW_ESTIMATES)
    M.inv_e = __fdividef(1.f, e0);
#else
    M.inv_e = rcp_nr(e0);
#endif
    M.rho = M.R * M.inv_e;
    // grad eps = (1/cs^2) sum_i w_i e_i eps~_i and sum_i e_i f_i = sum_i e_i h_i,
    // both over opposite pairs: eps~_i - eps~_opp(i) is exact in FP32 for
    // neighbouring porosities within a factor 2 (Sterbenz), so the small
    // gradient keeps full relative precision
#pragma unroll
    for (int c = 0; c < D; ++c) { M.ge[c] = 0.f; M.j[c] = 0.f; }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int k = L::opp(i);
        const float de = 3.f * L::w(i) * (et[i] - et[k]);
        const float dh = h[i] - h[k];
        if (L::ex(i)) { M.ge[0] += L::ex(i) * de; M.j[0] += L::ex(i) * dh; }
        if (L::ey(i)) { M.ge[1] += L::ey(i) * de; M.j[1] += L::ey(i) * dh; }
        if (D == 3 && L::ez(i)) { M.ge[2] += L::ez(i) * de; M.j[2] += L::ez(i) * dh; }
    }
    drag<false>(d, e0, M.inv_e, M.alpha, M.beta);
    const float pc = M.rho * (1.f / 3.f);
    float mm2 = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        M.Pc[c] = pc * M.ge[c];
        M.m[c] = M.j[c] + 0.5f * (M.Pc[c] + M.R * d.g[c]);
        mm2 += M.m[c] * M.m[c];
    }
    // Eq. 1moment with the drag: (R + alpha/2 + beta/2 |u|) u = m, solved exactly
    M.a = M.R + 0.5f * M.alpha;
    M.b = 0.5f * M.beta;
    // square roots and the reciprocal through the hardware approximations
    // (relative error ~1e-7, far below the FP32 rounding of the populations)
#if defined(VANS_IEEE_MATH)
    M.mm = sqrtf(mm2);
    M.sq = sqrtf(M.a * M.a + 4.f * M.b * M.mm);
    M.D = M.a + M.sq;
    M.s = __fdiv_rn(2.f, M.D);
#elif defined(VANS_RAW_ESTIMATES)
    M.mm = mm2 > 0.f ? mm2 * rsqrtf(mm2) : 0.f;
    const float q2 = M.a * M.a + 4.f * M.b * M.mm;
    M.sq = q2 * rsqrtf(q2);
    M.D = M.a + M.sq;
    M.s = __fdividef(2.f, M.D);
#else
    M.mm = mm2 > 0.f ? sqrt_nr(mm2) : 0.f;
    M.sq = sqrt_nr(M.a * M.a + 4.f * M.b * M.mm);
    M.D = M.a + M.sq;
    M.s = 2.f * rcp_nr(M.D);
#endif
    M.un = M.mm * M.s;
    const float kd = M.alpha + M.beta * M.un;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        M.u[c] = M.m[c] * M.s;
        M.V[c] = M.Pc[c] + M.R * d.g[c] - kd * M.u[c];
    }
}

// ---------------------------------------------------------- collision ----
// f*_i = f_i - (f_i - f^eq_i)/tau + P_i + F_i (the final LBE), in deviation
// form: with A_i = f^eq_i/w_i - eps(x) = dl + R (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)
// (Eq. d2q9eq) and S_i/w_i = (1 - 1/(2tau)) (3 (e_i - u) + 9 (e_i.u) e_i).V
// (Eqs. pi and Fi), the stored value is
//   o_i = (1 - omega) h_i + w_i [omega A_i + S_i/w_i + (eps(x) - eps~_i)].
// Directions come in opposite pairs +c/-c, which share the even part of A and
// S and flip the sign of the odd part.  eps(x) - eps~_i is formed first (exact
// for porosities within a factor 2): adding eps(x) ~ 0.5 to the O(1e-3) terms
// and subtracting eps~_i afterwards would cost 3e-8 absolute per population.
template <int Q>
__device__ __forceinline__ void collide(const VDom &d, const float h[Q], float e0, const float et[Q],
                                        float o[Q], Macro<Q> *Mout = nullptr) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    Macro<Q> M;
    macro<Q>(d, h, e0, et, M);
    if (Mout) *Mout = M;
    const float om = d.omega, ct = d.ctau, om1 = 1.f - om;
    float uu = 0.f, uV = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) { uu += M.u[c] * M.u[c]; uV += M.u[c] * M.V[c]; }
    const float symc = om * (M.dl - 1.5f * M.R * uu) - 3.f * ct * uV;
    const float omR = om * M.R;
    o[0] = om1 * h[0] + L::w(0) * symc;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;               // handle each pair once, from its first member
        const int j = L::opp(i);
        float eu = 0.f, eV = 0.f;
        if (L::ex(i)) { eu += L::ex(i) * M.u[0]; eV += L::ex(i) * M.V[0]; }
        if (L::ey(i)) { eu += L::ey(i) * M.u[1]; eV += L::ey(i) * M.V[1]; }
        if (D == 3 && L::ez(i)) { eu += L::ez(i) * M.u[2]; eV += L::ez(i) * M.V[2]; }
        const float sym = symc + 4.5f * omR * eu * eu + 9.f * ct * eu * eV;
        const float anti = 3.f * (omR * eu + ct * eV);
        o[i] = om1 * h[i] + L::w(i) * ((sym + anti) + (e0 - et[i]));
        o[j] = om1 * h[j] + L::w(j) * ((sym - anti) + (e0 - et[j]));
    }
}

// ------------------------------------------------- plates on nodes ----
// The non-equilibrium extrapolation scheme of the paper's validation runs
// (wall_kind 1): rows 0 and ny-1 are nodes on the plates.  A plate node x_b
// takes f^eq(eps_b, rho_f, u_b) plus the non-equilibrium part of its fluid
// neighbour x_f, n_i = f_i(x_f) - f^eq_i(eps_f, rho_f, u_f), and relaxes towards
// f^eq(eps_b, rho_f, u_b) with no source term, so its post-collision value is
// f^eq_i(eps_b, rho_f, u_b) + (1 - omega) n_i.  From the neighbour's moments M
// (h_i = f_i(x_f) - w_i eps_f, dl = sum h, R = eps_f rho_f) and with
// A_i, B_i the bracket of Eq. d2q9eq minus one at u_f and at u_b,
//   n_i = h_i - w_i (dl + R A_i),
//   f^eq_i(eps_b, rho_f, u_b) - w_i e_ref = w_i [(eps_b - e_ref) + eps_b dl / eps_f
//                                               + eps_b rho_f B_i],
// all small differences, formed before any O(1) term is added.

// index of the lattice direction (ex, ey, ez) (0 when there is none)
template <int Q>
__host__ __device__ constexpr int dir_index(int ex, int ey, int ez) {
    for (int j = 0; j < Q; ++j)
        if (Lat<Q>::ex(j) == ex && Lat<Q>::ey(j) == ey && Lat<Q>::ez(j) == ez) return j;
    return 0;
}

// 3 e_i.v + 4.5 (e_i.v)^2 - 1.5 v.v
template <int Q>
__device__ __forceinline__ float eq_bracket(int i, const float v[3]) {
    using L = Lat<Q>;
    float ev = 0.f, vv = 0.f;
    if (L::ex(i)) ev += L::ex(i) * v[0];
    if (L::ey(i)) ev += L::ey(i) * v[1];
    if (L::D == 3 && L::ez(i)) ev += L::ez(i) * v[2];
#pragma unroll
    for (int c = 0; c < L::D; ++c) vv += v[c] * v[c];
    return 3.f * ev + 4.5f * ev * ev - 1.5f * vv;
}

// value of direction i at the plate node, minus w_i e_ref, with the neighbour's
// non-equilibrium part scaled by keep (1 - omega: post-collision; 1: the
// populations the node holds before its collision)
template <int Q>
__device__ __forceinline__ float plate_value(const VDom &d, int i, float h_i, const Macro<Q> &M,
                                             float eb, float eref, const float ub[3], float keep) {
    using L = Lat<Q>;
    const float A = eq_bracket<Q>(i, M.u), B = eq_bracket<Q>(i, ub);
    const float neq = h_i - L::w(i) * (M.dl + M.R * A);
    (void)d;
    return L::w(i) * ((eb - eref) + eb * M.dl * M.inv_e + eb * M.rho * B) + keep * neq;
}

// Store the inward populations of the plate nodes next to fluid row y: lo
// (directions with e_y > 0) into row 0 when y == 1, hi (e_y < 0) into row
// ny-1 when y == ny-2, V cells per thread from column x0, halo columns included.
template <int Q, int V>
__device__ __forceinline__ void store_plates(const VDom &d, float *__restrict__ fout, int y, int z,
                                             int x0, bool plo, bool phi, const float lo[Q][V],
                                             const float hi[Q][V]) {
    using L = Lat<Q>;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (!(side ? phi : plo)) continue;
        const long long rb = row_offset(d, side ? y + 1 : y - 1, z);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (side ? L::ey(i) >= 0 : L::ey(i) <= 0) continue;
            const float *v = side ? hi[i] : lo[i];
            st_masked<V>(fout + i * d.plane + rb, x0, d.nx, v);
            if (x0 == 0 && L::ex(i) < 0) store_halo_hi<Q>(fout + i * d.plane + rb, d.nx, v[0]);
#pragma unroll
            for (int c = 0; c < V; ++c)
                if (x0 + c == d.nx - 1 && L::ex(i) > 0) store_halo_lo<Q>(fout + i * d.plane + rb, v[c]);
        }
    }
}

}  // namespace vans
