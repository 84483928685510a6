// vans_adjoint_tma.cu -- the reverse step with a bulk-copy pipeline.
//
// Same arithmetic as k_step_adjoint (vans_aux.cu): for every cell, the
// transposed step.  The cell's pulled populations f^t, its porosity neighbours
// and lambda^{t+1} at the cell come in, the vector-Jacobian product of the
// collision (collide_vjp_t, Eqs. d2q9eq, pi, Fi, 0moment, 1moment) gives
// lambda^t for the populations the cell pulled, which go back to where they
// were pulled from (the transpose of the pull: a permutation of the state's
// entries, so every entry is written once), and the eps / grad-eps partials
// are added into compensated accumulators.
//
// The register-load kernel waits for all of a row's loads and then computes
// ~1300 instructions per cell with nothing in flight.  Here persistent CTAs
// take tiles b, b + G, ... (one row segment of TW cells each); a producer warp
// stages the Q state rows of the pull, the porosity rows and the Q lambda rows
// of each tile with 1-D bulk copies, `stages` tiles ahead; each compute warp
// releases a stage as soon as it has read it into registers.  The accumulator
// words of a tile are loaded before the tile's wait, so their latency hides
// behind it.
#include "vans_adjoint.cuh"
#include "vans_pipeline.cuh"

namespace vans {

// One staged tile of the reverse step (the compute warps): read the stage into
// registers, release it, then the vector-Jacobian product of each cell, the
// compensated accumulation and the scatter of lambda.  EDGE = false: the
// tile's row touches no wall, so the wall flags are false at compile time.
template <int Q, int NT, int CPT, typename T, bool EDGE, class Rel>
__device__ __forceinline__ void adjoint_tile(const VDom &d, const float *__restrict__ sb,
                                             const float *__restrict__ lin, float *__restrict__ lout,
                                             float *__restrict__ grad, const Nb3 &Y, const Nb3 &Z,
                                             int y, int z, int xs, int tid,
                                             float (&gs)[CPT][1 + Lat<Q>::D],
                                             float (&gc)[CPT][1 + Lat<Q>::D], Rel &&release) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NE = EpsRows<Q>::N;
    const long long nc = (1 + D) * d.cells;
    const long long ro = row_offset(d, y, z);
    auto ywall = [&](int k) { return EDGE && Y.wall[k]; };
    auto zwall = [&](int k) { return EDGE && Z.wall[k]; };
    float h[CPT][Q], et[CPT][Q], mu[CPT][Q];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const int xl = tid + cc * NT;
        const int x = xs + xl;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = ywall(1 - L::ey(i)) || zwall(1 - L::ez(i));
            h[cc][i] = sb[i * SEG + kLead + xl + (bb ? 0 : -L::ex(i))];
        }
        const float e0 = sb[(Q + eps_slot<Q>(0, 0)) * SEG + kLead + xl];
        et[cc][0] = e0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool wall = ywall(1 + L::ey(i)) || zwall(1 + L::ez(i));
            et[cc][i] = wall ? e0
                             : sb[(Q + eps_slot<Q>(L::ey(i), L::ez(i))) * SEG + kLead + xl + L::ex(i)];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // lambda of the population this cell sends along e_i; across the
            // periodic x seam the scatter of the step after left it in the
            // halo column on the other side, outside this tile's segment
            const bool wall_out = ywall(1 + L::ey(i)) || zwall(1 + L::ez(i));
            float v = sb[(Q + NE + i) * SEG + kLead + xl];
            if (!wall_out && L::ex(i) > 0 && x == d.nx - 1) v = lin[i * d.plane + ro - 1];
            if (!wall_out && L::ex(i) < 0 && x == 0) v = lin[i * d.plane + ro + d.nx];
            mu[cc][i] = v;
        }
    }
    release();
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const int x = xs + tid + cc * NT;
        if (x >= d.nx) continue;
        const float e0 = et[cc][0];
        float hh[Q], ll[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) hh[i] = h[cc][i];
        if (EDGE) apply_moving_wall<Q>(d, Y.wall[2], Z, e0, hh);
        T ebar, gbar[3];
        collide_vjp_t<Q, T>(d, hh, e0, et[cc], mu[cc], ll, ebar, gbar);
        if (EDGE && d.moving && Y.wall[2]) {
            // the populations this cell sends into the moving wall come back
            // as their opposites with a gain that is linear in eps(x)
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ey(i) > 0 && !zwall(1 + L::ez(i)))
                    ebar += (T)wall_gain<Q>(d, L::opp(i), 1.f) * (T)mu[cc][i];
        }
        const long long m = ((long long)z * d.ny + y) * d.nx + x;
        acc2_reg_term(gs[cc][0], gc[cc][0], ebar);
#pragma unroll
        for (int c = 0; c < D; ++c) acc2_reg_term(gs[cc][1 + c], gc[cc][1 + c], gbar[c]);
#pragma unroll
        for (int c = 0; c <= D; ++c) {
            grad[c * d.cells + m] = gs[cc][c];
            grad[nc + c * d.cells + m] = gc[cc][c];
        }
        // lambda^t goes back to the entry the pull read (the transposed pull)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ey = L::ey(i), ez = L::ez(i);
            const bool bb = ywall(1 - ey) || zwall(1 - ez);
            if (bb)
                lout[L::opp(i) * d.plane + ro + x] = ll[i];
            else
                lout[i * d.plane + row_offset(d, Y.r[1 - ey], Z.r[1 - ez]) + x - L::ex(i)] = ll[i];
        }
    }
}

template <int Q, int NT, int CPT, typename T>
__global__ void __launch_bounds__(NT + 32) k_adjoint_tma(const VDom d, const float *__restrict__ st,
                                                         const float *__restrict__ lin,
                                                         float *__restrict__ lout,
                                                         float *__restrict__ grad, int ntx,
                                                         int ntiles, int stages) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NE = EpsRows<Q>::N;
    constexpr int NS = 2 * Q + NE;      // state rows, porosity rows, lambda rows
    constexpr int NCW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    const int tid = threadIdx.x;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int n = (ntiles - b + G - 1) / G;          // tiles of this CTA
    if (n <= 0) return;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= NT) {                                  // producer warp
        if (tid != NT) return;
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < n; ++k) {
            const int s = k % stages;
            if (k >= stages) {
                ok = mbar_wait_bounded(&empty[s], (uint32_t)(((k / stages) - 1) & 1));
                if (!ok) break;
                fence_proxy_async_smem();
            }
            const int t = b + k * G;
            const int row = t / ntx, xs = (t - row * ntx) * TW;
            float *sb = buf + s * (NS * SEG);
            const uint32_t bytes = issue_tile<Q, TW>(d, st, row, xs, sb, &full[s], Q);
            const long long ro = row_offset(d, row % d.ny, row / d.ny);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                bulk_g2s(sb + (Q + NE + i) * SEG, lin + i * d.plane + ro + xs - kLead, bytes, &full[s]);
            issued = k + 1;
        }
        if (!ok) {
            // a compute warp gave up: flag it and let the copies in flight land
            if (d.status) atomicOr(d.status, 2);
            const int first = issued > stages ? issued - stages : 0;
            for (int j = first; j < issued; ++j)
                mbar_wait_bounded(&full[j % stages], (uint32_t)((j / stages) & 1));
        }
        return;
    }

    const int lane = tid & 31;
    const long long nc = (1 + D) * d.cells;           // compensation words follow the sums
    int s = 0;
    uint32_t par = 0;
    for (int k = 0; k < n; ++k) {
        const int t = b + k * G;
        const int row = t / ntx, xs = (t - row * ntx) * TW;
        int y, z;
        Nb3 Y, Z;
        row_nbs<Q>(d, row, y, z, Y, Z);
        // accumulator words of this tile's cells, loaded before the wait
        float gs[CPT][1 + D], gc[CPT][1 + D];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const int x = xs + tid + cc * NT;
            if (x < d.nx) {
                const long long m = ((long long)z * d.ny + y) * d.nx + x;
#pragma unroll
                for (int c = 0; c <= D; ++c) {
                    gs[cc][c] = grad[c * d.cells + m];
                    gc[cc][c] = grad[nc + c * d.cells + m];
                }
            }
        }
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], par))) {
            if (lane == 0 && d.status) atomicOr(d.status, 2);
            return;
        }
        const float *sb = buf + s * (NS * SEG);
        uint64_t *const emp = &empty[s];
        auto release = [&] {
            __syncwarp();                             // every lane's reads precede the arrive
            if (lane == 0) mbar_arrive(emp);
        };
        if (Y.wall[0] || Y.wall[2] || Z.wall[0] || Z.wall[2])
            adjoint_tile<Q, NT, CPT, T, true>(d, sb, lin, lout, grad, Y, Z, y, z, xs, tid, gs, gc,
                                              release);
        else
            adjoint_tile<Q, NT, CPT, T, false>(d, sb, lin, lout, grad, Y, Z, y, z, xs, tid, gs, gc,
                                               release);
        if (++s == stages) { s = 0; par ^= 1u; }
    }
}

template <int Q, int NT, int CPT, typename T>
static cudaError_t launch_adj_tma_t(const VDom &d, const float *state, const float *lam_in,
                                    float *lam_out, float *grad, int stages, cudaStream_t s) {
    constexpr int TW = NT * CPT;
    constexpr int NS = 2 * Q + EpsRows<Q>::N;
    const size_t smem = kBarBytes + (size_t)stages * NS * (TW + 2 * kLead) * sizeof(float);
    if (stages < 2 || stages > kBarBytes / 16 || smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = k_adjoint_tma<Q, NT, CPT, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT + 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int ntx = (d.nx + TW - 1) / TW;
    const long long ntiles = (long long)ntx * d.rows;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * occ;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT + 32, smem, s>>>(d, state, lam_in, lam_out, grad, ntx, (int)ntiles,
                                               stages);
    return cudaGetLastError();
}

// L.warps -> compute warps (2 or 4), L.cpt -> cells per thread per tile (D2Q9
// 1 or 2, D3Q19 1), L.rows -> pipeline stages
cudaError_t launch_adjoint_tma(int q, const VDom &d, const float *state, const float *lam_in,
                               float *lam_out, float *grad, int fp64, Launch L, cudaStream_t s) {
    const int nt = 32 * L.warps;
#define VANS_ADJ_CASE(QQ, NTT, CC)                                                              \
    if (q == QQ && nt == NTT && L.cpt == CC)                                                    \
        return fp64 ? launch_adj_tma_t<QQ, NTT, CC, double>(d, state, lam_in, lam_out, grad, L.rows, s) \
                    : launch_adj_tma_t<QQ, NTT, CC, float>(d, state, lam_in, lam_out, grad, L.rows, s);
    VANS_ADJ_CASE(9, 64, 1)
    VANS_ADJ_CASE(9, 128, 1)
    VANS_ADJ_CASE(9, 128, 2)
    VANS_ADJ_CASE(19, 128, 1)
#undef VANS_ADJ_CASE
    return cudaErrorInvalidValue;
}

}  // namespace vans
