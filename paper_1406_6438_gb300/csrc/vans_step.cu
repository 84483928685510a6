// vans_step.cu -- the fused collide-and-stream step (the hot path).
//
// One kernel does the whole update of the final LBE with P_i and F_i for every
// cell it owns: pull the Q populations from the previous step's buffer (periodic
// wrap through the halo columns, half-way bounce-back at walls), form eps*rho and
// the implicit velocity of Eq. 1moment (drag solved in closed form), build
// f^eq (Eq. d2q9eq), P_i (Eq. pi) and F_i (Eq. Fi), relax and store.  Each
// population is read once from HBM and written once; eps comes through L1/L2.
//
// Thread mapping: a warp covers 32*CPT consecutive cells of one row (y for
// D2Q9, a (y,z) line for D3Q19); each lane owns CPT cells and loads them with
// one aligned vector load per direction.  The +-1 column shift of the pull is
// done with a warp shuffle, so every global load is an aligned vector load.
#include "vans_device.cuh"

namespace vans {

// Outputs of a monitoring step (vans_step_monitored): rho and u of the state
// the step reads, and reductions into stats = {max |u - u_prev|, max |u|,
// diverged (1.0f), emissions}.
struct Monitor {
    float *rho;
    float *u;
    float *stats;
    float *part;     // kMonSlots partial maxima of stats[0..2] each, [stat][slot]
};

__device__ __forceinline__ void atomic_max_nonneg(float *a, float v) {
    // non-negative floats order like their bit patterns
    atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
}

// PL: the instance handles plates on nodes (wall_kind 1); the others carry
// none of that code (it would raise their register count).
template <int Q, int CPT, bool EDGE, bool EMIT = false, bool PL = false>
__device__ __forceinline__ void step_row(const VDom &d, const float *__restrict__ fin,
                                         float *__restrict__ fout, int y, int z, int x0, int lane,
                                         const Monitor *mon = nullptr) {
    using L = Lat<Q>;
    // plates on nodes: a plate row is written by its fluid neighbour row
    const bool nee = PL && EDGE && d.nee;
    if (nee && (y == 0 || y == d.ny - 1)) return;
    const bool plo = nee && y == 1, phi = nee && y == d.ny - 2;
    const Nb3 Y = nb3<EDGE>(y, d.ny, d.wall_y);
    Nb3 Z;
    if (Q == 19) {
        Z = nb3<EDGE>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }

    // S1: pull.  h_i(x) = stored deviation at x - e_i, or the opposite
    // direction of x itself when x - e_i lies past a wall.
    float h[Q][CPT];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long ro = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        ld_shift<CPT>(fin + si * d.plane + ro, x0, bb ? 0 : -ex, lane, h[i]);
    }

    // porosity of the cell and of its Q-1 neighbours (for grad eps and the
    // deviation shift), from the padded eps rows
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

    // the monitored step's previous u, loaded with the populations: read after
    // this thread's first moment stores, the loads (which may alias them) were
    // serialised behind them (1.7 ms for a 250 us step at 4096^2)
    float up[L::D][CPT];
    if (EMIT) {
        const long long nb = ((long long)z * d.ny + y) * d.nx + x0;
#pragma unroll
        for (int c = 0; c < L::D; ++c)
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                up[c][k] = (x0 + k < d.nx) ? mon->u[c * d.cells + nb + k] : 0.f;
    }

    float out[Q][CPT], lo[Q][CPT], hi[Q][CPT];   // lo / hi: the plate nodes below / above
    float dmax = 0.f, umax = 0.f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        float hh[Q], et[Q];
        const float e0 = E[1][1][k + 1];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            hh[i] = h[i][k];
            const bool wall = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
            et[i] = (i == 0 || wall) ? e0 : E[1 + L::ey(i)][1 + L::ez(i)][k + 1 + L::ex(i)];
        }
        if (EDGE) apply_moving_wall<Q>(d, Y.wall[2], Z, e0, hh);
        if (EMIT) {
            // S8 fused into the step: the moments of the state this step reads
            Macro<Q> M;
            macro<Q>(d, hh, e0, et, M);
            if (x0 + k < d.nx) {
                const long long n = ((long long)z * d.ny + y) * d.nx + x0 + k;
                mon->rho[n] = M.rho;
                float du2 = 0.f;
#pragma unroll
                for (int c = 0; c < L::D; ++c) {
                    du2 += (M.u[c] - up[c][k]) * (M.u[c] - up[c][k]);
                    mon->u[c * d.cells + n] = M.u[c];
                }
                dmax = fmaxf(dmax, sqrtf(du2));
                umax = fmaxf(umax, M.un);
                bad = bad || !isfinite(M.R) || !isfinite(M.un) || !(M.un < 0.5f);
            }
        }
        float o[Q];
        Macro<Q> M;
        collide<Q>(d, hh, e0, et, o, nee ? &M : nullptr);   // S2-S7
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i][k] = o[i];
        if (plo || phi) {
            // post-collision values the plate nodes send into this row, stored
            // against the porosity of the cell they stream to
            const float om1 = 1.f - d.omega, zero[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float enb = E[1][1 + L::ez(i)][k + 1 + L::ex(i)];
                if (plo && L::ey(i) > 0)
                    lo[i][k] = plate_value<Q>(d, i, hh[i], M, E[0][1][k + 1], enb, zero, om1);
                if (phi && L::ey(i) < 0)
                    hi[i][k] = plate_value<Q>(d, i, hh[i], M, E[2][1][k + 1], enb, d.uw, om1);
            }
        }
    }
    if (EMIT) {
        // warp maxima, one atomic per warp
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dmax = fmaxf(dmax, __shfl_xor_sync(VANS_FULL, dmax, off));
            umax = fmaxf(umax, __shfl_xor_sync(VANS_FULL, umax, off));
        }
        bad = __any_sync(VANS_FULL, bad);
        if (lane == 0) {
            // one of kMonSlots partial maxima per warp: with every warp on the
            // same three words the step took 634 us at 4096^2, 420 us spread
            const int slot = (int)((blockIdx.x * ((blockDim.x * blockDim.y) >> 5) +
                                    ((threadIdx.y * blockDim.x + threadIdx.x) >> 5)) &
                                   (kMonSlots - 1));
            atomic_max_nonneg(&mon->part[slot], bad ? 0.f : dmax);
            atomic_max_nonneg(&mon->part[kMonSlots + slot], bad ? 0.f : umax);
            if (bad) atomic_max_nonneg(&mon->part[2 * kMonSlots + slot], 1.f);
        }
    }

    const long long ro = row_offset(d, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_masked<CPT>(fout + i * d.plane + ro, x0, d.nx, out[i]);
    // halo copies: column nx mirrors column 0 for directions moving -x, column
    // -1 mirrors column nx-1 for directions moving +x
    if (x0 == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::ex(i) < 0) store_halo_hi<Q>(fout + i * d.plane + ro, d.nx, out[i][0]);
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if (x0 + k == d.nx - 1) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ex(i) > 0) store_halo_lo<Q>(fout + i * d.plane + ro, out[i][k]);
        }
    }
    if (plo || phi) store_plates<Q, CPT>(d, fout, y, z, x0, plo, phi, lo, hi);
}

template <int Q, int CPT, bool EMIT = false, bool PL = false>
__global__ void __launch_bounds__(256) k_step(const VDom d, const float *__restrict__ fin,
                                              float *__restrict__ fout, int nxb, Monitor mon = {}) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int wx = threadIdx.x >> 5;
    const int bx = blockIdx.x % nxb;
    const int by = blockIdx.x / nxb;
    const int r = by * blockDim.y + threadIdx.y;
    if (r >= d.rows) return;                               // whole warp
    const int xw = (bx * (blockDim.x >> 5) + wx) * 32 * CPT;
    if (xw >= d.nx) return;                                // whole warp
    const int x0 = xw + lane * CPT;
    const int y = r % d.ny, z = r / d.ny;
    const bool edge = (y == 0) || (y == d.ny - 1) || (PL && (y == 1 || y == d.ny - 2)) ||
                      (Q == 19 && (z == 0 || z == d.nz - 1));
    if (edge)
        step_row<Q, CPT, true, EMIT, PL>(d, fin, fout, y, z, x0, lane, &mon);
    else
        step_row<Q, CPT, false, EMIT, PL>(d, fin, fout, y, z, x0, lane, &mon);
    if (EMIT && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(&mon.stats[3], 1.f);
}

// Batched D2Q9: one persistent grid walks a flattened list of equal-shaped
// tiles drawn from all domains; each tile carries its domain index, whose
// descriptor (sizes, tau, drag constants, buffers) comes from a device table.
template <int CPT>
__global__ void __launch_bounds__(256) k_step_batched(const VDom *__restrict__ doms,
                                                      const Tile *__restrict__ tiles, int ntiles,
                                                      int parity) {
    const int lane = threadIdx.x & 31;
    const int wx = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const VDom d = doms[T.dom];
        const int r = T.row + threadIdx.y;
        const int xw = T.x0 + wx * 32 * CPT;
        if (r < d.rows && xw < d.nx) {                     // whole warp
            const int x0 = xw + lane * CPT;
            const float *fin = parity ? d.f[1] : d.f[0];
            float *fout = parity ? d.f[0] : d.f[1];
            if (r == 0 || r == d.ny - 1)
                step_row<9, CPT, true>(d, fin, fout, r, 0, x0, lane);
            else
                step_row<9, CPT, false>(d, fin, fout, r, 0, x0, lane);
        }
    }
}

template <int Q, int CPT>
static cudaError_t launch_step_t(const VDom &d, const float *fin, float *fout, Launch L,
                                 cudaStream_t stream) {
    const int cells_per_block_x = 32 * CPT * L.warps;
    const int nxb = (d.nx + cells_per_block_x - 1) / cells_per_block_x;
    const int nrb = (d.rows + L.rows - 1) / L.rows;
    const long long nblocks = (long long)nxb * nrb;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)nblocks), block(32 * L.warps, L.rows);
    const Monitor none{};
    return d.nee ? launch_pdl(k_step<Q, CPT, false, true>, grid, block, 0, stream, d, fin, fout, nxb, none)
                 : launch_pdl(k_step<Q, CPT, false, false>, grid, block, 0, stream, d, fin, fout, nxb, none);
}

cudaError_t launch_step(int q, const VDom &d, const float *fin, float *fout, Launch L,
                        cudaStream_t stream) {
    if (L.kind >= 1 && L.kind <= 7) return launch_step_tma(q, d, fin, fout, L, stream);
    if (L.kind == 8) return launch_step_cluster(q, d, fin, fout, 1, L, stream);
    if (L.kind != 0) return cudaErrorInvalidValue;
    if (q == 9) {
        switch (L.cpt) {
            case 1: return launch_step_t<9, 1>(d, fin, fout, L, stream);
            case 2: return launch_step_t<9, 2>(d, fin, fout, L, stream);
            case 4: return launch_step_t<9, 4>(d, fin, fout, L, stream);
        }
    } else if (q == 19) {
        switch (L.cpt) {
            case 1: return launch_step_t<19, 1>(d, fin, fout, L, stream);
            case 2: return launch_step_t<19, 2>(d, fin, fout, L, stream);
            case 4: return launch_step_t<19, 4>(d, fin, fout, L, stream);
        }
    }
    return cudaErrorInvalidValue;
}

// A monitoring step: the register-load kernel (D2Q9 4 cells per lane, D3Q19 2;
// 4 warps) with the moment outputs and reductions switched on.
cudaError_t launch_step_monitor(int q, const VDom &d, const float *fin, float *fout, float *rho,
                                float *u, float *stats, float *part, cudaStream_t stream) {
    constexpr int WARPS = 4;
    const int cpt = q == 9 ? 4 : 2;     // D3Q19: 2 cells per lane (4 took 176 registers)
    const int nxb = (d.nx + 32 * cpt * WARPS - 1) / (32 * cpt * WARPS);
    const long long nblocks = (long long)nxb * d.rows;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const Monitor mon{rho, u, stats, part};
    if (q == 9)
        k_step<9, 4, true><<<(unsigned)nblocks, 32 * WARPS, 0, stream>>>(d, fin, fout, nxb, mon);
    else if (q == 19)
        k_step<19, 2, true><<<(unsigned)nblocks, 32 * WARPS, 0, stream>>>(d, fin, fout, nxb, mon);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// stats[c] = max over the slots of part[c][slot], c = 0..2 (one block)
__global__ void k_monitor_finalize(const float *__restrict__ part, float *__restrict__ stats) {
    __shared__ float red[3][kMonSlots];
    for (int i = threadIdx.x; i < kMonSlots; i += blockDim.x)
        for (int c = 0; c < 3; ++c) red[c][i] = part[c * kMonSlots + i];
    __syncthreads();
    for (int w = kMonSlots / 2; w > 0; w >>= 1) {
        for (int i = threadIdx.x; i < w; i += blockDim.x)
            for (int c = 0; c < 3; ++c) red[c][i] = fmaxf(red[c][i], red[c][i + w]);
        __syncthreads();
    }
    if (threadIdx.x < 3) stats[threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_monitor_finalize(const float *part, float *stats, cudaStream_t stream) {
    k_monitor_finalize<<<1, 256, 0, stream>>>(part, stats);
    return cudaGetLastError();
}

int batched_blocks_per_sm(Launch L) {
    int n = 0;
    const int threads = 32 * L.warps * L.rows;
    cudaError_t e = cudaErrorInvalidValue;
    switch (L.cpt) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batched<1>, threads, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batched<2>, threads, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batched<4>, threads, 0); break;
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

cudaError_t launch_step_batched(const VDom *doms_dev, const Tile *tiles_dev, int ntiles, int parity,
                                Launch L, int grid, cudaStream_t stream) {
    dim3 block(32 * L.warps, L.rows);
    switch (L.cpt) {
        case 1: k_step_batched<1><<<grid, block, 0, stream>>>(doms_dev, tiles_dev, ntiles, parity); break;
        case 2: k_step_batched<2><<<grid, block, 0, stream>>>(doms_dev, tiles_dev, ntiles, parity); break;
        case 4: k_step_batched<4><<<grid, block, 0, stream>>>(doms_dev, tiles_dev, ntiles, parity); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vans
