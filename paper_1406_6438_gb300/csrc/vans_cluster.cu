// vans_cluster.cu -- many steps in one launch for domains that fit in the
// shared memory of one thread-block cluster (launch kind 8).
//
// A small domain (the 128x64 channel, the 80x80 Couette case) is a few
// hundred KB of populations: one step is a few microseconds of launch
// overhead around less than a microsecond of work.  Here one cluster of up to
// 16 CTAs holds the whole state in its distributed shared memory for the
// whole run: CTA k owns a band of consecutive rows (row = z * ny + y) and keeps
// two copies of its band, the populations the step reads and the ones it
// writes, each row with its halo columns -1 and nx.  A step is the same pull,
// collision and store as every other kernel here (the functions of
// vans_device.cuh, so the same arithmetic); a pull that crosses into another
// band reads the owning CTA's shared memory through the cluster's
// distributed shared memory window.  One cluster barrier per step separates
// the writes of step t from the reads of step t + 1; because the two copies
// alternate, the writes of step t + 1 (into the copy read at step t) also
// come after every read of step t.  The band is loaded from the state buffer
// `fin` at the start and written back to `fout` at the end (columns -1 .. nx
// of every row and direction, the library's padded layout).
#include <cooperative_groups.h>

#include "vans_device.cuh"

namespace cg = cooperative_groups;

namespace vans {

namespace {

constexpr int kClusterMax = 16;
constexpr int kClusterSmemMax = 227 * 1024;

// floats per row copy in shared memory: columns -1 .. nx, rounded up to 4
__host__ __device__ inline int cluster_row_floats(int nx) { return (nx + 2 + 3) & ~3; }

// cells per thread at most: D2Q9 2, D3Q19 1 (its 19 addresses and porosities
// per cell stay in registers for the whole launch)
template <int Q> struct CellsMax { static constexpr int N = (Q == 9) ? 2 : 1; };

// Address, in the cluster's shared-memory window, of `local` (a shared-memory
// address of this CTA) in the shared memory of CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const float *local, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ float ld_cluster(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" :: "r"(addr), "f"(v) : "memory");
}

}  // namespace

// Every thread keeps at most CellsMax<Q>::N cells of its CTA's band for the
// whole launch.  What a cell's update needs besides the populations does not
// change from step to step, so it is formed once, before the first step: the
// address (in the cluster's shared-memory window, so in the shared memory of
// the CTA that owns the row) of each of the Q entries its pull reads, and its
// own and its neighbours' porosities.  A step is then Q loads, the collision
// and Q stores per cell.
// PL (plates on nodes, wall_kind 1): rows 0 and ny-1 are plate nodes and are
// not stepped; the fluid row next to a plate writes the plate node's inward
// populations (f^eq of the plate plus this cell's non-equilibrium part,
// relaxed), as the other step kernels do, into the plate row's entries, which
// may lie in the neighbouring CTA's band (a store through the cluster window).
template <int Q, int NT, bool PL>
__global__ void __launch_bounds__(NT) k_step_cluster(const VDom d, const float *fin, float *fout,
                                                     int nsteps, int band) {
    using L = Lat<Q>;
    constexpr int kCellsMax = CellsMax<Q>::N;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int sp = cluster_row_floats(d.nx);
    const long long copy = (long long)Q * band * sp;     // floats of one copy of a band
    extern __shared__ __align__(16) float sm[];
    const int r0 = rank * band;
    const int nr = max(0, min(band, d.rows - r0));
    const int nx = d.nx;

    // the band's rows of the state buffer, columns -1 .. nx
    for (long long t = threadIdx.x; t < (long long)Q * nr * (nx + 2); t += NT) {
        const int c = (int)(t % (nx + 2));
        const long long pr = t / (nx + 2);
        const int rl = (int)(pr % nr), i = (int)(pr / nr);
        sm[((long long)i * band + rl) * sp + c] =
            fin[i * d.plane + (long long)(r0 + rl) * d.pitch + d.off - 1 + c];
    }

    // per cell, fixed for the launch: pull addresses (copy 0), porosities,
    // the row offset of its stores, and whether it sits under a moving wall
    uint32_t src[kCellsMax][Q];
    float e0[kCellsMax], et[kCellsMax][Q];
    int dst[kCellsMax], xs[kCellsMax];
    bool top[kCellsMax], live[kCellsMax];
    Nb3 Zs[kCellsMax];
    // plates on nodes: sides (bit 0 the plate below, bit 1 the plate above:
    // both for the one fluid row between plates 2 rows apart), and each plate
    // row's entry of this column (copy 0, plane 0, cluster window)
    int pside[kCellsMax];
    uint32_t pdst[kCellsMax][2];
#pragma unroll
    for (int k = 0; k < kCellsMax; ++k) {
        const int t = threadIdx.x + k * NT;
        live[k] = t < nr * nx;
        const int tt = live[k] ? t : 0;
        const int rl = tt / nx, x = tt - rl * nx;
        const int r = r0 + rl, y = r % d.ny, z = r / d.ny;
        pside[k] = 0;
        pdst[k][0] = pdst[k][1] = 0;
        if (PL) {
            if (y == 0 || y == d.ny - 1) live[k] = false;          // plate node: not stepped
            if (live[k]) {
                pside[k] = (y == 1 ? 1 : 0) | (y == d.ny - 2 ? 2 : 0);
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (!(pside[k] & (1 << side))) continue;
                    const int rp = side == 0 ? r - 1 : r + 1, owner = rp / band;
                    pdst[k][side] =
                        cluster_addr(sm + (long long)(rp - owner * band) * sp + 1 + x, owner);
                }
            }
        }
        const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
        Nb3 Z;
        if (Q == 19) {
            Z = nb3<true>(z, d.nz, d.wall_z);
        } else {
            Z.r[0] = Z.r[1] = Z.r[2] = 0;
            Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
        }
        Zs[k] = Z;
        top[k] = Y.wall[2];
        xs[k] = x;
        dst[k] = rl * sp + 1 + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // the entry at x - e_i of row (y - e_y, z - e_z), or the opposite
            // direction of this cell past a wall; that row lives in the band
            // of CTA row / band
            const int ey = L::ey(i), ez = L::ez(i);
            const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
            const int sr = bb ? r : Z.r[1 - ez] * d.ny + Y.r[1 - ey];
            const int owner = sr / band;
            const int plane = bb ? L::opp(i) : i;
            const int col = bb ? x : x - L::ex(i);
            src[k][i] = cluster_addr(sm + ((long long)plane * band + (sr - owner * band)) * sp +
                                         col + 1, owner);
        }
        e0[k] = live[k] ? __ldg(d.eps + row_offset(d, y, z) + x) : 1.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
            et[k][i] = (i == 0 || wall || !live[k])
                           ? e0[k]
                           : __ldg(d.eps + row_offset(d, Y.r[1 + L::ey(i)], Z.r[1 + L::ez(i)]) + x +
                                   L::ex(i));
        }
    }
    cl.sync();

    int b = 0;
    for (int s = 0; s < nsteps; ++s) {
        const uint32_t cur = (uint32_t)(b * copy * sizeof(float));   // the copy read this step
        float *nxt = sm + (b ^ 1) * copy;
#pragma unroll
        for (int k = 0; k < kCellsMax; ++k) {
            if (!live[k]) continue;
            float h[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i] = ld_cluster(src[k][i] + cur);
            apply_moving_wall<Q>(d, top[k], Zs[k], e0[k], h);
            float o[Q];
            Macro<Q> M;
            collide<Q>(d, h, e0[k], et[k], o, (PL && pside[k]) ? &M : nullptr);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float *row = nxt + (long long)i * band * sp + dst[k];   // this cell's column
                row[0] = o[i];
                if (xs[k] == 0 && L::ex(i) < 0) row[nx] = o[i];         // halo copies of the wrap
                if (xs[k] == nx - 1 && L::ex(i) > 0) row[-nx] = o[i];
            }
            if (PL && pside[k]) {
                // the plate node's populations toward this row: e_y > 0 from
                // the plate below, e_y < 0 from the plate above, each stored
                // against the porosity of the row cell it streams to
                constexpr int jym = dir_index<Q>(0, -1, 0), jyp = dir_index<Q>(0, 1, 0);
                constexpr int jxp = dir_index<Q>(1, 0, 0), jxm = dir_index<Q>(-1, 0, 0);
                constexpr int jzp = dir_index<Q>(0, 0, 1), jzm = dir_index<Q>(0, 0, -1);
                const float om1 = 1.f - d.omega, zero[3] = {0.f, 0.f, 0.f};
                const uint32_t next = (uint32_t)((b ^ 1) * copy * sizeof(float));
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int ey = L::ey(i);
                    if (ey == 0 || !(pside[k] & (ey > 0 ? 1 : 2))) continue;
                    const bool lo = ey > 0;
                    const int ex = L::ex(i), ez = L::ez(i);
                    const float enb = ex > 0 ? et[k][jxp] : ex < 0 ? et[k][jxm]
                                    : ez > 0 ? et[k][jzp] : ez < 0 ? et[k][jzm] : e0[k];
                    const float v = plate_value<Q>(d, i, h[i], M, lo ? et[k][jym] : et[k][jyp], enb,
                                                   lo ? zero : d.uw, om1);
                    const uint32_t a = pdst[k][lo ? 0 : 1] + next +
                                       (uint32_t)((long long)i * band * sp * sizeof(float));
                    st_cluster(a, v);
                    if (xs[k] == 0 && ex < 0) st_cluster(a + (uint32_t)(nx * sizeof(float)), v);
                    if (xs[k] == nx - 1 && ex > 0) st_cluster(a - (uint32_t)(nx * sizeof(float)), v);
                }
            }
        }
        cl.sync();
        b ^= 1;
    }

    const float *res = sm + b * copy;
    for (long long t = threadIdx.x; t < (long long)Q * nr * (nx + 2); t += NT) {
        const int c = (int)(t % (nx + 2));
        const long long pr = t / (nx + 2);
        const int rl = (int)(pr % nr), i = (int)(pr / nr);
        fout[i * d.plane + (long long)(r0 + rl) * d.pitch + d.off - 1 + c] =
            res[((long long)i * band + rl) * sp + c];
    }
}

// Rows per CTA and CTAs of the cluster for a cluster of at most cmax CTAs.
static void cluster_shape(const VDom &d, int cmax, int &band, int &ctas) {
    band = (d.rows + cmax - 1) / cmax;
    ctas = (d.rows + band - 1) / band;
}

size_t cluster_smem_bytes(int q, const VDom &d, int cmax) {
    int band = 0, ctas = 0;
    cluster_shape(d, cmax, band, ctas);
    return 2 * (size_t)q * band * cluster_row_floats(d.nx) * sizeof(float);
}

bool cluster_fits(int q, const VDom &d, int cmax, int warps) {
    if (cmax < 1 || cmax > kClusterMax) return false;
    int band = 0, ctas = 0;
    cluster_shape(d, cmax, band, ctas);
    const int cells_max = (q == 9) ? CellsMax<9>::N : CellsMax<19>::N;
    if ((long long)band * d.nx > (long long)cells_max * 32 * warps) return false;
    return cluster_smem_bytes(q, d, cmax) <= (size_t)kClusterSmemMax;
}

template <int Q, int NT>
static cudaError_t launch_cluster_t(const VDom &d, const float *fin, float *fout, int nsteps,
                                    int cmax, cudaStream_t stream) {
    int band = 0, ctas = 0;
    cluster_shape(d, cmax, band, ctas);
    const size_t smem = cluster_smem_bytes(Q, d, cmax);
    auto kern = d.nee ? k_step_cluster<Q, NT, true> : k_step_cluster<Q, NT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ctas > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    e = cudaLaunchKernelEx(&cfg, kern, d, fin, fout, nsteps, band);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// kind 8: `warps` warps per CTA (8 or 16), `rows` = the largest cluster (2..16)
cudaError_t launch_step_cluster(int q, const VDom &d, const float *fin, float *fout, int nsteps,
                                Launch L, cudaStream_t stream) {
    if (nsteps < 1) return cudaErrorInvalidValue;
    if (!cluster_fits(q, d, L.rows, L.warps)) return cudaErrorInvalidValue;
    if (q == 9) {
        if (L.warps == 8) return launch_cluster_t<9, 256>(d, fin, fout, nsteps, L.rows, stream);
        if (L.warps == 16) return launch_cluster_t<9, 512>(d, fin, fout, nsteps, L.rows, stream);
    } else if (q == 19) {
        if (L.warps == 8) return launch_cluster_t<19, 256>(d, fin, fout, nsteps, L.rows, stream);
        if (L.warps == 16) return launch_cluster_t<19, 512>(d, fin, fout, nsteps, L.rows, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vans
