// vans_step_tma.cu -- the fused step with a bulk-copy (TMA) pipeline.
//
// Same arithmetic as k_step (vans_step.cu) -- pull, moments, implicit velocity,
// f^eq + P_i + F_i, relax, store -- but the loads no longer come from the
// threads.  A persistent CTA owns a contiguous run of tiles (TW cells of one
// row); one elected thread streams the Q source-row segments and the porosity
// rows of the next tiles into shared memory with 1-D cp.async.bulk copies that
// complete on an mbarrier, while all threads compute the current tile from
// shared memory.  Copies therefore stay in flight through the compute phase,
// which is what limited the register-load version (one load phase per warp,
// then ~1100 instructions with nothing in flight).  Shared-memory reads are
// unit-stride across a warp (no bank conflicts) and the +-1 column shift of the
// pull is just an offset.  Stores go straight to global memory, 128 bytes per
// warp instruction.
#include "vans_device.cuh"
#include "vans_tma.cuh"

namespace vans {

template <int Q> struct EpsRows;
template <> struct EpsRows<9> { static constexpr int N = 3; };    // dy = -1, 0, 1
template <> struct EpsRows<19> { static constexpr int N = 9; };   // (dy, dz) in {-1,0,1}^2

template <int Q>
__host__ __device__ constexpr int eps_slot(int dy, int dz) {
    return Q == 9 ? dy + 1 : (dz + 1) * 3 + (dy + 1);
}

template <int Q>
__device__ __forceinline__ void row_nbs(const VDom &d, int row, int &y, int &z, Nb3 &Y, Nb3 &Z) {
    y = row % d.ny;
    z = row / d.ny;
    Y = nb3<true>(y, d.ny, d.wall_y);
    if (Q == 19) {
        Z = nb3<true>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }
}

constexpr int kBarBytes = 128;   // room for up to 16 mbarriers in front of the stages

// Issue the bulk copies of the tile (row, xs) into stage buffer sb (one thread).
template <int Q, int TW>
__device__ __forceinline__ void issue_tile(const VDom &d, const float *__restrict__ fin, int row,
                                           int xs, float *sb, uint64_t *bar) {
    using L = Lat<Q>;
    constexpr int SEG = TW + 8;
    constexpr int NS = Q + EpsRows<Q>::N;
    int y, z;
    Nb3 Y, Z;
    row_nbs<Q>(d, row, y, z, Y, Z);
    const int nval = min(TW, d.nx - xs);
    // columns xs-4 .. xs+round4(nval)+3: the cells, the +-1 neighbours (halo
    // columns included) and 16-byte alignment on both ends
    const uint32_t bytes = (uint32_t)((((nval + 3) & ~3) + 8) * 4);
    mbar_arrive_expect_tx(bar, bytes * NS);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long ro = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        bulk_g2s(sb + i * SEG, fin + si * d.plane + ro + xs - 4, bytes, bar);
    }
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if (Q == 9 && dz != 0) continue;
            const float *src = d.eps + row_offset(d, Y.r[1 + dy], Z.r[1 + dz]) + xs - 4;
            bulk_g2s(sb + (Q + eps_slot<Q>(dy, dz)) * SEG, src, bytes, bar);
        }
    (void)NS;
}

template <int Q, int NT, int CPT>
__global__ void __launch_bounds__(NT) k_step_tma(const VDom d, const float *__restrict__ fin,
                                                 float *__restrict__ fout, int ntx, int ntiles,
                                                 int stages) {
    using L = Lat<Q>;
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 8;
    constexpr int NS = Q + EpsRows<Q>::N;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    const int tid = threadIdx.x;
    const int t0 = (int)((long long)blockIdx.x * ntiles / gridDim.x);
    const int t1 = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
    const int n = t1 - t0;
    if (n <= 0) return;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // tile cursors (row, column block) advanced one tile at a time: the
    // consumer's for tile t0 + k, thread 0's producer one `stages` tiles ahead
    int row = t0 / ntx, xt = t0 - (t0 / ntx) * ntx;
    int prow = row, pxt = xt;
    if (tid == 0) {
        const int pre = n < stages ? n : stages;
        for (int k = 0; k < pre; ++k) {
            issue_tile<Q, TW>(d, fin, prow, pxt * TW, buf + k * (NS * SEG), &bars[k]);
            if (++pxt == ntx) { pxt = 0; ++prow; }
        }
    }

    int k = 0, s = 0;
    uint32_t par = 0;
    bool ok = true;
    for (; k < n; ++k) {
        ok = __syncthreads_and(mbar_wait_bounded(&bars[s], par));
        if (!ok) break;
        const float *sb = buf + s * (NS * SEG);
        const int xs = xt * TW;
        int y, z;
        Nb3 Y, Z;
        row_nbs<Q>(d, row, y, z, Y, Z);
        const long long ro = row_offset(d, y, z);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int xl = tid + c * NT;
            const int x = xs + xl;
            float h[Q], et[Q], o[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = Y.wall[1 - L::ey(i)] || Z.wall[1 - L::ez(i)];
                h[i] = sb[i * SEG + 4 + xl + (bb ? 0 : -L::ex(i))];
            }
            const float e0 = sb[(Q + eps_slot<Q>(0, 0)) * SEG + 4 + xl];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool wall = Y.wall[1 + L::ey(i)] || Z.wall[1 + L::ez(i)];
                et[i] = (i == 0 || wall)
                            ? e0
                            : sb[(Q + eps_slot<Q>(L::ey(i), L::ez(i))) * SEG + 4 + xl + L::ex(i)];
            }
            collide<Q>(d, h, e0, et, o);
            if (x < d.nx) {
#pragma unroll
                for (int i = 0; i < Q; ++i) fout[i * d.plane + ro + x] = o[i];
                if (x == 0) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ex(i) < 0) fout[i * d.plane + ro + d.nx] = o[i];
                }
                if (x == d.nx - 1) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ex(i) > 0) fout[i * d.plane + ro - 1] = o[i];
                }
            }
        }
        __syncthreads();                 // everyone is done reading stage s
        if (tid == 0 && k + stages < n) {
            fence_proxy_async_smem();
            issue_tile<Q, TW>(d, fin, prow, pxt * TW, buf + s * (NS * SEG), &bars[s]);
            if (++pxt == ntx) { pxt = 0; ++prow; }
        }
        if (++xt == ntx) { xt = 0; ++row; }
        if (++s == stages) { s = 0; par ^= 1u; }
    }
    if (!ok) {
        // a copy did not land within the time limit: flag it, then give the
        // copies already issued into this CTA's shared memory a bounded chance
        // to finish before the CTA exits
        if (tid == 0) {
            if (d.status) atomicOr(d.status, 2);
            const int last = (k + stages < n) ? k + stages : n;
            for (int j = k; j < last; ++j)
                mbar_wait_bounded(&bars[j % stages], (uint32_t)((j / stages) & 1));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// D2Q9 variant with a porosity ring.  Each CTA walks a vertical strip: one
// column block xt and a run of consecutive rows r0..r1-1, so tile k needs the
// eps rows r0+k-1, r0+k, r0+k+1 and only r0+k+1 is new.  The eps rows live in
// a ring of stages+2 row slots next to the population stages; the producer
// loads the one new row with each tile (the first tile also loads its two
// predecessors), so each eps row leaves HBM once per strip instead of three
// times.  Ring slot of eps row r0-1+j is j mod (stages+2); the slot a new row
// overwrites was last read by tile k-stages, which has finished when tile k is
// issued.
template <int TW>
__device__ __forceinline__ void issue_tile_ring(const VDom &d, const float *__restrict__ fin, int row,
                                                int xs, int k, int r0, float *sb, float *ring,
                                                int rslots, uint64_t *bar) {
    using L = Lat<9>;
    constexpr int SEG = TW + 8;
    const int y = row;
    const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
    const int nval = min(TW, d.nx - xs);
    const uint32_t bytes = (uint32_t)((((nval + 3) & ~3) + 8) * 4);
    const int neps = (k == 0) ? 3 : 1;
    mbar_arrive_expect_tx(bar, bytes * (9 + neps));
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ey = L::ey(i);
        const bool bb = Y.wall[1 - ey];
        const int si = bb ? L::opp(i) : i;
        const long long ro = (long long)(bb ? y : Y.r[1 - ey]) * d.pitch + VANS_OFF;
        bulk_g2s(sb + i * SEG, fin + si * d.plane + ro + xs - 4, bytes, bar);
    }
    for (int j = (k == 0 ? 0 : k + 2); j <= k + 2; ++j) {
        int ry = r0 - 1 + j;                      // eps row r0-1+j, wrapped into [0, ny)
        ry = ry < 0 ? ry + d.ny : (ry >= d.ny ? ry - d.ny : ry);
        bulk_g2s(ring + (j % rslots) * SEG, d.eps + (long long)ry * d.pitch + VANS_OFF + xs - 4, bytes,
                 bar);
    }
}

template <int NT, int CPT>
__global__ void __launch_bounds__(NT) k_step_tma_ring(const VDom d, const float *__restrict__ fin,
                                                      float *__restrict__ fout, int ntx, int per_col,
                                                      int stages) {
    using L = Lat<9>;
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 8;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    float *ring = buf + stages * 9 * SEG;
    const int rslots = stages + 2;
    const int tid = threadIdx.x;
    // strip of this CTA: column block xt, rows [r0, r1)
    const int xt = blockIdx.x % ntx;
    const int c = blockIdx.x / ntx;
    const int r0 = (int)((long long)c * d.ny / per_col);
    const int r1 = (int)((long long)(c + 1) * d.ny / per_col);
    const int n = r1 - r0;
    if (n <= 0) return;
    const int xs = xt * TW;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
        const int pre = n < stages ? n : stages;
        for (int k = 0; k < pre; ++k)
            issue_tile_ring<TW>(d, fin, r0 + k, xs, k, r0, buf + k * 9 * SEG, ring, rslots, &bars[k]);
    }
    int k = 0, s = 0;
    uint32_t par = 0;
    bool ok = true;
    for (; k < n; ++k) {
        ok = __syncthreads_and(mbar_wait_bounded(&bars[s], par));
        if (!ok) break;
        const float *sb = buf + s * 9 * SEG;
        const float *em = ring + (k % rslots) * SEG;          // eps row y-1
        const float *e0r = ring + ((k + 1) % rslots) * SEG;   // eps row y
        const float *ep = ring + ((k + 2) % rslots) * SEG;    // eps row y+1
        const int y = r0 + k;
        const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
        const long long ro = (long long)y * d.pitch + VANS_OFF;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const int xl = tid + cc * NT;
            const int x = xs + xl;
            float h[9], et[9], o[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const bool bb = Y.wall[1 - L::ey(i)];
                h[i] = sb[i * SEG + 4 + xl + (bb ? 0 : -L::ex(i))];
            }
            const float e0 = e0r[4 + xl];
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int ey = L::ey(i);
                const float *er = ey > 0 ? ep : (ey < 0 ? em : e0r);
                et[i] = Y.wall[1 + ey] ? e0 : er[4 + xl + L::ex(i)];
            }
            et[0] = e0;
            collide<9>(d, h, e0, et, o);
            if (x < d.nx) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fout[i * d.plane + ro + x] = o[i];
                if (x == 0) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (L::ex(i) < 0) fout[i * d.plane + ro + d.nx] = o[i];
                }
                if (x == d.nx - 1) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (L::ex(i) > 0) fout[i * d.plane + ro - 1] = o[i];
                }
            }
        }
        __syncthreads();
        if (tid == 0 && k + stages < n) {
            fence_proxy_async_smem();
            issue_tile_ring<TW>(d, fin, r0 + k + stages, xs, k + stages, r0, buf + s * 9 * SEG, ring,
                                rslots, &bars[s]);
        }
        if (++s == stages) { s = 0; par ^= 1u; }
    }
    if (!ok) {
        if (tid == 0) {
            if (d.status) atomicOr(d.status, 2);
            const int last = (k + stages < n) ? k + stages : n;
            for (int j = k; j < last; ++j)
                mbar_wait_bounded(&bars[j % stages], (uint32_t)((j / stages) & 1));
        }
        __syncthreads();
    }
}

template <int NT, int CPT>
static cudaError_t launch_ring_t(const VDom &d, const float *fin, float *fout, int stages,
                                 cudaStream_t stream) {
    constexpr int TW = NT * CPT;
    const size_t smem = kBarBytes + (size_t)(stages * 9 + stages + 2) * (TW + 8) * sizeof(float);
    if (stages < 2 || stages > 16 || smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = k_step_tma_ring<NT, CPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int ntx = (d.nx + TW - 1) / TW;
    // strips per column block: fill the machine, at most one row per strip
    int per_col = (sms * occ) / ntx;
    if (per_col < 1) per_col = 1;
    if (per_col > d.ny) per_col = d.ny;
    const long long grid = (long long)per_col * ntx;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)grid, NT, smem, stream>>>(d, fin, fout, ntx, per_col, stages);
    return cudaGetLastError();
}

template <int Q, int NT, int CPT>
static size_t tma_smem_bytes(int stages) {
    constexpr int TW = NT * CPT;
    constexpr int NS = Q + EpsRows<Q>::N;
    return kBarBytes + (size_t)stages * NS * (TW + 8) * sizeof(float);
}

template <int Q, int NT, int CPT>
static cudaError_t launch_tma_t(const VDom &d, const float *fin, float *fout, int stages,
                                cudaStream_t stream) {
    constexpr int TW = NT * CPT;
    const size_t smem = tma_smem_bytes<Q, NT, CPT>(stages);
    if (stages < 2 || stages > 16 || smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = k_step_tma<Q, NT, CPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int ntx = (d.nx + TW - 1) / TW;
    const long long ntiles = (long long)ntx * d.rows;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * occ;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT, smem, stream>>>(d, fin, fout, ntx, (int)ntiles, stages);
    return cudaGetLastError();
}

// L.warps -> threads per CTA (32 * warps), L.cpt -> cells per thread per tile,
// L.rows -> pipeline stages; kind 2 selects the D2Q9 porosity-ring variant
cudaError_t launch_step_tma(int q, const VDom &d, const float *fin, float *fout, Launch L,
                            cudaStream_t stream) {
    const int nt = 32 * L.warps;
    if (L.kind == 2) {
        if (q != 9) return cudaErrorInvalidValue;
        if (nt == 128 && L.cpt == 2) return launch_ring_t<128, 2>(d, fin, fout, L.rows, stream);
        if (nt == 128 && L.cpt == 4) return launch_ring_t<128, 4>(d, fin, fout, L.rows, stream);
        if (nt == 256 && L.cpt == 1) return launch_ring_t<256, 1>(d, fin, fout, L.rows, stream);
        if (nt == 256 && L.cpt == 2) return launch_ring_t<256, 2>(d, fin, fout, L.rows, stream);
        return cudaErrorInvalidValue;
    }
#define VANS_TMA_CASE(QQ, NTT, CC)                              \
    if (q == QQ && nt == NTT && L.cpt == CC)                    \
        return launch_tma_t<QQ, NTT, CC>(d, fin, fout, L.rows, stream);
    VANS_TMA_CASE(9, 128, 2)
    VANS_TMA_CASE(9, 128, 4)
    VANS_TMA_CASE(9, 256, 1)
    VANS_TMA_CASE(9, 256, 2)
    VANS_TMA_CASE(19, 128, 1)
    VANS_TMA_CASE(19, 128, 2)
    VANS_TMA_CASE(19, 256, 1)
#undef VANS_TMA_CASE
    return cudaErrorInvalidValue;
}

}  // namespace vans
