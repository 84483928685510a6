// vans_step_tma.cu -- the fused step with a bulk-copy (TMA) pipeline.
//
// Same arithmetic as k_step (vans_step.cu) -- pull, moments, implicit velocity,
// f^eq + P_i + F_i, relax, store -- but the loads no longer come from the
// threads: one elected thread streams the Q source-row segments of a row tile
// and its porosity rows into shared memory with 1-D cp.async.bulk copies that
// complete on an mbarrier (transaction bytes), `stages` tiles ahead, while the
// compute threads work on the current tile from shared memory.  Copies stay in
// flight through the compute phase, which is what limited the register-load
// kernel (one load phase per warp, then ~1100 instructions with nothing in
// flight).  Shared-memory reads are unit-stride across a warp and the +-1
// column shift of the pull is an offset.  The launch kinds of this file:
//
//   2  k_step_tma_ring: each CTA walks a strip of consecutive rows of one
//      column block and keeps the porosity rows in a shared-memory ring (each
//      row leaves HBM once per strip); thread 0 refills a stage after a block
//      barrier.
//   4, 5  kind 2 warp-specialised: a producer warp refills a stage when every
//      compute warp has released it on an "empty" mbarrier, which each warp
//      does right after reading the stage into registers; 4 strided cells, 5
//      each thread on V adjacent cells (16- or 8-byte shared loads and global
//      stores).
//   6, 7  k_step_tma_ilv: persistent CTAs take tiles b, b+G, ... of the
//      row-major order (the whole grid sweeps one band of rows), warp-
//      specialised as 4/5; 6 strided cells, 7 adjacent cells.
//
// (Kinds 1 -- a pipeline over contiguous runs of tiles with the porosity rows
// staged per tile -- and 3 -- kind 2 with adjacent cells -- were never the
// fastest at any measured size and are not built.)
//
// The batched step (kinds 2, 4-7 over many domains) uses the same tile bodies
// with a strip table or an interleaved tile table; plates-on-nodes instances
// (wall_kind 1) exist for a subset of the launch shapes.
#include "vans_pipeline.cuh"

namespace vans {


// ---------------------------------------------------------------------------
// Variant with a porosity ring.  Each CTA walks one strip: a column block xt,
// one z plane and a run of consecutive rows y0..y1-1, so tile k (row y0+k)
// needs the eps rows at y-1, y, y+1 (times z-1, z, z+1 for D3Q19) and only the
// y+1 ones are new.  The eps rows live in a ring of stages+2 slots (a slot
// holds the NZR = 1 or 3 z-rows of one y) beside the population stages; the
// producer loads one slot per tile (the first tile also loads its two
// predecessors), so each eps row leaves HBM once per strip instead of three
// (D2Q9) or nine (D3Q19) times.  Slot of y-position y0-1+j is j mod (stages+2);
// the slot a new position overwrites was last read by tile k-stages, which has
// finished when tile k is issued.
template <int Q, int TW>
__device__ __forceinline__ void issue_tile_ring(const VDom &d, const float *__restrict__ fin, int y,
                                                int z, int xs, int k, int y0, float *sb, float *ring,
                                                int rslots, uint64_t *bar) {
    using L = Lat<Q>;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NZR = (Q == 9) ? 1 : 3;
    const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
    Nb3 Z;
    if (Q == 19) {
        Z = nb3<true>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }
    const int nval = min(TW, d.nx - xs);
    const uint32_t bytes = seg_bytes(nval);
    const int jfirst = (k == 0) ? 0 : k + 2;
    mbar_arrive_expect_tx(bar, bytes * (Q + NZR * (k + 3 - jfirst)));
    const uint64_t again = l2_evict_last();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long ro = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        bulk_g2s(sb + i * SEG, fin + si * d.plane + ro + xs - kLead, bytes, bar);
    }
    for (int j = jfirst; j <= k + 2; ++j) {
        int ry = y0 - 1 + j;                      // y-position y0-1+j, wrapped into [0, ny)
        ry = ry < 0 ? ry + d.ny : (ry >= d.ny ? ry - d.ny : ry);
        float *slot = ring + (j % rslots) * (NZR * SEG);
#pragma unroll
        for (int dz = 0; dz < NZR; ++dz) {
            const int rz = (Q == 9) ? 0 : Z.r[dz];
            bulk_g2s_hint(slot + dz * SEG, d.eps + row_offset(d, ry, rz) + xs - kLead, bytes, bar,
                          again);
        }
    }
}

// Compute of one staged tile with each thread on V consecutive cells (D2Q9:
// V = 4, D3Q19: V = 2), columns x0l..x0l+V-1 of the tile: each population row
// comes in one or two aligned V-wide shared loads (8 or 16 bytes) and each
// output row leaves in one V-wide global store.  Segment position p holds
// column xs - kLead + p.
template <int Q, int NT, int V, bool EDGE, bool PL, bool RAG, bool WRAP, class Rel>
__device__ __forceinline__ void ring_tile_vec(const VDom &d, const float *__restrict__ sb,
                                              const float *const ey_slot[3], const Nb3 &Y,
                                              const Nb3 &Z, float *__restrict__ fout, int y, int z,
                                              int xs, int tid, Rel &&release) {
    using L = Lat<Q>;
    static_assert(V == 2 || V == 4, "2 or 4 cells per thread");
    constexpr int SEG = NT * V + 2 * kLead;
    constexpr int NZ = (Q == 9) ? 1 : 3;      // z-rows per ring slot
    // plates on nodes (PL instances only): a plate row is written by its
    // fluid neighbour row
    const bool nee = PL && EDGE && d.nee;
    if (nee && (y == 0 || y == d.ny - 1)) {
        release();
        return;
    }
    const bool plo = nee && y == 1, phi = nee && y == d.ny - 2;
    const long long ro = row_offset(d, y, z);
    const int x0l = V * tid;
    // RAG (batched instances): a warp whose cells all lie past the last column
    // (the ragged last tile of a row) has nothing to compute or store
    if (RAG && xs + V * (tid & ~31) >= d.nx) {
        release();
        return;
    }
    auto ywall = [&](int k) { return EDGE && Y.wall[k]; };
    auto zwall = [&](int k) { return EDGE && Z.wall[k]; };
    auto vload = [&](const float *row, int p, float out[V]) {
        if constexpr (V == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(row + p);
            out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
        } else {
            const float2 t = *reinterpret_cast<const float2 *>(row + p);
            out[0] = t.x; out[1] = t.y;
        }
    };
    float h[Q][V];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *row = sb + i * SEG;
        const bool bb = ywall(1 - L::ey(i)) || zwall(1 - L::ez(i));
        const int s = bb ? 0 : -L::ex(i);
        float B[V];
        vload(row, x0l + kLead, B);
        if (s == 0) {
#pragma unroll
            for (int c = 0; c < V; ++c) h[i][c] = B[c];
        } else if (s < 0) {
            float A[V];
            vload(row, x0l + kLead - V, A);
            h[i][0] = (WRAP && x0l == 0) ? row[kLead + d.nx - 1] : A[V - 1];
#pragma unroll
            for (int c = 1; c < V; ++c) h[i][c] = B[c - 1];
        } else {
            float C[V];
            vload(row, x0l + kLead + V, C);
#pragma unroll
            for (int c = 0; c < V - 1; ++c) h[i][c] = B[c + 1];
            h[i][V - 1] = (WRAP && x0l + V == d.nx) ? row[kLead] : C[0];
        }
    }
    // eps rows (y + dy, z + dz) at columns x0l-1 .. x0l+V; a D3Q19 corner row
    // (dy, dz both nonzero) is only read at dx = 0
    float E[3][NZ][V + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int q = 0; q < NZ; ++q) {
            const float *row = ey_slot[r] + q * SEG;
            float B[V];
            vload(row, x0l + kLead, B);
#pragma unroll
            for (int c = 0; c < V; ++c) E[r][q][c + 1] = B[c];
            const bool side = (Q == 9) || r == 1 || q == 1;
            if (side) {
                float A[V], C[V];
                vload(row, x0l + kLead - V, A);
                vload(row, x0l + kLead + V, C);
                E[r][q][0] = (WRAP && x0l == 0) ? row[kLead + d.nx - 1] : A[V - 1];
                E[r][q][V + 1] = (WRAP && x0l + V == d.nx) ? row[kLead] : C[0];
            } else {
                E[r][q][0] = E[r][q][V + 1] = 0.f;    // never read
            }
        }
    }
    release();                  // the stage is no longer read
    constexpr int ZC = (Q == 9) ? 0 : 1;    // the z-row of dz = 0
    float out[Q][V], lo[Q][V], hi[Q][V];    // lo / hi: the plate nodes below / above
#pragma unroll
    for (int c = 0; c < V; ++c) {
        float hh[Q], et[Q], o[Q];
        const float e0 = E[1][ZC][c + 1];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            hh[i] = h[i][c];
            const bool wall = ywall(1 + L::ey(i)) || zwall(1 + L::ez(i));
            et[i] = (i == 0 || wall) ? e0 : E[1 + L::ey(i)][ZC + L::ez(i)][c + 1 + L::ex(i)];
        }
        if (EDGE) apply_moving_wall<Q>(d, Y.wall[2], Z, e0, hh);
        Macro<Q> M;
        collide<Q>(d, hh, e0, et, o, nee ? &M : nullptr);
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i][c] = o[i];
        if (plo || phi) {
            const float om1 = 1.f - d.omega, zero[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float enb = E[1][ZC + L::ez(i)][c + 1 + L::ex(i)];
                if (plo && L::ey(i) > 0)
                    lo[i][c] = plate_value<Q>(d, i, hh[i], M, E[0][ZC][c + 1], enb, zero, om1);
                if (phi && L::ey(i) < 0)
                    hi[i][c] = plate_value<Q>(d, i, hh[i], M, E[2][ZC][c + 1], enb, d.uw, om1);
            }
        }
    }
    const int x0 = xs + x0l;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_masked<V>(fout + i * d.plane + ro, x0, d.nx, out[i]);
    if (x0 == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::ex(i) < 0) store_halo_hi<Q>(fout + i * d.plane + ro, d.nx, out[i][0]);
    }
#pragma unroll
    for (int c = 0; c < V; ++c) {
        if (x0 + c == d.nx - 1) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::ex(i) > 0) store_halo_lo<Q>(fout + i * d.plane + ro, out[i][c]);
        }
    }
    if (plo || phi) store_plates<Q, V>(d, fout, y, z, x0, plo, phi, lo, hi);
}

// Compute and store one staged tile of the ring pipeline (all NT threads).
// Every shared-memory read of the tile comes first, into registers; then
// release() (the caller's way to hand the stage back to the producer), then
// the collisions and the global stores.
// EDGE = false: the tile's row touches no wall (the wall flags are known to be
// false at compile time, which drops the per-direction selects).  PL: the
// instance handles plates on nodes (wall_kind 1); the others carry none of that
// code (it would raise their register count).  RAG (the batched instances,
// whose domains end in ragged tiles): warps past the row's last column skip the
// tile; the single-domain instances measured slower with the test in place.
template <int Q, int NT, int CPT, bool VEC, bool EDGE, bool PL, bool RAG, class Rel,
          bool WRAP = false>
__device__ __forceinline__ void ring_tile(const VDom &d, const float *__restrict__ sb,
                                          const float *const ey_slot[3], const Nb3 &Y, const Nb3 &Z,
                                          float *__restrict__ fout, int y, int z, int xs, int tid,
                                          Rel &&release) {
    using L = Lat<Q>;
    constexpr int SEG = NT * CPT + 2 * kLead;
    if constexpr (VEC) {
        ring_tile_vec<Q, NT, CPT, EDGE, PL, RAG, WRAP>(d, sb, ey_slot, Y, Z, fout, y, z, xs, tid,
                                                        release);
    } else {
        // plates on nodes (PL instances only): a plate row is written by its
        // fluid neighbour row
        const bool nee = PL && EDGE && d.nee;
        if (nee && (y == 0 || y == d.ny - 1)) {
            release();
            return;
        }
        const bool plo = nee && y == 1, phi = nee && y == d.ny - 2;
        const long long ro = row_offset(d, y, z);
        auto ywall = [&](int k) { return EDGE && Y.wall[k]; };
        auto zwall = [&](int k) { return EDGE && Z.wall[k]; };
        float h[CPT][Q], et[CPT][Q];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const int xl = tid + cc * NT;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = ywall(1 - L::ey(i)) || zwall(1 - L::ez(i));
                h[cc][i] = sb[i * SEG + kLead + xl + (bb ? 0 : -L::ex(i))];
            }
            const float e0 = ey_slot[1][(Q == 9 ? 0 : 1) * SEG + kLead + xl];
            et[cc][0] = e0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int ey = L::ey(i), ez = L::ez(i);
                const bool wall = ywall(1 + ey) || zwall(1 + ez);
                et[cc][i] =
                    wall ? e0 : ey_slot[1 + ey][(Q == 9 ? 0 : 1 + ez) * SEG + kLead + xl + L::ex(i)];
            }
        }
        release();
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const int x = xs + tid + cc * NT;
            if (RAG && xs + (tid & ~31) + cc * NT >= d.nx) continue;   // whole warp past nx
            float o[Q];
            if (EDGE) apply_moving_wall<Q>(d, Y.wall[2], Z, et[cc][0], h[cc]);
            Macro<Q> M;
            collide<Q>(d, h[cc], et[cc][0], et[cc], o, nee ? &M : nullptr);
            if (plo || phi) {
                // eps of the plate node (the cell below / above) and of the row
                // cells its populations stream to (x + ex, z + ez of this row),
                // all among this cell's neighbour porosities
                constexpr int jxp = dir_index<Q>(1, 0, 0), jxm = dir_index<Q>(-1, 0, 0);
                constexpr int jzp = dir_index<Q>(0, 0, 1), jzm = dir_index<Q>(0, 0, -1);
                constexpr int jym = dir_index<Q>(0, -1, 0), jyp = dir_index<Q>(0, 1, 0);
                const float om1 = 1.f - d.omega, zero[3] = {0.f, 0.f, 0.f};
                float lo[Q][1], hi[Q][1];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int ex = L::ex(i), ez = L::ez(i);
                    const float enb = ex > 0 ? et[cc][jxp] : ex < 0 ? et[cc][jxm]
                                    : ez > 0 ? et[cc][jzp] : ez < 0 ? et[cc][jzm] : et[cc][0];
                    if (plo && L::ey(i) > 0)
                        lo[i][0] = plate_value<Q>(d, i, h[cc][i], M, et[cc][jym], enb, zero, om1);
                    if (phi && L::ey(i) < 0)
                        hi[i][0] = plate_value<Q>(d, i, h[cc][i], M, et[cc][jyp], enb, d.uw, om1);
                }
                store_plates<Q, 1>(d, fout, y, z, x, plo, phi, lo, hi);
            }
            if (x < d.nx) {
#pragma unroll
                for (int i = 0; i < Q; ++i) fout[i * d.plane + ro + x] = o[i];
                if (x == 0) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ex(i) < 0) store_halo_hi<Q>(fout + i * d.plane + ro, d.nx, o[i]);
                }
                if (x == d.nx - 1) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (L::ex(i) > 0) store_halo_lo<Q>(fout + i * d.plane + ro, o[i]);
                }
            }
        }
    }
}

template <int Q>
__device__ __forceinline__ Nb3 plane_nbs(const VDom &d, int z) {
    Nb3 Z;
    if (Q == 19) {
        Z = nb3<true>(z, d.nz, d.wall_z);
    } else {
        Z.r[0] = Z.r[1] = Z.r[2] = 0;
        Z.wall[0] = Z.wall[1] = Z.wall[2] = false;
    }
    return Z;
}

// One strip of tiles: column block starting at xs, plane z, rows [y0, y1).
// VEC (D2Q9, CPT = 4): the contiguous 4-cells-per-thread compute above.
// Thread 0 refills a stage after a CTA barrier says every thread is done with it.
template <int Q, int NT, int CPT, bool VEC = false, bool PL = false, bool RAG = false>
__device__ __forceinline__ void ring_strip(const VDom &d, const float *__restrict__ fin,
                                           float *__restrict__ fout, int xs, int z, int y0, int y1,
                                           int stages, unsigned char *smem) {
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NZR = (Q == 9) ? 1 : 3;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    float *ring = buf + stages * Q * SEG;
    const int rslots = stages + 2;
    const int tid = threadIdx.x;
    const int n = y1 - y0;
    if (n <= 0) return;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
        const int pre = n < stages ? n : stages;
        for (int k = 0; k < pre; ++k)
            issue_tile_ring<Q, TW>(d, fin, y0 + k, z, xs, k, y0, buf + k * Q * SEG, ring, rslots,
                                   &bars[k]);
    }
    const Nb3 Z = plane_nbs<Q>(d, z);
    const bool zedge = Z.wall[0] || Z.wall[2];
    int k = 0, s = 0, j0 = 0;
    uint32_t par = 0;
    bool ok = true;
    for (; k < n; ++k) {
        ok = __syncthreads_and(mbar_wait_bounded(&bars[s], par));
        if (!ok) break;
        const float *sb = buf + s * Q * SEG;
        const int j1 = (j0 + 1 == rslots) ? 0 : j0 + 1, j2 = (j1 + 1 == rslots) ? 0 : j1 + 1;
        const float *ey_slot[3] = {ring + j0 * (NZR * SEG),    // y-1: ring slot k mod rslots
                                   ring + j1 * (NZR * SEG),    // y
                                   ring + j2 * (NZR * SEG)};   // y+1
        j0 = j1;
        const int y = y0 + k;
        const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
        // (D3Q19 keeps one body: a second copy of its larger tile code measured slower)
        if (Q == 19 || zedge || Y.wall[0] || Y.wall[2] || (PL && (y <= 1 || y >= d.ny - 2)))
            ring_tile<Q, NT, CPT, VEC, true, PL, RAG>(d, sb, ey_slot, Y, Z, fout, y, z, xs, tid,
                                                      [] {});
        else
            ring_tile<Q, NT, CPT, VEC, false, PL, RAG>(d, sb, ey_slot, Y, Z, fout, y, z, xs, tid,
                                                       [] {});
        __syncthreads();
        if (tid == 0 && k + stages < n) {
            fence_proxy_async_smem();
            issue_tile_ring<Q, TW>(d, fin, y0 + k + stages, z, xs, k + stages, y0, buf + s * Q * SEG,
                                   ring, rslots, &bars[s]);
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

// Warp-specialised form of the strip: NT compute threads plus one producer
// warp.  Stage s has a "full" barrier (the bulk copies' transaction count) and
// an "empty" barrier that each compute warp arrives on as soon as its lanes
// have read the stage into registers (before the collisions and the stores);
// lane 0 of the producer warp refills a stage as soon as its empty phase
// completes.  No CTA-wide barrier sits in the loop, so a compute warp
// that finishes a tile moves on to the next staged one without waiting for the
// others.  Stage reuse is the same as above: tile k+stages (and the eps ring
// slot it loads, last read by tile k) is issued after every warp is done with
// tile k.  stages <= kBarBytes / 16.
template <int Q, int NT, int CPT, bool VEC = false, bool PL = false, bool RAG = false>
__device__ __forceinline__ void ring_strip_ws(const VDom &d, const float *__restrict__ fin,
                                              float *__restrict__ fout, int xs, int z, int y0, int y1,
                                              int stages, unsigned char *smem) {
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NZR = (Q == 9) ? 1 : 3;
    constexpr int NCW = NT / 32;          // compute warps
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    float *ring = buf + stages * Q * SEG;
    const int rslots = stages + 2;
    const int tid = threadIdx.x;
    const int n = y1 - y0;
    if (n <= 0) return;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= NT) {                      // producer warp
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
            issue_tile_ring<Q, TW>(d, fin, y0 + k, z, xs, k, y0, buf + s * Q * SEG, ring, rslots,
                                   &full[s]);
            issued = k + 1;
        }
        if (!ok) {
            // a compute warp gave up: flag it and let the copies in flight land
            // before the CTA's shared memory goes away
            if (d.status) atomicOr(d.status, 2);
            const int first = issued > stages ? issued - stages : 0;
            for (int j = first; j < issued; ++j)
                mbar_wait_bounded(&full[j % stages], (uint32_t)((j / stages) & 1));
        }
        return;
    }
    const int lane = tid & 31;
    const Nb3 Z = plane_nbs<Q>(d, z);
    const bool zedge = Z.wall[0] || Z.wall[2];
    int s = 0, j0 = 0;
    uint32_t par = 0;
    for (int k = 0; k < n; ++k) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], par))) {
            if (lane == 0 && d.status) atomicOr(d.status, 2);
            return;
        }
        const float *sb = buf + s * Q * SEG;
        const int j1 = (j0 + 1 == rslots) ? 0 : j0 + 1, j2 = (j1 + 1 == rslots) ? 0 : j1 + 1;
        const float *ey_slot[3] = {ring + j0 * (NZR * SEG), ring + j1 * (NZR * SEG),
                                   ring + j2 * (NZR * SEG)};
        j0 = j1;
        const int y = y0 + k;
        const Nb3 Y = nb3<true>(y, d.ny, d.wall_y);
        uint64_t *const emp = &empty[s];
        auto release = [&] {
            __syncwarp();       // every lane's reads of the stage precede the arrive
            if (lane == 0) mbar_arrive(emp);
        };
        if (Q == 19 || zedge || Y.wall[0] || Y.wall[2] || (PL && (y <= 1 || y >= d.ny - 2)))
            ring_tile<Q, NT, CPT, VEC, true, PL, RAG>(d, sb, ey_slot, Y, Z, fout, y, z, xs, tid,
                                                      release);
        else
            ring_tile<Q, NT, CPT, VEC, false, PL, RAG>(d, sb, ey_slot, Y, Z, fout, y, z, xs, tid,
                                                       release);
        if (++s == stages) { s = 0; par ^= 1u; }
    }
}

template <int Q, int NT, int CPT, bool VEC = false, bool WS = false, bool PL = false>
__global__ void __launch_bounds__(WS ? NT + 32 : NT) k_step_tma_ring(const VDom d,
                                                                      const float *__restrict__ fin,
                                                                      float *__restrict__ fout,
                                                                      int ntx, int per_y, int stages) {
    extern __shared__ __align__(128) unsigned char smem[];
    // strip of this CTA: column block xt, plane z, rows [y0, y1)
    const int xt = blockIdx.x % ntx;
    const int rem = blockIdx.x / ntx;
    const int z = rem % d.nz;
    const int yc = rem / d.nz;
    const int y0 = (int)((long long)yc * d.ny / per_y);
    const int y1 = (int)((long long)(yc + 1) * d.ny / per_y);
    if constexpr (WS)
        ring_strip_ws<Q, NT, CPT, VEC, PL>(d, fin, fout, xt * NT * CPT, z, y0, y1, stages, smem);
    else
        ring_strip<Q, NT, CPT, VEC, PL>(d, fin, fout, xt * NT * CPT, z, y0, y1, stages, smem);
}

// Interleaved persistent step.  CTA b of G takes tiles b, b + G, b + 2G, ...
// of a tile order (row-major for one domain; domain after domain for a batch),
// so at any moment the whole grid works on one band of neighbouring rows: the
// DRAM sees each population plane as one advancing window instead of one
// stream per CTA, no CTA restarts its pipeline between runs of rows, and the
// porosity rows a tile shares with the tiles of the rows above and below (3
// per tile in D2Q9, 9 in D3Q19, copied with the population rows into the
// stage) come mostly from L2.  Warp-specialised like ring_strip_ws: NT compute
// threads + one producer warp, full/empty barriers per stage, release as soon
// as a warp's lanes have read the stage.  stages <= kBarBytes / 16.
//
// A cursor walks this CTA's tiles: load() fetches the current tile's
// description (for a batch, its table entry and its domain's descriptor, into
// registers), dom(), fin(), fout(), row(), xs() describe it and next() moves G
// tiles on.
struct IlvCursor {             // one domain: (row, column block), no table
    const VDom *d;
    const float *f_in;
    float *f_out;
    int row_, xt, ntx, drow, dxt;
    __device__ IlvCursor(const VDom &dd, const float *fi, float *fo, int b, int G, int ntx_)
        : d(&dd), f_in(fi), f_out(fo), row_(b / ntx_), xt(b - (b / ntx_) * ntx_), ntx(ntx_),
          drow(G / ntx_), dxt(G - (G / ntx_) * ntx_) {}
    __device__ void load(int) {}
    __device__ const VDom &dom() const { return *d; }
    __device__ const float *fin() const { return f_in; }
    __device__ float *fout() const { return f_out; }
    __device__ int row() const { return row_; }
    __device__ int xs(int TW) const { return xt * TW; }
    __device__ void next() {
        row_ += drow;
        xt += dxt;
        if (xt >= ntx) { xt -= ntx; ++row_; }
    }
};

struct IlvBatchCursor {        // a batch: tile table {dom, row, x0}, descriptor per domain
    const VDom *doms;
    const Tile *tiles;
    int t, G, parity;
    Tile T;
    VDom D;                    // register copy of the current tile's descriptor
    __device__ IlvBatchCursor(const VDom *ds, const Tile *ts, int b, int G_, int par)
        : doms(ds), tiles(ts), t(b), G(G_), parity(par) {}
    __device__ void load(int ntiles) {
        if (t < ntiles) {
            T = tiles[t];
            D = doms[T.dom];
        }
    }
    __device__ const VDom &dom() const { return D; }
    __device__ const float *fin() const { return parity ? D.f[1] : D.f[0]; }
    __device__ float *fout() const { return parity ? D.f[0] : D.f[1]; }
    __device__ int row() const { return T.row; }
    __device__ int xs(int) const { return T.x0; }
    __device__ void next() { t += G; }
};

template <int Q, int NT, int CPT, bool VEC, bool PL, bool RAG, class Cur, bool WRAP = false>
__device__ __forceinline__ void ilv_run(Cur cur, const int *status, int ntiles, int stages,
                                        unsigned char *smem) {
    constexpr int TW = NT * CPT;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NS = Q + EpsRows<Q>::N;
    constexpr int NZR = (Q == 9) ? 1 : 3;
    constexpr int NCW = NT / 32;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    float *buf = reinterpret_cast<float *>(smem + kBarBytes);
    const int tid = threadIdx.x;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const int n = (ntiles - b + G - 1) / G;        // tiles of this CTA
    if (n <= 0) return;
    int *const st = const_cast<int *>(status);

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= NT) {                      // producer warp
        if (tid != NT) return;
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < n; ++k) {
            const int s = k % stages;
            cur.load(ntiles);                         // (its latency hides behind the wait)
            if (k >= stages) {
                ok = mbar_wait_bounded(&empty[s], (uint32_t)(((k / stages) - 1) & 1));
                if (!ok) break;
                fence_proxy_async_smem();
            }
            issue_tile<Q, TW, WRAP>(cur.dom(), cur.fin(), cur.row(), cur.xs(TW),
                                    buf + s * (NS * SEG), &full[s]);
            issued = k + 1;
            cur.next();
        }
        if (!ok) {
            if (st) atomicOr(st, 2);
            const int first = issued > stages ? issued - stages : 0;
            for (int j = first; j < issued; ++j)
                mbar_wait_bounded(&full[j % stages], (uint32_t)((j / stages) & 1));
        }
        return;
    }
    const int lane = tid & 31;
    int s = 0;
    uint32_t par = 0;
    for (int k = 0; k < n; ++k) {
        cur.load(ntiles);                             // descriptor loads overlap the wait
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], par))) {
            if (lane == 0 && st) atomicOr(st, 2);
            return;
        }
        const VDom &d = cur.dom();
        int y, z;
        Nb3 Y, Z;
        row_nbs<Q>(d, cur.row(), y, z, Y, Z);
        const float *sb = buf + s * (NS * SEG);
        const float *ey_slot[3] = {sb + Q * SEG, sb + (Q + NZR) * SEG, sb + (Q + 2 * NZR) * SEG};
        uint64_t *const emp = &empty[s];
        auto release = [&] {
            __syncwarp();       // every lane's reads of the stage precede the arrive
            if (lane == 0) mbar_arrive(emp);
        };
        const int xs = cur.xs(TW);
        // (D3Q19 too: here a second copy of the tile code, for the rows away
        // from walls, is faster -- 256^3 duct 0.937 -> 0.969 of the copy
        // bandwidth -- unlike in the strip kernels)
        if (Y.wall[0] || Y.wall[2] || Z.wall[0] || Z.wall[2] ||
            (PL && (y <= 1 || y >= d.ny - 2)))
            ring_tile<Q, NT, CPT, VEC, true, PL, RAG, decltype(release) &, WRAP>(
                d, sb, ey_slot, Y, Z, cur.fout(), y, z, xs, tid, release);
        else
            ring_tile<Q, NT, CPT, VEC, false, PL, RAG, decltype(release) &, WRAP>(
                d, sb, ey_slot, Y, Z, cur.fout(), y, z, xs, tid, release);
        cur.next();
        if (++s == stages) { s = 0; par ^= 1u; }
    }
}

template <int Q, int NT, int CPT, bool VEC, bool PL = false, bool WRAP = false>
__global__ void __launch_bounds__(NT + 32) k_step_tma_ilv(const VDom d, const float *__restrict__ fin,
                                                           float *__restrict__ fout, int ntx,
                                                           int ntiles, int stages) {
    extern __shared__ __align__(128) unsigned char smem[];
    ilv_run<Q, NT, CPT, VEC, PL, false, IlvCursor, WRAP>(
        IlvCursor(d, fin, fout, (int)blockIdx.x, (int)gridDim.x, ntx), d.status, ntiles, stages, smem);
}

// Batched D2Q9, interleaved: the tile table lists every (domain, row, column
// block) of the batch, domain after domain, row-major within a domain.
template <int NT, int CPT, bool VEC>
__global__ void __launch_bounds__(NT + 32) k_step_ilv_batched(const VDom *__restrict__ doms,
                                                               const Tile *__restrict__ tiles,
                                                               int ntiles, int parity, int stages,
                                                               int *status,
                                                               unsigned long long *prof) {
    extern __shared__ __align__(128) unsigned char smem[];
    prof_begin(prof);
    ilv_run<9, NT, CPT, VEC, false, true>(
        IlvBatchCursor(doms, tiles, (int)blockIdx.x, (int)gridDim.x, parity), status, ntiles,
        stages, smem);
    prof_end(prof);
}

// Dynamic shared memory to request for a kernel that needs `need` bytes so
// that at most `ctas` of its CTAs fit on one SM (0: as many as fit).  Fewer
// CTAs mean fewer row segments in flight: past a point, more outstanding
// copies of the 19 (or 9) direction planes lower the DRAM throughput.
static size_t cap_smem(size_t need, int ctas) {
    if (ctas <= 0) return need;
    int dev = 0, per_sm = 0, reserved = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // just too large for ctas + 1 CTAs per SM, small enough for ctas
    size_t share = (size_t)(per_sm / (ctas + 1) - reserved + 128) & ~(size_t)127;
    if (share > (size_t)optin) share = (size_t)optin;
    return need > share ? need : share;
}

template <int Q, int NT, int CPT, bool VEC, bool PL = false>
static cudaError_t launch_ilv_t(const VDom &d, const float *fin, float *fout, int stages, int ctas,
                                cudaStream_t stream) {
    constexpr int TW = NT * CPT;
    constexpr int NS = Q + EpsRows<Q>::N;
    const size_t smem = kBarBytes + (size_t)stages * NS * (TW + 2 * kLead) * sizeof(float);
    if (stages < 2 || stages > kBarBytes / 16 || smem > 227 * 1024) return cudaErrorInvalidValue;
    const size_t smem_req = cap_smem(smem, ctas);
    // D3Q19 rows that are one tile, nx a multiple of 8, x periodic within the
    // domain (not a slab): cells-only staging
    constexpr bool kWrapOk = Q == 19 && VEC && !PL;
    const bool wrap = kWrapOk && d.nx <= TW && (d.nx & 7) == 0 && d.off == 32 && d.xwrap;
    auto kern = wrap ? k_step_tma_ilv<Q, NT, CPT, VEC, PL, kWrapOk>
                     : k_step_tma_ilv<Q, NT, CPT, VEC, PL, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT + 32, smem_req);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int ntx = (d.nx + TW - 1) / TW;
    const long long ntiles = (long long)ntx * d.rows;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * occ;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT + 32, smem_req, stream>>>(d, fin, fout, ntx, (int)ntiles, stages);
    return cudaGetLastError();
}

// Batched D2Q9: CTA b takes strip b of a table built on the host (domain,
// column block, rows y0..y1-1; largest strips first) and advances it with the
// porosity-ring pipeline, using that domain's descriptor and buffers.
template <int NT, int CPT, bool VEC = false, bool WS = false>
__global__ void __launch_bounds__(WS ? NT + 32 : NT) k_step_ring_batched(
    const VDom *__restrict__ doms, const Tile *__restrict__ strips, int parity, int stages,
    unsigned long long *prof) {
    extern __shared__ __align__(128) unsigned char smem[];
    prof_begin(prof);
    const Tile S = strips[blockIdx.x];   // {dom, y0, x0, y1}
    const VDom d = doms[S.dom];
    const float *fin = parity ? d.f[1] : d.f[0];
    float *fout = parity ? d.f[0] : d.f[1];
    if constexpr (WS)
        ring_strip_ws<9, NT, CPT, VEC, false, true>(d, fin, fout, S.x0, 0, S.row, S.pad, stages, smem);
    else
        ring_strip<9, NT, CPT, VEC, false, true>(d, fin, fout, S.x0, 0, S.row, S.pad, stages, smem);
    prof_end(prof);
}

// Strips per (column block, plane): the smallest count whose grid fills the
// resident CTA slots to >= 95 % in its last wave, else the best fill found.
static int pick_per_y(int ncol, int ny, long long resident) {
    int best = 1;
    double best_eff = 0.0;
    for (int p = 1; p <= ny; ++p) {
        const long long grid = (long long)ncol * p;
        const long long waves = (grid + resident - 1) / resident;
        const double eff = (double)grid / (double)(waves * resident);
        if (eff >= 0.95) return p;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = p;
        }
        if (grid > 64 * resident) break;
    }
    return best;
}

template <int Q, int NT, int CPT, bool VEC = false, bool WS = false, bool PL = false>
static cudaError_t launch_ring_t(const VDom &d, const float *fin, float *fout, int stages, int ctas,
                                 cudaStream_t stream) {
    constexpr int TW = NT * CPT;
    constexpr int NZR = (Q == 9) ? 1 : 3;
    const size_t smem =
        kBarBytes + (size_t)(stages * Q + (stages + 2) * NZR) * (TW + 2 * kLead) * sizeof(float);
    const int max_stages = WS ? kBarBytes / 16 : kBarBytes / 8;
    if (stages < 2 || stages > max_stages || smem > 227 * 1024) return cudaErrorInvalidValue;
    const size_t smem_req = cap_smem(smem, ctas);
    auto kern = k_step_tma_ring<Q, NT, CPT, VEC, WS, PL>;
    constexpr int nthreads = WS ? NT + 32 : NT;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nthreads, smem_req);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int ntx = (d.nx + TW - 1) / TW;
    const int ncol = ntx * d.nz;
    const int per_y = pick_per_y(ncol, d.ny, (long long)sms * occ);
    const long long grid = (long long)ncol * per_y;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)grid, nthreads, smem_req, stream>>>(d, fin, fout, ntx, per_y, stages);
    return cudaGetLastError();
}

template <int NT, int CPT, bool VEC = false, bool WS = false>
static cudaError_t launch_ring_batched_t(const VDom *doms, const Tile *strips, int nstrips, int parity,
                                         int stages, int ctas, cudaStream_t stream,
                                         unsigned long long *prof) {
    constexpr int TW = NT * CPT;
    const size_t smem = kBarBytes + (size_t)(stages * 9 + (stages + 2)) * (TW + 2 * kLead) * sizeof(float);
    const int max_stages = WS ? kBarBytes / 16 : kBarBytes / 8;
    if (stages < 2 || stages > max_stages || smem > 227 * 1024 || nstrips < 1)
        return cudaErrorInvalidValue;
    const size_t smem_req = cap_smem(smem, ctas);
    auto kern = k_step_ring_batched<NT, CPT, VEC, WS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
    if (e != cudaSuccess) return e;
    kern<<<nstrips, WS ? NT + 32 : NT, smem_req, stream>>>(doms, strips, parity, stages, prof);
    return cudaGetLastError();
}

template <int NT, int CPT, bool VEC>
static cudaError_t launch_ilv_batched_t(const VDom *doms, const Tile *tiles, int ntiles, int parity,
                                        int stages, int ctas, int *status, cudaStream_t stream,
                                        unsigned long long *prof) {
    constexpr int TW = NT * CPT;
    const size_t smem = kBarBytes + (size_t)stages * 12 * (TW + 2 * kLead) * sizeof(float);
    if (stages < 2 || stages > kBarBytes / 16 || smem > 227 * 1024 || ntiles < 1)
        return cudaErrorInvalidValue;
    const size_t smem_req = cap_smem(smem, ctas);
    auto kern = k_step_ilv_batched<NT, CPT, VEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT + 32, smem_req);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * occ;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, NT + 32, smem_req, stream>>>(doms, tiles, ntiles, parity, stages, status,
                                                         prof);
    return cudaGetLastError();
}

// kind 2: ring strips; 4: the same, warp-specialised; 5: warp-specialised with
// 4 contiguous cells per thread
cudaError_t launch_ring_batched(const VDom *doms, const Tile *strips, int nstrips, int parity,
                                Launch L, int *status, cudaStream_t stream,
                                unsigned long long *prof) {
    const int nt = 32 * L.warps;
    const int st = L.rows;
    if (L.kind == 6) {     // interleaved tile table, strided cells
        if (nt == 128 && L.cpt == 2)
            return launch_ilv_batched_t<128, 2, false>(doms, strips, nstrips, parity, st, L.ctas, status, stream, prof);
        if (nt == 256 && L.cpt == 2)
            return launch_ilv_batched_t<256, 2, false>(doms, strips, nstrips, parity, st, L.ctas, status, stream, prof);
        return cudaErrorInvalidValue;
    }
    if (L.kind == 7) {     // interleaved tile table, 4 consecutive cells
        if (nt == 64 && L.cpt == 4)
            return launch_ilv_batched_t<64, 4, true>(doms, strips, nstrips, parity, st, L.ctas, status, stream, prof);
        if (nt == 128 && L.cpt == 4)
            return launch_ilv_batched_t<128, 4, true>(doms, strips, nstrips, parity, st, L.ctas, status, stream, prof);
        return cudaErrorInvalidValue;
    }
    if (L.kind == 5) {
        if (nt == 64 && L.cpt == 4)
            return launch_ring_batched_t<64, 4, true, true>(doms, strips, nstrips, parity, st, L.ctas, stream, prof);
        if (nt == 128 && L.cpt == 4)
            return launch_ring_batched_t<128, 4, true, true>(doms, strips, nstrips, parity, st, L.ctas, stream, prof);
        return cudaErrorInvalidValue;
    }
    if (L.kind != 2 && L.kind != 4) return cudaErrorInvalidValue;
    const bool ws = L.kind == 4;
#define VANS_RB_CASE(NTT, CC)                                                                   \
    if (nt == NTT && L.cpt == CC)                                                               \
        return ws ? launch_ring_batched_t<NTT, CC, false, true>(doms, strips, nstrips, parity, st, L.ctas, \
                                                               stream, prof)                        \
                  : launch_ring_batched_t<NTT, CC>(doms, strips, nstrips, parity, st, L.ctas, stream, prof);
    VANS_RB_CASE(128, 2)
    VANS_RB_CASE(128, 4)
    VANS_RB_CASE(256, 1)
    VANS_RB_CASE(256, 2)
#undef VANS_RB_CASE
    return cudaErrorInvalidValue;
}

// L.warps -> compute threads per CTA (32 * warps), L.cpt -> cells per thread
// per tile, L.rows -> pipeline stages; kind 2 the porosity ring, 4 and 5 its
// warp-specialised forms (one extra producer warp; 5 with contiguous cells),
// 6 and 7 the interleaved tiles.
// The launch shapes with a plates-on-nodes instance (wall_kind 1).
static bool plate_shape(int q, const Launch &L) {
    const int nt = 32 * L.warps;
    if (q == 9)
        return (L.kind == 2 && nt == 128 && (L.cpt == 2 || L.cpt == 4)) ||
               ((L.kind == 5 || L.kind == 7) && L.cpt == 4 && (nt == 64 || nt == 128));
    return (L.kind == 2 && nt == 128 && L.cpt == 1) ||
           ((L.kind == 5 || L.kind == 7) && nt == 128 && L.cpt == 2);
}

bool launch_has_plates(int q, Launch L) { return L.kind == 0 || L.kind == 8 || plate_shape(q, L); }

static cudaError_t launch_plates(int q, const VDom &d, const float *fin, float *fout, Launch L,
                                 cudaStream_t stream) {
    const int nt = 32 * L.warps;
    const int st = L.rows;
    if (!plate_shape(q, L)) return cudaErrorInvalidValue;
    if (q == 9) {
        if (L.kind == 2)
            return L.cpt == 2 ? launch_ring_t<9, 128, 2, false, false, true>(d, fin, fout, st, L.ctas, stream)
                              : launch_ring_t<9, 128, 4, false, false, true>(d, fin, fout, st, L.ctas, stream);
        if (L.kind == 5)
            return nt == 64 ? launch_ring_t<9, 64, 4, true, true, true>(d, fin, fout, st, L.ctas, stream)
                            : launch_ring_t<9, 128, 4, true, true, true>(d, fin, fout, st, L.ctas, stream);
        return nt == 64 ? launch_ilv_t<9, 64, 4, true, true>(d, fin, fout, st, L.ctas, stream)
                        : launch_ilv_t<9, 128, 4, true, true>(d, fin, fout, st, L.ctas, stream);
    }
    if (L.kind == 2) return launch_ring_t<19, 128, 1, false, false, true>(d, fin, fout, st, L.ctas, stream);
    if (L.kind == 5) return launch_ring_t<19, 128, 2, true, true, true>(d, fin, fout, st, L.ctas, stream);
    return launch_ilv_t<19, 128, 2, true, true>(d, fin, fout, st, L.ctas, stream);
}

cudaError_t launch_step_tma(int q, const VDom &d, const float *fin, float *fout, Launch L,
                            cudaStream_t stream) {
    if (d.nee) return launch_plates(q, d, fin, fout, L, stream);
    const int nt = 32 * L.warps;
    if (L.kind == 6) {                  // interleaved tiles, strided cells per thread
        if (q == 9 && nt == 128 && L.cpt == 2) return launch_ilv_t<9, 128, 2, false>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 9 && nt == 256 && L.cpt == 2) return launch_ilv_t<9, 256, 2, false>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 128 && L.cpt == 1) return launch_ilv_t<19, 128, 1, false>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 256 && L.cpt == 1) return launch_ilv_t<19, 256, 1, false>(d, fin, fout, L.rows, L.ctas, stream);
        return cudaErrorInvalidValue;
    }
    if (L.kind == 7) {                  // interleaved tiles, consecutive cells per thread
        if (q == 9 && nt == 64 && L.cpt == 4) return launch_ilv_t<9, 64, 4, true>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 9 && nt == 128 && L.cpt == 4) return launch_ilv_t<9, 128, 4, true>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 64 && L.cpt == 2) return launch_ilv_t<19, 64, 2, true>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 128 && L.cpt == 2) return launch_ilv_t<19, 128, 2, true>(d, fin, fout, L.rows, L.ctas, stream);
        // 192-, 320- and 384-cell tiles: D3Q19 rows up to that many cells
        // are one tile, staged cells-only (an 8-warp, 512-cell instance, one
        // CTA per SM, measured 0.80 of the copy bandwidth at 512^3 against
        // 0.86 for kind 4, and is not built)
        if (q == 19 && nt == 96 && L.cpt == 2) return launch_ilv_t<19, 96, 2, true>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 160 && L.cpt == 2) return launch_ilv_t<19, 160, 2, true>(d, fin, fout, L.rows, L.ctas, stream);
        if (q == 19 && nt == 192 && L.cpt == 2) return launch_ilv_t<19, 192, 2, true>(d, fin, fout, L.rows, L.ctas, stream);
        return cudaErrorInvalidValue;
    }
    if (L.kind == 5) {                  // warp-specialised ring, consecutive cells per thread
        if (q == 19 && L.cpt == 2) {
            if (nt == 64) return launch_ring_t<19, 64, 2, true, true>(d, fin, fout, L.rows, L.ctas, stream);
            if (nt == 128) return launch_ring_t<19, 128, 2, true, true>(d, fin, fout, L.rows, L.ctas, stream);
        }
        if (q == 9 && L.cpt == 4) {
            if (nt == 64) return launch_ring_t<9, 64, 4, true, true>(d, fin, fout, L.rows, L.ctas, stream);
            if (nt == 128) return launch_ring_t<9, 128, 4, true, true>(d, fin, fout, L.rows, L.ctas, stream);
        }
        return cudaErrorInvalidValue;
    }
    if (L.kind == 2 || L.kind == 4) {
        const bool ws = L.kind == 4;
#define VANS_RING_CASE(QQ, NTT, CC)                                                     \
        if (q == QQ && nt == NTT && L.cpt == CC)                                        \
            return ws ? launch_ring_t<QQ, NTT, CC, false, true>(d, fin, fout, L.rows, L.ctas, stream) \
                      : launch_ring_t<QQ, NTT, CC>(d, fin, fout, L.rows, L.ctas, stream);
        VANS_RING_CASE(9, 128, 2)
        VANS_RING_CASE(9, 128, 4)
        VANS_RING_CASE(9, 256, 1)
        VANS_RING_CASE(9, 256, 2)
        VANS_RING_CASE(19, 128, 1)
        VANS_RING_CASE(19, 128, 2)
        VANS_RING_CASE(19, 256, 1)
#undef VANS_RING_CASE
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace vans
