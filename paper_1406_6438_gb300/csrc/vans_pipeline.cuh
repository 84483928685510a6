// vans_pipeline.cuh -- staging helpers shared by the bulk-copy pipelined
// kernels (the forward step and the reverse step): the slots of the porosity
// rows in a stage, the row neighbours of a tile, and the copies of one row tile
// into a shared-memory stage.
#pragma once

#include "vans_device.cuh"
#include "vans_tma.cuh"

namespace vans {

template <int Q> struct EpsRows;
template <> struct EpsRows<9> { static constexpr int N = 3; };    // dy = -1, 0, 1
template <> struct EpsRows<19> { static constexpr int N = 9; };   // (dy, dz) in {-1,0,1}^2

// Stage slot of the porosity row (y + dy, z + dz): D2Q9 dy + 1; D3Q19 the
// three z-rows of one dy side by side, (dy + 1) * 3 + dz + 1 (the layout of
// the ring slots, so the same tile compute reads both)
template <int Q>
__host__ __device__ constexpr int eps_slot(int dy, int dz) {
    return Q == 9 ? dy + 1 : (dy + 1) * 3 + (dz + 1);
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

// A staged row segment of the tile at column xs holds columns xs - kLead ..
// xs + TW + kLead - 1: the +-1 neighbours of the tile's cells (halo columns
// included), from and to whole 32-byte sectors (column 0 starts a sector, so
// column xs - kLead starts one too); a stage slot is TW + 2 kLead floats.
constexpr int kLead = 8;

// bytes of the copy of one staged row segment with nval cells
__host__ __device__ constexpr uint32_t seg_bytes(int nval) {
    return (uint32_t)(((nval + kLead - 1) / kLead * kLead + 2 * kLead) * 4);
}

// Issue the bulk copies of the tile (row, xs) into stage buffer sb (one
// thread): the Q population rows the pull reads and the porosity rows.  The
// barrier's transaction count also covers `extra` further copies of the same
// size, which the caller issues; the size of each copy is returned.
// WRAP (rows that are one tile, nx a multiple of 8, column 0 on a 128-byte
// line): only the cells are copied, whole lines and no halo columns, which the
// compute then takes from the other end of the staged row (the periodic x wrap:
// every write of a halo entry also writes its mirror there); a segment with
// halos touches one more 128-byte line per row, 12 % more reads on 256-cell
// rows.
template <int Q, int TW, bool WRAP = false>
__device__ __forceinline__ uint32_t issue_tile(const VDom &d, const float *__restrict__ fin, int row,
                                               int xs, float *sb, uint64_t *bar, int extra = 0) {
    using L = Lat<Q>;
    constexpr int SEG = TW + 2 * kLead;
    constexpr int NS = Q + EpsRows<Q>::N;
    int y, z;
    Nb3 Y, Z;
    row_nbs<Q>(d, row, y, z, Y, Z);
    const int nval = min(TW, d.nx - xs);
    const uint32_t bytes = WRAP ? (uint32_t)(nval * 4) : seg_bytes(nval);
    const int c0 = WRAP ? xs : xs - kLead;        // first column copied
    const int s0 = WRAP ? kLead : 0;              // its place in the stage row
    mbar_arrive_expect_tx(bar, bytes * (NS + extra));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ey = L::ey(i), ez = L::ez(i);
        const bool bb = Y.wall[1 - ey] || Z.wall[1 - ez];
        const int si = bb ? L::opp(i) : i;
        const long long ro = bb ? row_offset(d, y, z) : row_offset(d, Y.r[1 - ey], Z.r[1 - ez]);
        bulk_g2s(sb + i * SEG + s0, fin + si * d.plane + ro + c0, bytes, bar);
    }
    // the porosity rows are read again by the tiles of the neighbouring rows:
    // keep them in L2 longest
    const uint64_t again = l2_evict_last();
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if (Q == 9 && dz != 0) continue;
            const float *src = d.eps + row_offset(d, Y.r[1 + dy], Z.r[1 + dz]) + c0;
            bulk_g2s_hint(sb + (Q + eps_slot<Q>(dy, dz)) * SEG + s0, src, bytes, bar, again);
        }
    return bytes;
}

}  // namespace vans
