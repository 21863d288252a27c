// Ghost-cell boundary conditions (arXiv:2305.00762, Sec. 3: ghost-cell
// approach) for one padded state; shared by the single-grid and the batched
// ghost kernels.
#pragma once

#include <cuda_runtime.h>

#include "gbr_internal.h"

namespace gbr {

// Source index of ghost coordinate k on an axis of n interior cells, and
// whether the normal / tangential velocity changes sign (kinds: 0 periodic,
// 1 transmissive, 2 no-slip wall, 3 symmetry; custom sides are resolved to
// one of 1-3 before).
__device__ __forceinline__ int ghost_src(int k, int n, int lo, int hi, bool& flip_n, bool& flip_t)
{
    flip_n = false;
    flip_t = false;
    if (k >= 0 && k < n) return k;
    const int bc = k < 0 ? lo : hi;
    if (bc == 0) return ((k % n) + n) % n;
    if (bc == 1) return k < 0 ? 0 : n - 1;
    flip_n = true;
    flip_t = (bc == 2);
    return k < 0 ? -1 - k : 2 * n - 1 - k;
}

// Number of ghost cells of a grid: 6 full rows below and above, 6 cells left
// and right of every interior row.
__host__ __device__ __forceinline__ long long ghost_count(const Grid& g)
{
    return 2LL * kGhost * (g.nx + 2 * kGhost) + 2LL * kGhost * g.ny;
}

constexpr int kBcCustom = 4, kBcFixed = 5, kBcHalo = 6;

// Kind of a custom side beside the cell with tangential index k (centre at
// (k + 1/2) h along the side) at time t; for kBcFixed also its state.
__device__ __forceinline__ int side_kind(const SideBC& S, int k, double h, double t, const double*& state)
{
    const bool lo = (k + 0.5) * h < S.s0 + S.speed * t;
    state = lo ? S.qlo : S.qhi;
    return lo ? S.kind_lo : S.kind_hi;
}

// Fill ghost cell number id (0 <= id < ghost_count) of the padded state q. A
// corner ghost takes the y image of the x image of an interior cell, so the
// velocity sign flips of both axes compose. The ghost rows of a halo side
// (south / north of one slab of a grid split along y) hold the neighbouring
// slab's interior rows, written before the fill: their interior columns are
// left alone and their west / east ghosts follow the x rule of their own row,
// as for an interior row. With custom sides (sides != null,
// boundary time t), a south / north ghost whose side is fixed there takes the
// fixed state; otherwise the source row is found first and a west / east
// side is resolved at that row (a fixed state is then mirrored across the
// south / north side like any x image).
__device__ __forceinline__ void fill_ghost(const Grid& g, double* q, const int bc[4], long long id,
                                           const SideBC* sides = nullptr, double dx = 0.0, double dy = 0.0,
                                           double t = 0.0)
{
    const int nx = g.nx, ny = g.ny, W = nx + 2 * kGhost;
    const long long band = (long long)kGhost * W;
    int gx, gy;
    if (id < band) {
        gy = (int)(id / W);
        gx = (int)(id - (long long)gy * W);
    } else if (id < 2 * band) {
        const long long k = id - band;
        gy = ny + kGhost + (int)(k / W);
        gx = (int)(k - (long long)(k / W) * W);
    } else {
        const long long k = id - 2 * band;
        gy = kGhost + (int)(k / (2 * kGhost));
        const int c = (int)(k - (long long)(k / (2 * kGhost)) * (2 * kGhost));
        gx = c < kGhost ? c : nx + c;
    }
    const int j = gx - kGhost, i = gy - kGhost;
    const bool halo_row = (i < 0 && bc[2] == kBcHalo) || (i >= ny && bc[3] == kBcHalo);
    if (halo_row && j >= 0 && j < nx) return;
    const long long d = (long long)gy * g.pitch + gx;
    const long long pl = g.plane;
    int ky[2] = {bc[2], bc[3]}, kx[2] = {bc[0], bc[1]};
    if (sides && (i < 0 || i >= ny) && bc[i < 0 ? 2 : 3] == kBcCustom) {
        const double* st;
        const int k = side_kind(sides[i < 0 ? 2 : 3], j, dx, t, st);
        if (k == kBcFixed) {
            for (int m = 0; m < 4; ++m) q[d + m * pl] = st[m];
            return;
        }
        ky[i < 0 ? 0 : 1] = k;
    }
    bool fnx, ftx, fny = false, fty = false;
    const int is = halo_row ? i : ghost_src(i, ny, ky[0], ky[1], fny, fty);
    if (sides && (j < 0 || j >= nx) && bc[j < 0 ? 0 : 1] == kBcCustom) {
        const double* st;
        const int k = side_kind(sides[j < 0 ? 0 : 1], is, dy, t, st);
        if (k == kBcFixed) {
            q[d] = st[0];
            q[d + pl] = fty ? -st[1] : st[1];
            q[d + 2 * pl] = fny ? -st[2] : st[2];
            q[d + 3 * pl] = st[3];
            return;
        }
        kx[j < 0 ? 0 : 1] = k;
    }
    const int js = ghost_src(j, nx, kx[0], kx[1], fnx, ftx);
    const bool flip_u = fnx != fty;  // x momentum: normal to x faces, tangential to y faces
    const bool flip_v = ftx != fny;
    const long long s = (long long)(is + kGhost) * g.pitch + (js + kGhost);
    q[d] = q[s];
    q[d + pl] = flip_u ? -q[s + pl] : q[s + pl];
    q[d + 2 * pl] = flip_v ? -q[s + 2 * pl] : q[s + 2 * pl];
    q[d + 3 * pl] = q[s + 3 * pl];
}

}  // namespace gbr
