// Ghost-cell boundary conditions (arXiv:2305.00762, Sec. 3: ghost-cell
// approach) for one padded state; shared by the single-grid and the batched
// ghost kernels.
#pragma once

#include <cuda_runtime.h>

#include "gbr_internal.h"

namespace gbr {

// Source index of ghost coordinate k on an axis of n interior cells, and
// whether the normal / tangential velocity changes sign (kinds: 0 periodic,
// 1 transmissive, 2 no-slip wall, 3 symmetry).
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

// Fill ghost cell number id (0 <= id < ghost_count) of the padded state q. A
// corner ghost takes the y image of the x image of an interior cell, so the
// velocity sign flips of both axes compose.
__device__ __forceinline__ void fill_ghost(const Grid& g, double* q, const int bc[4], long long id)
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
    bool fnx, ftx, fny, fty;
    const int js = ghost_src(j, nx, bc[0], bc[1], fnx, ftx);
    const int is = ghost_src(i, ny, bc[2], bc[3], fny, fty);
    const bool flip_u = fnx != fty;  // x momentum: normal to x faces, tangential to y faces
    const bool flip_v = ftx != fny;
    const long long d = (long long)gy * g.pitch + gx;
    const long long s = (long long)(is + kGhost) * g.pitch + (js + kGhost);
    const long long pl = g.plane;
    q[d] = q[s];
    q[d + pl] = flip_u ? -q[s + pl] : q[s + pl];
    q[d + 2 * pl] = flip_v ? -q[s + 2 * pl] : q[s + 2 * pl];
    q[d + 3 * pl] = q[s + 3 * pl];
}

}  // namespace gbr
