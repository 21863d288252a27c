// Ghost-cell fill and CFL wavespeed reduction (arXiv:2305.00762, Sec. 3
// ghost-cell boundaries; Sec. 2.5 time step).
#include <cuda_runtime.h>

#include "gbr_internal.h"

namespace gbr {

// Source index of ghost coordinate k on an axis of n interior cells, and
// whether the normal / tangential velocity changes sign (GBR_BC_* kinds:
// 0 periodic, 1 transmissive, 2 no-slip wall, 3 symmetry).
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

// One thread per ghost cell of the padded frame. A corner ghost takes the y
// image of the x image of an interior cell, so the velocity sign flips of
// both axes compose.
__global__ void ghost_kernel(const GhostParams P)
{
    const int nx = P.g.nx, ny = P.g.ny, W = nx + 2 * kGhost;
    const long long band = (long long)kGhost * W;
    const long long total = 2 * band + 2LL * kGhost * ny;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id == 0 && P.mode != 0) {
        DevScalars* d = P.ds;
        double dt = P.dt;
        if (P.mode == 2) {
            const double lam = __longlong_as_double((long long)d->lam[P.cur]);
            dt = fmin(P.cfl / lam, P.dt_max);
        }
        d->dt = dt;
        d->t += dt;
        d->lam[P.next] = 0ull;
    }
    if (id >= total) return;
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
    const int js = ghost_src(j, nx, P.bc[0], P.bc[1], fnx, ftx);
    const int is = ghost_src(i, ny, P.bc[2], P.bc[3], fny, fty);
    const bool flip_u = fnx != fty;  // x momentum: normal to x faces, tangential to y faces
    const bool flip_v = ftx != fny;
    const long long d = (long long)gy * P.g.pitch + gx;
    const long long s = (long long)(is + kGhost) * P.g.pitch + (js + kGhost);
    const long long pl = P.g.plane;
    double* q = P.q;
    q[d] = q[s];
    q[d + pl] = flip_u ? -q[s + pl] : q[s + pl];
    q[d + 2 * pl] = flip_v ? -q[s + 2 * pl] : q[s + 2 * pl];
    q[d + 3 * pl] = q[s + 3 * pl];
}

cudaError_t launch_ghosts(const GhostParams& p, cudaStream_t s)
{
    const long long total = 2LL * kGhost * (p.g.nx + 2 * kGhost) + 2LL * kGhost * p.g.ny;
    const int nt = 256;
    const unsigned nb = (unsigned)((total + nt - 1) / nt);
    ghost_kernel<<<nb, nt, 0, s>>>(p);
    return cudaGetLastError();
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// lambda = max over interior cells of max((|u|+c)/dx, (|v|+c)/dy, 4 nu/dx^2,
// 4 nu/dy^2): grid-stride per thread, warp shuffle, block, one atomic max on
// the bit pattern (valid for non-negative doubles).
__global__ void wavespeed_kernel(const Grid g, const Physics ph, const double* __restrict__ q,
                                 unsigned long long* lam)
{
    const long long n = (long long)g.nx * g.ny;
    const double idx_ = 1.0 / ph.dx, idy = 1.0 / ph.dy;
    double m = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / g.nx), j = (int)(e - (long long)i * g.nx);
        const long long o = (long long)(i + kGhost) * g.pitch + (j + kGhost);
        const double r = q[o], ir = 1.0 / r;
        const double u = q[o + g.plane] * ir, v = q[o + 2 * g.plane] * ir;
        const double p = (ph.gamma - 1.0) * (q[o + 3 * g.plane] - 0.5 * r * (u * u + v * v));
        const double c = sqrt(ph.gamma * p * ir);
        double l = fmax((fabs(u) + c) * idx_, (fabs(v) + c) * idy);
        if (ph.mu > 0.0) {
            const double nu4 = 4.0 * ph.mu * ir;
            l = fmax(l, fmax(nu4 * idx_ * idx_, nu4 * idy * idy));
        }
        m = fmax(m, l);
    }
    __shared__ double red[32];
    m = warp_max_d(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        v = warp_max_d(v);
        if (threadIdx.x == 0) atomicMax(lam, (unsigned long long)__double_as_longlong(v));
    }
}

cudaError_t launch_wavespeed(const Grid& g, const Physics& ph, const double* q, unsigned long long* lam,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(lam, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)g.nx * g.ny;
    int nb = (int)((n + 255) / 256);
    if (nb > 152 * 8) nb = 152 * 8;
    wavespeed_kernel<<<nb, 256, 0, s>>>(g, ph, q, lam);
    return cudaGetLastError();
}

}  // namespace gbr
