// Ghost-cell fill and CFL wavespeed reduction (arXiv:2305.00762, Sec. 3
// ghost-cell boundaries; Sec. 2.5 time step).
#include <cuda_runtime.h>

#include "ghost.cuh"
#include "gbr_internal.h"
#include "stage_kernel.cuh"

namespace gbr {

// One thread per ghost cell of the padded frame; its first thread also does
// the per-step scalar bookkeeping of GhostParams::mode.
__global__ void ghost_kernel(const GhostParams P)
{
    const long long total = ghost_count(P.g);
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
        d->ts[P.next] = d->ts[P.cur] + dt;
        d->lam[P.next] = 0ull;
    }
    if (id >= total) return;
    // Boundary time of this stage: the step's start time ts[cur] (not written
    // by this launch) plus c_stage dt (dt was written by an earlier launch
    // whenever c_stage != 0).
    const double t = P.ds->ts[P.cur] + (P.c_stage != 0.0 ? P.c_stage * P.ds->dt : 0.0);
    fill_ghost(P.g, P.q, P.bc, id, P.side, P.dx, P.dy, t);
}

// Simulated time of the current state: the reported time and the step start
// time (slot cur) that time-dependent boundaries read.
__global__ void set_time_kernel(DevScalars* d, int cur, double t)
{
    d->t = t;
    d->ts[cur] = t;
}

cudaError_t launch_set_time(DevScalars* d, int cur, double t, cudaStream_t s)
{
    set_time_kernel<<<1, 1, 0, s>>>(d, cur, t);
    return cudaGetLastError();
}

cudaError_t launch_ghosts(const GhostParams& p, cudaStream_t s)
{
    const long long total = ghost_count(p.g);
    const int nt = 256;
    const unsigned nb = (unsigned)((total + nt - 1) / nt);
    ghost_kernel<<<nb, nt, 0, s>>>(p);
    return cudaGetLastError();
}

// Ghost cells of buffer `buf` of every grid of a batch (one thread per ghost
// cell of the whole batch); with mode 2 the first ncases threads also form
// each grid's dt, advance its time and clear its wavespeed slot; with mode 3
// they take each grid's dt from dts[] instead (a grid at dt = 0 keeps its
// time and its wavespeed, and its stages are skipped).
__global__ void batch_ghost_kernel(const BatchCase* __restrict__ cases, int ncases, long long total, int buf,
                                   int mode, double cfl, const double* __restrict__ dts)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode == 2 && id < ncases) {
        DevScalars* d = cases[id].ds;
        const double lam = __longlong_as_double((long long)d->lam[0]);
        const double rem = cases[id].t_end - d->t;
        const double dt = rem > 0.0 ? fmin(cfl / lam, rem) : 0.0;
        d->dt = dt;
        d->t += dt;
        d->lam[0] = 0ull;
    }
    if (mode == 3 && id < ncases) {
        DevScalars* d = cases[id].ds;
        const double dt = dts[id];
        d->dt = dt;
        if (dt > 0.0) {
            d->t += dt;
            d->lam[0] = 0ull;
        }
    }
    if (id >= total) return;
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cases[mid].ghost_begin <= id) lo = mid;
        else hi = mid - 1;
    }
    const BatchCase& C = cases[lo];
    fill_ghost(C.g, C.q[buf], C.bc, id - C.ghost_begin);
}

cudaError_t launch_batch_ghosts(const BatchCase* cases, int ncases, long long total_ghosts, int buf, int mode,
                                double cfl, cudaStream_t s, const double* dts)
{
    long long n = total_ghosts > ncases ? total_ghosts : ncases;
    const int nt = 256;
    batch_ghost_kernel<<<(unsigned)((n + nt - 1) / nt), nt, 0, s>>>(cases, ncases, total_ghosts, buf, mode, cfl,
                                                                     dts);
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
// Standalone CFL wavespeed of a padded state in the precision T of the
// stage arithmetic (the same per-cell function as the stage epilogue).
template <typename T>
__global__ void wavespeed_kernel(const Grid g, const Physics ph, const double* __restrict__ q,
                                 unsigned long long* lam)
{
    const long long n = (long long)g.nx * g.ny;
    const T gamma = T(ph.gamma), gm1 = T(ph.gm1), mu = T(ph.mu);
    const T idx_ = T(ph.inv_dx), idy = T(ph.inv_dy);
    double m = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / g.nx), j = (int)(e - (long long)i * g.nx);
        const long long o = (long long)(i + kGhost) * g.pitch + (j + kGhost);
        m = fmax(m, cell_wavespeed<T>(q[o], q[o + g.plane], q[o + 2 * g.plane], q[o + 3 * g.plane], gamma, gm1, mu,
                                      idx_, idy));
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
                             int precision, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(lam, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)g.nx * g.ny;
    int nb = (int)((n + 255) / 256);
    if (nb > 152 * 8) nb = 152 * 8;
    if (precision == 32)
        wavespeed_kernel<float><<<nb, 256, 0, s>>>(g, ph, q, lam);
    else
        wavespeed_kernel<double><<<nb, 256, 0, s>>>(g, ph, q, lam);
    return cudaGetLastError();
}

}  // namespace gbr
