// Per-stage kernel of a batch of independent grids: every CTA walks the
// batch's tile list (tile = blockIdx.x + k gridDim.x; a persistent grid of
// resident CTAs, or one CTA per tile when the grid covers the list), finds
// the tile's grid and runs the same fused tile body as the single-grid
// kernel, with that grid's own dt, wavespeed slot and error word. Grids
// whose dt is zero (stopped at their end time) are skipped.
#pragma once

#include "stage_kernel.cuh"

namespace gbr {

__device__ __forceinline__ int batch_case_of(const BatchCase* cases, int ncases, int tile)
{
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cases[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Register budgets for the CTAs per SM that shared memory allows: three in
// FP32 (80 registers, the single-grid FP32 kernel's count), two in FP64.
template <typename T, int BX, int BY, int NT, bool LEARNED>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 2) batch_stage_kernel(const BatchCase* __restrict__ cases, int ncases,
                                                         int total_tiles, int stage, const SensorDev* sensor)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const double ca = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
    const double cbc = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const BatchCase& C = cases[batch_case_of(cases, ncases, tile)];
        if (C.ds->dt == 0.0) continue;  // uniform over the CTA
        const int local = tile - C.tile_begin;
        const int ty = local / C.tiles_x, tx = local - ty * C.tiles_x;
        StageParams P;
        P.g = C.g;
        P.ph = C.ph;
        P.q = C.q[stage];
        P.qn = C.q[0];
        P.qout = C.q[(stage + 1) % 3];
        P.res = nullptr;
        P.sigx = nullptr;
        P.sigy = nullptr;
        P.lam_out = stage == 2 ? &C.ds->lam[0] : nullptr;
        P.err = &C.ds->err;
        P.dt_ptr = &C.ds->dt;
        P.dt = 0.0;
        P.ca = ca;
        P.cb = cbc;
        P.cc = cbc;
        P.sensor = sensor;
        P.dec = C.dec;
        P.stall_bytes = 0;
        P.stall_mma = 0;
        stage_tile<T, BX, BY, NT, false, LEARNED>(P, tx * BX, ty * BY, smem_raw);
    }
}

// Persistent grid size: resident CTAs per SM x SMs (computed once per
// device; the first call on a device also raises the kernel's dynamic
// shared-memory limit there, so it must happen outside stream capture).
template <typename T, int BX, int BY, int NT, bool LEARNED>
cudaError_t batch_blocks(int* out)
{
    using L = TileLayout<BX, BY, false>;
    constexpr size_t smem = L::template total_bytes<T, NT, LEARNED>();
    static PerDevice<int> blocks;
    return blocks.get(out, [&](int* v) {
        auto kern = batch_stage_kernel<T, BX, BY, NT, LEARNED>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        *v = (per_sm > 0 ? per_sm : 1) * sms;
        return cudaSuccess;
    });
}

// total_tiles < 0: only prepare the kernel (batch_blocks), launch nothing.
template <typename T, int BX, int BY, int NT, bool LEARNED = false>
cudaError_t launch_batch_t(const BatchCase* cases, int ncases, int total_tiles, int stage, cudaStream_t s,
                           const SensorDev* sensor = nullptr, bool per_tile = false)
{
    using L = TileLayout<BX, BY, false>;
    constexpr size_t smem = L::template total_bytes<T, NT, LEARNED>();
    int blocks = 0;
    cudaError_t e = batch_blocks<T, BX, BY, NT, LEARNED>(&blocks);
    if (e != cudaSuccess || total_tiles <= 0) return e;
    const int grid = (per_tile || total_tiles < blocks) ? total_tiles : blocks;
    batch_stage_kernel<T, BX, BY, NT, LEARNED><<<grid, NT, smem, s>>>(cases, ncases, total_tiles, stage, sensor);
    return cudaGetLastError();
}

}  // namespace gbr
