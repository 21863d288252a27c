// Learned discontinuity sensor: a 50 -> 32 -> 32 -> 1 perceptron (ReLU,
// ReLU, sigmoid) on a 5 x 5 stencil of normalised density and pressure
// differences, evaluated on the tensor cores (BF16 operands, FP32
// accumulation). It stands in for the per-cell test of the density detector
// of arXiv:2305.00762, Sec. 2.4 (Eq. detector); the plain detector remains
// the fallback where the network is unsure and the source of its labels.
//
// Features of cell c (stencil offset k = (dy+2)*5 + (dx+2), dy, dx in
// [-2, 2]): f_k = (rho_k - rho_c) / (max_k' |rho_k' - rho_c| + 1e-3) and
// f_{25+k} likewise for p; f_50..f_63 = 0. The 1e-3 floor makes density and
// pressure variations far below the detector's epsilon scale read as flat.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbr {

constexpr int kSensorIn = 50;
constexpr int kSensorK = 64;      // padded input width
constexpr int kSensorH = 32;      // hidden width
// Row pitches of the transposed weights: padded so that the eight row groups
// of a B-fragment load fall in different shared-memory banks.
constexpr int kW1Pitch = kSensorK + 8;
constexpr int kW2Pitch = kSensorH + 8;
constexpr float kSensorFloor = 1e-3f;
constexpr float kSensorLo = 0.3f;  // p < lo: smooth
constexpr float kSensorHi = 0.7f;  // p > hi: discontinuity; otherwise the plain detector decides
// Soft training target of a cell: 1 / (1 + exp((psi_min - 1/2) / tau)), with
// psi_min = min(psi_x, psi_y) of Eq. detector, stored in units of 1/255. A
// cell whose psi lies within 0.8 tau of the threshold gets a target inside
// the fallback band, so the network learns to leave it to the plain detector.
constexpr double kSensorTau = 0.02;
// Host weight vector: W1[50][32], b1[32], W2[32][32], b2[32], w3[32], b3.
constexpr int kSensorParams = kSensorIn * kSensorH + kSensorH + kSensorH * kSensorH + kSensorH + kSensorH + 1;

// Device copy used by the kernels: W1 and W2 transposed (n-major, k
// contiguous) and rounded to BF16; biases and the output layer in FP32.
struct SensorDev {
    __nv_bfloat16 w1t[kSensorH * kW1Pitch];  // [n][k], k >= 50 zero
    __nv_bfloat16 w2t[kSensorH * kW2Pitch];  // [n][k]
    float b1[kSensorH], b2[kSensorH], w3[kSensorH], b3, pad[3];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
    return *reinterpret_cast<const uint32_t*>(&v);
}

// D = A B + C for one 16x8x16 tile (A row-major 16x16 BF16, B column-major
// 16x8 BF16, C/D 16x8 FP32) on the tensor cores.
__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Copy the sensor weights into shared memory (all threads of the block).
__device__ __forceinline__ void load_sensor(SensorDev* dst, const SensorDev* src)
{
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SensorDev) / 4); i += blockDim.x) d[i] = s[i];
}

// Normalisation denominators of one cell from its 5x5 neighbourhood:
// rho at r[dy*st + dx], p at p[...] (pointers at the cell).
__device__ __forceinline__ void sensor_scales(const float* r, const float* p, int st, float& sr, float& sp)
{
    const float rc = r[0], pc = p[0];
    float mr = 0.f, mp = 0.f;
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
            mr = fmaxf(mr, fabsf(r[dy * st + dx] - rc));
            mp = fmaxf(mp, fabsf(p[dy * st + dx] - pc));
        }
    sr = 1.f / (mr + kSensorFloor);
    sp = 1.f / (mp + kSensorFloor);
}

// Feature k of a cell (0 <= k < 64) given its scales.
__device__ __forceinline__ float sensor_feature(const float* r, const float* p, int st, float sr, float sp, int k)
{
    if (k < 25) {
        const int dy = k / 5 - 2, dx = k % 5 - 2;
        return (r[dy * st + dx] - r[0]) * sr;
    }
    if (k < 50) {
        const int kk = k - 25, dy = kk / 5 - 2, dx = kk % 5 - 2;
        return (p[dy * st + dx] - p[0]) * sp;
    }
    return 0.f;
}

// The network on 16 cells of one warp. Row i (0..15) is the cell whose
// density / pressure pointers are rho_of(i), p_of(i) (a functor returning the
// pointers). Returns, for the two rows this lane holds (lane/4 and lane/4+8),
// the outputs p (valid in every lane of a quad).
template <typename CellPtrs>
__device__ __forceinline__ void sensor_warp16(const SensorDev& W, CellPtrs cells, int st, float& out_lo,
                                              float& out_hi)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *rl, *pl, *rh, *ph;
    cells(g, rl, pl);
    cells(g + 8, rh, ph);
    // Normalisation denominators: the four lanes of a quad hold the same two
    // cells; each takes every fourth neighbour and the quad combines the
    // maxima (a maximum does not depend on the order).
    float mrl = 0.f, mpl = 0.f, mrh = 0.f, mph = 0.f;
    {
        const float rcl = rl[0], pcl = pl[0], rch = rh[0], pch = ph[0];
#pragma unroll
        for (int k = t; k < 25; k += 4) {
            const int o = (k / 5 - 2) * st + (k % 5 - 2);
            mrl = fmaxf(mrl, fabsf(rl[o] - rcl));
            mpl = fmaxf(mpl, fabsf(pl[o] - pcl));
            mrh = fmaxf(mrh, fabsf(rh[o] - rch));
            mph = fmaxf(mph, fabsf(ph[o] - pch));
        }
#pragma unroll
        for (int m = 1; m <= 2; m <<= 1) {
            mrl = fmaxf(mrl, __shfl_xor_sync(0xffffffffu, mrl, m));
            mpl = fmaxf(mpl, __shfl_xor_sync(0xffffffffu, mpl, m));
            mrh = fmaxf(mrh, __shfl_xor_sync(0xffffffffu, mrh, m));
            mph = fmaxf(mph, __shfl_xor_sync(0xffffffffu, mph, m));
        }
    }
    const float srl = 1.f / (mrl + kSensorFloor), spl = 1.f / (mpl + kSensorFloor);
    const float srh = 1.f / (mrh + kSensorFloor), sph = 1.f / (mph + kSensorFloor);
    // layer 1: [16 x 64] x [64 x 32]
    float acc1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = W.b1[8 * nt + 2 * t], b1 = W.b1[8 * nt + 2 * t + 1];
        acc1[nt][0] = b0;
        acc1[nt][1] = b1;
        acc1[nt][2] = b0;
        acc1[nt][3] = b1;
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int k0 = 16 * ks + 2 * t, k1 = k0 + 8;
        uint32_t a[4];
        a[0] = pack_bf16(sensor_feature(rl, pl, st, srl, spl, k0), sensor_feature(rl, pl, st, srl, spl, k0 + 1));
        a[1] = pack_bf16(sensor_feature(rh, ph, st, srh, sph, k0), sensor_feature(rh, ph, st, srh, sph, k0 + 1));
        a[2] = pack_bf16(sensor_feature(rl, pl, st, srl, spl, k1), sensor_feature(rl, pl, st, srl, spl, k1 + 1));
        a[3] = pack_bf16(sensor_feature(rh, ph, st, srh, sph, k1), sensor_feature(rh, ph, st, srh, sph, k1 + 1));
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const __nv_bfloat16* wb = W.w1t + (8 * nt + g) * kW1Pitch;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wb + k0);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wb + k1);
            mma_bf16_16816(acc1[nt], a, b0, b1);
        }
    }
    // ReLU, round to BF16: the accumulator tiles of columns 16ks..16ks+15 are
    // exactly the A fragment of layer 2's k-step ks.
    uint32_t a2[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        a2[ks][0] = pack_bf16(fmaxf(acc1[2 * ks][0], 0.f), fmaxf(acc1[2 * ks][1], 0.f));
        a2[ks][1] = pack_bf16(fmaxf(acc1[2 * ks][2], 0.f), fmaxf(acc1[2 * ks][3], 0.f));
        a2[ks][2] = pack_bf16(fmaxf(acc1[2 * ks + 1][0], 0.f), fmaxf(acc1[2 * ks + 1][1], 0.f));
        a2[ks][3] = pack_bf16(fmaxf(acc1[2 * ks + 1][2], 0.f), fmaxf(acc1[2 * ks + 1][3], 0.f));
    }
    // layer 2: [16 x 32] x [32 x 32], then the 32 -> 1 output layer
    float zl = 0.f, zh = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        float acc[4] = {W.b2[n0], W.b2[n0 + 1], W.b2[n0], W.b2[n0 + 1]};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const __nv_bfloat16* wb = W.w2t + (8 * nt + g) * kW2Pitch;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wb + 16 * ks + 2 * t);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wb + 16 * ks + 8 + 2 * t);
            mma_bf16_16816(acc, a2[ks], b0, b1);
        }
        zl += fmaxf(acc[0], 0.f) * W.w3[n0] + fmaxf(acc[1], 0.f) * W.w3[n0 + 1];
        zh += fmaxf(acc[2], 0.f) * W.w3[n0] + fmaxf(acc[3], 0.f) * W.w3[n0 + 1];
    }
    zl += __shfl_xor_sync(0xffffffffu, zl, 1);
    zl += __shfl_xor_sync(0xffffffffu, zl, 2);
    zh += __shfl_xor_sync(0xffffffffu, zh, 1);
    zh += __shfl_xor_sync(0xffffffffu, zh, 2);
    out_lo = 1.f / (1.f + expf(-(zl + W.b3)));
    out_hi = 1.f / (1.f + expf(-(zh + W.b3)));
}

}  // namespace gbr
