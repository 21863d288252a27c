// Learned discontinuity sensor: a 50 -> 32 -> 32 -> 1 perceptron (ReLU,
// ReLU, sigmoid) on a 5 x 5 stencil of normalised density and pressure
// differences, evaluated on the tcgen05 tensor cores (BF16 operands, FP32
// accumulation in tensor memory; sensor.cu). It stands in for the per-cell test of the density detector
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
// Row pitches of the transposed weights in the device copy (the kernels
// re-order them into the tensor cores' core-matrix layout in shared memory).
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

}  // namespace gbr
