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

// Four 8x8 BF16 matrices from shared memory, one row address per lane (lanes
// 8j..8j+7 give the rows of matrix j); lane l receives row l/4, columns
// 2(l%4), 2(l%4)+1 of each: the B fragments of mma m16n8k16 when the rows are
// the n index and the columns 8 consecutive k of a [n][k] weight array.
__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* row)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(row));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// Copy the sensor weights into shared memory (all threads of the block).
__device__ __forceinline__ void load_sensor(SensorDev* dst, const SensorDev* src)
{
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SensorDev) / 4); i += blockDim.x) d[i] = s[i];
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
// density / pressure pointers are rho_of(i), p_of(i) and whose normalisation
// scales 1/(max|q_k - q_c| + floor) are sr, sp (a functor returning the
// pointers and the scales). Returns, for the two rows this lane holds (lane/4
// and lane/4+8), the outputs p (valid in every lane of a quad).
template <typename CellPtrs>
__device__ __forceinline__ void sensor_warp16(const SensorDev& W, CellPtrs cells, int st, float& out_lo,
                                              float& out_hi)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *rl, *pl, *rh, *ph;
    float srl, spl, srh, sph;
    cells(g, rl, pl, srl, spl);
    cells(g + 8, rh, ph, srh, sph);
    // B fragments: lane l addresses row (l & 7) of matrix l >> 3; matrices 0, 1
    // are k-halves of n-tile 2np, matrices 2, 3 those of n-tile 2np + 1.
    const int bn = 8 * (lane >> 4) + (lane & 7), bk = 8 * ((lane >> 3) & 1);
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
        for (int np = 0; np < 2; ++np) {
            uint32_t b[4];
            ldmatrix_x4(b[0], b[1], b[2], b[3], W.w1t + (16 * np + bn) * kW1Pitch + 16 * ks + bk);
            mma_bf16_16816(acc1[2 * np], a, b[0], b[1]);
            mma_bf16_16816(acc1[2 * np + 1], a, b[2], b[3]);
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
    for (int np = 0; np < 2; ++np) {
        float acc[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n0 = 8 * (2 * np + h) + 2 * t;
            acc[h][0] = W.b2[n0];
            acc[h][1] = W.b2[n0 + 1];
            acc[h][2] = W.b2[n0];
            acc[h][3] = W.b2[n0 + 1];
        }
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t b[4];
            ldmatrix_x4(b[0], b[1], b[2], b[3], W.w2t + (16 * np + bn) * kW2Pitch + 16 * ks + bk);
            mma_bf16_16816(acc[0], a2[ks], b[0], b[1]);
            mma_bf16_16816(acc[1], a2[ks], b[2], b[3]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // n-tiles in order 0..3, as the output layer's sum
            const int n0 = 8 * (2 * np + h) + 2 * t;
            zl += fmaxf(acc[h][0], 0.f) * W.w3[n0] + fmaxf(acc[h][1], 0.f) * W.w3[n0 + 1];
            zh += fmaxf(acc[h][2], 0.f) * W.w3[n0] + fmaxf(acc[h][3], 0.f) * W.w3[n0 + 1];
        }
    }
    zl += __shfl_xor_sync(0xffffffffu, zl, 1);
    zl += __shfl_xor_sync(0xffffffffu, zl, 2);
    zh += __shfl_xor_sync(0xffffffffu, zh, 1);
    zh += __shfl_xor_sync(0xffffffffu, zh, 2);
    out_lo = 1.f / (1.f + expf(-(zl + W.b3)));
    out_hi = 1.f / (1.f + expf(-(zh + W.b3)));
}

}  // namespace gbr
