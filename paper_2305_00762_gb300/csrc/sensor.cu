// Learned discontinuity sensor: per-cell evaluation and dataset extraction on
// a padded state, and the hand-written training kernels (BF16 operands, FP32
// accumulation, binary cross-entropy, Adam).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "gbr_internal.h"
#include "sensor.cuh"
#include "stage_kernel.cuh"

namespace gbr {

// ---------------------------------------------------------------------------
// Weight packing (host): W1[50][32], b1[32], W2[32][32], b2[32], w3[32], b3.
// ---------------------------------------------------------------------------
void pack_sensor(const float* w, SensorDev* out)
{
    memset(out, 0, sizeof(*out));
    const float* W1 = w;
    const float* b1 = W1 + kSensorIn * kSensorH;
    const float* W2 = b1 + kSensorH;
    const float* b2 = W2 + kSensorH * kSensorH;
    const float* w3 = b2 + kSensorH;
    const float b3 = w3[kSensorH];
    for (int n = 0; n < kSensorH; ++n) {
        for (int k = 0; k < kSensorK; ++k)
            out->w1t[n * kW1Pitch + k] = __float2bfloat16_rn(k < kSensorIn ? W1[k * kSensorH + n] : 0.f);
        for (int k = 0; k < kSensorH; ++k) out->w2t[n * kW2Pitch + k] = __float2bfloat16_rn(W2[k * kSensorH + n]);
        out->b1[n] = b1[n];
        out->b2[n] = b2[n];
        out->w3[n] = w3[n];
    }
    out->b3 = b3;
}

// ---------------------------------------------------------------------------
// Per-cell sensor output, decisions, features and plain labels of a padded
// state. A tile covers kTX x kTY cells of one of two index spaces: the
// interior cells (origin = padded cell kGhost, extent nx x ny), or the
// decision region (origin = padded cell 3, extent (nx + 6) x (ny + 6): every
// cell whose detector flag a stage tile reads).
// ---------------------------------------------------------------------------
constexpr int kTX = 32, kTY = 24, kH = 2, kRW = kTX + 2 * kH, kRH = kTY + 2 * kH;
constexpr int kDecOrigin = 3;

struct SensorTileParams {
    Grid g;
    double gamma;
    const double* q;        // padded state, ghosts filled
    const SensorDev* w;     // weights (eval, decisions) or nullptr
    float* prob;            // [ny][nx] network output, or nullptr
    __nv_bfloat16* feat;    // [ny*nx][64] features, or nullptr
    unsigned char* label;   // [ny*nx] plain-detector label, or nullptr
    unsigned char* target;  // [ny*nx] soft target in units of 1/255, or nullptr
    unsigned char* dec;     // decision-region mode: decisions (padded layout), else nullptr
    int stall;              // failure-detection test: withhold the first MMA batch (its wait gives up)
};

// The staged region of one tile and the per-cell normalisation scales.
struct SensorRegion {
    float sr[kRH * kRW], sp[kRH * kRW];  // staged rho, p (tile + 2-cell halo)
    float hr[2 * kRH * kTX], hp[2 * kRH * kTX];  // max, then min, over 5 columns
    float scr[kTY * kTX], scp[kTY * kTX];  // per-cell normalisation scales
};

// Stage the tile's region as FP32 rho, p exactly as the FP32 stage kernel
// stages its primitives (clamped to the padded extent; clamped cells feed no
// output), and, if `scales`, each cell's normalisation scales. Every thread of
// the block takes part (block-wide barriers inside).
__device__ void sensor_scales(SensorRegion& S);

__device__ void sensor_stage(const SensorTileParams& P, const int tx0, const int ty0, const int org, bool scales,
                             SensorRegion& S)
{
    const int nx = P.g.nx, ny = P.g.ny;
    const float gm1 = (float)(P.gamma - 1.0);
    for (int idx = threadIdx.x; idx < kRH * kRW; idx += blockDim.x) {
        const int ry = idx / kRW, rx = idx - ry * kRW;
        const int gx = min(tx0 + rx + org - kH, nx + 2 * kGhost - 1);
        const int gy = min(ty0 + ry + org - kH, ny + 2 * kGhost - 1);
        const long long o = (long long)gy * P.g.pitch + gx;
        float r, u, v, pr;
        prims_of(P.q[o], P.q[o + P.g.plane], P.q[o + 2 * P.g.plane], P.q[o + 3 * P.g.plane], gm1, r, u, v, pr);
        S.sr[idx] = r;
        S.sp[idx] = pr;
    }
    __syncthreads();
    if (scales) sensor_scales(S);
}

__device__ void sensor_scales(SensorRegion& S)
{
    // Normalisation scales 1/(max_k |q_k - q_c| + floor) over each cell's
    // 5 x 5 window, from separable window maxima and minima: rounding is
    // monotone, so max_k RN(q_k - q_c) = RN(max_k q_k - q_c) (likewise for the
    // minimum) and the scales are those of the direct 25-term maximum, bit
    // for bit.
    for (int idx = threadIdx.x; idx < kRH * kTX; idx += blockDim.x) {
        const int ry = idx / kTX, cx = idx - ry * kTX;
        const float* r = S.sr + ry * kRW + cx;
        const float* p = S.sp + ry * kRW + cx;
        float rmx = r[0], rmn = r[0], pmx = p[0], pmn = p[0];
#pragma unroll
        for (int d = 1; d < 5; ++d) {
            rmx = fmaxf(rmx, r[d]);
            rmn = fminf(rmn, r[d]);
            pmx = fmaxf(pmx, p[d]);
            pmn = fminf(pmn, p[d]);
        }
        S.hr[idx] = rmx;
        S.hr[kRH * kTX + idx] = rmn;
        S.hp[idx] = pmx;
        S.hp[kRH * kTX + idx] = pmn;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kTY * kTX; c += blockDim.x) {
        const int cy = c / kTX, cx = c - cy * kTX;
        float rmx = S.hr[c], rmn = S.hr[kRH * kTX + c], pmx = S.hp[c], pmn = S.hp[kRH * kTX + c];
#pragma unroll
        for (int d = 1; d < 5; ++d) {
            const int o = c + d * kTX;
            rmx = fmaxf(rmx, S.hr[o]);
            rmn = fminf(rmn, S.hr[kRH * kTX + o]);
            pmx = fmaxf(pmx, S.hp[o]);
            pmn = fminf(pmn, S.hp[kRH * kTX + o]);
        }
        const float rc = S.sr[(cy + kH) * kRW + cx + kH], pc = S.sp[(cy + kH) * kRW + cx + kH];
        const float mr = fmaxf(0.f, fmaxf(rmx - rc, rc - rmn)), mp = fmaxf(0.f, fmaxf(pmx - pc, pc - pmn));
        S.scr[c] = 1.f / (mr + kSensorFloor);
        S.scp[c] = 1.f / (mp + kSensorFloor);
    }
    __syncthreads();
}

// Dataset extraction on one tile: BF16 features of each interior cell (for
// training), the plain detector's label and its soft target (FP64, Eq.
// detector).
__device__ void sensor_dataset_tile(const SensorTileParams& P, const int tx0, const int ty0, SensorRegion& S)
{
    const int nx = P.g.nx, ny = P.g.ny;
    sensor_stage(P, tx0, ty0, kGhost, P.feat != nullptr, S);
    if (P.feat) {  // one cell per thread, 64 features each
        for (int c = threadIdx.x; c < kTX * kTY; c += blockDim.x) {
            const int cy = c / kTX, cx = c - cy * kTX, i = ty0 + cy, j = tx0 + cx;
            if (i >= ny || j >= nx) continue;
            const float* r = S.sr + (cy + kH) * kRW + (cx + kH);
            const float* p = S.sp + (cy + kH) * kRW + (cx + kH);
            const float s1 = S.scr[c], s2 = S.scp[c];
            uint32_t* out = reinterpret_cast<uint32_t*>(P.feat + ((long long)i * nx + j) * kSensorK);
            for (int k = 0; k < kSensorK; k += 2)
                out[k / 2] = pack_bf16(sensor_feature(r, p, kRW, s1, s2, k), sensor_feature(r, p, kRW, s1, s2, k + 1));
        }
    }
    if (P.label || P.target) {  // plain detector in FP64 on the density (Eq. detector)
        for (int c = threadIdx.x; c < kTX * kTY; c += blockDim.x) {
            const int cy = c / kTX, cx = c - cy * kTX, i = ty0 + cy, j = tx0 + cx;
            if (i >= ny || j >= nx) continue;
            const double* r = P.q + (long long)(i + kGhost) * P.g.pitch + (j + kGhost);
            if (P.label) {
                const bool tr = trouble_cell<double>(r, 1) || trouble_cell<double>(r, P.g.pitch);
                P.label[(long long)i * nx + j] = tr ? 1 : 0;
            }
            if (P.target) {
                const double psi = fmin(detector_psi(r, 1), detector_psi(r, P.g.pitch));
                const double tt = 1.0 / (1.0 + exp((psi - 0.5) / kSensorTau));
                P.target[(long long)i * nx + j] = (unsigned char)floor(255.0 * tt + 0.5);
            }
        }
    }
}

__global__ void __launch_bounds__(256) sensor_dataset_kernel(const SensorTileParams P)
{
    __shared__ SensorRegion S;
    sensor_dataset_tile(P, blockIdx.x * kTX, blockIdx.y * kTY, S);
}

// ---------------------------------------------------------------------------
// The network on the fifth-generation tensor cores (tcgen05): one CTA of G
// warpgroups (128 G threads) per 32 x 24 tile, one thread per cell, 6/G
// rounds; warpgroup g's 128 cells of a round are the M = 128 rows of its own
// MMAs, on its own 64 tensor-memory columns.
// A thread writes its cell's 64 features (50 + zero padding, BF16 pairs) into
// its own tensor-memory lane; one thread issues the layer-1 MMAs
// (M = 128 cells, N = 32, K = 64: four K = 16 steps, A from tensor memory, B
// = W1^T from shared memory through a matrix descriptor, FP32 accumulation in
// tensor memory); each thread reads its cell's 32 accumulators back, adds the
// bias, applies ReLU, rounds to BF16 and writes them as layer 2's A; layer 2
// (K = 32) runs the same way; the 32 -> 1 output is a per-thread dot product.
// Tensor memory per warpgroup: 64 columns, A at [0, 32) (layer 1's features,
// then layer 2's inputs once layer 1's MMAs are done) and D at [32, 64)
// (layer 1's accumulators, then layer 2's once every thread has read them).
// The shared memory of a CTA is sized so that at most 8/G CTAs fit on an SM
// (228 KB), so their allocations (64 G columns each, 512 per SM) never wait
// on one another. Every mbarrier wait is bounded; on a timeout the CTA reports
// kErrTimeout, skips its remaining rounds and still frees its columns.
// ---------------------------------------------------------------------------
constexpr int kTcGroups = 2;  // warpgroups per CTA (measured fastest of 1, 2 and 4)
// shared memory per CTA for G warpgroups: more than 228 KB / (8/G + 1) with
// the 1 KB the runtime reserves per CTA, so no more than 8/G CTAs fit
template <int G>
constexpr size_t tc_smem_bytes() { return G == 4 ? 80 * 1024 : (G == 2 ? 56 * 1024 : 28 * 1024); }

// Tensor copy of a tile's FP64 region: x from the region's first column
// rounded down to even (16-byte aligned), 2 columns wider than the region.
constexpr int kRawW = kRW + 2;
constexpr size_t kRawBytes = sizeof(double) * 4 * kRawW * kRH;
constexpr size_t kRegionScratch = sizeof(SensorRegion) - sizeof(float) * 2 * kRH * kRW;  // hr .. scp

struct TcSmem {
    // W1^T [32 n][64 k] and W2^T [32 n][32 k], BF16, K-major in 8 x 8 core
    // matrices (8 rows of 16 bytes, 128 contiguous bytes each), core matrix
    // (n/8, k/8) at ((n/8) * KG + k/8) * 128 bytes, KG = k-groups per row.
    alignas(128) __nv_bfloat16 w1c[kSensorH * kSensorK];
    alignas(128) __nv_bfloat16 w2c[kSensorH * kSensorH];
    float b1[kSensorH], b2[kSensorH], w3[kSensorH], b3;
    alignas(8) unsigned long long mbar, tma_bar;
    unsigned taddr;
    // the tensor copy lands on R.hr .. R.scp and the tail after them (free
    // until the window maxima are formed, after the conversion)
    alignas(128) SensorRegion R;
    unsigned char raw_tail[kRawBytes > kRegionScratch ? kRawBytes - kRegionScratch : 1];
};
static_assert(sizeof(TcSmem) <= tc_smem_bytes<kTcGroups>(), "tcgen05 sensor tile exceeds its shared memory");
static_assert((sizeof(float) * 2 * kRH * kRW) % 128 == 0, "the copy's landing area must stay 128-byte aligned");
static_assert(kRawW % 2 == 0 && kRawW <= 256 && kRH <= 256, "tensor copy box: 16-byte rows, at most 256 wide");

// Warp 0 waits for the MMAs' completion; the block barrier then releases the
// other warps (which read the accumulators after their own fence). True on
// every thread if the wait succeeded.
__device__ __forceinline__ bool tc_wait_mmas(unsigned long long* bar, unsigned parity)
{
    bool done = true;
    if ((threadIdx.x >> 5) == 0) done = mbar_wait_parity_bounded(bar, parity);
    return __syncthreads_and(done) != 0;
}

// Set-up of a CTA: the weights in core-matrix order (read by the MMAs through
// the async proxy) and 64 G tensor-memory columns (warp 0). The MMA mbarrier
// is initialised by the kernel before. Returns the columns' base address.
template <int G>
__device__ uint32_t tc_setup(const SensorDev* w, TcSmem& S)
{
    constexpr int kThreads = 128 * G;
    const int tid = threadIdx.x;
    for (int i = tid; i < kSensorH * kSensorK; i += kThreads) {
        const int n = i / kSensorK, k = i - n * kSensorK;
        S.w1c[core_index(n, k, kSensorK / 8)] = w->w1t[n * kW1Pitch + k];
    }
    for (int i = tid; i < kSensorH * kSensorH; i += kThreads) {
        const int n = i / kSensorH, k = i - n * kSensorH;
        S.w2c[core_index(n, k, kSensorH / 8)] = w->w2t[n * kW2Pitch + k];
    }
    if (tid < kSensorH) {
        S.b1[tid] = w->b1[tid];
        S.b2[tid] = w->b2[tid];
        S.w3[tid] = w->w3[tid];
    }
    if (tid == 0) S.b3 = w->b3;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.taddr)),
                     "r"(kColsPerGroup * G)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return S.taddr;
}

// Release of the CTA's tensor-memory columns (after its last wait).
template <int G>
__device__ void tc_teardown(uint32_t tm)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kColsPerGroup * G)
                     : "memory");
    }
}

// One 32 x 24 tile whose region and scales are staged: 6/G rounds of both
// layers. `phase` is the mbarrier's next parity (two completions per round).
// False if a bounded wait gave up (uniform over the CTA; the remaining rounds
// are skipped).
template <int G>
__device__ bool tc_tile(const SensorTileParams& P, const int tx0, const int ty0, TcSmem& S, const uint32_t tm,
                        unsigned& phase)
{
    constexpr int kThreads = 128 * G;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool decide = P.dec != nullptr;
    const int org = decide ? kDecOrigin : kGhost;
    const int ni = decide ? P.g.ny + 2 * kDecOrigin : P.g.ny;
    const int nj = decide ? P.g.nx + 2 * kDecOrigin : P.g.nx;
    // this warp's quarter of the lanes, in its warpgroup's columns
    const uint32_t lanes = ((uint32_t)((warp & 3) * 32) << 16) + kColsPerGroup * (uint32_t)(warp >> 2);
    const uint64_t d1 = tc_smem_desc(S.w1c, 128, 128 * (kSensorK / 8));
    const uint64_t d2 = tc_smem_desc(S.w2c, 128, 128 * (kSensorH / 8));
    for (int round = 0; round < kTX * kTY / kThreads; ++round) {
        const int c = round * kThreads + tid, cy = c / kTX, cx = c - cy * kTX;
        const float* r = S.R.sr + (cy + kH) * kRW + (cx + kH);
        const float* p = S.R.sp + (cy + kH) * kRW + (cx + kH);
        const float sr = S.R.scr[c], sp = S.R.scp[c];
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // features 32 half .. 32 half + 31
            uint32_t a[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = 32 * half + 2 * j;
                a[j] = pack_bf16(sensor_feature(r, p, kRW, sr, sp, k), sensor_feature(r, p, kRW, sr, sp, k + 1));
            }
            tc_st16(tm + lanes + kColA + 16 * half, a);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && !(P.stall && round == 0)) {
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int ks = 0; ks < kSensorK / 16; ++ks)
                    tc_mma(tm + kColsPerGroup * g + kColD, tm + kColsPerGroup * g + kColA + 8 * ks,
                           d1 + (uint64_t)((256 * ks) >> 4), ks > 0);
            tc_commit(&S.mbar);
        }
        if (!tc_wait_mmas(&S.mbar, phase)) return false;
        phase ^= 1u;
        tc_fence_after();
        uint32_t h[16];
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // hidden units 16 half .. 16 half + 15
            uint32_t d[16];
            tc_ld16(tm + lanes + kColD + 16 * half, d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = 16 * half + 2 * j;
                h[8 * half + j] = pack_bf16(fmaxf(__uint_as_float(d[2 * j]) + S.b1[n], 0.f),
                                            fmaxf(__uint_as_float(d[2 * j + 1]) + S.b1[n + 1], 0.f));
            }
        }
        tc_st16(tm + lanes + kColA, h);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int ks = 0; ks < kSensorH / 16; ++ks)
                    tc_mma(tm + kColsPerGroup * g + kColD, tm + kColsPerGroup * g + kColA + 8 * ks,
                           d2 + (uint64_t)((256 * ks) >> 4), ks > 0);
            tc_commit(&S.mbar);
        }
        if (!tc_wait_mmas(&S.mbar, phase)) return false;
        phase ^= 1u;
        tc_fence_after();
        float z = 0.f;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t d[16];
            tc_ld16(tm + lanes + kColD + 16 * half, d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = 16 * half + j;
                z += fmaxf(__uint_as_float(d[j]) + S.b2[n], 0.f) * S.w3[n];
            }
        }
        const float pv = 1.f / (1.f + expf(-(z + S.b3)));
        const int i = ty0 + cy, j = tx0 + cx;
        if (i < ni && j < nj) {
            if (decide)
                P.dec[(long long)(i + org) * P.g.pitch + (j + org)] = pv > kSensorHi ? 1 : (pv < kSensorLo ? 0 : 2);
            else
                P.prob[(long long)i * P.g.nx + j] = pv;
        }
    }
    return true;
}

// One CTA per tile of one grid. The region arrives by one tensor copy (tmap:
// box kRawW x kRH x 4 of the padded state), issued before the weights are
// staged and the tensor memory is allocated, so the three overlap.
template <int G>
__global__ void __launch_bounds__(128 * G, 8 / G)
    sensor_tc_kernel(const SensorTileParams P, unsigned* err, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw);
    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * kTY;
    const int org = P.dec ? kDecOrigin : kGhost;
    const int gx0 = tx0 + org - kH, gy0 = ty0 + org - kH;  // padded coordinates of region cell (0, 0)
    const int xa = gx0 & ~1, ox = gx0 - xa;                // 16-byte aligned copy origin
    double* raw = reinterpret_cast<double*>(S.R.hr);
    const bool tma = (smem_addr(raw) & 127u) == 0;         // uniform: the copy needs 128-byte alignment
    if (tid == 0) {
        mbar_init(&S.mbar, 1);
        mbar_init(&S.tma_bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tma && tid == 0) {
        mbar_arrive_expect_tx(&S.tma_bar, (unsigned)kRawBytes);
        tma_load_3d(raw, &tmap, xa, gy0, 0, &S.tma_bar);
    }
    const uint32_t tm = tc_setup<G>(P.w, S);
    bool ok = true;
    if (tma) {
        ok = __syncthreads_and(mbar_wait_bounded(&S.tma_bar)) != 0;
        if (!ok) {
            // One more bounded wait for the copy before the CTA leaves; leaving
            // is safe only once its bytes have landed (a copy still in flight
            // would write into shared memory another CTA may own). The timeout
            // bit the CTA sets keeps every later result of the context
            // untrusted until gbr_set_state.
            mbar_wait_bounded(&S.tma_bar);
        } else {
            // cells beyond the padded extent read as zero and only feed
            // outputs that are never stored
            const float gm1 = (float)(P.gamma - 1.0);
            constexpr int plane = kRawW * kRH;
            for (int idx = tid; idx < kRH * kRW; idx += blockDim.x) {
                const int ry = idx / kRW, rx = idx - ry * kRW;
                const int o = ry * kRawW + rx + ox;
                float r, u, v, pr;
                prims_of(raw[o], raw[plane + o], raw[2 * plane + o], raw[3 * plane + o], gm1, r, u, v, pr);
                S.R.sr[idx] = r;
                S.R.sp[idx] = pr;
            }
            __syncthreads();
            sensor_scales(S.R);
        }
    } else {
        sensor_stage(P, tx0, ty0, org, true, S.R);
    }
    unsigned phase = 0;
    if (ok) ok = tc_tile<G>(P, tx0, ty0, S, tm, phase);
    tc_teardown<G>(tm);
    if (!ok && tid == 0 && err) atomicOr(err, kErrTimeout);
}

// Decision pass over every running case of a batch: one CTA per sensor tile
// of the concatenated tile list (a persistent loop over tiles measured twice
// as slow: its CTAs move through the staging and MMA phases in step). A CTA
// of a stopped case returns before it allocates anything.
template <int G>
__global__ void __launch_bounds__(128 * G, 8 / G)
    batch_sensor_tc_kernel(const BatchCase* __restrict__ cases, int ncases, int buf, const SensorDev* w)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw);
    const int tile = blockIdx.x;
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cases[mid].dtile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    const BatchCase& C = cases[lo];
    if (C.ds->dt == 0.0) return;  // stopped case; uniform over the CTA
    const int local = tile - C.dtile_begin;
    const int ty = local / C.dtiles_x, tx = local - ty * C.dtiles_x;
    SensorTileParams P;
    P.g = C.g;
    P.gamma = C.ph.gamma;
    P.q = C.q[buf];
    P.w = w;
    P.prob = nullptr;
    P.feat = nullptr;
    P.label = nullptr;
    P.target = nullptr;
    P.dec = C.dec;
    P.stall = 0;
    if (threadIdx.x == 0) mbar_init(&S.mbar, 1);
    const uint32_t tm = tc_setup<G>(w, S);  // its barriers order the initialisation
    sensor_stage(P, tx * kTX, ty * kTY, kDecOrigin, true, S.R);
    unsigned phase = 0;
    const bool ok = tc_tile<G>(P, tx * kTX, ty * kTY, S, tm, phase);
    tc_teardown<G>(tm);
    if (!ok && threadIdx.x == 0) atomicOr(&C.ds->err, kErrTimeout);
}

static cudaError_t launch_sensor_tc(const SensorTileParams& P, dim3 grid, unsigned* err, cudaStream_t s)
{
    constexpr size_t smem = tc_smem_bytes<kTcGroups>();
    static PerDevice<int> configured;  // the shared-memory limit is raised once per device
    int ok = 0;
    cudaError_t e = configured.get(&ok, [](int* v) {
        *v = 1;
        return cudaFuncSetAttribute(sensor_tc_kernel<kTcGroups>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    if ((e = encode_state_map(P.g, P.q, kRawW, kRH, &map)) != cudaSuccess) return e;
    sensor_tc_kernel<kTcGroups><<<grid, 128 * kTcGroups, smem, s>>>(P, err, map);
    return cudaGetLastError();
}

cudaError_t launch_sensor_tile(const Grid& g, double gamma, const double* q, const SensorDev* w, float* prob,
                               void* feat_bf16, unsigned char* label, unsigned char* target, unsigned* err,
                               cudaStream_t s)
{
    SensorTileParams P;
    P.g = g;
    P.gamma = gamma;
    P.q = q;
    P.w = w;
    P.prob = prob;
    P.feat = static_cast<__nv_bfloat16*>(feat_bf16);
    P.label = label;
    P.target = target;
    P.dec = nullptr;
    P.stall = 0;
    dim3 grid((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY);
    if (prob) {
        if (!w || feat_bf16 || label || target) return cudaErrorInvalidValue;
        return launch_sensor_tc(P, grid, err, s);
    }
    sensor_dataset_kernel<<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

void sensor_decide_tiles(const Grid& g, int* tiles_x, int* tiles)
{
    const int tx = (g.nx + 2 * kDecOrigin + kTX - 1) / kTX, ty = (g.ny + 2 * kDecOrigin + kTY - 1) / kTY;
    *tiles_x = tx;
    *tiles = tx * ty;
}

cudaError_t launch_sensor_decide(const Grid& g, double gamma, const double* q, const SensorDev* w,
                                 unsigned char* dec, unsigned* err, int stall, cudaStream_t s)
{
    if (!w || !dec) return cudaErrorInvalidValue;
    SensorTileParams P;
    P.g = g;
    P.gamma = gamma;
    P.q = q;
    P.w = w;
    P.prob = nullptr;
    P.feat = nullptr;
    P.label = nullptr;
    P.target = nullptr;
    P.dec = dec;
    P.stall = stall;
    int tx, tiles;
    sensor_decide_tiles(g, &tx, &tiles);
    return launch_sensor_tc(P, dim3(tx, tiles / tx), err, s);
}

cudaError_t launch_batch_sensor_decide(const BatchCase* cases, int ncases, int total_tiles, int buf,
                                       const SensorDev* w, cudaStream_t s)
{
    constexpr size_t smem = tc_smem_bytes<kTcGroups>();
    auto kern = batch_sensor_tc_kernel<kTcGroups>;
    static PerDevice<int> configured;  // the shared-memory limit is raised once per device
    int ok = 0;
    cudaError_t e = configured.get(&ok, [&](int* v) {
        *v = 1;
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    if (total_tiles <= 0) return cudaSuccess;  // prepare only (or nothing to do)
    kern<<<total_tiles, 128 * kTcGroups, smem, s>>>(cases, ncases, buf, w);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Training: one kernel accumulates the gradient of a mini-batch, one applies
// Adam. Operands are BF16-rounded (features as stored, weights and the first
// hidden layer rounded), products accumulate in FP32.
// ---------------------------------------------------------------------------
constexpr int kTrainWarps = 4;
constexpr int kXP = kSensorIn + 1;  // row pitches of the per-warp scratch (odd: no bank conflicts)
constexpr int kHP = kSensorH + 1;
// dynamic shared memory of the gradient kernel, in floats
constexpr int kOffW1 = 0;
constexpr int kOffW2 = kOffW1 + kSensorIn * kSensorH;
constexpr int kOffB1 = kOffW2 + kSensorH * kSensorH;
constexpr int kOffB2 = kOffB1 + kSensorH;
constexpr int kOffW3 = kOffB2 + kSensorH;
constexpr int kOffB3 = kOffW3 + kSensorH;
constexpr int kOffG = kOffB3 + 4;
constexpr int kOffWarp = kOffG + ((kSensorParams + 3) / 4) * 4;
constexpr int kWarpFloats = 32 * kXP + 4 * 32 * kHP + 32;  // x, h1, dh1, dh2, h2, dz
constexpr int kTrainSmemFloats = kOffWarp + kTrainWarps * kWarpFloats;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct TrainParams {
    const __nv_bfloat16* X;  // [n][64]
    const unsigned char* y;  // [n] targets in units of 1/255
    long long n;
    int batch;               // samples per step
    unsigned long long seed;
    int step;
    float pos_weight;        // loss weight of label-1 samples
    const float* w;          // FP32 master parameters (host layout)
    float* grad;             // accumulated gradient (host layout), zeroed by Adam
    float* loss;             // [steps] summed loss of each step
};

__global__ void __launch_bounds__(kTrainWarps * 32) sensor_grad_kernel(const TrainParams P)
{
    extern __shared__ float sm[];
    float* const W1 = sm + kOffW1;
    float* const W2 = sm + kOffW2;
    float* const b1 = sm + kOffB1;
    float* const b2 = sm + kOffB2;
    float* const w3 = sm + kOffW3;
    float* const gacc = sm + kOffG;
    const float* pw = P.w;
    for (int i = threadIdx.x; i < kSensorIn * kSensorH; i += blockDim.x) W1[i] = bf16r(pw[i]);
    for (int i = threadIdx.x; i < kSensorH * kSensorH; i += blockDim.x)
        W2[i] = bf16r(pw[kSensorIn * kSensorH + kSensorH + i]);
    for (int i = threadIdx.x; i < kSensorH; i += blockDim.x) {
        b1[i] = pw[kSensorIn * kSensorH + i];
        b2[i] = pw[kSensorIn * kSensorH + kSensorH + kSensorH * kSensorH + i];
        w3[i] = pw[kSensorIn * kSensorH + 2 * kSensorH + kSensorH * kSensorH + i];
    }
    if (threadIdx.x == 0) sm[kOffB3] = pw[kSensorParams - 1];
    for (int i = threadIdx.x; i < kSensorParams; i += blockDim.x) gacc[i] = 0.f;
    __syncthreads();
    const float b3s = sm[kOffB3];
    float* const wbase = sm + kOffWarp + (threadIdx.x >> 5) * kWarpFloats;
    float* const xsw = wbase;                       // [32][kXP]
    float* const h1sw = xsw + 32 * kXP;             // [32][kHP]
    float* const d1sw = h1sw + 32 * kHP;
    float* const d2sw = d1sw + 32 * kHP;
    float* const h2sw = d2sw + 32 * kHP;
    float* const dzsw = h2sw + 32 * kHP;            // [32]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* xr = xsw + lane * kXP;
    float* h1r = h1sw + lane * kHP;
    float* d1r = d1sw + lane * kHP;
    float* d2r = d2sw + lane * kHP;
    float* h2r = h2sw + lane * kHP;
    float aW1[kSensorIn], aW2[kSensorH], ab1 = 0.f, ab2 = 0.f, aw3 = 0.f, ab3 = 0.f, lsum = 0.f;
#pragma unroll
    for (int k = 0; k < kSensorIn; ++k) aW1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < kSensorH; ++k) aW2[k] = 0.f;

    const int per_block = kTrainWarps * 32;
    for (int base = blockIdx.x * per_block; base < P.batch; base += gridDim.x * per_block) {
        const int s_id = base + warp * 32 + lane;
        const bool valid = s_id < P.batch;
        // sample (with replacement) by a counter-based hash of (seed, step, s_id)
        const unsigned long long hsh = splitmix64(P.seed ^ ((unsigned long long)P.step * 0x100000001ull + s_id));
        const long long idx = (long long)(hsh % (unsigned long long)P.n);
        const __nv_bfloat16* xin = P.X + idx * kSensorK;
        for (int k = 0; k < kSensorIn; ++k) xr[k] = valid ? __bfloat162float(xin[k]) : 0.f;
        const float yv = valid ? (float)P.y[idx] * (1.f / 255.f) : 0.f;
        // forward
        for (int n = 0; n < kSensorH; ++n) {
            float a = b1[n];
            for (int k = 0; k < kSensorIn; ++k) a = fmaf(xr[k], W1[k * kSensorH + n], a);
            h1r[n] = bf16r(fmaxf(a, 0.f));
        }
        float z = b3s;
        for (int n = 0; n < kSensorH; ++n) {
            float a = b2[n];
            for (int k = 0; k < kSensorH; ++k) a = fmaf(h1r[k], W2[k * kSensorH + n], a);
            a = fmaxf(a, 0.f);
            h2r[n] = a;
            z = fmaf(a, w3[n], z);
        }
        const float p = 1.f / (1.f + expf(-z));
        const float wt = valid ? 1.f + (P.pos_weight - 1.f) * yv : 0.f;
        // binary cross-entropy from the logit: softplus(z) - y z
        const float l = fmaxf(z, 0.f) - yv * z + log1pf(expf(-fabsf(z)));
        lsum += wt * l;
        const float dz = wt * (p - yv);
        // backward
        for (int n = 0; n < kSensorH; ++n) d2r[n] = h2r[n] > 0.f ? dz * w3[n] : 0.f;
        for (int k = 0; k < kSensorH; ++k) {
            float a = 0.f;
            for (int n = 0; n < kSensorH; ++n) a = fmaf(d2r[n], W2[k * kSensorH + n], a);
            d1r[k] = h1r[k] > 0.f ? a : 0.f;
        }
        dzsw[lane] = dz;
        __syncwarp();
        // lane n accumulates column n of every weight gradient over the 32 samples
        const int n = lane;
        for (int s = 0; s < 32; ++s) {
            const float* xs_s = xsw + s * kXP;
            const float* h1_s = h1sw + s * kHP;
            const float d1 = d1sw[s * kHP + n], d2 = d2sw[s * kHP + n];
#pragma unroll
            for (int k = 0; k < kSensorIn; ++k) aW1[k] = fmaf(xs_s[k], d1, aW1[k]);
#pragma unroll
            for (int k = 0; k < kSensorH; ++k) aW2[k] = fmaf(h1_s[k], d2, aW2[k]);
            ab1 += d1;
            ab2 += d2;
            aw3 = fmaf(h2sw[s * kHP + n], dzsw[s], aw3);
            ab3 += dzsw[s];
        }
        __syncwarp();
    }
    // block reduction in shared memory, then one global add per parameter
    const int n = lane;
#pragma unroll
    for (int k = 0; k < kSensorIn; ++k) atomicAdd(&gacc[k * kSensorH + n], aW1[k]);
    atomicAdd(&gacc[kSensorIn * kSensorH + n], ab1);
#pragma unroll
    for (int k = 0; k < kSensorH; ++k) atomicAdd(&gacc[kSensorIn * kSensorH + kSensorH + k * kSensorH + n], aW2[k]);
    atomicAdd(&gacc[kSensorIn * kSensorH + kSensorH + kSensorH * kSensorH + n], ab2);
    atomicAdd(&gacc[kSensorIn * kSensorH + 2 * kSensorH + kSensorH * kSensorH + n], aw3);
    if (lane == 0) atomicAdd(&gacc[kSensorParams - 1], ab3);
    // the loss of the step
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __syncthreads();
    for (int i = threadIdx.x; i < kSensorParams; i += blockDim.x) atomicAdd(&P.grad[i], gacc[i]);
    if (lane == 0) atomicAdd(&P.loss[P.step], lsum);
}

// Adam (Kingma and Ba, 2015) on the mean gradient of the step; clears it.
__global__ void sensor_adam_kernel(float* w, float* grad, float* m, float* v, int step, float lr, float inv_batch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kSensorParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i] * inv_batch;
    grad[i] = 0.f;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)(step + 1)));
    const float vh = vi / (1.f - powf(b2, (float)(step + 1)));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
}

cudaError_t launch_sensor_train(const void* X_bf16, const unsigned char* y, long long n, int steps, int batch,
                                float lr, float pos_weight, unsigned long long seed, float* w, float* grad,
                                float* m, float* v, float* loss, cudaStream_t s)
{
    const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(X_bf16);
    const int per_block = kTrainWarps * 32;
    const int blocks = (batch + per_block - 1) / per_block;
    const size_t smem = sizeof(float) * kTrainSmemFloats;
    cudaError_t e = cudaFuncSetAttribute(sensor_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < steps; ++k) {
        TrainParams P;
        P.X = X;
        P.y = y;
        P.n = n;
        P.batch = batch;
        P.seed = seed;
        P.step = k;
        P.pos_weight = pos_weight;
        P.w = w;
        P.grad = grad;
        P.loss = loss;
        sensor_grad_kernel<<<blocks, per_block, smem, s>>>(P);
        sensor_adam_kernel<<<(kSensorParams + 255) / 256, 256, 0, s>>>(w, grad, m, v, k, lr, 1.f / batch);
    }
    return cudaGetLastError();
}

}  // namespace gbr
