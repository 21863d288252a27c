// Internal declarations shared by the host C-ABI (gbr_api.cu) and the kernel
// translation units. Not part of the public interface (include/gbr.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace gbr {

// Per-device launch set-up (kernel attributes and occupancy-derived grid
// sizes are properties of a kernel on one device). PerDevice<V> holds one
// value per device ordinal below kDeviceSlots; `get` computes it with `make`
// on the current device the first time and returns the stored value after
// (a race between threads computes the same value twice, harmlessly).
constexpr int kDeviceSlots = 64;
template <typename V>
struct PerDevice {
    std::atomic<V> val[kDeviceSlots];  // zero: not computed yet
    template <typename F>
    cudaError_t get(V* out, F make)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kDeviceSlots) return make(out);
        V v = val[dev].load(std::memory_order_acquire);
        if (v == V(0)) {
            if ((e = make(&v)) != cudaSuccess) return e;
            val[dev].store(v, std::memory_order_release);
        }
        *out = v;
        return cudaSuccess;
    }
};

constexpr int kGhost = 6;  // ghost layers per side (Sec. 2.3, LC bound reach)

// Device-resident scalars of one solver context.
struct DevScalars {
    unsigned long long lam[2];  // CFL wavespeed of a state, bits of a double >= 0
    double dt;                  // step size used by the current step
    double t;                   // simulated time since the last set_state
    unsigned int err;           // bit 0: non-physical stage state, bit 1: a bounded wait gave up
    unsigned int pad;
    double ts[2];               // time at the start of the step, slot cur (read by time-dependent boundaries)
};

// A GBR_BC_CUSTOM side on the device: kinds below / above the split point
// s0 + speed t along the side, fixed states as conservative vectors.
struct SideBC {
    int kind_lo, kind_hi;
    double s0, speed;
    double qlo[4], qhi[4];
};

// Padded state geometry: plane m of a state starts at base + m * plane; the
// interior cell (j, i) sits at (i + 6) * pitch + (j + 6).
struct Grid {
    int nx, ny;
    int pitch;        // elements per padded row (>= nx + 12)
    long long plane;  // elements per component plane
};

struct Physics {
    double gamma, mu, Pr, dx, dy;
    int order;  // 7: MEG7 (alpha = 38/7, beta = 3/190); 4: the alpha = 4, beta = 0 member
    int cons;   // 0: MEG7-prim (reconstruct U); 1: MEG7-cons (reconstruct Q)
    int riemann;  // 0: HLLC; 1: shock-stable HLLC-LM (Fleischmann et al. 2020)
    // Derived once on the host (derive_physics), so that no kernel thread
    // spends FP64 divisions on them: gamma - 1, 1/(gamma - 1), the heat
    // conduction coefficient mu / (Pr (gamma - 1)), 1/dx, 1/dy.
    double gm1, igm1, kq, inv_dx, inv_dy;
};

// Fill the derived members of ph from gamma, mu, Pr, dx, dy.
inline void derive_physics(Physics& ph)
{
    ph.gm1 = ph.gamma - 1.0;
    ph.igm1 = 1.0 / (ph.gamma - 1.0);
    ph.kq = ph.mu / (ph.Pr * (ph.gamma - 1.0));
    ph.inv_dx = 1.0 / ph.dx;
    ph.inv_dy = 1.0 / ph.dy;
}

struct SensorDev;

// One fused residual (+ stage update) pass, Secs. 2.1-2.5.
struct StageParams {
    Grid g;
    Physics ph;
    const double* q;         // stage input state (padded, ghosts filled)
    const double* qn;        // Q^n (padded) for the RK combination (may equal qout)
    double* qout;            // output state (padded) or nullptr (residual only)
    double* res;             // dense residual [4][ny][nx] or nullptr
    unsigned char* sigx;     // optional x-face flags [ny][nx+1]
    unsigned char* sigy;     // optional y-face flags [ny+1][nx]
    unsigned long long* lam_out;  // optional wavespeed of qout (atomic max)
    unsigned int* err;       // error word
    const double* dt_ptr;    // device dt (used when non-null)
    double dt;               // host dt otherwise
    double ca, cb, cc;       // qout = ca * qn + cb * q + cc * dt * Res
    const SensorDev* sensor; // learned-sensor weights (FP32 form) or nullptr
    const unsigned char* dec;  // learned-sensor decisions of padded cells [3, n+9) (pitch g.pitch), with sensor
    unsigned stall_bytes;    // failure-detection test hook: extra bytes the tile staging waits for (0)
    unsigned stall_mma;      // failure-detection test hook: the fused sensor withholds its first MMA batch (0)
};

// Ghost fill of one padded state, plus the per-step scalar bookkeeping done
// by its first thread (mode 1: add dt to t and clear lam[next]; mode 2: form
// dt = min(cfl / lam[cur], dt_max) on the device first).
struct GhostParams {
    Grid g;
    double* q;
    int bc[4];  // west, east, south, north
    DevScalars* ds;
    int mode;
    int cur, next;
    double dt, cfl, dt_max;
    SideBC side[4];     // GBR_BC_CUSTOM sides
    double dx, dy;      // cell sizes (positions along custom sides)
    double c_stage;     // stage abscissa: the boundary time is ts[cur] + c_stage dt
};

// One grid of a batch, as the device sees it. tiles_x / tile_begin describe
// the current tile shape: tile t of the batch belongs to the case with the
// largest tile_begin <= t.
struct BatchCase {
    Grid g;
    Physics ph;
    int bc[4];
    double* q[3];        // Q^n, Q^(1), Q^(2) (padded)
    unsigned char* dec;  // learned-sensor decisions (padded layout) or nullptr
    int dtiles_x, dtile_begin;  // sensor-pass tiles of this case: per row, first batch tile
    DevScalars* ds;      // lam[0] = wavespeed of Q^n, dt, t, err
    double t_end;        // the case stops (dt = 0) once t reaches t_end
    int tiles_x, tiles;  // tiles of this case for the current tile shape
    int tile_begin;      // first batch tile of this case
    long long ghost_begin;  // first batch ghost cell of this case
};

struct TileShape {
    int bx, by;
};

cudaError_t launch_ghosts(const GhostParams& p, cudaStream_t s);
cudaError_t launch_set_time(DevScalars* d, int cur, double t, cudaStream_t s);
// Ghost cells of buffer `buf` (0, 1, 2) of every case; with mode 2 the first
// ncases threads also form each case's dt = min(cfl / lam, t_end - t), advance
// its time and clear its wavespeed slot; with mode 3 each case's dt is
// dts[k] (device array; a case at dt = 0 is left as it is).
cudaError_t launch_batch_ghosts(const BatchCase* cases, int ncases, long long total_ghosts, int buf, int mode,
                                double cfl, cudaStream_t s, const double* dts = nullptr);
// Candidate tile shapes of the persistent batch kernel (returns the count).
int batch_tile_shapes_f64(const TileShape** shapes);
int batch_tile_shapes_f32(const TileShape** shapes);
// One kernel over all tiles of all cases for RK stage `stage` (0, 1, 2):
// per_tile = false, a persistent grid (resident CTAs x SMs) whose CTAs walk
// the tile list; true, one CTA per tile.
cudaError_t launch_batch_stage_f64(int shape, const BatchCase* cases, int ncases, int total_tiles, int stage,
                                   cudaStream_t s, bool per_tile = false);
cudaError_t launch_batch_stage_f32(int shape, const BatchCase* cases, int ncases, int total_tiles, int stage,
                                   cudaStream_t s, const SensorDev* sensor = nullptr, bool per_tile = false);
// Learned sensor (sensor.cu): host packing of the weight vector, per-cell
// evaluation / dataset extraction on a padded state, training.
void pack_sensor(const float* w, SensorDev* out);
// Tensor map of a padded FP64 state for the stage kernels' tile staging:
// 3-D (x over the nx + 12 padded columns, y over the ny + 12 padded rows,
// the 4 fields), box box_w x box_h x 4, out-of-range cells read as zero.
// Host-only; encodings are cached per (state, grid, box).
cudaError_t encode_state_map(const Grid& g, const double* q, int box_w, int box_h, CUtensorMap* out);

// Network outputs (prob, on the tcgen05 tensor cores), dataset features,
// labels and targets of one padded state (ghosts filled). A bounded wait of
// the tensor-core pass that gives up sets kErrTimeout in *err.
cudaError_t launch_sensor_tile(const Grid& g, double gamma, const double* q, const SensorDev* w, float* prob,
                               void* feat_bf16, unsigned char* label, unsigned char* target, unsigned* err,
                               cudaStream_t s);
// The learned sensor's decision pass of one padded state (ghosts filled), on
// the tcgen05 tensor cores: dec[y * pitch + x] for padded cells x in
// [3, nx + 9), y in [3, ny + 9): 1 = discontinuity (p > 0.7), 0 = smooth
// (p < 0.3), 2 = unsure. A wait that gives up sets kErrTimeout in *err;
// stall != 0 (failure-detection test) withholds the first MMA batch so that
// its bounded wait gives up.
cudaError_t launch_sensor_decide(const Grid& g, double gamma, const double* q, const SensorDev* w,
                                 unsigned char* dec, unsigned* err, int stall, cudaStream_t s);
// Sensor-pass tiles of a grid (the tile grid over its decision region).
void sensor_decide_tiles(const Grid& g, int* tiles_x, int* tiles);
// The decision pass of buffer `buf` of every running case of a batch (one
// CTA per sensor tile; total_tiles = sum of the cases' sensor-pass tiles; a
// negative count only prepares the kernel, outside stream capture).
cudaError_t launch_batch_sensor_decide(const BatchCase* cases, int ncases, int total_tiles, int buf,
                                       const SensorDev* w, cudaStream_t s);
cudaError_t launch_sensor_train(const void* X_bf16, const unsigned char* y, long long n, int steps, int batch,
                                float lr, float pos_weight, unsigned long long seed, float* w, float* grad, float* m,
                                float* v, float* loss, cudaStream_t s);
cudaError_t launch_wavespeed(const Grid& g, const Physics& ph, const double* q, unsigned long long* lam,
                             int precision, cudaStream_t s);
cudaError_t launch_stage_f64(const StageParams& p, cudaStream_t s);
cudaError_t launch_stage_f32(const StageParams& p, cudaStream_t s);
cudaError_t launch_stage_cons_f64(const StageParams& p, cudaStream_t s);
cudaError_t launch_stage_cons_f32(const StageParams& p, cudaStream_t s);

}  // namespace gbr
