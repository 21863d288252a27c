// Host implementation of the batch part of the C ABI (include/gbr.h).
#include <cuda_runtime.h>
#include <string.h>

#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbr.h"
#include "ghost.cuh"
#include "gbr_internal.h"
#include "sensor.cuh"

using namespace gbr;

struct gbr_batch {
    int n;
    int device;
    cudaStream_t stream;      // caller's stream (launches, graph replays)
    cudaStream_t capture;     // internal stream used to capture graphs
    std::vector<BatchCase> cases;  // host copy of the descriptors
    BatchCase* d_cases;
    DevScalars* d_scal;
    double* pool;             // all padded states
    int precision;
    int shape;                // index into the precision's tile-shape table
    int per_tile;             // 1: one CTA per tile; 0: a persistent grid walking the tiles
    int total_tiles;
    long long total_ghosts;
    bool dirty;               // descriptors need uploading
    // cached graph
    cudaGraphExec_t graph;
    int g_nsteps, g_precision, g_shape, g_per_tile;
    double g_cfl;
    int g_sensor;
    int timing;
    SensorDev* d_sensor;      // learned-sensor weights (null until set)
    int sensor;               // 1: use them (FP32 only)
    unsigned char* dec_pool;  // the cases' learned-sensor decisions (padded layouts)
    int total_dtiles;         // sensor-pass tiles of all cases
    double* d_dt;             // caller-supplied per-case dt of gbr_batch_step (n doubles)
};

namespace {

int st(cudaError_t e)
{
    if (e == cudaSuccess) return GBR_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GBR_ERR_NOMEM : GBR_ERR_CUDA;
}

#define TRY(expr)                       \
    do {                                \
        int rc_ = st(expr);             \
        if (rc_ != GBR_OK) return rc_;  \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int shapes(int precision, const TileShape** s)
{
    return precision == 32 ? batch_tile_shapes_f32(s) : batch_tile_shapes_f64(s);
}

// Tile decomposition of every case for the current shape.
void retile(gbr_batch* b)
{
    const TileShape* sh;
    shapes(b->precision, &sh);
    const TileShape t = sh[b->shape];
    int begin = 0;
    for (auto& c : b->cases) {
        c.tiles_x = (c.g.nx + t.bx - 1) / t.bx;
        c.tiles = c.tiles_x * ((c.g.ny + t.by - 1) / t.by);
        c.tile_begin = begin;
        begin += c.tiles;
    }
    b->total_tiles = begin;
    b->dirty = true;
}

int upload(gbr_batch* b)
{
    if (!b->dirty) return GBR_OK;
    TRY(cudaMemcpyAsync(b->d_cases, b->cases.data(), sizeof(BatchCase) * b->n, cudaMemcpyHostToDevice, b->stream));
    b->dirty = false;
    return GBR_OK;
}

const SensorDev* sensor_of(gbr_batch* b) { return (b->precision == 32 && b->sensor) ? b->d_sensor : nullptr; }

// Stage k of every running case; with the learned sensor, its decision pass
// over the stage's input state first.
int stage(gbr_batch* b, int k, cudaStream_t s)
{
    const SensorDev* w = sensor_of(b);
    if (w) TRY(launch_batch_sensor_decide(b->d_cases, b->n, b->total_dtiles, k, w, s));
    cudaError_t e = b->precision == 32
                        ? launch_batch_stage_f32(b->shape, b->d_cases, b->n, b->total_tiles, k, s, w, b->per_tile)
                        : launch_batch_stage_f64(b->shape, b->d_cases, b->n, b->total_tiles, k, s, b->per_tile);
    return st(e);
}

// One RK3 step of every case (Eq. rk): ghost fill + batch stage kernel,
// three times; the first ghost fill forms each case's dt on the device
// (mode 2: CFL) or takes it from b->d_dt (mode 3: the caller's dt).
int enqueue_step(gbr_batch* b, double cfl, cudaStream_t s, int mode = 2)
{
    int rc;
    for (int k = 0; k < 3; ++k) {
        TRY(launch_batch_ghosts(b->d_cases, b->n, b->total_ghosts, k, k == 0 ? mode : 0, cfl, s, b->d_dt));
        if ((rc = stage(b, k, s)) != GBR_OK) return rc;
    }
    return GBR_OK;
}

void drop_graph(gbr_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

int check_errors(gbr_batch* b, std::vector<DevScalars>& h)
{
    h.resize(b->n);
    TRY(cudaMemcpyAsync(h.data(), b->d_scal, sizeof(DevScalars) * b->n, cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    for (const auto& d : h)
        if (d.err & 1u) return GBR_ERR_NONPHYSICAL;
    return GBR_OK;
}

// Body of gbr_batch_step_cfl (arguments already checked).
int batch_step_cfl(gbr_batch* b, double cfl, int nsteps)
{
    DeviceGuard dg(b->device);
    int rc = upload(b);
    if (rc != GBR_OK) return rc;
    if (!b->graph || b->g_nsteps != nsteps || b->g_cfl != cfl || b->g_precision != b->precision ||
        b->g_shape != b->shape || b->g_per_tile != b->per_tile || b->g_sensor != (sensor_of(b) != nullptr)) {
        drop_graph(b);
        // first-use kernel setup outside the capture (a negative tile count
        // prepares the stage kernel without launching it)
        TRY(b->precision == 32 ? launch_batch_stage_f32(b->shape, b->d_cases, b->n, -1, 0, b->stream, sensor_of(b))
                               : launch_batch_stage_f64(b->shape, b->d_cases, b->n, -1, 0, b->stream));
        if (sensor_of(b)) TRY(launch_batch_sensor_decide(b->d_cases, b->n, -1, 0, sensor_of(b), b->stream));
        // The descriptors must be on the device before the capture stream
        // replays anything: order the capture stream after the caller's.
        TRY(cudaStreamSynchronize(b->stream));
        TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
        int erc = GBR_OK;
        for (int s = 0; s < nsteps && erc == GBR_OK; ++s) erc = enqueue_step(b, cfl, b->capture);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (erc != GBR_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return erc != GBR_OK ? erc : GBR_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return st(e);
        }
        b->g_nsteps = nsteps;
        b->g_cfl = cfl;
        b->g_precision = b->precision;
        b->g_shape = b->shape;
        b->g_per_tile = b->per_tile;
        b->g_sensor = sensor_of(b) != nullptr;
    }
    return st(cudaGraphLaunch(b->graph, b->stream));
}

}  // namespace

extern "C" {

int gbr_batch_create(int n, const int* nx, const int* ny, const double* dx, const double* dy, const int* bc,
                     double gamma, gbr_batch** out)
{
    if (!out) return GBR_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !nx || !ny || !dx || !dy || !bc || !(gamma > 1.0)) return GBR_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        if (nx[k] < GBR_GHOST || ny[k] < GBR_GHOST || !(dx[k] > 0.0) || !(dy[k] > 0.0)) return GBR_ERR_ARG;
        if ((long long)nx[k] * ny[k] > (1LL << 31)) return GBR_ERR_ARG;
        for (int s = 0; s < 4; ++s)
            if (bc[4 * k + s] < GBR_BC_PERIODIC || bc[4 * k + s] > GBR_BC_SYMMETRY) return GBR_ERR_ARG;
        if ((bc[4 * k] == GBR_BC_PERIODIC) != (bc[4 * k + 1] == GBR_BC_PERIODIC)) return GBR_ERR_ARG;
        if ((bc[4 * k + 2] == GBR_BC_PERIODIC) != (bc[4 * k + 3] == GBR_BC_PERIODIC)) return GBR_ERR_ARG;
    }
    gbr_batch* b = new (std::nothrow) gbr_batch();
    if (!b) return GBR_ERR_NOMEM;
    b->n = n;
    b->precision = 64;
    b->per_tile = 1;  // measured faster than the persistent grid on the 64-grid ensemble
    b->cases.resize(n);
    int rc = st(cudaGetDevice(&b->device));
    long long total = 0, ghosts = 0;
    int dtiles = 0;
    for (int k = 0; k < n && rc == GBR_OK; ++k) {
        BatchCase& c = b->cases[k];
        memset(&c, 0, sizeof(c));
        c.g.nx = nx[k];
        c.g.ny = ny[k];
        c.g.pitch = ((nx[k] + 2 * kGhost + 15) / 16) * 16;
        c.g.plane = (((long long)c.g.pitch * (ny[k] + 2 * kGhost) + 15) / 16) * 16;
        c.ph.gamma = gamma;
        c.ph.mu = 0.0;
        c.ph.Pr = 1.0;
        c.ph.dx = dx[k];
        c.ph.dy = dy[k];
        c.ph.order = 7;
        derive_physics(c.ph);
        for (int s = 0; s < 4; ++s) c.bc[s] = bc[4 * k + s];
        c.t_end = 1e300;
        c.ghost_begin = ghosts;
        ghosts += ghost_count(c.g);
        int dtx = 0, dt = 0;
        sensor_decide_tiles(c.g, &dtx, &dt);
        c.dtiles_x = dtx;
        c.dtile_begin = dtiles;
        dtiles += dt;
        total += 12 * c.g.plane;  // 3 states x 4 planes
    }
    b->total_ghosts = ghosts;
    b->total_dtiles = dtiles;
    if (rc == GBR_OK) rc = st(cudaMalloc(&b->pool, sizeof(double) * (size_t)total));
    if (rc == GBR_OK) rc = st(cudaMemset(b->pool, 0, sizeof(double) * (size_t)total));
    if (rc == GBR_OK) rc = st(cudaMalloc(&b->d_scal, sizeof(DevScalars) * n));
    if (rc == GBR_OK) rc = st(cudaMemset(b->d_scal, 0, sizeof(DevScalars) * n));
    if (rc == GBR_OK) rc = st(cudaMalloc(&b->d_cases, sizeof(BatchCase) * n));
    if (rc == GBR_OK) rc = st(cudaMalloc(&b->d_dt, sizeof(double) * n));
    if (rc == GBR_OK) rc = st(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    if (rc != GBR_OK) {
        gbr_batch_destroy(b);
        return rc;
    }
    long long off = 0;
    for (int k = 0; k < n; ++k) {
        BatchCase& c = b->cases[k];
        for (int s = 0; s < 3; ++s) c.q[s] = b->pool + off + (long long)s * 4 * c.g.plane;
        off += 12 * c.g.plane;
        c.ds = b->d_scal + k;
    }
    retile(b);
    if ((rc = upload(b)) != GBR_OK || (rc = st(cudaStreamSynchronize(b->stream))) != GBR_OK) {
        gbr_batch_destroy(b);
        return rc;
    }
    *out = b;
    return GBR_OK;
}

int gbr_batch_destroy(gbr_batch* b)
{
    if (!b) return GBR_OK;
    DeviceGuard dg(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graph(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->pool);
    cudaFree(b->d_scal);
    cudaFree(b->d_cases);
    cudaFree(b->d_dt);
    cudaFree(b->d_sensor);
    cudaFree(b->dec_pool);
    cudaGetLastError();
    delete b;
    return GBR_OK;
}

int gbr_batch_set_stream(gbr_batch* b, void* stream)
{
    if (!b) return GBR_ERR_ARG;
    b->stream = (cudaStream_t)stream;
    return GBR_OK;
}

int gbr_batch_set_option(gbr_batch* b, int key, double val)
{
    if (!b) return GBR_ERR_ARG;
    if (key == GBR_OPT_PRECISION) {
        if (val != 64.0 && val != 32.0) return GBR_ERR_ARG;
        if ((int)val != b->precision) {
            b->precision = (int)val;
            b->shape = 0;
            retile(b);
        }
        return GBR_OK;
    }
    if (key == GBR_OPT_SENSOR) {
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        if (val == 1.0 && !b->d_sensor) return GBR_ERR_STATE;
        b->sensor = (int)val;
        return GBR_OK;
    }
    if (key == GBR_OPT_TIMING) {
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        b->timing = (int)val;
        return GBR_OK;
    }
    if (key == GBR_OPT_RIEMANN) {  // every case; the descriptors go up before the next launch
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        for (BatchCase& c : b->cases) c.ph.riemann = (int)val;
        b->dirty = true;
        return GBR_OK;
    }
    if (key == GBR_OPT_LAUNCH) {  // a cached graph of the other form is re-captured
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        b->per_tile = (int)val;
        return GBR_OK;
    }
    return GBR_ERR_ARG;
}

int gbr_batch_set_state(gbr_batch* b, int k, const double* Q, int on_device)
{
    if (!b || !Q || k < 0 || k >= b->n) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    const BatchCase& c = b->cases[k];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int m = 0; m < 4; ++m)
        TRY(cudaMemcpy2DAsync(c.q[0] + m * c.g.plane + (long long)kGhost * c.g.pitch + kGhost,
                              sizeof(double) * c.g.pitch, Q + (size_t)m * c.g.nx * c.g.ny, sizeof(double) * c.g.nx,
                              sizeof(double) * c.g.nx, c.g.ny, kind, b->stream));
    TRY(cudaMemsetAsync(c.ds, 0, sizeof(DevScalars), b->stream));
    TRY(launch_wavespeed(c.g, c.ph, c.q[0], &c.ds->lam[0], b->precision, b->stream));
    if (!on_device) TRY(cudaStreamSynchronize(b->stream));
    return GBR_OK;
}

int gbr_batch_get_state(gbr_batch* b, int k, double* Q, int on_device)
{
    if (!b || !Q || k < 0 || k >= b->n) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    const BatchCase& c = b->cases[k];
    for (int m = 0; m < 4; ++m)
        TRY(cudaMemcpy2DAsync(Q + (size_t)m * c.g.nx * c.g.ny, sizeof(double) * c.g.nx,
                              c.q[0] + m * c.g.plane + (long long)kGhost * c.g.pitch + kGhost,
                              sizeof(double) * c.g.pitch, sizeof(double) * c.g.nx, c.g.ny,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (!on_device) TRY(cudaStreamSynchronize(b->stream));
    return GBR_OK;
}

int gbr_batch_set_end_times(gbr_batch* b, const double* t_end)
{
    if (!b || !t_end) return GBR_ERR_ARG;
    for (int k = 0; k < b->n; ++k)
        if (!(t_end[k] >= 0.0)) return GBR_ERR_ARG;
    for (int k = 0; k < b->n; ++k) b->cases[k].t_end = t_end[k];
    b->dirty = true;
    return GBR_OK;
}

int gbr_batch_step_cfl(gbr_batch* b, double cfl, int nsteps)
{
    if (!b || !(cfl > 0.0) || nsteps < 1) return GBR_ERR_ARG;
    nvtxRangePushA("gbr batch steps");
    const int rc = batch_step_cfl(b, cfl, nsteps);
    nvtxRangePop();
    return rc;
}

int gbr_batch_step(gbr_batch* b, const double* dt_per_case)
{
    if (!b || !dt_per_case) return GBR_ERR_ARG;
    for (int k = 0; k < b->n; ++k)
        if (!(dt_per_case[k] >= 0.0) || !(dt_per_case[k] < 1e300)) return GBR_ERR_ARG;
    nvtxRangePushA("gbr batch step");
    DeviceGuard dg(b->device);
    int rc = upload(b);
    // the host array is staged by the copy before the call returns
    if (rc == GBR_OK)
        rc = st(cudaMemcpyAsync(b->d_dt, dt_per_case, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream));
    if (rc == GBR_OK) rc = enqueue_step(b, 0.0, b->stream, 3);
    nvtxRangePop();
    return rc;
}

int gbr_batch_get_times(gbr_batch* b, double* t, double* dt)
{
    if (!b) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    std::vector<DevScalars> h;
    int rc = check_errors(b, h);
    if (rc == GBR_ERR_CUDA || rc == GBR_ERR_NOMEM) return rc;
    for (int k = 0; k < b->n; ++k) {
        if (t) t[k] = h[k].t;
        if (dt) dt[k] = h[k].dt;
    }
    return rc;
}

int gbr_batch_autotune(gbr_batch* b, int trials, int* choice, int* bx, int* by)
{
    if (!b || trials < 1) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    const TileShape* sh;
    const int ns = shapes(b->precision, &sh);
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    int rc = GBR_OK;
    // Stage-1 launches read Q^n and write Q^(1) only: the states are kept.
    // The case dt words must be non-zero for tiles to run: use the stored dt
    // of the last step, or a tiny positive dt if no step was taken yet.
    std::vector<DevScalars> h(b->n);
    rc = st(cudaMemcpyAsync(h.data(), b->d_scal, sizeof(DevScalars) * b->n, cudaMemcpyDeviceToHost, b->stream));
    if (rc == GBR_OK) rc = st(cudaStreamSynchronize(b->stream));
    std::vector<DevScalars> tuned = h;
    for (auto& d : tuned)
        if (!(d.dt > 0.0)) d.dt = 1e-12;
    if (rc == GBR_OK)
        rc = st(cudaMemcpyAsync(b->d_scal, tuned.data(), sizeof(DevScalars) * b->n, cudaMemcpyHostToDevice,
                                b->stream));
    // candidate c: shape c % ns, launch form c / ns (0 persistent, 1 one CTA per tile)
    for (int c = 0; c < 2 * ns && rc == GBR_OK; ++c) {
        b->shape = c % ns;
        b->per_tile = c / ns;
        retile(b);
        if ((rc = upload(b)) != GBR_OK) break;
        rc = st(launch_batch_ghosts(b->d_cases, b->n, b->total_ghosts, 0, 0, 0.0, b->stream));
        if (rc == GBR_OK) rc = stage(b, 0, b->stream);  // warm-up and first-use setup
        if (rc != GBR_OK) break;
        rc = st(cudaEventRecord(e0, b->stream));
        for (int r = 0; r < trials && rc == GBR_OK; ++r) rc = stage(b, 0, b->stream);
        if (rc == GBR_OK) rc = st(cudaEventRecord(e1, b->stream));
        if (rc == GBR_OK) rc = st(cudaEventSynchronize(e1));
        float ms = 0.f;
        if (rc == GBR_OK) rc = st(cudaEventElapsedTime(&ms, e0, e1));
        if (rc == GBR_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // restore the scalars (dt, t, error word) and select the winner
    int rc2 = st(cudaMemcpyAsync(b->d_scal, h.data(), sizeof(DevScalars) * b->n, cudaMemcpyHostToDevice, b->stream));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape = best % ns;
    b->per_tile = best / ns;
    retile(b);
    if (rc == GBR_OK) rc = rc2;
    if (rc == GBR_OK) rc = upload(b);
    if (rc == GBR_OK) rc = st(cudaStreamSynchronize(b->stream));
    if (choice) *choice = best;
    if (bx) *bx = sh[best % ns].bx;
    if (by) *by = sh[best % ns].by;
    return rc;
}

int gbr_batch_set_sensor_weights(gbr_batch* b, const float* w, int n)
{
    if (!b || !w || n != kSensorParams) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    SensorDev h;
    pack_sensor(w, &h);
    if (!b->d_sensor) TRY(cudaMalloc(&b->d_sensor, sizeof(SensorDev)));
    if (!b->dec_pool) {
        size_t bytes = 0;
        for (const auto& c : b->cases) bytes += (size_t)c.g.pitch * (c.g.ny + 2 * kGhost);
        TRY(cudaMalloc(&b->dec_pool, bytes));
        TRY(cudaMemsetAsync(b->dec_pool, 2, bytes, b->stream));  // "unsure" outside the written regions
        size_t off = 0;
        for (auto& c : b->cases) {
            c.dec = b->dec_pool + off;
            off += (size_t)c.g.pitch * (c.g.ny + 2 * kGhost);
        }
        b->dirty = true;
        const int rc = upload(b);
        if (rc != GBR_OK) return rc;
    }
    TRY(cudaMemcpyAsync(b->d_sensor, &h, sizeof(SensorDev), cudaMemcpyHostToDevice, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    return GBR_OK;
}

int gbr_batch_sync(gbr_batch* b)
{
    if (!b) return GBR_ERR_ARG;
    DeviceGuard dg(b->device);
    std::vector<DevScalars> h;
    return check_errors(b, h);
}

}  // extern "C"
