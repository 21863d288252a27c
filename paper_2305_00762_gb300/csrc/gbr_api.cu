// Host implementation of the C ABI declared in include/gbr.h.
#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbr.h"
#include "gbr_internal.h"
#include "sensor.cuh"

using namespace gbr;

struct gbr_ctx {
    Grid g;
    Physics ph;
    int bc[4];
    int device;
    cudaStream_t stream;
    double* Qn;   // current state (padded)
    double* Qa;   // stage buffers (padded)
    double* Qb;
    double* R;    // residual scratch [4][ny][nx]
    DevScalars* ds;
    unsigned char* sigx;
    unsigned char* sigy;
    int precision;
    int record_flags;
    int sensor;
    int have_state;
    int lam_cur;
    int stage_next;  // next stage of a step run stage by stage (gbr_step_stage): 0 = no step in progress
    int step_mode;   // that step's dt: 1 = host value step_dt, 2 = CFL on the device
    double step_dt;
    // launch timing (GBR_OPT_TIMING)
    int timing;
    std::vector<cudaEvent_t> ev;   // pairs: start, stop
    std::vector<int> ev_class;
    int ev_used;
    int launches[GBR_KERNEL_CLASSES];
    int dropped;
    int stall_test;  // GBR_OPT_STALL_TEST
    SideBC side[4];  // GBR_BC_CUSTOM sides (transmissive until gbr_set_side)
    // learned sensor
    SensorDev* d_sensor;
    float* prob;          // per-cell sensor output scratch
    unsigned char* dec;   // learned-sensor decisions of the stage input (padded layout)
};

namespace {

struct DeviceGuard {  // make the context's device current for one call
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

// NVTX range of a host call (visible in Nsight timelines; a no-op without a
// profiler attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return GBR_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GBR_ERR_NOMEM : GBR_ERR_CUDA;
}

#define GBR_TRY(expr)                         \
    do {                                      \
        int rc_ = cuda_status(expr);          \
        if (rc_ != GBR_OK) return rc_;        \
    } while (0)

bool bc_ok(const gbr_bc* bc)
{
    const int k[4] = {bc->west, bc->east, bc->south, bc->north};
    bool halo = false, custom = false;
    for (int i = 0; i < 4; ++i) {
        if (k[i] < GBR_BC_PERIODIC || k[i] > GBR_BC_HALO || k[i] == GBR_BC_FIXED) return false;
        if (k[i] == GBR_BC_HALO && i < 2) return false;  // slabs split along y only
        halo |= k[i] == GBR_BC_HALO;
        custom |= k[i] == GBR_BC_CUSTOM;
    }
    if (halo && custom) return false;
    if ((bc->west == GBR_BC_PERIODIC) != (bc->east == GBR_BC_PERIODIC)) return false;
    if ((bc->south == GBR_BC_PERIODIC) != (bc->north == GBR_BC_PERIODIC)) return false;
    return bc->dx > 0.0 && bc->dy > 0.0;
}

int copy_state(gbr_ctx* c, double* dst_padded, const double* src, cudaMemcpyKind kind)
{
    for (int m = 0; m < 4; ++m) {
        GBR_TRY(cudaMemcpy2DAsync(dst_padded + m * c->g.plane + (long long)kGhost * c->g.pitch + kGhost,
                                  sizeof(double) * c->g.pitch, src + (size_t)m * c->g.nx * c->g.ny,
                                  sizeof(double) * c->g.nx, sizeof(double) * c->g.nx, c->g.ny, kind,
                                  c->stream));
    }
    return GBR_OK;
}

int read_back_errors(gbr_ctx* c, DevScalars* host)
{
    GBR_TRY(cudaMemcpyAsync(host, c->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    GBR_TRY(cudaStreamSynchronize(c->stream));
    if (host->err & 2u) return GBR_ERR_TIMEOUT;
    return (host->err & 1u) ? GBR_ERR_NONPHYSICAL : GBR_OK;
}

constexpr int kMaxTimed = 65536;

// Bracket one launch with events when timing is on.
struct Timed {
    gbr_ctx* c;
    int slot = -1;
    Timed(gbr_ctx* c_, int cls) : c(c_)
    {
        if (!c->timing) return;
        c->launches[cls]++;
        if (c->ev_used >= kMaxTimed) {
            c->dropped++;
            return;
        }
        if ((int)c->ev.size() < 2 * (c->ev_used + 1)) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
                cudaGetLastError();
                c->dropped++;
                return;
            }
            c->ev.push_back(a);
            c->ev.push_back(b);
            c->ev_class.push_back(cls);
        }
        slot = c->ev_used++;
        c->ev_class[slot] = cls;
        cudaEventRecord(c->ev[2 * slot], c->stream);
    }
    ~Timed()
    {
        if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], c->stream);
    }
};

int ghosts(gbr_ctx* c, double* q, int mode, double dt, double cfl, double dt_max, double c_stage = 0.0)
{
    Timed tm(c, GBR_KERNEL_GHOST);
    GhostParams p;
    memset(&p, 0, sizeof(p));
    p.g = c->g;
    p.q = q;
    for (int k = 0; k < 4; ++k) p.side[k] = c->side[k];
    p.dx = c->ph.dx;
    p.dy = c->ph.dy;
    p.c_stage = c_stage;
    for (int k = 0; k < 4; ++k) p.bc[k] = c->bc[k];
    p.ds = c->ds;
    p.mode = mode;
    p.cur = c->lam_cur;
    p.next = 1 - c->lam_cur;
    p.dt = dt;
    p.cfl = cfl;
    p.dt_max = dt_max;
    return cuda_status(launch_ghosts(p, c->stream));
}

StageParams stage_params(gbr_ctx* c, const double* q)
{
    StageParams p;
    memset(&p, 0, sizeof(p));
    p.g = c->g;
    p.ph = c->ph;
    p.q = q;
    p.qn = c->Qn;
    p.err = &c->ds->err;
    p.sigx = c->record_flags ? c->sigx : nullptr;
    p.sigy = c->record_flags ? c->sigy : nullptr;
    p.sensor = (c->sensor && c->precision == 32) ? c->d_sensor : nullptr;
    p.stall_bytes = c->stall_test == 1 ? 16u : 0u;
    return p;
}

int stage(gbr_ctx* c, const StageParams& p)
{
    Range r("gbr stage");
    Timed tm(c, GBR_KERNEL_STAGE);  // includes the learned sensor's decision pass
    if (c->precision == 32 && p.sensor) {
        StageParams q = p;
        if (c->sensor == 2) {  // the network fused into the stage kernel
            q.dec = nullptr;
            q.stall_mma = c->stall_test == 2 ? 1u : 0u;
            return cuda_status(launch_stage_f32(q, c->stream));
        }
        q.dec = c->dec;  // a separate decision pass, then the stage
        cudaError_t e =
            launch_sensor_decide(c->g, c->ph.gamma, p.q, p.sensor, c->dec, p.err, c->stall_test == 2, c->stream);
        if (e == cudaSuccess) e = launch_stage_f32(q, c->stream);
        return cuda_status(e);
    }
    cudaError_t e = (c->precision == 32) ? launch_stage_f32(p, c->stream) : launch_stage_f64(p, c->stream);
    return cuda_status(e);
}

// Input state of RK stage k (0, 1, 2).
double* stage_input(gbr_ctx* c, int k) { return k == 0 ? c->Qn : (k == 1 ? c->Qa : c->Qb); }

// Stage k of Eq. rk: Q1 = Qn + dt R(Qn); Q2 = 3/4 Qn + 1/4 Q1 + 1/4 dt R(Q1);
// Qn+1 = 1/3 Qn + 2/3 Q2 + 2/3 dt R(Q2): the ghost fill of the stage's input
// (the first one forms the step's scalars: mode 1 with the host dt, mode 2
// with dt from the CFL condition on the device; the stage times of the
// boundaries are t, t + dt, t + dt/2) and the fused stage pass. dt is a host
// value (mode 1) or the device word formed by the first ghost fill (mode 2).
int rk3_stage(gbr_ctx* c, int k, int mode, double dt, double cfl, double dt_max)
{
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    static const double c_stage[3] = {0.0, 1.0, 0.5};
    int rc;
    double* in = stage_input(c, k);
    if ((rc = ghosts(c, in, k == 0 ? mode : 0, dt, cfl, dt_max, c_stage[k])) != GBR_OK) return rc;
    StageParams p = stage_params(c, in);
    p.qout = k == 2 ? c->Qn : stage_input(c, k + 1);  // stage 3: each cell reads its own Q^n before writing it
    p.dt = dt;
    p.dt_ptr = (mode == 2) ? &c->ds->dt : nullptr;
    p.ca = ca[k];
    p.cb = cb[k];
    p.cc = cb[k];
    if (k == 2) p.lam_out = &c->ds->lam[1 - c->lam_cur];
    if ((rc = stage(c, p)) != GBR_OK) return rc;
    if (k == 2) c->lam_cur = 1 - c->lam_cur;
    return GBR_OK;
}

int rk3_step(gbr_ctx* c, int mode, double dt, double cfl, double dt_max)
{
    Range r("gbr step");
    int rc;
    for (int k = 0; k < 3; ++k)
        if ((rc = rk3_stage(c, k, mode, dt, cfl, dt_max)) != GBR_OK) return rc;
    return GBR_OK;
}

// The wavespeed words of up to kLambdaMax contexts on one device, passed by
// value to the reduction kernel.
constexpr int kLambdaMax = 256;
struct LambdaWords {
    unsigned long long* w[kLambdaMax];
    int n;
};

// One thread: the largest word (the largest non-negative double) written back
// to every context.
__global__ void lambda_max_kernel(const LambdaWords W)
{
    unsigned long long m = 0ull;
    for (int i = 0; i < W.n; ++i) m = *W.w[i] > m ? *W.w[i] : m;
    for (int i = 0; i < W.n; ++i) *W.w[i] = m;
}

}  // namespace

extern "C" {

int gbr_create(int nx, int ny, double gamma, double mu, double Pr, const gbr_bc* bc, gbr_ctx** out)
{
    if (!out || !bc) return GBR_ERR_ARG;
    *out = nullptr;
    if (nx < kGhost || ny < kGhost || !(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0) || !bc_ok(bc))
        return GBR_ERR_ARG;
    if ((long long)nx * ny > (1LL << 31)) return GBR_ERR_ARG;
    gbr_ctx* c = new (std::nothrow) gbr_ctx();  // value-initialised: scalars zero
    if (!c) return GBR_ERR_NOMEM;
    c->g.nx = nx;
    c->g.ny = ny;
    c->g.pitch = ((nx + 2 * kGhost + 15) / 16) * 16;
    c->g.plane = (((long long)c->g.pitch * (ny + 2 * kGhost) + 15) / 16) * 16;
    c->ph.gamma = gamma;
    c->ph.mu = mu;
    c->ph.Pr = Pr;
    c->ph.dx = bc->dx;
    c->ph.dy = bc->dy;
    c->ph.order = 7;
    derive_physics(c->ph);
    c->bc[0] = bc->west;
    c->bc[1] = bc->east;
    c->bc[2] = bc->south;
    c->bc[3] = bc->north;
    for (int k = 0; k < 4; ++k) {
        c->side[k].kind_lo = c->side[k].kind_hi = GBR_BC_TRANSMISSIVE;
        c->side[k].s0 = 0.0;
        c->side[k].speed = 0.0;
    }
    c->precision = 64;
    c->stream = 0;
    int rc = cuda_status(cudaGetDevice(&c->device));
    const size_t sbytes = sizeof(double) * 4 * (size_t)c->g.plane;
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&c->Qn, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&c->Qa, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&c->Qb, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&c->R, sizeof(double) * 4 * (size_t)nx * ny));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&c->ds, sizeof(DevScalars)));
    if (rc == GBR_OK) rc = cuda_status(cudaMemset(c->Qn, 0, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMemset(c->Qa, 0, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMemset(c->Qb, 0, sbytes));
    if (rc == GBR_OK) rc = cuda_status(cudaMemset(c->ds, 0, sizeof(DevScalars)));
    if (rc != GBR_OK) {
        gbr_destroy(c);
        return rc;
    }
    *out = c;
    return GBR_OK;
}

int gbr_destroy(gbr_ctx* c)
{
    if (!c) return GBR_OK;
    DeviceGuard dg(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    cudaFree(c->Qn);
    cudaFree(c->Qa);
    cudaFree(c->Qb);
    cudaFree(c->R);
    cudaFree(c->ds);
    cudaFree(c->sigx);
    cudaFree(c->sigy);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    cudaFree(c->d_sensor);
    cudaFree(c->prob);
    cudaFree(c->dec);
    cudaGetLastError();
    delete c;
    return GBR_OK;
}

int gbr_set_stream(gbr_ctx* c, void* stream)
{
    if (!c) return GBR_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return GBR_OK;
}

int gbr_set_state(gbr_ctx* c, const double* Q, int on_device)
{
    if (!c || !Q) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    int rc = copy_state(c, c->Qn, Q, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (rc != GBR_OK) return rc;
    GBR_TRY(cudaMemsetAsync(c->ds, 0, sizeof(DevScalars), c->stream));
    c->lam_cur = 0;
    c->stage_next = 0;
    {
        Timed tm(c, GBR_KERNEL_WAVESPEED);
        GBR_TRY(launch_wavespeed(c->g, c->ph, c->Qn, &c->ds->lam[0], c->precision, c->stream));
    }
    if (!on_device) GBR_TRY(cudaStreamSynchronize(c->stream));
    c->have_state = 1;
    return GBR_OK;
}

int gbr_get_state(gbr_ctx* c, double* Q, int on_device)
{
    if (!c || !Q) return GBR_ERR_ARG;
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    for (int m = 0; m < 4; ++m) {
        GBR_TRY(cudaMemcpy2DAsync(Q + (size_t)m * c->g.nx * c->g.ny, sizeof(double) * c->g.nx,
                                  c->Qn + m * c->g.plane + (long long)kGhost * c->g.pitch + kGhost,
                                  sizeof(double) * c->g.pitch, sizeof(double) * c->g.nx, c->g.ny,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
    if (on_device) return GBR_OK;
    DevScalars h;
    return read_back_errors(c, &h);
}

int gbr_residual(gbr_ctx* c, double* res, int on_device)
{
    if (!c || !res) return GBR_ERR_ARG;
    Range r("gbr residual");
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    int rc = ghosts(c, c->Qn, 0, 0, 0, 0);
    if (rc != GBR_OK) return rc;
    StageParams p = stage_params(c, c->Qn);
    p.res = on_device ? res : c->R;
    if ((rc = stage(c, p)) != GBR_OK) return rc;
    if (on_device) return GBR_OK;
    GBR_TRY(cudaMemcpyAsync(res, c->R, sizeof(double) * 4 * (size_t)c->g.nx * c->g.ny, cudaMemcpyDeviceToHost,
                            c->stream));
    DevScalars h;
    rc = read_back_errors(c, &h);  // synchronises
    if (rc == GBR_ERR_TIMEOUT || rc == GBR_ERR_CUDA) return rc;
    return GBR_OK;  // the non-physical flag concerns stage updates, not the residual
}

int gbr_step(gbr_ctx* c, double dt)
{
    if (!c || !(dt > 0.0)) return GBR_ERR_ARG;
    if (!c->have_state || c->stage_next != 0) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    return rk3_step(c, 1, dt, 0.0, 0.0);
}

int gbr_step_cfl(gbr_ctx* c, double cfl, double dt_max)
{
    if (!c || !(cfl > 0.0) || !(dt_max > 0.0)) return GBR_ERR_ARG;
    if (!c->have_state || c->stage_next != 0) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    return rk3_step(c, 2, 0.0, cfl, dt_max);
}

int gbr_step_stage(gbr_ctx* c, int k, double dt, double cfl, double dt_max)
{
    if (!c || k < 0 || k > 2) return GBR_ERR_ARG;
    if (k == 0 && !(dt > 0.0) && !(dt == 0.0 && cfl > 0.0 && dt_max > 0.0)) return GBR_ERR_ARG;
    if (!c->have_state || c->stage_next != k) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    Range r("gbr step stage");
    if (k == 0) {
        c->step_mode = dt > 0.0 ? 1 : 2;
        c->step_dt = dt;
    }
    const int rc = rk3_stage(c, k, c->step_mode, c->step_dt, cfl, dt_max);
    if (rc != GBR_OK) return rc;
    c->stage_next = (k + 1) % 3;
    return GBR_OK;
}

int gbr_halo_copy(gbr_ctx* c, int side, int dir, double* buf, int on_device)
{
    if (!c || !buf || (side != 2 && side != 3) || (dir != 0 && dir != 1)) return GBR_ERR_ARG;
    if (dir == 1 && c->bc[side] != GBR_BC_HALO) return GBR_ERR_ARG;
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    const int nx = c->g.nx, ny = c->g.ny;
    // padded row of the first of the six rows
    const int row = dir == 0 ? (side == 2 ? kGhost : ny) : (side == 2 ? 0 : ny + kGhost);
    double* q = stage_input(c, c->stage_next) + (long long)row * c->g.pitch + kGhost;
    const size_t spitch = sizeof(double) * c->g.pitch, bpitch = sizeof(double) * nx;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (dir == 0 ? cudaMemcpyDeviceToHost
                                                                           : cudaMemcpyHostToDevice);
    for (int m = 0; m < 4; ++m) {
        double* b = buf + (size_t)m * kGhost * nx;
        double* s = q + m * c->g.plane;
        if (dir == 0) GBR_TRY(cudaMemcpy2DAsync(b, bpitch, s, spitch, bpitch, kGhost, kind, c->stream));
        else GBR_TRY(cudaMemcpy2DAsync(s, spitch, b, bpitch, bpitch, kGhost, kind, c->stream));
    }
    if (!on_device) GBR_TRY(cudaStreamSynchronize(c->stream));
    return GBR_OK;
}

int gbr_lambda_word(gbr_ctx* c, unsigned long long** word)
{
    if (!c || !word) return GBR_ERR_ARG;
    *word = &c->ds->lam[c->lam_cur];
    return GBR_OK;
}

int gbr_lambda_max(gbr_ctx* const* ctx, int n)
{
    if (!ctx || n < 1 || n > kLambdaMax) return GBR_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctx[i] || ctx[i]->device != ctx[0]->device || ctx[i]->stage_next != 0) return GBR_ERR_ARG;
    DeviceGuard dg(ctx[0]->device);
    LambdaWords W;
    memset(&W, 0, sizeof(W));
    W.n = n;
    for (int i = 0; i < n; ++i) W.w[i] = &ctx[i]->ds->lam[ctx[i]->lam_cur];
    lambda_max_kernel<<<1, 1, 0, ctx[0]->stream>>>(W);
    return cuda_status(cudaGetLastError());
}

int gbr_get_time(gbr_ctx* c, double* t)
{
    if (!c || !t) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    DevScalars h;
    int rc = read_back_errors(c, &h);
    *t = h.t;
    return rc;
}

int gbr_max_wavespeed(gbr_ctx* c, double* lambda)
{
    if (!c || !lambda) return GBR_ERR_ARG;
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    DevScalars h;
    int rc = read_back_errors(c, &h);
    if (rc == GBR_ERR_CUDA || rc == GBR_ERR_NOMEM) return rc;
    unsigned long long bits = h.lam[c->lam_cur];
    double v;
    memcpy(&v, &bits, sizeof(v));
    *lambda = v;
    return rc;
}

int gbr_set_time(gbr_ctx* c, double t)
{
    if (!c || !std::isfinite(t)) return GBR_ERR_ARG;
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    return cuda_status(launch_set_time(c->ds, c->lam_cur, t, c->stream));
}

int gbr_set_side(gbr_ctx* c, int side, const gbr_side* sd)
{
    if (!c || !sd || side < 0 || side > 3 || c->bc[side] != GBR_BC_CUSTOM) return GBR_ERR_ARG;
    const int kinds[2] = {sd->kind_lo, sd->kind_hi};
    const double* prim[2] = {sd->lo, sd->hi};
    SideBC b;
    memset(&b, 0, sizeof(b));
    for (int h = 0; h < 2; ++h) {
        const int k = kinds[h];
        if (k != GBR_BC_TRANSMISSIVE && k != GBR_BC_NOSLIP_WALL && k != GBR_BC_SYMMETRY && k != GBR_BC_FIXED)
            return GBR_ERR_ARG;
        double* q = h ? b.qhi : b.qlo;
        if (k == GBR_BC_FIXED) {
            const double r = prim[h][0], u = prim[h][1], v = prim[h][2], p = prim[h][3];
            if (!(r > 0.0) || !(p > 0.0) || !std::isfinite(u) || !std::isfinite(v)) return GBR_ERR_ARG;
            q[0] = r;
            q[1] = r * u;
            q[2] = r * v;
            q[3] = p / (c->ph.gamma - 1.0) + 0.5 * r * (u * u + v * v);
        }
    }
    if (!std::isfinite(sd->s0) || !std::isfinite(sd->speed)) return GBR_ERR_ARG;
    b.kind_lo = sd->kind_lo;
    b.kind_hi = sd->kind_hi;
    b.s0 = sd->s0;
    b.speed = sd->speed;
    c->side[side] = b;
    return GBR_OK;
}

int gbr_set_option(gbr_ctx* c, int key, double val)
{
    if (!c) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    switch (key) {
    case GBR_OPT_PRECISION:
        if (val != 64.0 && val != 32.0) return GBR_ERR_ARG;
        c->precision = (int)val;
        return GBR_OK;
    case GBR_OPT_RECORD_FLAGS:
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        if (val == 1.0 && !c->sigx) {
            GBR_TRY(cudaMalloc(&c->sigx, (size_t)c->g.ny * (c->g.nx + 1)));
            GBR_TRY(cudaMalloc(&c->sigy, (size_t)(c->g.ny + 1) * c->g.nx));
            GBR_TRY(cudaMemset(c->sigx, 0, (size_t)c->g.ny * (c->g.nx + 1)));
            GBR_TRY(cudaMemset(c->sigy, 0, (size_t)(c->g.ny + 1) * c->g.nx));
        }
        c->record_flags = (int)val;
        return GBR_OK;
    case GBR_OPT_SENSOR:
        if (val != 0.0 && val != 1.0 && val != 2.0) return GBR_ERR_ARG;
        if (val != 0.0 && !c->d_sensor) return GBR_ERR_STATE;
        c->sensor = (int)val;
        return GBR_OK;
    case GBR_OPT_ORDER:
        if (val != 7.0 && val != 4.0) return GBR_ERR_ARG;
        if (val == 4.0 && c->ph.cons) return GBR_ERR_UNSUPPORTED;
        c->ph.order = (int)val;
        return GBR_OK;
    case GBR_OPT_VARIABLES:
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        if (val == 1.0 && c->ph.order != 7) return GBR_ERR_UNSUPPORTED;
        c->ph.cons = (int)val;
        return GBR_OK;
    case GBR_OPT_STALL_TEST:
        if (val != 0.0 && val != 1.0 && val != 2.0) return GBR_ERR_ARG;
        c->stall_test = (int)val;
        return GBR_OK;
    case GBR_OPT_RIEMANN:
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        c->ph.riemann = (int)val;
        return GBR_OK;
    case GBR_OPT_TIMING:
        if (val != 0.0 && val != 1.0) return GBR_ERR_ARG;
        c->timing = (int)val;
        c->ev_used = 0;
        c->dropped = 0;
        for (int k = 0; k < GBR_KERNEL_CLASSES; ++k) c->launches[k] = 0;
        return GBR_OK;
    default:
        return GBR_ERR_ARG;
    }
}

int gbr_get_timing(gbr_ctx* c, double* ms, int* launches, int* dropped)
{
    if (!c || !ms || !launches) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    GBR_TRY(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < GBR_KERNEL_CLASSES; ++k) {
        ms[k] = 0.0;
        launches[k] = c->launches[k];
        c->launches[k] = 0;
    }
    for (int s = 0; s < c->ev_used; ++s) {
        float t = 0.f;
        GBR_TRY(cudaEventElapsedTime(&t, c->ev[2 * s], c->ev[2 * s + 1]));
        ms[c->ev_class[s]] += t;
    }
    if (dropped) *dropped = c->dropped;
    c->ev_used = 0;
    c->dropped = 0;
    return GBR_OK;
}

int gbr_get_flags(gbr_ctx* c, unsigned char* sigx, unsigned char* sigy, int on_device)
{
    if (!c || !sigx || !sigy) return GBR_ERR_ARG;
    if (!c->sigx) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    GBR_TRY(cudaMemcpyAsync(sigx, c->sigx, (size_t)c->g.ny * (c->g.nx + 1), k, c->stream));
    GBR_TRY(cudaMemcpyAsync(sigy, c->sigy, (size_t)(c->g.ny + 1) * c->g.nx, k, c->stream));
    if (!on_device) GBR_TRY(cudaStreamSynchronize(c->stream));
    return GBR_OK;
}

int gbr_set_sensor_weights(gbr_ctx* c, const float* w, int n)
{
    if (!c || !w || n != kSensorParams) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    SensorDev h;
    pack_sensor(w, &h);
    if (!c->d_sensor) GBR_TRY(cudaMalloc(&c->d_sensor, sizeof(SensorDev)));
    if (!c->dec) {
        const size_t bytes = (size_t)c->g.pitch * (c->g.ny + 2 * kGhost);
        GBR_TRY(cudaMalloc(&c->dec, bytes));
        GBR_TRY(cudaMemsetAsync(c->dec, 2, bytes, c->stream));  // "unsure" outside the written region
    }
    GBR_TRY(cudaMemcpyAsync(c->d_sensor, &h, sizeof(SensorDev), cudaMemcpyHostToDevice, c->stream));
    GBR_TRY(cudaStreamSynchronize(c->stream));
    return GBR_OK;
}

int gbr_sensor_eval(gbr_ctx* c, float* prob, int on_device)
{
    if (!c || !prob) return GBR_ERR_ARG;
    if (!c->have_state || !c->d_sensor) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    int rc = ghosts(c, c->Qn, 0, 0, 0, 0);
    if (rc != GBR_OK) return rc;
    const size_t n = (size_t)c->g.nx * c->g.ny;
    float* out = prob;
    if (!on_device) {
        if (!c->prob) GBR_TRY(cudaMalloc(&c->prob, sizeof(float) * n));
        out = c->prob;
    }
    GBR_TRY(launch_sensor_tile(c->g, c->ph.gamma, c->Qn, c->d_sensor, out, nullptr, nullptr, nullptr, &c->ds->err,
                               c->stream));
    if (!on_device) {
        GBR_TRY(cudaMemcpyAsync(prob, c->prob, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
        DevScalars h;
        rc = read_back_errors(c, &h);  // synchronises
        if (rc == GBR_ERR_TIMEOUT || rc == GBR_ERR_CUDA) return rc;
    }
    return GBR_OK;
}

int gbr_sensor_dataset(gbr_ctx* c, void* features, unsigned char* labels, unsigned char* targets)
{
    if (!c || (!features && !labels && !targets)) return GBR_ERR_ARG;
    if (!c->have_state) return GBR_ERR_STATE;
    DeviceGuard dg(c->device);
    int rc = ghosts(c, c->Qn, 0, 0, 0, 0);
    if (rc != GBR_OK) return rc;
    return cuda_status(
        launch_sensor_tile(c->g, c->ph.gamma, c->Qn, nullptr, nullptr, features, labels, targets, nullptr, c->stream));
}

int gbr_sensor_train(const void* features, const unsigned char* targets, long long n, int steps, int batch,
                     double lr, double pos_weight, unsigned long long seed, float* w, float* loss, void* stream)
{
    if (!features || !targets || !w || n < 1 || steps < 1 || batch < 1 || !(lr > 0.0) || !(pos_weight > 0.0))
        return GBR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *dw = nullptr, *dg = nullptr, *dm = nullptr, *dv = nullptr, *dl = nullptr;
    const size_t pb = sizeof(float) * kSensorParams;
    int rc = cuda_status(cudaMalloc(&dw, pb));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&dg, pb));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&dm, pb));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&dv, pb));
    if (rc == GBR_OK) rc = cuda_status(cudaMalloc(&dl, sizeof(float) * steps));
    if (rc == GBR_OK) rc = cuda_status(cudaMemcpyAsync(dw, w, pb, cudaMemcpyHostToDevice, s));
    if (rc == GBR_OK) rc = cuda_status(cudaMemsetAsync(dg, 0, pb, s));
    if (rc == GBR_OK) rc = cuda_status(cudaMemsetAsync(dm, 0, pb, s));
    if (rc == GBR_OK) rc = cuda_status(cudaMemsetAsync(dv, 0, pb, s));
    if (rc == GBR_OK) rc = cuda_status(cudaMemsetAsync(dl, 0, sizeof(float) * steps, s));
    if (rc == GBR_OK)
        rc = cuda_status(launch_sensor_train(features, targets, n, steps, batch, (float)lr, (float)pos_weight, seed,
                                             dw, dg, dm, dv, dl, s));
    if (rc == GBR_OK) rc = cuda_status(cudaMemcpyAsync(w, dw, pb, cudaMemcpyDeviceToHost, s));
    if (rc == GBR_OK && loss) rc = cuda_status(cudaMemcpyAsync(loss, dl, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
    if (rc == GBR_OK) rc = cuda_status(cudaStreamSynchronize(s));
    cudaFree(dw);
    cudaFree(dg);
    cudaFree(dm);
    cudaFree(dv);
    cudaFree(dl);
    return rc;
}

int gbr_sync(gbr_ctx* c)
{
    if (!c) return GBR_ERR_ARG;
    DeviceGuard dg(c->device);
    DevScalars h;
    return read_back_errors(c, &h);
}

const char* gbr_error_string(int status)
{
    switch (status) {
    case GBR_OK: return "ok";
    case GBR_ERR_ARG: return "invalid argument";
    case GBR_ERR_CUDA: return "CUDA runtime error";
    case GBR_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or non-finite)";
    case GBR_ERR_TIMEOUT: return "bounded device wait timed out";
    case GBR_ERR_STATE: return "call out of order (no state set)";
    case GBR_ERR_NOMEM: return "device allocation failed";
    case GBR_ERR_UNSUPPORTED: return "unsupported option or mode";
    default: return "unknown status";
    }
}

}  // extern "C"
