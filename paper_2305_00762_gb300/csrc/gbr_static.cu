// gbr_step_static: one TVD-RK3 step of a caller-owned device state that
// allocates no device memory.
//
// Why it exists. gbr_step works on buffers that gbr_create allocates with
// cudaMalloc. Some callers cannot allocate at run time: a host application
// that owns all device memory through its own pool and forbids plugins to call
// cudaMalloc; a real-time loop that must not enter the driver's allocator
// (cudaMalloc can synchronise the device and take unbounded time); a process
// running close to the memory limit, where an allocation could fail halfway
// through a run. For them this entry point takes its scratch -- the padded
// copy of the input, the two Runge-Kutta stage states and the error word --
// from one file-scope __device__ array of fixed size that every GPU loading
// the library holds until the process exits.
//
// The kernels are the ones gbr_step launches; only where their scratch lives
// differs. The paper has no counterpart to this entry point.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/gbr.h"
#include "gbr_internal.h"

using namespace gbr;

// Scratch of gbr_step_static (GBR_STATIC_SCRATCH_DOUBLES doubles = 8 MiB):
// [0, 32): a DevScalars block (the error word is cleared by every call);
// then three padded FP64 states of 4 planes each (Q^n, Q^(1), Q^(2)).
static __device__ __align__(256) double g_static_scratch[GBR_STATIC_SCRATCH_DOUBLES];

namespace {

constexpr long long kHeader = 32;  // doubles reserved for the DevScalars block
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices];  // device address of the array, per device

// Once per device, with that device current: the device address of the
// array. In host code the name g_static_scratch is only a host-side stand-in
// and must never be passed to a kernel. Devices with an ordinal of
// kMaxDevices or more are not served (GBR_ERR_UNSUPPORTED).
int scratch_address(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return GBR_ERR_CUDA;
    }
    if (dev >= kMaxDevices) return GBR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GBR_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GBR_OK;
}

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return GBR_OK;
    cudaGetLastError();
    return GBR_ERR_CUDA;
}

}  // namespace

extern "C" int gbr_step_static(const double* Q_in, double* Q_out, int nx, int ny, double gamma, double mu,
                               double Pr, const gbr_bc* bc, double dt, void* stream)
{
    if (!Q_in || !Q_out || !bc) return GBR_ERR_ARG;
    if (nx < GBR_GHOST || ny < GBR_GHOST || !(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0) || !(dt > 0.0))
        return GBR_ERR_ARG;
    const int kinds[4] = {bc->west, bc->east, bc->south, bc->north};
    for (int k = 0; k < 4; ++k)
        if (kinds[k] < GBR_BC_PERIODIC || kinds[k] > GBR_BC_SYMMETRY) return GBR_ERR_ARG;
    if ((bc->west == GBR_BC_PERIODIC) != (bc->east == GBR_BC_PERIODIC) ||
        (bc->south == GBR_BC_PERIODIC) != (bc->north == GBR_BC_PERIODIC) || !(bc->dx > 0.0) || !(bc->dy > 0.0))
        return GBR_ERR_ARG;

    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.pitch = ((nx + 2 * kGhost + 15) / 16) * 16;
    g.plane = (((long long)g.pitch * (ny + 2 * kGhost) + 15) / 16) * 16;
    if (kHeader + 12 * g.plane > (long long)GBR_STATIC_SCRATCH_DOUBLES) return GBR_ERR_ARG;  // too large

    double* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != GBR_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    DevScalars* ds = reinterpret_cast<DevScalars*>(base);
    double* Qn = base + kHeader;
    double* Q1 = Qn + 4 * g.plane;
    double* Q2 = Q1 + 4 * g.plane;

    Physics ph{};  // value-initialised: MEG7-prim, HLLC
    ph.gamma = gamma;
    ph.mu = mu;
    ph.Pr = Pr;
    ph.dx = bc->dx;
    ph.dy = bc->dy;
    ph.order = 7;
    derive_physics(ph);

    // The array keeps the previous call's contents: clear the error word.
    if ((rc = status_of(cudaMemsetAsync(ds, 0, sizeof(DevScalars), s))) != GBR_OK) return rc;
    for (int m = 0; m < 4; ++m) {
        rc = status_of(cudaMemcpy2DAsync(Qn + m * g.plane + (long long)kGhost * g.pitch + kGhost,
                                         sizeof(double) * g.pitch, Q_in + (size_t)m * nx * ny, sizeof(double) * nx,
                                         sizeof(double) * nx, ny, cudaMemcpyDeviceToDevice, s));
        if (rc != GBR_OK) return rc;
    }

    GhostParams gp;
    memset(&gp, 0, sizeof(gp));
    gp.g = g;
    gp.bc[0] = bc->west;
    gp.bc[1] = bc->east;
    gp.bc[2] = bc->south;
    gp.bc[3] = bc->north;
    gp.ds = ds;
    gp.mode = 0;

    StageParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.g = g;
    sp.ph = ph;
    sp.qn = Qn;
    sp.err = &ds->err;
    sp.dt = dt;

    // Eq. rk with the same three fused passes as gbr_step.
    const double* in[3] = {Qn, Q1, Q2};
    double* out[3] = {Q1, Q2, Qn};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int k = 0; k < 3; ++k) {
        gp.q = const_cast<double*>(in[k]);
        if ((rc = status_of(launch_ghosts(gp, s))) != GBR_OK) return rc;
        sp.q = in[k];
        sp.qout = out[k];
        sp.ca = ca[k];
        sp.cb = cb[k];
        sp.cc = cc[k];
        if ((rc = status_of(launch_stage_f64(sp, s))) != GBR_OK) return rc;
    }
    for (int m = 0; m < 4; ++m) {
        rc = status_of(cudaMemcpy2DAsync(Q_out + (size_t)m * nx * ny, sizeof(double) * nx,
                                         Qn + m * g.plane + (long long)kGhost * g.pitch + kGhost,
                                         sizeof(double) * g.pitch, sizeof(double) * nx, ny,
                                         cudaMemcpyDeviceToDevice, s));
        if (rc != GBR_OK) return rc;
    }
    unsigned int err = 0;
    if ((rc = status_of(cudaMemcpyAsync(&err, &ds->err, sizeof(err), cudaMemcpyDeviceToHost, s))) != GBR_OK)
        return rc;
    if ((rc = status_of(cudaStreamSynchronize(s))) != GBR_OK) return rc;
    if (err & 2u) return GBR_ERR_TIMEOUT;
    return (err & 1u) ? GBR_ERR_NONPHYSICAL : GBR_OK;
}
