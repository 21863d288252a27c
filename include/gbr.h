/*
 * gbr.h -- C ABI of the GB300 (sm_103a) library for the seventh-order
 * gradient-based reconstruction scheme MEG7-prim of Chamarthi, "Efficient
 * high-order gradient-based reconstruction for compressible flows"
 * (arXiv:2305.00762): the per-Runge-Kutta-stage residual of the 2D
 * compressible Navier-Stokes equations on a uniform Cartesian grid.
 *
 * Conventions shared by every entry point
 * --------------------------------------
 * State layout. A state Q is the conservative vector (rho, rho u, rho v, E)
 * (Sec. 1, Eq. CNS-base) of the nx * ny interior cells, structure of arrays,
 * float64: Q[m * ny * nx + i * nx + j] for component m = 0..3, row i (y) and
 * column j (x), x fastest. Residuals use the same layout. Cell (j, i) has
 * centre (x0 + (j + 1/2) dx, y0 + (i + 1/2) dy).
 *
 * Pointers. Arguments named "on_device" select whether a buffer pointer is a
 * device pointer (1; it must be usable on the context's device and stream) or
 * host memory (0; pageable or pinned). The library only reads or writes
 * caller buffers during the call (host buffers) or in stream order before the
 * next synchronising call (device buffers); it keeps no caller pointer.
 *
 * Ownership. Every device buffer the solver needs (three padded states, the
 * residual scratch, reduction words) is allocated by gbr_create with
 * cudaMalloc and freed by gbr_destroy.
 *
 * Errors. Every call returns int: GBR_OK (0) or a negative gbr_status. No
 * call aborts, traps or prints. Errors raised asynchronously on the device
 * (a non-physical state; a tile-staging wait that gave up, GBR_ERR_TIMEOUT)
 * are reported by the next synchronising call (gbr_max_wavespeed,
 * gbr_get_state with a host buffer, gbr_sync) and stay set until
 * gbr_set_state. Calls with a NULL context or out-of-range arguments return
 * GBR_ERR_ARG and change nothing.
 *
 * Streams. All work is issued on the context's stream (the legacy default
 * stream until gbr_set_stream). Host-buffer transfers synchronise that stream.
 */
#ifndef GBR_H
#define GBR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Ghost layers per side. Sec. 2.3: the LC bound at face j+1/2 uses d_{j-1},
 * which uses Phi'_{j-2}, which uses Phi_{j-5}; face j-1/2 adds one cell. */
#define GBR_GHOST 6

typedef enum {
    GBR_OK = 0,
    GBR_ERR_ARG = -1,         /* NULL pointer, bad size or value */
    GBR_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    GBR_ERR_NONPHYSICAL = -3, /* a stage produced rho <= 0, p <= 0 or a non-finite value */
    GBR_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    GBR_ERR_STATE = -5,       /* call out of order (e.g. no state set yet) */
    GBR_ERR_NOMEM = -6,       /* device allocation failed */
    GBR_ERR_UNSUPPORTED = -7  /* option or mode not available */
} gbr_status;

/* Boundary conditions by ghost cells (Sec. 3, "ghost cell approach"; the
 * kinds used by Examples 1, 9 and 10). Periodic must be paired on opposite
 * sides. */
typedef enum {
    GBR_BC_PERIODIC = 0,     /* wrap around */
    GBR_BC_TRANSMISSIVE = 1, /* zero gradient: copy of the nearest interior cell */
    GBR_BC_NOSLIP_WALL = 2,  /* mirror; both velocity components change sign */
    GBR_BC_SYMMETRY = 3,     /* mirror; the normal velocity changes sign */
    /* The side is described by gbr_set_side (single-grid solvers only;
     * transmissive until set): fixed inflow states, and kinds that change
     * along the side at a point that may move with time, as the double Mach
     * reflection of Woodward and Colella needs (Example 8). */
    GBR_BC_CUSTOM = 4,
    /* Only inside gbr_side: ghost cells hold a fixed primitive state. */
    GBR_BC_FIXED = 5,
    /* South or north side of one slab of a grid split along y into slabs
     * (single-grid solvers only; not with GBR_BC_CUSTOM sides): its six ghost
     * rows are interior rows of the neighbouring slab, written by the caller
     * with gbr_halo_copy before every stage (gbr_step_stage). The library
     * fills only the west / east ghost cells of those rows, by the west /
     * east rule, as it does for interior rows. */
    GBR_BC_HALO = 6
} gbr_bc_kind;

/* Boundary kinds per side and the uniform cell sizes (the grid is
 * [x0, x0 + nx dx] x [y0, y0 + ny dy]; only dx, dy enter the scheme). */
typedef struct {
    int west, east, south, north; /* gbr_bc_kind */
    double dx, dy;                /* > 0 */
} gbr_bc;

/* A GBR_BC_CUSTOM side. Cells along the side are split at the tangential
 * coordinate s0 + speed * t (t: the stage's simulated time, see gbr_step;
 * coordinates of cell centres measured from the grid's lower-left corner,
 * i.e. (j + 1/2) dx along the south and north sides, (i + 1/2) dy along the
 * west and east sides). Ghost cells beside cells below the split point take
 * kind_lo, the others kind_hi: GBR_BC_TRANSMISSIVE, GBR_BC_NOSLIP_WALL,
 * GBR_BC_SYMMETRY, or GBR_BC_FIXED with the primitive state lo / hi
 * (rho > 0, u, v, p > 0). A corner ghost cell takes the south / north side's
 * fixed state if that side is fixed there, else the image across that side
 * of the west / east ghost cell (which is itself fixed or an image). */
typedef struct {
    int kind_lo, kind_hi;
    double s0, speed;
    double lo[4], hi[4];
} gbr_side;

/* Options for gbr_set_option. */
typedef enum {
    /* Arithmetic of the stencil, reconstruction and flux work: 64 (default)
     * or 32. The stage accumulation and the positivity check stay FP64. */
    GBR_OPT_PRECISION = 0,
    /* 1: record the detector flag sigma of every face of the next residual
     * or stage evaluation (read back with gbr_get_flags); 0: off (default). */
    GBR_OPT_RECORD_FLAGS = 1,
    /* Discontinuity sensor: 0 = the density detector of Sec. 2.4 (default);
     * 1 = the learned sensor evaluated by a separate decision pass before
     * each stage (the form batches use; the faster one); 2 = the learned
     * sensor's network evaluated inside the FP32 stage kernel on the tile it
     * has staged. Both take the same decisions; they need
     * gbr_set_sensor_weights first (else GBR_ERR_STATE), act in precision 32
     * only, and keep the density detector as fallback. */
    GBR_OPT_SENSOR = 2,
    /* 1: bracket every kernel launch with CUDA events on the context's
     * stream (read back with gbr_get_timing); 0: off (default). */
    GBR_OPT_TIMING = 3,
    /* Order of the gradient-based reconstruction: 7 (default; MEG7, alpha =
     * 38/7, beta = 3/190 in Eqs. good_6tth-order_scheme_flux and alpha-beta,
     * Eqs. grb, flux-full, flux-right) or 4 (the alpha = 4, beta = 0 member of
     * the same family, Sec. 3 Eq. fourth for the flux reconstruction). The MP
     * limiter, detector, Riemann solver and viscous flux are unchanged. */
    GBR_OPT_ORDER = 4,
    /* Reconstructed variables: 0 = primitive (MEG7-prim, default), 1 =
     * conservative (MEG7-cons: Q and its gradients projected with the
     * eigenvectors of the conservative flux Jacobian; the viscous terms take
     * their velocity and temperature gradients from the conservative ones by
     * the chain rule of Sec. 2.2). Order 7 only; the learned sensor is not
     * used with it (the density detector decides). */
    GBR_OPT_VARIABLES = 5,
    /* Failure-detection test hook: 1 makes every single-grid stage launch
     * wait for 16 bytes more than its tile copy delivers, so each CTA's
     * bounded staging wait gives up (after a few seconds) and the next
     * synchronising call reports GBR_ERR_TIMEOUT; the copy itself completes,
     * nothing faults, and gbr_set_state clears the error. 2: the learned
     * sensor's decision pass (FP32 with the sensor on) withholds its first
     * batch of tensor-core MMAs, so each CTA's bounded wait for their
     * completion gives up (no MMA is in flight; its tensor memory is freed)
     * and the next synchronising call reports GBR_ERR_TIMEOUT in the same
     * way. 0: off (default). */
    GBR_OPT_STALL_TEST = 6,
    /* Riemann solver of Eq. Riemann_revisit: 0 = HLLC (default); 1 = the
     * shock-stable HLLC of Fleischmann, Adami and Adams (2020), which
     * Examples 7 and 8 use against the carbuncle: the HLLC-LM flux, whose
     * acoustic terms |S_L|(Q*_L - Q_L) and |S_R|(Q_R - Q*_R) are scaled by
     * phi = sin(pi/2 min(1, Ma / 0.1)), Ma = max(|u_L|/c_L, |u_R|/c_R) over
     * the face-normal velocities. Faces at Ma >= 0.1 (every supersonic face)
     * keep plain HLLC. All precisions and reconstructions; batches too. */
    GBR_OPT_RIEMANN = 7,
    /* Batches only: launch form of the stage kernel, 1 = one CTA per tile
     * (default), 0 = a persistent grid of resident CTAs walking the tile
     * list. The same results either way; gbr_batch_autotune sets it. */
    GBR_OPT_LAUNCH = 8
} gbr_option;

/* Kernel classes reported by gbr_get_timing. */
typedef enum {
    GBR_KERNEL_STAGE = 0, /* fused residual + stage update (or residual only) */
    GBR_KERNEL_GHOST = 1, /* ghost-cell fill (+ per-step scalars) */
    GBR_KERNEL_WAVESPEED = 2, /* standalone CFL wavespeed reduction */
    GBR_KERNEL_CLASSES = 3
} gbr_kernel_class;

typedef struct gbr_ctx gbr_ctx; /* opaque, library-owned */

/* Create a solver for nx x ny interior cells (nx, ny >= GBR_GHOST) of an
 * ideal gas with ratio of specific heats gamma > 1 (Eq. pressure), constant
 * dynamic viscosity mu >= 0 (mu = 0: Euler) and Prandtl number Pr > 0
 * (Eqs. visc, visc-interface). bc: boundary kinds and cell sizes (read during
 * the call only). On success *out owns device memory of about
 * 3 * 32 (nx + 12)(ny + 12) + 32 nx ny bytes on the current CUDA device. */
int gbr_create(int nx, int ny, double gamma, double mu, double Pr, const gbr_bc *bc, gbr_ctx **out);

/* Free the context and its device memory (after synchronising its stream).
 * NULL is accepted and ignored. */
int gbr_destroy(gbr_ctx *ctx);

/* Issue all later work on `stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream; NULL = legacy default stream). */
int gbr_set_stream(gbr_ctx *ctx, void *stream);

/* Copy the state Q ([4][ny][nx], float64) into the solver (Sec. 1: the
 * conservative cell-centre point values). The state's CFL wavespeed is
 * computed on the device right away. */
int gbr_set_state(gbr_ctx *ctx, const double *Q, int on_device);

/* Copy the current state out ([4][ny][nx], float64). With a host buffer the
 * call synchronises and reports pending device errors. */
int gbr_get_state(gbr_ctx *ctx, double *Q, int on_device);

/* Res(Q) of the current state, Eqs. eqn-differencing_residual and deriv:
 * Res = -(F_{j+1/2} - F_{j-1/2})/dx - (G_{i+1/2} - G_{i-1/2})/dy with the
 * MEG7 convective flux (Secs. 2.2-2.4) and the alpha-damping viscous flux
 * (Sec. 2.1). res: [4][ny][nx] float64. With a host buffer the call
 * synchronises and reports GBR_ERR_TIMEOUT if the tile staging gave up. */
int gbr_residual(gbr_ctx *ctx, double *res, int on_device);

/* One third-order TVD Runge-Kutta step of size dt > 0 (Sec. 2.5, Eq. rk):
 * three fused residual + stage-update passes. Every stage state is checked
 * for rho > 0, p > 0 and finiteness in FP64; a failure is reported as
 * GBR_ERR_NONPHYSICAL by the next synchronising call. The new state's CFL
 * wavespeed is reduced in the last stage. Asynchronous. */
int gbr_step(gbr_ctx *ctx, double dt);

/* One RK3 step with dt = min(cfl / lambda(Q^n), dt_max) formed on the device
 * (Sec. 2.5), so that consecutive steps need no host synchronisation; the
 * simulated time advances by that dt (gbr_get_time). cfl > 0, dt_max > 0. */
int gbr_step_cfl(gbr_ctx *ctx, double cfl, double dt_max);

/* Describe side `side` (0 west, 1 east, 2 south, 3 north), which must have
 * been created as GBR_BC_CUSTOM. Read during the call; applies to all later
 * ghost fills. The RK stages of a step from time t with step dt see the
 * boundary at t, t + dt and t + dt/2 (the stage abscissae of Eq. rk). */
int gbr_set_side(gbr_ctx *ctx, int side, const gbr_side *s);

/* Set the simulated time of the current state (gbr_set_state resets it to
 * 0): the time GBR_BC_CUSTOM sides see, e.g. when a run resumes from a
 * saved state. Asynchronous, in stream order. */
int gbr_set_time(gbr_ctx *ctx, double t);

/* Simulated time accumulated by gbr_step / gbr_step_cfl since the last
 * gbr_set_state (synchronises). */
int gbr_get_time(gbr_ctx *ctx, double *t);

/* lambda = max over cells of max((|u|+c)/dx, (|v|+c)/dy, 4 nu/dx^2,
 * 4 nu/dy^2), c = sqrt(gamma p / rho), nu = mu / rho (Sec. 2.5: dt =
 * CFL / lambda). Synchronises; returns pending device errors. */
int gbr_max_wavespeed(gbr_ctx *ctx, double *lambda);

/* ----------------------------------------------------------------------
 * One grid split along y into slabs (one context per slab, e.g. one per GPU).
 * Eq. deriv's residual reaches six cells in each direction (reading of the
 * LC bound, see GBR_GHOST), so before each Runge-Kutta stage every slab needs
 * the six boundary rows of each neighbour at that stage. A step of a slab is
 * then: for k = 0, 1, 2: copy the six rows next to each GBR_BC_HALO side out
 * of every neighbour (gbr_halo_copy, dir 0) and into this slab's ghost rows
 * (dir 1), then gbr_step_stage(k); after stage 2, the wavespeeds of all slabs
 * are reduced to their maximum (gbr_lambda_word / gbr_lambda_max) so that
 * the next CFL step takes one dt everywhere (Sec. 2.5). With identical
 * inputs the slabs reproduce the single-grid step bit for bit.
 * ---------------------------------------------------------------------- */

/* Stage k (0, 1, 2) of a TVD-RK3 step (Eq. rk): the ghost fill of the
 * stage's input state and the fused residual + stage-update pass, as gbr_step
 * runs them. k = 0 starts a step: dt > 0 gives a fixed step; dt = 0 forms
 * dt = min(cfl / lambda, dt_max) on the device (cfl, dt_max > 0), lambda the
 * current wavespeed word. k = 1, 2 continue the step (dt, cfl, dt_max
 * ignored). Stages must come in the order 0, 1, 2 (else GBR_ERR_STATE).
 * Asynchronous. */
int gbr_step_stage(gbr_ctx *ctx, int k, double dt, double cfl, double dt_max);

/* Halo rows of the state the next gbr_step_stage reads. side: 2 south, 3
 * north. dir 0 (pack): copy the six interior rows next to that side (rows
 * 0..5 for south, ny-6..ny-1 for north, interior columns only) into buf;
 * dir 1 (unpack): copy buf into the six ghost rows beyond that side (rows
 * -6..-1 for south, ny..ny+5 for north; the side must be GBR_BC_HALO). buf:
 * [4][6][nx] float64, x fastest, rows in increasing y, on the device
 * (on_device = 1) or host. Device copies are asynchronous on the context's
 * stream; host copies synchronise it. */
int gbr_halo_copy(gbr_ctx *ctx, int side, int dir, double *buf, int on_device);

/* Device address of the context's current wavespeed word (the bits of a
 * double >= 0, so the largest word is the largest value): a max all-reduce
 * of these words across slabs after each step (e.g. NCCL, unsigned 64-bit
 * max) makes every slab's next CFL step use the global wavespeed. */
int gbr_lambda_word(gbr_ctx *ctx, unsigned long long **word);

/* The same reduction for 1 <= n <= 256 contexts on one device, between
 * steps: after it, each context's wavespeed word holds the maximum over the
 * n. Issued on ctx[0]'s stream (order the other contexts' streams before
 * it); GBR_ERR_ARG for contexts on different devices or in mid-step. */
int gbr_lambda_max(gbr_ctx *const *ctx, int n);

/* Set an option (gbr_option). Returns GBR_ERR_ARG for an unknown key or a
 * bad value, GBR_ERR_UNSUPPORTED for a mode that cannot run. */
int gbr_set_option(gbr_ctx *ctx, int key, double val);

/* Detector flags of the last evaluation made with GBR_OPT_RECORD_FLAGS on
 * (Eqs. detector and buffer): sigx [ny][nx+1] for the x faces j-1/2 .. nx-1/2
 * of every row, sigy [ny+1][nx] for the y faces; 1 = smooth (flux
 * reconstruction), 0 = discontinuity (MEG7 states). During a full step the
 * flags of the last stage are kept. */
int gbr_get_flags(gbr_ctx *ctx, unsigned char *sigx, unsigned char *sigy, int on_device);

/* Event timing recorded since the option was set or the last call:
 * ms[k] = summed device time (milliseconds) and launches[k] = launch count of
 * kernel class k (arrays of GBR_KERNEL_CLASSES entries, host memory).
 * Synchronises, then clears the record. At most 65536 launches are kept;
 * later ones are counted in launches[] but not timed (*dropped > 0). */
int gbr_get_timing(gbr_ctx *ctx, double *ms, int *launches, int *dropped);

/* ----------------------------------------------------------------------
 * Learned discontinuity sensor. A perceptron 50 -> 32 -> 32 -> 1 (ReLU, ReLU,
 * sigmoid) on the 5 x 5 stencil of density and pressure differences of a
 * cell, each field divided by (its largest absolute difference + 1e-3),
 * replaces the per-cell density-detector test of Sec. 2.4 (Eq. detector) in
 * the FP32 form: output < 0.3 marks smooth flow (no plain test is run), in
 * [0.3, 0.7] the plain detector decides (per direction), and > 0.7 marks a
 * discontinuity whose direction the plain per-direction tests assign (both
 * directions if neither test marks the cell). The buffer of Eq. buffer is
 * unchanged. The network runs on the tcgen05 tensor cores (BF16 operands,
 * FP32 accumulation in tensor memory), in a decision pass launched before
 * each FP32 stage (GBR_OPT_SENSOR = 1), or inside the FP32 stage kernel on
 * the cells the stage has staged (GBR_OPT_SENSOR = 2).
 * Weight vector (GBR_SENSOR_PARAMS floats): W1[50][32], b1[32], W2[32][32],
 * b2[32], w3[32], b3, with h1 = relu(x W1 + b1) rounded to BF16,
 * h2 = relu(h1 W2 + b2), p = 1/(1 + exp(-(h2 . w3 + b3))).
 * ---------------------------------------------------------------------- */
#define GBR_SENSOR_PARAMS 2721

/* Load sensor weights (host array of n = GBR_SENSOR_PARAMS floats). Enable
 * them with gbr_set_option(ctx, GBR_OPT_SENSOR, 1) (FP32 precision). */
int gbr_set_sensor_weights(gbr_ctx *ctx, const float *w, int n);

/* Network output p per interior cell of the current state ([ny][nx] float32),
 * computed from FP32 primitives as the FP32 stage kernel stages them, by the
 * same tcgen05 tensor-core pass that forms the stage's decisions. Errors:
 * GBR_ERR_STATE without a state or weights; GBR_ERR_TIMEOUT if a bounded
 * device wait gave up (reported here with host buffers, else by the next
 * synchronising call). */
int gbr_sensor_eval(gbr_ctx *ctx, float *prob, int on_device);

/* Training data from the current state (device buffers): features[ny*nx][64]
 * BF16 (row-major cells, zero-padded past 50); labels[ny*nx] = 1 where the
 * plain detector marks the cell (psi_x < 0.5 or psi_y < 0.5, FP64), else 0;
 * targets[ny*nx] = round(255 / (1 + exp((psi_min - 0.5) / 0.02))) with
 * psi_min = min(psi_x, psi_y) in FP64, the soft training target in units of
 * 1/255 (a cell within 0.016 of the threshold gets a target inside the
 * fallback band [0.3, 0.7]). Any of the three may be NULL, not all.
 * Asynchronous. */
int gbr_sensor_dataset(gbr_ctx *ctx, void *features, unsigned char *labels, unsigned char *targets);

/* Train the sensor on n samples (device buffers as written by
 * gbr_sensor_dataset; targets in units of 1/255, hard labels as 0 / 255):
 * `steps` Adam steps (learning rate lr) on mini-batches of `batch` samples
 * drawn with replacement by a counter-based hash of (seed, step, slot);
 * binary cross-entropy against target t with sample weight
 * 1 + (pos_weight - 1) t; BF16 operands, FP32 accumulation. w (host,
 * GBR_SENSOR_PARAMS floats) holds the initial weights on entry and the
 * trained ones on return; loss (host, `steps` floats, may be NULL) receives
 * each step's summed loss. Allocates temporary device memory; synchronises
 * `stream`. */
int gbr_sensor_train(const void *features, const unsigned char *targets, long long n, int steps, int batch,
                     double lr, double pos_weight, unsigned long long seed, float *w, float *loss, void *stream);

/* Wait for the context's stream and report pending device errors. */
int gbr_sync(gbr_ctx *ctx);

/* ----------------------------------------------------------------------
 * Batches: many independent inviscid grids of uneven size stepped together.
 * Every RK stage of every grid runs in one kernel launch over the batch's
 * tile list (one CTA per tile, or a persistent grid of resident CTAs that
 * walks the list, whichever gbr_batch_autotune measured faster; one CTA per
 * tile until then); each grid advances with its own
 * dt = min(cfl / lambda_k, t_end_k - t_k) formed on the device, so a call to
 * gbr_batch_step_cfl replays a CUDA graph of its nsteps steps without any
 * host synchronisation. Grids, gas and the scheme are as for gbr_create with
 * mu = 0; each grid's state is set and read like gbr_set_state /
 * gbr_get_state. Device memory: about 96 (nx+12)(ny+12) bytes per grid.
 * ---------------------------------------------------------------------- */
typedef struct gbr_batch gbr_batch; /* opaque, library-owned */

/* Create a batch of n >= 1 grids: grid k has nx[k] x ny[k] interior cells
 * (>= GBR_GHOST), cell sizes dx[k], dy[k] > 0 and boundary kinds
 * bc[4k .. 4k+3] (west, east, south, north: GBR_BC_PERIODIC to
 * GBR_BC_SYMMETRY; custom sides are for single-grid solvers only); all share
 * gamma > 1 (inviscid).
 * Host arrays, read during the call only. Precision defaults to 64. */
int gbr_batch_create(int n, const int *nx, const int *ny, const double *dx, const double *dy, const int *bc,
                     double gamma, gbr_batch **out);

/* Free the batch and its device memory (NULL accepted). */
int gbr_batch_destroy(gbr_batch *b);

/* Issue all later work of the batch on `stream` (NULL = legacy default). */
int gbr_batch_set_stream(gbr_batch *b, void *stream);

/* GBR_OPT_PRECISION (64 or 32, as for a single grid), GBR_OPT_SENSOR,
 * GBR_OPT_TIMING or GBR_OPT_RIEMANN (for every case), GBR_OPT_LAUNCH. */
int gbr_batch_set_option(gbr_batch *b, int key, double val);

/* Set grid k's state ([4][ny_k][nx_k] float64); resets its time to 0 and
 * computes its CFL wavespeed on the device. */
int gbr_batch_set_state(gbr_batch *b, int k, const double *Q, int on_device);

/* Copy grid k's state out (synchronises for host buffers). */
int gbr_batch_get_state(gbr_batch *b, int k, double *Q, int on_device);

/* Per-grid end times t_end[0..n-1] (host array; default: unbounded). A grid
 * whose time reached its t_end takes no further steps (dt = 0, no work). */
int gbr_batch_set_end_times(gbr_batch *b, const double *t_end);

/* nsteps >= 1 TVD-RK3 steps of every grid at its own CFL time step
 * (cfl > 0). The launch sequence (batched ghost fills and stage kernels) is
 * captured once into a CUDA graph per (nsteps, cfl, precision, tile shape,
 * launch form) and replayed. Asynchronous. */
int gbr_batch_step_cfl(gbr_batch *b, double cfl, int nsteps);

/* One TVD-RK3 step (Sec. 2.5, Eq. rk) of every grid at the caller's step
 * size: grid k advances by dt_per_case[k] >= 0 (host array of n finite
 * values, read during the call only); a grid at dt 0 is skipped (state, time
 * and wavespeed unchanged). For callers that run their own time control, e.g.
 * a common dt = CFL / max_k lambda_k, or fixed steps compared with a
 * reference. End times (gbr_batch_set_end_times) are not applied here. The
 * launches are issued directly (no graph) on the batch's stream;
 * asynchronous. GBR_ERR_ARG for a NULL pointer or a negative or non-finite
 * dt (nothing runs). */
int gbr_batch_step(gbr_batch *b, const double *dt_per_case);

/* Per-grid time t[k] and last step size dt[k] (host arrays of n entries, either
 * may be NULL). Synchronises; returns GBR_ERR_NONPHYSICAL if any grid's stage
 * produced rho <= 0, p <= 0 or a non-finite value. */
int gbr_batch_get_times(gbr_batch *b, double *t, double *dt);

/* Time every candidate tile shape of the current precision, each in both
 * launch forms (a persistent grid of resident CTAs walking the tile list, or
 * one CTA per tile), on the batch's own grids (`trials` launches of the
 * first RK stage each, which leave the states untouched) and keep the
 * fastest; *choice (may be NULL) receives its index, shape + S * form with S
 * the number of shapes and form 0 persistent, 1 one CTA per tile, and *bx,
 * *by (may be NULL) its shape. */
int gbr_batch_autotune(gbr_batch *b, int trials, int *choice, int *bx, int *by);

/* Sensor weights of the batch (as gbr_set_sensor_weights); enable with
 * gbr_batch_set_option(b, GBR_OPT_SENSOR, 1) in FP32 precision. */
int gbr_batch_set_sensor_weights(gbr_batch *b, const float *w, int n);

/* Wait for the batch's stream; reports pending device errors. */
int gbr_batch_sync(gbr_batch *b);

/* Capacity of the scratch array of gbr_step_static, in doubles (8 MiB). */
#define GBR_STATIC_SCRATCH_DOUBLES (1 << 20)

/* One TVD-RK3 step of size dt (the same kernels and result as gbr_step) of a
 * caller-owned device state, without allocating any device memory. The paper
 * has no counterpart to this entry point; it is for callers that cannot
 * call cudaMalloc at run time -- a host application that owns all device
 * memory through its own pool and forbids plugins to allocate, a real-time
 * loop that must not enter the driver's allocator (cudaMalloc may
 * synchronise the device and take unbounded time), a process running close
 * to its memory limit.
 *
 * Q_in, Q_out: device pointers, [4][ny][nx] float64 (layout as above); they
 * may be the same buffer. The grid, gas and boundary arguments mean what they
 * mean for gbr_create; dt > 0; stream: a cudaStream_t (NULL = legacy default
 * stream). The call is synchronous: it waits for the stream and returns
 * GBR_ERR_NONPHYSICAL if a stage produced rho <= 0, p <= 0 or a non-finite
 * value (the step is still completed and written).
 *
 * Scratch: a file-scope __device__ array of GBR_STATIC_SCRATCH_DOUBLES
 * doubles, held by every GPU that loads the library until the process exits.
 * A grid needs 32 + 12 * roundup16(roundup16(nx + 12) * (ny + 12)) doubles of
 * it, which admits up to about 270 x 270 cells (256 x 256 fits); a larger
 * grid returns GBR_ERR_ARG and nothing runs. Devices with ordinal 64 or more
 * return GBR_ERR_UNSUPPORTED.
 *
 * First call on a device. It looks up the array's device address for that
 * device (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture. With CUDA's default lazy module loading,
 * the code and the array are also loaded onto the device at that first call
 * (or at the first call of any other entry point there): the driver then
 * reserves device memory for the 8 MiB array and the kernels' code, which
 * takes time and can fail near the memory limit (GBR_ERR_CUDA). Callers that
 * must not see that should make one warm-up call at start-up, or run with
 * CUDA_MODULE_LOADING=EAGER. After that, calls allocate nothing: no
 * cudaMalloc, cudaFree or allocating library routine is called.
 *
 * All calls share the one array and each clears what must start at zero;
 * calls that overlap on the GPU (several host threads or streams at once)
 * race on it, so serialise them. */
int gbr_step_static(const double *Q_in, double *Q_out, int nx, int ny, double gamma, double mu, double Pr,
                    const gbr_bc *bc, double dt, void *stream);

/* Static text for a gbr_status value. */
const char *gbr_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GBR_H */
