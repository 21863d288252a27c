"""Thin ctypes binding of the C ABI in include/gbr.h (argument marshalling
only; every step of the method runs in the CUDA library libgbr.so).

Functions keep the C names. Array arguments may be numpy arrays (host) or
torch CUDA tensors (device); the binding passes their pointers and the
matching on_device flag. The library must have been built
(``paper_2305_00762_gb300.build.build()``); there is no fallback path, so a
missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GBR_OK, GBR_ERR_ARG, GBR_ERR_CUDA, GBR_ERR_NONPHYSICAL = 0, -1, -2, -3
GBR_ERR_TIMEOUT, GBR_ERR_STATE, GBR_ERR_NOMEM, GBR_ERR_UNSUPPORTED = -4, -5, -6, -7
GBR_BC_PERIODIC, GBR_BC_TRANSMISSIVE, GBR_BC_NOSLIP_WALL, GBR_BC_SYMMETRY = 0, 1, 2, 3
GBR_BC_CUSTOM, GBR_BC_FIXED, GBR_BC_HALO = 4, 5, 6
GBR_OPT_PRECISION, GBR_OPT_RECORD_FLAGS, GBR_OPT_SENSOR, GBR_OPT_TIMING, GBR_OPT_ORDER = 0, 1, 2, 3, 4
GBR_OPT_VARIABLES, GBR_OPT_STALL_TEST, GBR_OPT_RIEMANN, GBR_OPT_LAUNCH = 5, 6, 7, 8
GBR_KERNEL_STAGE, GBR_KERNEL_GHOST, GBR_KERNEL_WAVESPEED, GBR_KERNEL_CLASSES = 0, 1, 2, 3
GBR_GHOST = 6
GBR_STATIC_SCRATCH_DOUBLES = 1 << 20
GBR_SENSOR_PARAMS = 2721

_lib = None


class GbrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} ({status})")


class gbr_bc(ctypes.Structure):
    _fields_ = [("west", ctypes.c_int), ("east", ctypes.c_int), ("south", ctypes.c_int),
                ("north", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class gbr_side(ctypes.Structure):
    _fields_ = [("kind_lo", ctypes.c_int), ("kind_hi", ctypes.c_int), ("s0", ctypes.c_double),
                ("speed", ctypes.c_double), ("lo", ctypes.c_double * 4), ("hi", ctypes.c_double * 4)]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libgbr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} missing (run paper_2305_00762_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    sig = {
        "gbr_create": (ip, [ip, ip, dp, dp, dp, ctypes.POINTER(gbr_bc), ctypes.POINTER(vp)]),
        "gbr_destroy": (ip, [vp]),
        "gbr_set_stream": (ip, [vp, vp]),
        "gbr_set_state": (ip, [vp, vp, ip]),
        "gbr_get_state": (ip, [vp, vp, ip]),
        "gbr_residual": (ip, [vp, vp, ip]),
        "gbr_step": (ip, [vp, dp]),
        "gbr_step_cfl": (ip, [vp, dp, dp]),
        "gbr_get_time": (ip, [vp, ctypes.POINTER(dp)]),
        "gbr_max_wavespeed": (ip, [vp, ctypes.POINTER(dp)]),
        "gbr_set_option": (ip, [vp, ip, dp]),
        "gbr_set_side": (ip, [vp, ip, ctypes.POINTER(gbr_side)]),
        "gbr_set_time": (ip, [vp, dp]),
        "gbr_get_flags": (ip, [vp, vp, vp, ip]),
        "gbr_get_timing": (ip, [vp, ctypes.POINTER(dp), ctypes.POINTER(ip), ctypes.POINTER(ip)]),
        "gbr_sync": (ip, [vp]),
        "gbr_step_static": (ip, [vp, vp, ip, ip, dp, dp, dp, ctypes.POINTER(gbr_bc), dp, vp]),
        "gbr_step_stage": (ip, [vp, ip, dp, dp, dp]),
        "gbr_halo_copy": (ip, [vp, ip, ip, vp, ip]),
        "gbr_lambda_word": (ip, [vp, ctypes.POINTER(vp)]),
        "gbr_lambda_max": (ip, [ctypes.POINTER(vp), ip]),
        "gbr_batch_create": (ip, [ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(dp),
                                  ctypes.POINTER(dp), ctypes.POINTER(ip), dp, ctypes.POINTER(vp)]),
        "gbr_batch_destroy": (ip, [vp]),
        "gbr_batch_set_stream": (ip, [vp, vp]),
        "gbr_batch_set_option": (ip, [vp, ip, dp]),
        "gbr_batch_set_state": (ip, [vp, ip, vp, ip]),
        "gbr_batch_get_state": (ip, [vp, ip, vp, ip]),
        "gbr_batch_set_end_times": (ip, [vp, ctypes.POINTER(dp)]),
        "gbr_batch_step_cfl": (ip, [vp, dp, ip]),
        "gbr_batch_step": (ip, [vp, ctypes.POINTER(ctypes.c_double)]),
        "gbr_batch_get_times": (ip, [vp, ctypes.POINTER(dp), ctypes.POINTER(dp)]),
        "gbr_batch_autotune": (ip, [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]),
        "gbr_batch_sync": (ip, [vp]),
        "gbr_batch_set_sensor_weights": (ip, [vp, ctypes.POINTER(ctypes.c_float), ip]),
        "gbr_set_sensor_weights": (ip, [vp, ctypes.POINTER(ctypes.c_float), ip]),
        "gbr_sensor_eval": (ip, [vp, vp, ip]),
        "gbr_sensor_dataset": (ip, [vp, vp, vp, vp]),
        "gbr_sensor_train": (ip, [vp, vp, ctypes.c_longlong, ip, ip, dp, dp, ctypes.c_ulonglong,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), vp]),
        "gbr_error_string": (ctypes.c_char_p, [ip]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def error_string(status: int) -> str:
    return load().gbr_error_string(int(status)).decode()


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(rc: int, what: str, allow=()):
    if rc != GBR_OK and rc not in allow:
        raise GbrError(rc, what)
    return rc


def gbr_create(nx, ny, gamma, mu, Pr, bc, dx, dy):
    b = gbr_bc(*[int(k) for k in bc], float(dx), float(dy))
    out = ctypes.c_void_p()
    _check(load().gbr_create(int(nx), int(ny), float(gamma), float(mu), float(Pr), ctypes.byref(b),
                             ctypes.byref(out)), "gbr_create")
    return out


def gbr_destroy(ctx):
    return _check(load().gbr_destroy(ctx), "gbr_destroy")


def gbr_set_stream(ctx, stream):
    return _check(load().gbr_set_stream(ctx, ctypes.c_void_p(int(stream or 0))), "gbr_set_stream")


def _expect(a, dtype, shape):
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
    name = str(a.dtype)
    if dtype not in name:
        raise ValueError(f"expected {dtype} data, got {name}")


def gbr_set_state(ctx, Q, nx, ny):
    _expect(Q, "float64", (4, ny, nx))
    p, dev = _ptr(Q)
    return _check(load().gbr_set_state(ctx, p, dev), "gbr_set_state")


def gbr_get_state(ctx, Q, nx, ny, allow=()):
    _expect(Q, "float64", (4, ny, nx))
    p, dev = _ptr(Q)
    return _check(load().gbr_get_state(ctx, p, dev), "gbr_get_state", allow)


def gbr_residual(ctx, R, nx, ny):
    _expect(R, "float64", (4, ny, nx))
    p, dev = _ptr(R)
    return _check(load().gbr_residual(ctx, p, dev), "gbr_residual")


def gbr_step(ctx, dt):
    return _check(load().gbr_step(ctx, float(dt)), "gbr_step")


def gbr_step_cfl(ctx, cfl, dt_max):
    return _check(load().gbr_step_cfl(ctx, float(cfl), float(dt_max)), "gbr_step_cfl")


def gbr_get_time(ctx, allow=()):
    t = ctypes.c_double()
    _check(load().gbr_get_time(ctx, ctypes.byref(t)), "gbr_get_time", allow)
    return t.value


def gbr_max_wavespeed(ctx, allow=()):
    lam = ctypes.c_double()
    rc = _check(load().gbr_max_wavespeed(ctx, ctypes.byref(lam)), "gbr_max_wavespeed", allow)
    return lam.value, rc


def gbr_set_option(ctx, key, val):
    return _check(load().gbr_set_option(ctx, int(key), float(val)), "gbr_set_option")


def gbr_set_side(ctx, side, kind_lo, kind_hi, s0=0.0, speed=0.0, lo=(1.0, 0.0, 0.0, 1.0), hi=(1.0, 0.0, 0.0, 1.0)):
    """Describe a GBR_BC_CUSTOM side (see gbr_side in gbr.h); lo, hi are
    primitive states (rho, u, v, p) used by GBR_BC_FIXED."""
    sd = gbr_side(int(kind_lo), int(kind_hi), float(s0), float(speed), (ctypes.c_double * 4)(*lo),
                  (ctypes.c_double * 4)(*hi))
    return _check(load().gbr_set_side(ctx, int(side), ctypes.byref(sd)), "gbr_set_side")


def gbr_get_flags(ctx, sigx, sigy, nx, ny):
    _expect(sigx, "uint8", (ny, nx + 1))
    _expect(sigy, "uint8", (ny + 1, nx))
    px, dx_ = _ptr(sigx)
    py, dy_ = _ptr(sigy)
    if dx_ != dy_:
        raise ValueError("flag buffers must both be host or both device")
    return _check(load().gbr_get_flags(ctx, px, py, dx_), "gbr_get_flags")


def gbr_get_timing(ctx):
    """{class: (total_ms, launches)} since the last call, and the number of
    launches that were counted but not timed."""
    ms = (ctypes.c_double * GBR_KERNEL_CLASSES)()
    n = (ctypes.c_int * GBR_KERNEL_CLASSES)()
    dropped = ctypes.c_int()
    _check(load().gbr_get_timing(ctx, ms, n, ctypes.byref(dropped)), "gbr_get_timing")
    names = ("stage", "ghost", "wavespeed")
    return {names[k]: (ms[k], n[k]) for k in range(GBR_KERNEL_CLASSES)}, dropped.value


def gbr_sync(ctx, allow=()):
    return _check(load().gbr_sync(ctx), "gbr_sync", allow)


def static_scratch_doubles(nx, ny):
    """Doubles of the static scratch array gbr_step_static needs for an
    nx x ny grid (it rejects grids above GBR_STATIC_SCRATCH_DOUBLES)."""
    pitch = (nx + 2 * GBR_GHOST + 15) // 16 * 16
    plane = (pitch * (ny + 2 * GBR_GHOST) + 15) // 16 * 16
    return 32 + 12 * plane


def gbr_step_static(Q_in, Q_out, nx, ny, gamma, mu, Pr, bc, dx, dy, dt, stream=0, allow=()):
    """One RK3 step of device tensors Q_in -> Q_out ([4][ny][nx] float64)
    that allocates no device memory (scratch in the library's static array).
    Raises ValueError for a grid beyond the array's capacity."""
    _expect(Q_in, "float64", (4, ny, nx))
    _expect(Q_out, "float64", (4, ny, nx))
    pin, din = _ptr(Q_in)
    pout, dout = _ptr(Q_out)
    if not (din and dout):
        raise ValueError("gbr_step_static takes device buffers")
    need = static_scratch_doubles(nx, ny)
    if need > GBR_STATIC_SCRATCH_DOUBLES:
        raise ValueError(f"grid {nx}x{ny} needs {need} doubles of static scratch; the library holds "
                         f"{GBR_STATIC_SCRATCH_DOUBLES} (about 270 x 270 cells at most)")
    b = gbr_bc(*[int(k) for k in bc], float(dx), float(dy))
    rc = load().gbr_step_static(pin, pout, int(nx), int(ny), float(gamma), float(mu), float(Pr),
                                ctypes.byref(b), float(dt), ctypes.c_void_p(int(stream or 0)))
    return _check(rc, "gbr_step_static", allow)


def _fvec(w, n):
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float32)).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} weights, got {a.size}")
    return a


def gbr_set_sensor_weights(ctx, w):
    a = _fvec(w, GBR_SENSOR_PARAMS)
    return _check(load().gbr_set_sensor_weights(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
                  "gbr_set_sensor_weights")


def gbr_sensor_eval(ctx, prob, nx, ny):
    _expect(prob, "float32", (ny, nx))
    p, dev = _ptr(prob)
    return _check(load().gbr_sensor_eval(ctx, p, dev), "gbr_sensor_eval")


def gbr_sensor_dataset(ctx, features, labels, targets=None):
    """features: device bfloat16 tensor [ncells, 64]; labels, targets: device
    uint8 tensors [ncells]; any of them may be None."""
    bufs = (features, labels, targets)
    for a in bufs:
        if a is not None and not _ptr(a)[1]:
            raise ValueError("gbr_sensor_dataset writes device buffers")
    pf, pl, pt = (_ptr(a)[0] if a is not None else None for a in bufs)
    return _check(load().gbr_sensor_dataset(ctx, pf, pl, pt), "gbr_sensor_dataset")


def gbr_sensor_train(features, targets, steps, batch, lr, pos_weight, seed, w0, stream=0):
    """Train from device features [n, 64] bf16 and targets [n] uint8 (units
    of 1/255); returns (trained weights, per-step loss)."""
    n = int(targets.shape[0])
    if tuple(features.shape) != (n, 64):
        raise ValueError("features must be [n, 64]")
    w = _fvec(w0, GBR_SENSOR_PARAMS).copy()
    loss = np.zeros(int(steps), np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load().gbr_sensor_train(_ptr(features)[0], _ptr(targets)[0], n, int(steps), int(batch), float(lr),
                                   float(pos_weight), int(seed) & (2**64 - 1), w.ctypes.data_as(fp),
                                   loss.ctypes.data_as(fp), ctypes.c_void_p(int(stream or 0))),
           "gbr_sensor_train")
    return w, loss


class Solver:
    """Convenience owner of one gbr context (marshalling only)."""

    def __init__(self, nx, ny, dx, dy, gamma=1.4, mu=0.0, Pr=0.72, bc=(GBR_BC_PERIODIC,) * 4,
                 precision=64, stream=None, order=7, cons=False, riemann=0):
        self.nx, self.ny = int(nx), int(ny)
        # construction arguments and custom sides, kept for checkpoints
        self.params = {"nx": int(nx), "ny": int(ny), "dx": float(dx), "dy": float(dy), "gamma": float(gamma),
                       "mu": float(mu), "Pr": float(Pr), "bc": tuple(int(k) for k in bc),
                       "precision": int(precision), "order": int(order), "cons": bool(cons),
                       "riemann": int(riemann)}
        self.sides = [None] * 4
        self.ctx = gbr_create(nx, ny, gamma, mu, Pr, bc, dx, dy)
        if stream is not None:
            gbr_set_stream(self.ctx, stream)
        if precision != 64:
            gbr_set_option(self.ctx, GBR_OPT_PRECISION, precision)
        if order != 7:
            gbr_set_option(self.ctx, GBR_OPT_ORDER, order)
        if cons:
            gbr_set_option(self.ctx, GBR_OPT_VARIABLES, 1)
        if riemann:
            gbr_set_option(self.ctx, GBR_OPT_RIEMANN, riemann)

    @classmethod
    def for_case(cls, case, **kw):
        s = cls(case.nx, case.ny, case.dx, case.dy, case.gamma, case.mu, case.Pr, case.bc, **kw)
        for k, sd in enumerate((case.meta or {}).get("sides", (None,) * 4)):
            if sd is not None:
                s.set_side(k, *sd)
        return s

    def set_side(self, k, kind_lo, kind_hi, s0=0.0, speed=0.0, lo=(1.0, 0.0, 0.0, 1.0), hi=(1.0, 0.0, 0.0, 1.0)):
        gbr_set_side(self.ctx, k, kind_lo, kind_hi, s0, speed, lo, hi)
        self.sides[k] = (int(kind_lo), int(kind_hi), float(s0), float(speed), tuple(map(float, lo)),
                         tuple(map(float, hi)))

    def close(self):
        if self.ctx is not None:
            gbr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, Q):
        gbr_set_state(self.ctx, Q, self.nx, self.ny)

    def get_state(self, out=None, allow=()):
        if out is None:
            out = np.empty((4, self.ny, self.nx))
        gbr_get_state(self.ctx, out, self.nx, self.ny, allow)
        return out

    def residual(self, out=None):
        if out is None:
            out = np.empty((4, self.ny, self.nx))
        gbr_residual(self.ctx, out, self.nx, self.ny)
        return out

    def step(self, dt):
        gbr_step(self.ctx, dt)

    def step_cfl(self, cfl, dt_max=1e300):
        gbr_step_cfl(self.ctx, cfl, dt_max)

    def time(self):
        return gbr_get_time(self.ctx)

    def set_time(self, t):
        _check(load().gbr_set_time(self.ctx, float(t)), "gbr_set_time")

    def max_wavespeed(self, allow=()):
        return gbr_max_wavespeed(self.ctx, allow)[0]

    def record_flags(self, on=True):
        gbr_set_option(self.ctx, GBR_OPT_RECORD_FLAGS, 1 if on else 0)

    def flags(self):
        sx = np.empty((self.ny, self.nx + 1), np.uint8)
        sy = np.empty((self.ny + 1, self.nx), np.uint8)
        gbr_get_flags(self.ctx, sx, sy, self.nx, self.ny)
        return sx, sy

    def timing(self, on=True):
        gbr_set_option(self.ctx, GBR_OPT_TIMING, 1 if on else 0)

    def set_sensor(self, w):
        """Load learned-sensor weights and switch the sensor on."""
        gbr_set_sensor_weights(self.ctx, w)
        gbr_set_option(self.ctx, GBR_OPT_SENSOR, 1)

    def sensor_eval(self):
        out = np.empty((self.ny, self.nx), np.float32)
        gbr_sensor_eval(self.ctx, out, self.nx, self.ny)
        return out

    def get_timing(self):
        return gbr_get_timing(self.ctx)

    def sync(self, allow=()):
        return gbr_sync(self.ctx, allow)

    # -- one slab of a grid split along y (see slab.py) --
    def step_stage(self, k, dt=0.0, cfl=0.0, dt_max=1e300):
        _check(load().gbr_step_stage(self.ctx, int(k), float(dt), float(cfl), float(dt_max)), "gbr_step_stage")

    def halo_copy(self, side, direction, buf):
        """direction 0: the six rows next to `side` into buf [4][6][nx];
        1: buf into the six ghost rows beyond `side` (a halo side)."""
        _expect(buf, "float64", (4, 6, self.nx))
        p, dev = _ptr(buf)
        _check(load().gbr_halo_copy(self.ctx, int(side), int(direction), ctypes.c_void_p(p), dev), "gbr_halo_copy")

    def lambda_word(self):
        """Device address of the current wavespeed word (uint64 bits of a double >= 0)."""
        w = ctypes.c_void_p()
        _check(load().gbr_lambda_word(self.ctx, ctypes.byref(w)), "gbr_lambda_word")
        return w.value


def lambda_max(solvers):
    """Reduce the wavespeed words of solvers on one device to their maximum."""
    arr = (ctypes.c_void_p * len(solvers))(*[s.ctx.value if isinstance(s.ctx, ctypes.c_void_p) else s.ctx
                                             for s in solvers])
    _check(load().gbr_lambda_max(arr, len(solvers)), "gbr_lambda_max")


class Batch:
    """Owner of one gbr batch of independent grids (marshalling only)."""

    def __init__(self, cases, precision=64, stream=None):
        L = load()
        n = len(cases)
        self.shapes = [(c.nx, c.ny) for c in cases]
        arr = lambda t, v: (t * len(v))(*v)
        nx = arr(ctypes.c_int, [c.nx for c in cases])
        ny = arr(ctypes.c_int, [c.ny for c in cases])
        dx = arr(ctypes.c_double, [c.dx for c in cases])
        dy = arr(ctypes.c_double, [c.dy for c in cases])
        bc = arr(ctypes.c_int, [int(k) for c in cases for k in c.bc])
        gamma = cases[0].gamma
        if any(c.gamma != gamma for c in cases) or any(c.mu != 0.0 for c in cases):
            raise ValueError("a batch shares one gamma and is inviscid")
        self.b = ctypes.c_void_p()
        _check(L.gbr_batch_create(n, nx, ny, dx, dy, bc, float(gamma), ctypes.byref(self.b)), "gbr_batch_create")
        self.n = n
        if stream is not None:
            _check(L.gbr_batch_set_stream(self.b, ctypes.c_void_p(int(stream))), "gbr_batch_set_stream")
        if precision != 64:
            self.set_option(GBR_OPT_PRECISION, precision)

    def set_option(self, key, val):
        _check(load().gbr_batch_set_option(self.b, int(key), float(val)), "gbr_batch_set_option")

    def close(self):
        if self.b is not None and self.b.value:
            load().gbr_batch_destroy(self.b)
        self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, k, Q):
        nx, ny = self.shapes[k]
        _expect(Q, "float64", (4, ny, nx))
        p, dev = _ptr(Q)
        _check(load().gbr_batch_set_state(self.b, int(k), p, dev), "gbr_batch_set_state")

    def get_state(self, k, out=None):
        nx, ny = self.shapes[k]
        if out is None:
            out = np.empty((4, ny, nx))
        _expect(out, "float64", (4, ny, nx))
        p, dev = _ptr(out)
        _check(load().gbr_batch_get_state(self.b, int(k), p, dev), "gbr_batch_get_state")
        return out

    def set_end_times(self, t_end):
        a = (ctypes.c_double * self.n)(*[float(x) for x in t_end])
        _check(load().gbr_batch_set_end_times(self.b, a), "gbr_batch_set_end_times")

    def step_cfl(self, cfl, nsteps=1):
        _check(load().gbr_batch_step_cfl(self.b, float(cfl), int(nsteps)), "gbr_batch_step_cfl")

    def step(self, dts):
        """One RK3 step of every grid at its own caller-supplied dt (0 skips)."""
        a = (ctypes.c_double * self.n)(*[float(x) for x in dts])
        _check(load().gbr_batch_step(self.b, a), "gbr_batch_step")

    def times(self, allow=()):
        t = (ctypes.c_double * self.n)()
        dt = (ctypes.c_double * self.n)()
        _check(load().gbr_batch_get_times(self.b, t, dt), "gbr_batch_get_times", allow)
        return np.array(t[:]), np.array(dt[:])

    def set_sensor(self, w):
        a = _fvec(w, GBR_SENSOR_PARAMS)
        _check(load().gbr_batch_set_sensor_weights(self.b, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                   a.size), "gbr_batch_set_sensor_weights")
        self.set_option(GBR_OPT_SENSOR, 1)

    def autotune(self, trials=3):
        c, bx, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().gbr_batch_autotune(self.b, int(trials), ctypes.byref(c), ctypes.byref(bx), ctypes.byref(by)),
               "gbr_batch_autotune")
        return c.value, (bx.value, by.value)

    def sync(self, allow=()):
        return _check(load().gbr_batch_sync(self.b), "gbr_batch_sync", allow)
