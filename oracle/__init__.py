"""Plain FP64 CPU oracle of the MEG7-prim residual (arXiv:2305.00762).

TEST INFRASTRUCTURE ONLY. ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers. The CUDA library in ``paper_2305_00762_gb300`` never imports this
package, and this package never imports it: the two share no code.

The arithmetic lives in ``meg7_oracle.c`` (plain loops, FP64,
``-ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
the scalar building blocks (each MP bound of Eq. mp-procedure on its own, the
characteristic eigenvector matrices), the detector, HLLC, the residual and
the RK3 step are pinned; the choices the paper leaves open (the state the
characteristic projection is frozen at, HLLC wave-speed bounds, 2D viscous
cross terms, ghost-layer count) are
"parity unpinned" with respect to the paper's intent, because the paper prints
no number that depends on them alone.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meg7_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmeg7_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_TRANSMISSIVE, BC_NOSLIP_WALL, BC_SYMMETRY = 0, 1, 2, 3
BC_CUSTOM, BC_FIXED = 4, 5  # a side described by Config.sides; inside it, a fixed primitive state
ERR_ARG, ERR_NONPHYSICAL = -1, -3
G = 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when the compiler supports it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Side(ctypes.Structure):
    _fields_ = [("kind_lo", ctypes.c_int), ("kind_hi", ctypes.c_int),
                ("s0", ctypes.c_double), ("speed", ctypes.c_double),
                ("lo", ctypes.c_double * 4), ("hi", ctypes.c_double * 4)]


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double),
                ("Pr", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("order", ctypes.c_int), ("cons", ctypes.c_int),
                ("t", ctypes.c_double), ("side", _Side * 4),
                ("riemann", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            u8 = ctypes.POINTER(ctypes.c_ubyte)
            cp = ctypes.POINTER(_Cfg)
            for name in ("or_grad6",):
                getattr(L, name).restype = ctypes.c_double
                getattr(L, name).argtypes = [dp]
            for name in ("or_grb_left", "or_grb_right", "or_meg7_left",
                         "or_meg7_right"):
                getattr(L, name).restype = ctypes.c_double
                getattr(L, name).argtypes = [dp, dp]
            L.or_grb_alphabeta_left.restype = ctypes.c_double
            L.or_grb_alphabeta_left.argtypes = [dp, dp, ctypes.c_double,
                                                ctypes.c_double]
            for name in ("or_flux_recon_left", "or_flux_recon_right",
                         "or_flux_recon4_left", "or_psi"):
                getattr(L, name).restype = ctypes.c_double
                getattr(L, name).argtypes = [dp]
            for name in ("or_hllc", "or_hllc_lm"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [ctypes.c_double, dp, dp, dp, dp, dp]
            L.or_residual.restype = ctypes.c_int
            L.or_residual.argtypes = [cp, dp, dp, u8, u8, u8]
            L.or_rk3_step.restype = ctypes.c_int
            L.or_rk3_step.argtypes = [cp, dp, ctypes.c_double]
            L.or_max_wavespeed.restype = ctypes.c_double
            L.or_max_wavespeed.argtypes = [cp, dp]
            L.or_fill_ghosts_padded.restype = ctypes.c_int
            L.or_fill_ghosts_padded.argtypes = [cp, dp]
            L.or_cons_eigenvectors.restype = None
            L.or_cons_eigenvectors.argtypes = [ctypes.c_double, dp, dp, dp]
            L.or_prim_eigenvectors.restype = None
            L.or_prim_eigenvectors.argtypes = [ctypes.c_double, dp, dp, dp]
            L.or_trouble_labels.restype = ctypes.c_int
            L.or_trouble_labels.argtypes = [cp, dp, u8]
            L.or_psi_min.restype = ctypes.c_int
            L.or_psi_min.argtypes = [cp, dp, dp]
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_ubyte)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _vec(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.shape != (n,):
        raise ValueError(f"expected {n} values, got shape {a.shape}")
    return a


@dataclass
class Config:
    """Grid and physics of one case (mirrors the CUDA library's arguments)."""
    nx: int
    ny: int
    dx: float
    dy: float
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 0.72
    bc: tuple = (BC_PERIODIC,) * 4   # west, east, south, north
    order: int = 7
    cons: int = 0                    # 1: MEG7-cons (conservative reconstruction)
    t: float = 0.0                   # time of the state (moving custom sides)
    # per side: None, or (kind_lo, kind_hi, s0, speed, lo (rho,u,v,p), hi) for BC_CUSTOM sides
    sides: tuple = (None, None, None, None)
    riemann: int = 0                 # 1: shock-stable HLLC-LM (reading R24)

    def c(self) -> _Cfg:
        sides = (_Side * 4)()
        for k, sd in enumerate(self.sides):
            if sd is not None:
                klo, khi, s0, speed, lo, hi = sd
                sides[k] = _Side(klo, khi, s0, speed, (ctypes.c_double * 4)(*lo), (ctypes.c_double * 4)(*hi))
            else:
                sides[k] = _Side(BC_TRANSMISSIVE, BC_TRANSMISSIVE, 0.0, 0.0)
        return _Cfg(self.nx, self.ny, self.dx, self.dy, self.gamma, self.mu,
                    self.Pr, (ctypes.c_int * 4)(*self.bc), self.order, self.cons, self.t, sides,
                    self.riemann)


# ---- scalar building blocks (pins) ----------------------------------------

def grad6(phi7):
    return lib().or_grad6(_dp(_vec(phi7, 7)))


def grb_left(phi5, dphi5):
    return lib().or_grb_left(_dp(_vec(phi5, 5)), _dp(_vec(dphi5, 5)))


def grb_right(phi5, dphi5):
    return lib().or_grb_right(_dp(_vec(phi5, 5)), _dp(_vec(dphi5, 5)))


def grb_alphabeta_left(phi5, dphi5, alpha, beta):
    return lib().or_grb_alphabeta_left(_dp(_vec(phi5, 5)), _dp(_vec(dphi5, 5)),
                                       float(alpha), float(beta))


def meg7_left(phi5, dphi5):
    return lib().or_meg7_left(_dp(_vec(phi5, 5)), _dp(_vec(dphi5, 5)))


def meg7_right(phi5, dphi5):
    return lib().or_meg7_right(_dp(_vec(phi5, 5)), _dp(_vec(dphi5, 5)))


def flux_recon_left(f9):
    return lib().or_flux_recon_left(_dp(_vec(f9, 9)))


def flux_recon_right(f9):
    return lib().or_flux_recon_right(_dp(_vec(f9, 9)))


def flux_recon4_left(f9):
    return lib().or_flux_recon4_left(_dp(_vec(f9, 9)))


def psi(rho5):
    return lib().or_psi(_dp(_vec(rho5, 5)))


def hllc(gamma, WL, WR, FL, FR, lm=False):
    """HLLC face flux (reading R7), or the shock-stable HLLC-LM (R24) if lm."""
    out = np.zeros(4)
    f = lib().or_hllc_lm if lm else lib().or_hllc
    f(float(gamma), _dp(_vec(WL, 4)), _dp(_vec(WR, 4)), _dp(_vec(FL, 4)), _dp(_vec(FR, 4)), _dp(out))
    return out


# ---- grid-level functions --------------------------------------------------

def _state(cfg: Config, Q) -> np.ndarray:
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    if Q.shape != (4, cfg.ny, cfg.nx):
        raise ValueError(f"state must be [4][ny][nx], got {Q.shape}")
    return Q


def residual(cfg: Config, Q, want_flags: bool = False, mask=None):
    """Res(Q) for the interior state Q ([4][ny][nx]); optionally the sigma
    flags of x faces ([ny][nx+1]) and y faces ([ny+1][nx]). With a boolean
    mask ([ny][nx]) only those cells are evaluated (others are NaN)."""
    Q = _state(cfg, Q)
    R = np.full_like(Q, np.nan) if mask is not None else np.zeros_like(Q)
    sx = np.zeros((cfg.ny, cfg.nx + 1), np.uint8) if want_flags else None
    sy = np.zeros((cfg.ny + 1, cfg.nx), np.uint8) if want_flags else None
    mk = None
    if mask is not None:
        mk = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        assert mk.shape == (cfg.ny, cfg.nx)
    rc = lib().or_residual(ctypes.byref(cfg.c()), _dp(Q), _dp(R), _u8(sx),
                           _u8(sy), _u8(mk))
    if rc != 0:
        raise RuntimeError(f"oracle residual failed: {rc}")
    return (R, sx, sy) if want_flags else R


def rk3_step(cfg: Config, Q, dt: float):
    """One TVD-RK3 step; returns (Q_new, status) with status 0 or -3."""
    Qn = _state(cfg, Q).copy()
    rc = lib().or_rk3_step(ctypes.byref(cfg.c()), _dp(Qn), float(dt))
    if rc not in (0, ERR_NONPHYSICAL):
        raise RuntimeError(f"oracle rk3 step failed: {rc}")
    return Qn, rc


def max_wavespeed(cfg: Config, Q) -> float:
    return lib().or_max_wavespeed(ctypes.byref(cfg.c()), _dp(_state(cfg, Q)))


def fill_ghosts_padded(cfg: Config, Qp) -> np.ndarray:
    Qp = np.ascontiguousarray(np.asarray(Qp, dtype=np.float64)).copy()
    assert Qp.shape == (4, cfg.ny + 2 * G, cfg.nx + 2 * G)
    rc = lib().or_fill_ghosts_padded(ctypes.byref(cfg.c()), _dp(Qp))
    if rc != 0:
        raise RuntimeError(f"oracle ghost fill failed: {rc}")
    return Qp


def cons_eigenvectors(gamma, w):
    """(L, R) eigenvector matrices of the conservative x-flux Jacobian at
    primitive state w = (rho, u, v, p), as the MEG7-cons face projection
    uses them (rows of L, columns of R)."""
    L = np.zeros(16)
    R = np.zeros(16)
    lib().or_cons_eigenvectors(float(gamma), _dp(_vec(w, 4)), _dp(L), _dp(R))
    return L.reshape(4, 4), R.reshape(4, 4)


def prim_eigenvectors(gamma, w):
    """(L, R) eigenvector matrices of the primitive-variable x-Jacobian at
    primitive state w = (rho, u, v, p), as the MEG7-prim face projection
    uses them (reading R2; rows of L, columns of R)."""
    L = np.zeros(16)
    R = np.zeros(16)
    lib().or_prim_eigenvectors(float(gamma), _dp(_vec(w, 4)), _dp(L), _dp(R))
    return L.reshape(4, 4), R.reshape(4, 4)


def trouble_labels(cfg: Config, Q) -> np.ndarray:
    """Plain-detector label per interior cell: psi_x < 0.5 or psi_y < 0.5."""
    Q = _state(cfg, Q)
    out = np.zeros((cfg.ny, cfg.nx), np.uint8)
    rc = lib().or_trouble_labels(ctypes.byref(cfg.c()), _dp(Q), _u8(out))
    if rc != 0:
        raise RuntimeError(f"oracle labels failed: {rc}")
    return out


def psi_min(cfg: Config, Q) -> np.ndarray:
    """min(psi_x, psi_y) of Eq. detector per interior cell, FP64."""
    Q = _state(cfg, Q)
    out = np.zeros((cfg.ny, cfg.nx))
    rc = lib().or_psi_min(ctypes.byref(cfg.c()), _dp(Q), _dp(out))
    if rc != 0:
        raise RuntimeError(f"oracle psi failed: {rc}")
    return out


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def run(cfg: Config, Q, t_end: float, cfl: float, max_steps: int = 10**9):
    """Advance to t_end with dt = min(cfl/lambda, t_end - t) per step
    (Sec. 2.5). Returns (Q, t, steps)."""
    import dataclasses
    Q = _state(cfg, Q).copy()
    t, n = 0.0, 0
    while t < t_end * (1 - 1e-14) and n < max_steps:
        dt = min(cfl / max_wavespeed(cfg, Q), t_end - t)
        Q, rc = rk3_step(dataclasses.replace(cfg, t=t), Q, dt)
        if rc != 0:
            raise RuntimeError("oracle: non-physical state")
        t += dt
        n += 1
    return Q, t, n
