"""Plain numpy restatement of the learned discontinuity sensor (features,
BF16 rounding, the 50 -> 32 -> 32 -> 1 network and its decision).

TEST INFRASTRUCTURE ONLY, like the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's baseline legs use it. It shares no code
with the CUDA kernels. Every array operation is float32 and rounds after each
operation; BF16 values are float32 numbers with the low 16 bits cleared by
round-to-nearest-even.

Definition (the same as the library's): for interior cell c with 5 x 5
neighbourhood offsets k = (dy+2)*5 + (dx+2),
    f_k      = (rho_k - rho_c) / (max_k' |rho_k' - rho_c| + 1e-3)
    f_{25+k} = (p_k - p_c)     / (max_k' |p_k' - p_c| + 1e-3)
with rho, p the FP32 primitives of the state (ghost cells by the boundary
conditions); x = bf16(f); h1 = bf16(relu(x W1 + b1)) with W1 in BF16;
h2 = relu(h1 W2 + b2) with W2 in BF16; p = 1 / (1 + exp(-(h2 . w3 + b3))).
Decision: 1 (discontinuity) if p > 0.7, 0 (smooth) if p < 0.3, else 2 (the
plain detector decides).
"""
from __future__ import annotations

import numpy as np

from . import G, Config, fill_ghosts_padded

N_IN, N_H = 50, 32
TAU = 0.02  # width of the soft training target around psi_c = 0.5
N_PARAMS = N_IN * N_H + N_H + N_H * N_H + N_H + N_H + 1
FLOOR = np.float32(1e-3)
LO, HI = 0.3, 0.7


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def unpack(w):
    w = np.asarray(w, dtype=np.float32).reshape(-1)
    assert w.size == N_PARAMS
    o = 0
    W1 = w[o:o + N_IN * N_H].reshape(N_IN, N_H); o += N_IN * N_H
    b1 = w[o:o + N_H]; o += N_H
    W2 = w[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = w[o:o + N_H]; o += N_H
    w3 = w[o:o + N_H]; o += N_H
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def prims_fp32(cfg: Config, Q):
    """FP32 density and pressure of the ghost-filled padded state."""
    Qp = np.zeros((4, cfg.ny + 2 * G, cfg.nx + 2 * G))
    Qp[:, G:G + cfg.ny, G:G + cfg.nx] = Q
    Qp = fill_ghosts_padded(cfg, Qp)
    f = np.float32
    r = Qp[0].astype(f)
    ir = f(1) / r
    u = Qp[1].astype(f) * ir
    v = Qp[2].astype(f) * ir
    p = f(cfg.gamma - 1.0) * (Qp[3].astype(f) - f(0.5) * r * (u * u + v * v))
    return r, p


def features(cfg: Config, Q) -> np.ndarray:
    """[ny*nx, 50] float32 features (before BF16 rounding)."""
    r, p = prims_fp32(cfg, Q)
    ny, nx = cfg.ny, cfg.nx
    out = np.zeros((ny * nx, N_IN), np.float32)
    for fi, a in enumerate((r, p)):
        c = a[G:G + ny, G:G + nx]
        diffs = [a[G + dy:G + dy + ny, G + dx:G + dx + nx] - c for dy in range(-2, 3) for dx in range(-2, 3)]
        m = np.zeros_like(c)
        for d in diffs:
            m = np.maximum(m, np.abs(d))
        s = np.float32(1) / (m + FLOOR)
        for k, d in enumerate(diffs):
            out[:, 25 * fi + k] = (d * s).reshape(-1)
    return out


def features_at(cfg: Config, Q, rows, cols, prims=None) -> np.ndarray:
    """Features of the listed cells ([n, 50] float32, as features()); rows
    and cols are interior indices and may reach 3 cells into the ghost
    layers. prims: the (rho, p) pair of prims_fp32, if already computed."""
    r, p = prims if prims is not None else prims_fp32(cfg, Q)
    rows = np.asarray(rows, dtype=np.int64) + G
    cols = np.asarray(cols, dtype=np.int64) + G
    out = np.zeros((rows.size, N_IN), np.float32)
    for fi, a in enumerate((r, p)):
        c = a[rows, cols]
        diffs = [a[rows + dy, cols + dx] - c for dy in range(-2, 3) for dx in range(-2, 3)]
        m = np.zeros_like(c)
        for d in diffs:
            m = np.maximum(m, np.abs(d))
        s = np.float32(1) / (m + FLOOR)
        for k, d in enumerate(diffs):
            out[:, 25 * fi + k] = d * s
    return out


def direction_flags(p, trouble_x, trouble_y):
    """Per-direction detector flags of cells under the learned sensor, from
    its output p and the plain per-direction tests: p < LO no flag; LO..HI
    the plain test of that direction; p > HI the plain tests give the
    direction, and a cell neither test marks is flagged in both."""
    d = decision(p)
    tx = np.asarray(trouble_x, dtype=bool)
    ty = np.asarray(trouble_y, dtype=bool)
    fx = np.where(d == 0, False, tx | ((d == 1) & ~ty))
    fy = np.where(d == 0, False, ty | ((d == 1) & ~tx))
    return fx, fy


def forward(x, w) -> np.ndarray:
    """Network output p for features x [n, 50] (rounded to BF16 here)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    xb = bf16_round(x)
    h1 = bf16_round(np.maximum(xb @ bf16_round(W1) + b1, 0).astype(np.float32))
    h2 = np.maximum(h1 @ bf16_round(W2) + b2, 0).astype(np.float32)
    z = (h2 @ w3 + b3).astype(np.float32)
    return (np.float32(1) / (np.float32(1) + np.exp(-z))).astype(np.float32)


def decision(p) -> np.ndarray:
    p = np.asarray(p)
    return np.where(p > HI, 1, np.where(p < LO, 0, 2)).astype(np.uint8)


def soft_target(psi_min, tau=TAU) -> np.ndarray:
    """Training target of a cell in units of 1/255 (uint8): 255 / (1 +
    exp((psi_min - 1/2) / tau)) rounded half up, in FP64; psi_min =
    min(psi_x, psi_y) of Eq. detector (oracle.psi_min)."""
    t = 1.0 / (1.0 + np.exp((np.asarray(psi_min, dtype=np.float64) - 0.5) / tau))
    return np.floor(255.0 * t + 0.5).astype(np.uint8)
