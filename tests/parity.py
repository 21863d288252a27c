"""Helpers for the GPU-vs-oracle parity tests.

Tolerance: FP64 results must match the oracle to 1e-12 relative per field.
For a state the scale is max|Q_m| (momenta share one scale, max |rho u|,
|rho v|). For a residual the scale is the size of the terms it is made of:
Eq. deriv forms Res as differences of face fluxes divided by the cell size,
so its rounding error is relative to max|F_m|/dx + max|G_m|/dy, not to
max|Res_m| (which can be orders of magnitude smaller where the fluxes nearly
cancel: the oracle itself moves such a residual by ~1e-11 of max|Res| under
one-ulp input perturbations). The detector flag sigma is the
one discontinuous decision of the scheme; a face whose oracle psi lies within
1e-12 of psi_c = 0.5 may legitimately flip under a different rounding order,
so the cells next to such a face are excluded from the field comparison and
the flip itself is accepted. Every other flag must agree exactly.
"""
import numpy as np

TOL64 = 1e-12


def psi_field(O, Qrow_rho):
    """psi_k of Eq. detector for a 1D array of densities (oracle scalar)."""
    out = np.full(Qrow_rho.shape, np.nan)
    for k in range(2, len(Qrow_rho) - 2):
        out[k] = O.psi(Qrow_rho[k - 2:k + 3])
    return out


def tie_faces_ok(O, cfg, Q, sx_g, sx_o, sy_g, sy_o, tol=1e-12):
    """Check that every flag mismatch is a tie; return a cell mask of the
    cells adjacent to mismatched faces (to exclude from field checks)."""
    G = 6
    Qp = np.zeros((4, cfg.ny + 2 * G, cfg.nx + 2 * G))
    Qp[:, G:G + cfg.ny, G:G + cfg.nx] = Q
    Qp = O.fill_ghosts_padded(cfg, Qp)
    rho = Qp[0]
    excl = np.zeros((cfg.ny, cfg.nx), bool)
    for (i, jf) in zip(*np.nonzero(sx_g != sx_o)):
        j = jf - 1   # face j+1/2
        row = rho[i + G]
        psis = [O.psi(row[j + k + G - 2:j + k + G + 3]) for k in range(-2, 4)]
        assert abs(min(psis) - 0.5) < tol, f"x-face flag mismatch at row {i}, face {jf}: psi {min(psis)}"
        for jj in (j, j + 1):
            if 0 <= jj < cfg.nx:
                excl[i, jj] = True
    for (iface, j) in zip(*np.nonzero(sy_g != sy_o)):
        i = iface - 1
        col = rho[:, j + G]
        psis = [O.psi(col[i + k + G - 2:i + k + G + 3]) for k in range(-2, 4)]
        assert abs(min(psis) - 0.5) < tol, f"y-face flag mismatch at face {iface}, col {j}: psi {min(psis)}"
        for ii in (i, i + 1):
            if 0 <= ii < cfg.ny:
                excl[ii, j] = True
    return excl


def state_scales(Q):
    s = [np.nanmax(np.abs(Q[m])) for m in range(4)]
    mom = max(s[1], s[2])
    return [s[0], mom, mom, s[3]]


def residual_scales(Q, dx, dy, gamma, R=None):
    """max|F_m|/dx + max|G_m|/dy of the cell convective fluxes of Q (Sec. 1),
    at least max|R_m|."""
    rho, mu, mv, E = Q
    u, v = mu / rho, mv / rho
    p = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v))
    F = [mu, mu * u + p, mu * v, u * (E + p)]
    G = [mv, mv * u, mv * v + p, v * (E + p)]
    out = []
    for m in range(4):
        s = np.abs(F[m]).max() / dx + np.abs(G[m]).max() / dy
        if R is not None:
            s = max(s, np.nanmax(np.abs(R[m])))
        out.append(s)
    return out


def field_errors(a, b, exclude=None, scales=None):
    """Max error per field relative to scales[m] (default max|b_m|)."""
    errs = []
    for m in range(a.shape[0]):
        d = np.abs(a[m] - b[m])
        if exclude is not None:
            d = np.where(exclude, 0.0, d)
        scale = scales[m] if scales is not None else np.nanmax(np.abs(b[m]))
        errs.append(float(np.nanmax(d) / scale) if scale > 0 else float(np.nanmax(d)))
    return errs


def assert_close(a, b, tol=TOL64, exclude=None, what="", scales=None):
    errs = field_errors(a, b, exclude, scales)
    assert max(errs) <= tol, f"{what}: per-field max rel err {errs} > {tol}"
    return errs


def assert_state_close(a, b, tol=TOL64, what=""):
    return assert_close(a, b, tol, what=what, scales=state_scales(b))


def assert_residual_close(R, Ro, Q, case, tol=TOL64, exclude=None, what=""):
    """Residual parity against the flux scale (the pass criterion); the error
    against max|Res_m| itself is printed beside it, so the margin is visible
    (pytest -s or -rP shows it)."""
    sc = residual_scales(Q, case.dx, case.dy, case.gamma, Ro)
    errs = assert_close(R, Ro, tol, exclude, what, sc)
    own = field_errors(R, Ro, exclude)
    print(f"[residual parity] {what}: max err / flux scale {max(errs):.2e}, "
          f"/ max|Res_m| {max(own):.2e} (per field {', '.join(f'{e:.1e}' for e in own)})")
    return errs
