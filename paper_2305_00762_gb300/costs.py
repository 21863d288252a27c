"""Algorithmic work of one cell-update (one interior cell through one RK
stage) of the MEG7-prim residual, used for roofline fractions.

Counts are of the method as defined (arXiv:2305.00762, Secs. 2.1-2.5), on the
smooth-region path (sigma = 1, MP condition satisfied, which is the common
case): each add, subtract, multiply, divide and square root counts as one
floating-point operation, comparisons and absolute values as none. Every
cell owns one x face and one y face, so a cell-update costs the per-cell work
plus two face evaluations plus its share of the stage update.
"""

# Per cell, both directions (done once per cell):
PER_CELL = {
    "cons_to_prim": 9,          # u = m/rho, v (2 div), p: 7
    "gradients_eq_six": 64,     # 8 flops x 4 primitives x 2 directions
    "detector_eq_detector": 36,  # a, b, 2ab+eps, a^2+b^2+eps, ratio; x and y
    "cell_fluxes": 18,          # E (6) + F^c (6) + G^c (6)
}

# Per face (x or y), Secs. 2.2-2.4:
PER_FACE = {
    "detector_buffer": 5,       # min over psi_{j-2..j+3}
    "eigen_setup": 12,          # mean state, c = sqrt(gamma p / rho), 1/c, rho/(2c), 1/(2c^2)
    "projection": 72,           # U and U' of 6 cells onto 4 left eigenvectors (sparse)
    "grb_left_right": 104,      # Eq. grb: 13 flops x 4 fields x 2 sides
    "mp_condition": 72,         # Eqs. alpha and mp5Condition: 9 flops x 8
    "back_projection": 14,      # right eigenvectors, 2 sides
    "prim_to_cons": 16,         # Q_L, Q_R
    "flux_reconstruction": 136,  # Eqs. flux-full / flux-right: 17 flops x 4 x 2
    "hllc": 122,                # Roe averages, wave speeds, star states, |A| dQ, central part
}

PER_FACE_VISCOUS = 50          # alpha-damping gradients of u, v, T; tau, q (Sec. 2.1)

PER_CELL_UPDATE = {
    "residual_eq_deriv": 20,    # 4 components: two differences, two scalings, one add
    "stage_update_fp64": 20,    # a Q^n + b Q^(k) + c dt Res, 4 components
    "positivity_fp64": 6,
    "wavespeed_share": 5,       # once per step (fused into stage 3)
}


def fp64_flop_per_cell_update(viscous: bool = False) -> int:
    face = sum(PER_FACE.values()) + (PER_FACE_VISCOUS if viscous else 0)
    return sum(PER_CELL.values()) + 2 * face + sum(PER_CELL_UPDATE.values())


def hbm_bytes_per_cell_update() -> float:
    """Compulsory HBM traffic of the fused stage with FP64 state (halo
    re-reads served from L2): stage 1 reads Q^n and writes Q^(1) (64 B),
    stages 2 and 3 read Q^(k) and Q^n and write (96 B each): 256/3 B."""
    return (64.0 + 96.0 + 96.0) / 3.0
