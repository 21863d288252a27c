"""Exact solution of the 1D Riemann problem for an ideal gas (written from the
gas dynamics: the pressure function of the two nonlinear waves, its root p*
by Newton iteration, then sampling of the self-similar solution at x/t)."""
import numpy as np


def _f(p, rho, pk, g):
    """Velocity jump across the K wave as a function of the star pressure, and
    its derivative: shock branch for p > pK, rarefaction branch otherwise."""
    c = np.sqrt(g * pk / rho)
    if p > pk:
        A, B = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(WL, WR, g=1.4):
    rL, uL, pL = WL
    rR, uR, pR = WR
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _f(p, rL, pL, g)
        fR, dR = _f(p, rR, pR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        p = max(1e-12, p - dp)
        if abs(dp) < 1e-14 * p:
            break
    fL, _ = _f(p, rL, pL, g)
    fR, _ = _f(p, rR, pR, g)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(WL, WR, xi, g=1.4):
    """(rho, u, p) at x/t = xi for each entry of the array xi."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    ps, us = star_state(WL, WR, g)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:
                S = uL - cL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                w = (rL, uL, pL) if s < S else (rL * (ps / pL + gm) / (gm * ps / pL + 1), us, ps)
            else:
                csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
                if s < uL - cL:
                    w = (rL, uL, pL)
                elif s > us - csL:
                    w = (rL * (ps / pL) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    r = rL * (c / cL) ** (2 / (g - 1))
                    w = (r, u, pL * (c / cL) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pR:
                S = uR + cR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                w = (rR, uR, pR) if s > S else (rR * (ps / pR + gm) / (gm * ps / pR + 1), us, ps)
            else:
                csR = cR * (ps / pR) ** ((g - 1) / (2 * g))
                if s > uR + cR:
                    w = (rR, uR, pR)
                elif s < us + csR:
                    w = (rR * (ps / pR) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    r = rR * (c / cR) ** (2 / (g - 1))
                    w = (r, u, pR * (c / cR) ** (2 * g / (g - 1)))
        out[:, n] = w
    return out
