"""Seeded synthetic inputs: the initial conditions of the benchmark cases.

This module is shared by the CUDA-path tests, the oracle tests and the
benchmark. It holds initial and exact solutions of the flows only, none of the
scheme's arithmetic. Every state is returned as conservative variables
(rho, rho u, rho v, E) in structure-of-arrays form ``[4][ny][nx]`` (x fastest),
float64, with cell centres at x_j = x0 + (j + 1/2) dx.

Cases (Sec. 3 of the paper, plus the synthetic ensemble members):

* ``isentropic_vortex`` -- Example 1 (order of accuracy), on a periodic square.
* ``riemann_2d``       -- Example 9 (Schulz-Rinne 2D Riemann problem).
* ``viscous_shock_tube`` -- Example 10 (Daru-Tenaud), Re = 1000.
* ``kelvin_helmholtz`` -- seeded periodic shear layer (ensemble member).
* ``entropy_wave``, ``free_stream``, ``shear_wave`` -- exact-solution checks.
* ``ensemble``         -- seeded table of uneven vortex / shear-layer cases.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BC_PERIODIC, BC_TRANSMISSIVE, BC_NOSLIP_WALL, BC_SYMMETRY = 0, 1, 2, 3


@dataclass
class Case:
    name: str
    Q: np.ndarray          # [4][ny][nx] conservative state, float64
    dx: float
    dy: float
    gamma: float
    mu: float
    Pr: float
    bc: tuple              # (west, east, south, north)
    t_end: float = 0.0
    cfl: float = 0.5
    meta: dict | None = None

    @property
    def nx(self) -> int:
        return self.Q.shape[2]

    @property
    def ny(self) -> int:
        return self.Q.shape[1]


def prim_to_cons(rho, u, v, p, gamma):
    """Ideal-gas conservative state from primitive fields (works on complex
    input too, for complex-step derivatives in tests)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def centres(n, lo, hi):
    d = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * d, d


# --------------------------------------------------------------------------
# Example 1: isentropic vortex
# --------------------------------------------------------------------------

def vortex_prims(X, Y, t=0.0, eps=5.0, gamma=1.4, centre=(5.0, 5.0),
                 period=(10.0, 10.0), u_inf=1.0, v_inf=1.0):
    """Exact primitive fields of the convected isentropic vortex at time t.

    The periodic problem's exact solution is its initial data translated by
    (u_inf, v_inf) t; the displacement from the vortex centre is taken as the
    minimum image inside one period, as in the initial data. X, Y may be
    complex (complex-step differentiation in tests)."""
    Lx, Ly = period
    xr = X - centre[0] - u_inf * t
    yr = Y - centre[1] - v_inf * t
    # minimum image on the real part only (keeps complex steps intact)
    xr = xr - Lx * np.round(np.real(xr) / Lx)
    yr = yr - Ly * np.round(np.real(yr) / Ly)
    r2 = xr * xr + yr * yr
    T = 1.0 - (gamma - 1.0) * eps ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    g = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = u_inf - g * yr
    v = v_inf + g * xr
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return rho, u, v, p


def isentropic_vortex(n, ny=None, eps=5.0, gamma=1.4, domain=(0.0, 10.0, 0.0, 10.0),
                      t=0.0, cfl=0.5, t_end=0.0):
    """Example 1 on a periodic box (default [0,10]^2 centred at (5,5); the
    paper's [-5,5]^2 is the same flow shifted)."""
    ny = n if ny is None else ny
    x0, x1, y0, y1 = domain
    xc, dx = centres(n, x0, x1)
    yc, dy = centres(ny, y0, y1)
    X, Y = np.meshgrid(xc, yc)
    centre = (0.5 * (x0 + x1), 0.5 * (y0 + y1))
    rho, u, v, p = vortex_prims(X, Y, t, eps, gamma, centre, (x1 - x0, y1 - y0))
    Q = prim_to_cons(rho, u, v, p, gamma)
    return Case("isentropic_vortex", np.ascontiguousarray(Q), dx, dy, gamma, 0.0, 0.72,
                (BC_PERIODIC,) * 4, t_end, cfl,
                {"eps": eps, "domain": domain, "centre": centre})


# --------------------------------------------------------------------------
# Example 9: 2D Riemann problem (Schulz-Rinne), quadrants split at (0.8, 0.8)
# --------------------------------------------------------------------------

def riemann_2d(n, ny=None, t_end=0.3, cfl=0.5, split=(0.8, 0.8)):
    ny = n if ny is None else ny
    xc, dx = centres(n, 0.0, 1.0)
    yc, dy = centres(ny, 0.0, 1.0)
    s11 = 4.0 / np.sqrt(11.0)
    states = {  # (rho, u, v, p) as printed in Example 9
        "ur": (1.5, 0.0, 0.0, 1.5),
        "ul": (33.0 / 62.0, s11, 0.0, 0.3),
        "ll": (77.0 / 558.0, s11, s11, 9.0 / 310.0),
        "lr": (33.0 / 62.0, 0.0, s11, 0.3),
    }
    # quadrant index 2*top + right: 0 = lower left, 1 = lower right,
    # 2 = upper left, 3 = upper right
    quad = (2 * (yc > split[1])[:, None] + (xc > split[0])[None, :]).astype(np.int8)
    table = np.array([states["ll"], states["lr"], states["ul"], states["ur"]]).T  # [4 fields][4 quadrants]
    prim = np.stack([table[m][quad] for m in range(4)])
    Q = prim_to_cons(*prim, 1.4)
    return Case("riemann_2d", np.ascontiguousarray(Q), dx, dy, 1.4, 0.0, 0.72,
                (BC_TRANSMISSIVE,) * 4, t_end, cfl, {"split": split})


# --------------------------------------------------------------------------
# Example 10: viscous shock tube (Daru-Tenaud), [0,1] x [0,0.5]
# --------------------------------------------------------------------------

def viscous_shock_tube(nx, ny=None, Re=1000.0, Pr=0.73, gamma=1.4, t_end=1.0, cfl=0.2):
    """Navier-Stokes shock tube on [0,1] x [0,0.5]: rho 120 / 1.2 split at
    x = 0.5, p = rho/gamma, at rest; mu = 1/Re; no-slip adiabatic walls west,
    east and south, a symmetry plane north. CFL 0.2 as in Sec. 2.5 (used for
    all of the paper's runs): on fine grids the viscous bound of the time step
    decides dt, and the alpha-damping heat-conduction operator is unstable
    under TVD-RK3 above CFL ~0.33 there."""
    ny = nx // 2 if ny is None else ny
    xc, dx = centres(nx, 0.0, 1.0)
    yc, dy = centres(ny, 0.0, 0.5)
    X, _ = np.meshgrid(xc, yc)
    left = X < 0.5
    rho = np.where(left, 120.0, 1.2)
    p = rho / gamma
    z = np.zeros_like(rho)
    Q = prim_to_cons(rho, z, z, p, gamma)
    return Case("viscous_shock_tube", np.ascontiguousarray(Q), dx, dy, gamma, 1.0 / Re, Pr,
                (BC_NOSLIP_WALL, BC_NOSLIP_WALL, BC_NOSLIP_WALL, BC_SYMMETRY), t_end, cfl)


# --------------------------------------------------------------------------
# Seeded shear layer and exact-solution checks
# --------------------------------------------------------------------------

def kelvin_helmholtz(n, rng, ny=None, amp=0.01, modes=4, cfl=0.5):
    """Periodic [0,1]^2 shear layer: rho = 2, u = -0.5 for |y - 1/2| < 1/4,
    else rho = 1, u = +0.5; p = 2.5; v = sum_m a_m sin(2 pi m x + phi_m),
    normalised to max |v| = amp. a_m, phi_m come from `rng`."""
    ny = n if ny is None else ny
    xc, dx = centres(n, 0.0, 1.0)
    yc, dy = centres(ny, 0.0, 1.0)
    X, Y = np.meshgrid(xc, yc)
    a = rng.uniform(0.2, 1.0, modes)
    ph = rng.uniform(0.0, 2 * np.pi, modes)
    xs = np.linspace(0.0, 1.0, 4096, endpoint=False)
    shape = sum(a[m] * np.sin(2 * np.pi * (m + 1) * xs + ph[m]) for m in range(modes))
    scale = amp / np.max(np.abs(shape))
    inner = np.abs(Y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    u = np.where(inner, -0.5, 0.5)
    v = scale * sum(a[m] * np.sin(2 * np.pi * (m + 1) * X + ph[m]) for m in range(modes))
    p = np.full_like(rho, 2.5)
    Q = prim_to_cons(rho, u, v, p, 1.4)
    return Case("kelvin_helmholtz", np.ascontiguousarray(Q), dx, dy, 1.4, 0.0, 0.72,
                (BC_PERIODIC,) * 4, 0.0, cfl, {"a": a, "phi": ph, "scale": scale})


def entropy_wave(n, amp=0.2, L=10.0, gamma=1.4):
    """rho = 1 + amp sin(2 pi (x + y)/L), u = v = p = 1: translates exactly."""
    xc, dx = centres(n, 0.0, L)
    X, Y = np.meshgrid(xc, xc)
    rho = 1.0 + amp * np.sin(2 * np.pi * (X + Y) / L)
    one = np.ones_like(rho)
    Q = prim_to_cons(rho, one, one, one, gamma)
    return Case("entropy_wave", np.ascontiguousarray(Q), dx, dx, gamma, 0.0, 0.72,
                (BC_PERIODIC,) * 4)


def free_stream(nx, ny, state=(1.3, 0.7, -0.4, 2.1), gamma=1.4, bc=(BC_PERIODIC,) * 4,
                dx=0.1, dy=0.07):
    rho, u, v, p = (np.full((ny, nx), s) for s in state)
    Q = prim_to_cons(rho, u, v, p, gamma)
    return Case("free_stream", np.ascontiguousarray(Q), dx, dy, gamma, 0.0, 0.72, bc)


def shear_wave(n, amp=1e-6, L=1.0, mu=1e-2, gamma=1.4, Pr=0.72, rho0=1.0, p0=1.0):
    """v = amp sin(2 pi x / L) on a uniform state at rest, periodic: to first
    order in amp it decays as exp(-(mu/rho0) k^2 t), k = 2 pi / L."""
    xc, dx = centres(n, 0.0, L)
    X, _ = np.meshgrid(xc, xc)
    rho = np.full_like(X, rho0)
    u = np.zeros_like(X)
    v = amp * np.sin(2 * np.pi * X / L)
    p = np.full_like(X, p0)
    Q = prim_to_cons(rho, u, v, p, gamma)
    return Case("shear_wave", np.ascontiguousarray(Q), dx, dx, gamma, mu, Pr,
                (BC_PERIODIC,) * 4, meta={"amp": amp, "k": 2 * np.pi / L})


def shock_tube(n, left, right, t_end, ny=8, x_split=0.5, gamma=1.4, cfl=0.5):
    """Example 2 (Sod, Lax) as an n x ny strip on [0,1] x [0, ny/n]:
    transmissive in x, periodic in y; left/right = (rho, u, p)."""
    xc, dx = centres(n, 0.0, 1.0)
    X = np.tile(xc, (ny, 1))
    prim = [np.where(X < x_split, left[k], right[k]) for k in range(3)]
    Q = prim_to_cons(prim[0], prim[1], np.zeros_like(X), prim[2], gamma)
    return Case("shock_tube", np.ascontiguousarray(Q), dx, dx, gamma, 0.0, 0.72,
                (BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_PERIODIC, BC_PERIODIC), t_end, cfl,
                {"left": left, "right": right, "x_split": x_split})


BC_CUSTOM, BC_FIXED = 4, 5   # a side described by meta["sides"]; a fixed primitive state


def double_mach(nx=1024, ny=None, t_end=0.2, cfl=0.5):
    """Example 8 (Woodward and Colella): [0,4] x [0,1], a Mach 10 shock at
    60 degrees to the wall, post-shock (8, 8.25 cos 30, -8.25 sin 30, 116.5),
    pre-shock (1.4, 0, 0, 1). Boundaries: post-shock inflow on the west,
    transmissive east, south post-shock for x < 1/6 and a reflecting wall
    (mirror, normal velocity reversed) beyond, north post-shock up to the
    exact shock position 1/6 + (1 + 20 t)/sqrt(3) and pre-shock beyond.
    meta["sides"][k] = (kind_lo, kind_hi, s0, speed, lo, hi) of a custom
    side, positions measured from the grid's lower-left corner."""
    ny = nx // 4 if ny is None else ny
    xc, dx = centres(nx, 0.0, 4.0)
    yc, dy = centres(ny, 0.0, 1.0)
    X, Y = np.meshgrid(xc, yc)
    c30, s30, r3 = np.cos(np.pi / 6), np.sin(np.pi / 6), np.sqrt(3.0)
    post = (8.0, 8.25 * c30, -8.25 * s30, 116.5)
    pre = (1.4, 0.0, 0.0, 1.0)
    behind = X < 1.0 / 6.0 + Y / r3
    prim = [np.where(behind, post[m], pre[m]) for m in range(4)]
    Q = prim_to_cons(*prim, 1.4)
    sides = ((BC_FIXED, BC_FIXED, 0.0, 0.0, post, post), None,
             (BC_FIXED, BC_SYMMETRY, 1.0 / 6.0, 0.0, post, pre),
             (BC_FIXED, BC_FIXED, 1.0 / 6.0 + 1.0 / r3, 20.0 / r3, post, pre))
    return Case("double_mach", np.ascontiguousarray(Q), dx, dy, 1.4, 0.0, 0.72,
                (BC_CUSTOM, BC_TRANSMISSIVE, BC_CUSTOM, BC_CUSTOM), t_end, cfl,
                {"sides": sides, "post": post, "pre": pre, "shock_speed": 10.0})


def shock_entropy_2d(nx=400, ny=None, t_end=1.8, cfl=0.5, theta=np.pi / 6):
    """Example 7: [-5,5] x [-1,1]; a Mach 3 shock at x = -4 with post-shock
    (3.857143, 2.629369, 0, 10.3333) runs into rho = 1 + 0.2 sin(10 x cos theta
    + 10 y sin theta), u = v = 0, p = 1. Boundaries: post-shock inflow on the
    west, transmissive elsewhere."""
    ny = nx // 5 if ny is None else ny
    xc, dx = centres(nx, -5.0, 5.0)
    yc, dy = centres(ny, -1.0, 1.0)
    X, Y = np.meshgrid(xc, yc)
    post = (3.857143, 2.629369, 0.0, 10.3333)
    behind = X < -4.0
    rho = np.where(behind, post[0], 1.0 + 0.2 * np.sin(10.0 * X * np.cos(theta) + 10.0 * Y * np.sin(theta)))
    u = np.where(behind, post[1], 0.0)
    p = np.where(behind, post[3], 1.0)
    Q = prim_to_cons(rho, u, np.zeros_like(rho), p, 1.4)
    sides = ((BC_FIXED, BC_FIXED, 0.0, 0.0, post, post), None, None, None)
    return Case("shock_entropy_2d", np.ascontiguousarray(Q), dx, dy, 1.4, 0.0, 0.72,
                (BC_CUSTOM, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE), t_end, cfl,
                {"sides": sides, "post": post, "theta": theta})


SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2)           # Example 2, Sod
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.14)   # Example 2, Lax (t = 0.14)


def odd_even_shock(nx, ny, mach=6.0, seed=94, noise=1e-6, x0=10, gamma=1.4):
    """Grid-aligned shock instability test (Quirk 1994) on a uniform grid of
    unit cells: a Mach `mach` shock at x = x0 cells moving in +x into gas at
    rest (rho 1.4, p 1), the Rankine-Hugoniot state behind it, and seeded
    relative density noise of size `noise` ahead of it. Transmissive west and
    east, symmetry planes south and north. A shock-stable flux keeps the rows
    alike; plain HLLC lets the noise grow into the carbuncle that Examples 7
    and 8 avoid with the shock-stable solver."""
    r1, p1 = 1.4, 1.0
    m2 = mach * mach
    r2 = r1 * (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)
    p2 = p1 * (2 * gamma * m2 - (gamma - 1)) / (gamma + 1)
    u2 = mach * np.sqrt(gamma * p1 / r1) * (1 - r1 / r2)
    rho = np.full((ny, nx), r1)
    u = np.zeros((ny, nx))
    p = np.full((ny, nx), p1)
    rho[:, :x0], u[:, :x0], p[:, :x0] = r2, u2, p2
    rho[:, x0:] *= 1 + noise * np.random.default_rng(seed).standard_normal((ny, nx - x0))
    Q = prim_to_cons(rho, u, np.zeros_like(u), p, gamma)
    return Case("odd_even_shock", np.ascontiguousarray(Q), 1.0, 1.0, gamma, 0.0, 0.72,
                (BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_SYMMETRY, BC_SYMMETRY), 0.0, 0.5,
                {"mach": mach, "shock_speed": mach * np.sqrt(gamma * p1 / r1)})


def ensemble(n_cases=64, seed=762, sizes=(256, 512, 1024, 2048)):
    """Seeded table of independent cases of uneven size: half isentropic
    vortices with strength U[1,5] on [0,10]^2, half shear layers."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cases):
        n = int(rng.choice(sizes))
        if k % 2 == 0:
            eps = float(rng.uniform(1.0, 5.0))
            out.append(("vortex", n, {"eps": eps}))
        else:
            out.append(("kh", n, {"seed": int(rng.integers(0, 2**31 - 1))}))
    return out


def make_ensemble_case(kind, n, params):
    if kind == "vortex":
        return isentropic_vortex(n, eps=params["eps"])
    return kelvin_helmholtz(n, np.random.default_rng(params["seed"]))
