"""Custom boundary sides of the oracle (fixed inflow states, kinds split at a
point that moves with time), as Examples 7 and 8 need: a uniform inflow is
preserved, the ghost frame of the double Mach reflection follows the exact
shock position, and the incident shock of Example 8 travels at its
Rankine-Hugoniot speed."""
import dataclasses

import numpy as np

from paper_2305_00762_gb300 import cases as C


def cfg_of(O, c, t=0.0):
    return O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc, t=t, sides=c.meta["sides"])


def test_uniform_inflow_is_preserved(oracle_mod):
    O = oracle_mod
    state = (1.3, 0.7, -0.2, 2.1)
    n = 24
    Q = C.prim_to_cons(*[np.full((n, n), v) for v in state], 1.4)
    sides = ((C.BC_FIXED, C.BC_FIXED, 0.0, 0.0, state, state), None,
             (C.BC_FIXED, C.BC_FIXED, 0.0, 0.0, state, state), None)
    cfg = O.Config(n, n, 0.1, 0.1, 1.4, 0.0, 0.72, (C.BC_CUSTOM, 1, C.BC_CUSTOM, 1), sides=sides)
    R = O.residual(cfg, Q)
    assert np.abs(R).max() < 1e-12


def test_double_mach_ghost_frame(oracle_mod):
    """At t = 0.05: north ghosts post-shock up to x_s(t) = 1/6 + (1 + 20 t)/sqrt(3)
    and pre-shock beyond; south ghosts post-shock for x < 1/6 and mirror
    images (v reversed) beyond; west ghosts post-shock; corners as their
    south / north side says where it is fixed."""
    O = oracle_mod
    c = C.double_mach(64, 16)
    t = 0.05
    g = O.G
    Qp = np.zeros((4, c.ny + 2 * g, c.nx + 2 * g))
    Qp[:, g:g + c.ny, g:g + c.nx] = c.Q
    P = O.fill_ghosts_padded(cfg_of(O, c, t), Qp)
    post = C.prim_to_cons(*[np.array(v) for v in c.meta["post"]], 1.4)
    pre = C.prim_to_cons(*[np.array(v) for v in c.meta["pre"]], 1.4)
    xj = (np.arange(-g, c.nx + g) + 0.5) * c.dx
    xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / np.sqrt(3.0)
    for row in range(c.ny + g, c.ny + 2 * g):        # north ghosts
        want = np.where(xj < xs, post[:, None], pre[:, None])
        assert np.array_equal(P[:, row, :], want)
    for k in range(g):                                 # south ghosts
        row = g - 1 - k
        src = P[:, g + k, :].copy()
        src[2] = -src[2]
        wall = xj >= 1.0 / 6.0
        assert np.array_equal(P[:, row, wall], src[:, wall])
        assert np.array_equal(P[:, row, ~wall], np.repeat(post[:, None], (~wall).sum(), axis=1))
    for col in range(g):                               # west ghosts, interior rows
        assert np.array_equal(P[:, g:g + c.ny, col], np.repeat(post[:, None], c.ny, axis=1))


def test_double_mach_incident_shock_speed(oracle_mod):
    """The incident shock, away from the wall, sits at the exact position
    x_s(y, t) = 1/6 + (y + 20 t)/sqrt(3) (shock speed 10 along its normal)
    after t = 0.03, to within two cells, on rows y in [0.6, 0.95]."""
    O = oracle_mod
    c = C.double_mach(160, 40)
    cfg = cfg_of(O, c)
    Q, t, steps = O.run(cfg, c.Q, 0.03, 0.5)
    assert abs(t - 0.03) < 1e-14
    yc = (np.arange(c.ny) + 0.5) * c.dy
    xc = (np.arange(c.nx) + 0.5) * c.dx
    checked = 0
    for i in np.nonzero((yc > 0.6) & (yc < 0.95))[0]:
        rho = Q[0, i]
        j = np.nonzero(rho < 0.5 * (8.0 + 1.4))[0][0]   # first cell ahead of the shock
        xs = 1.0 / 6.0 + (yc[i] + 20.0 * t) / np.sqrt(3.0)
        assert abs(xc[j] - xs) < 2 * c.dx, (yc[i], xc[j], xs)
        checked += 1
    assert checked >= 10
    p = 0.4 * (Q[3] - 0.5 * (Q[1] ** 2 + Q[2] ** 2) / Q[0])
    assert Q[0].min() > 0 and p.min() > 0


def test_stage_times_of_a_moving_side(oracle_mod):
    """One RK3 step from t with step dt sees the moving north side at t,
    t + dt and t + dt/2: it equals the three stages written out with those
    configurations."""
    O = oracle_mod
    c = C.double_mach(48, 12)
    t, dt = 0.02, 4e-4
    cfg = cfg_of(O, c, t)
    Q1, rc = O.rk3_step(cfg, c.Q, dt)
    assert rc == 0
    R0 = O.residual(cfg, c.Q)
    Qa = c.Q + dt * R0
    Ra = O.residual(dataclasses.replace(cfg, t=t + dt), Qa)
    Qb = 0.75 * c.Q + 0.25 * Qa + 0.25 * dt * Ra
    Rb = O.residual(dataclasses.replace(cfg, t=t + 0.5 * dt), Qb)
    Q2 = c.Q / 3.0 + 2.0 / 3.0 * Qb + 2.0 / 3.0 * dt * Rb
    assert np.abs(Q1 - Q2).max() <= 1e-13 * np.abs(Q2).max()
