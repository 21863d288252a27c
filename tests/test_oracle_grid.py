"""Pins of the oracle's 2D residual against exact solutions, invariants and
closed forms (arXiv:2305.00762, Secs. 1-2)."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C


def cfg_of(O, case, order=7):
    return O.Config(case.nx, case.ny, case.dx, case.dy, case.gamma, case.mu, case.Pr,
                    case.bc, order)


def test_free_stream_and_rest_state(oracle_mod):
    """A uniform moving state is an exact solution with periodic and
    transmissive boundaries; a uniform state at rest with every boundary
    type (walls and symmetry planes included, viscous too)."""
    O = oracle_mod
    for bc in ((0, 0, 0, 0), (1, 1, 1, 1), (0, 0, 1, 1)):
        c = C.free_stream(23, 17, bc=bc)
        R = O.residual(cfg_of(O, c), c.Q)
        assert np.abs(R).max() <= 1e-13
    for bc in ((2, 2, 2, 3), (3, 3, 3, 3), (2, 1, 3, 0)[:2] + (2, 3)):
        c = C.free_stream(19, 21, state=(0.8, 0.0, 0.0, 1.7), bc=bc)
        c.mu = 0.01
        R = O.residual(cfg_of(O, c), c.Q)
        assert np.abs(R).max() <= 1e-13


def test_periodic_conservation(oracle_mod):
    """Eq. deriv telescopes: on a periodic grid the domain sum of Res vanishes
    to roundoff, here on a discontinuous shear layer that exercises the
    detector (sigma = 0 faces) and the MP limiter."""
    O = oracle_mod
    c = C.kelvin_helmholtz(48, np.random.default_rng(3))
    R, sx, sy = O.residual(cfg_of(O, c), c.Q, want_flags=True)
    assert (sy == 0).sum() > 0 and (sy == 1).sum() > 0
    for m in range(4):
        scale = np.abs(R[m]).sum()
        assert abs(R[m].sum()) <= 1e-13 * scale


def test_transpose_symmetry_riemann(oracle_mod):
    """Example 9's data is symmetric under x <-> y with u <-> v; the
    dimension-by-dimension residual must be exactly symmetric too."""
    O = oracle_mod
    c = C.riemann_2d(40)
    R = O.residual(cfg_of(O, c), c.Q)
    assert np.array_equal(R[0], R[0].T)
    assert np.array_equal(R[3], R[3].T)
    assert np.array_equal(R[1], R[2].T)


def _vortex_dqdt(X, Y):
    h = 1e-30
    f = lambda X, Y: C.prim_to_cons(*C.vortex_prims(X, Y), 1.4)
    dx = np.imag(f(X + 1j * h, Y + 0j)) / h
    dy = np.imag(f(X + 0j, Y + 1j * h)) / h
    return -(dx + dy)   # the vortex translates with velocity (1, 1)


def test_residual_truncation_order_seven(oracle_mod):
    """Sec. 2.4: with flux reconstruction in smooth regions the scheme is
    genuinely seventh order: Res(Q_exact) - dQ/dt converges at ~7 on the
    isentropic vortex (Example 1), inside r < 3 of the centre."""
    O = oracle_mod
    errs = []
    for n in (64, 128, 256):
        c = C.isentropic_vortex(n)
        R, sx, sy = O.residual(cfg_of(O, c), c.Q, want_flags=True)
        assert sx.min() == 1 and sy.min() == 1   # smooth: no detector hits
        xc, _ = C.centres(n, 0.0, 10.0)
        X, Y = np.meshgrid(xc, xc)
        mask = np.hypot(X - 5, Y - 5) < 3
        errs.append(np.abs(R - _vortex_dqdt(X, Y))[:, mask].max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 6.5).all(), orders


def test_viscous_shear_wave_fourth_order(oracle_mod):
    """Sec. 2.1: the alpha-damping viscous scheme with sixth-order gradients
    is fourth order. For v = A sin(kx) at rest, Res(rho v) = mu v_xx;
    the relative error must fall at order ~4."""
    O = oracle_mod
    errs = []
    for n in (32, 64, 128):
        c = C.shear_wave(n, amp=1e-6, mu=1e-2)
        R = O.residual(cfg_of(O, c), c.Q)
        v = c.Q[2] / c.Q[0]
        exact = -c.mu * c.meta["k"] ** 2 * v
        errs.append(np.abs(R[2] - exact).max() / np.abs(exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 3.6).all() and (orders < 4.6).all(), (errs, orders)


def test_diagonal_shear_wave_cross_terms(oracle_mod):
    """Eq. visc in 2D: u = -A s, v = A s with s = sin(k(x+y)) is a
    divergence-free shear wave; the x- and y-face stresses (normal terms by
    alpha-damping, cross terms u_y, v_x, v_y, u_x from the cell-centre
    gradients) must add up to mu Lap(u) = -2 mu k^2 u. The tangential
    derivatives at a face are the mean of the two cell-centre values (the
    alpha-damping face gradient of Sec. 2.1 with the damping acting along the
    normal only), which is second order; a dropped or sign-flipped cross term
    would leave an O(1) error that does not converge."""
    O = oracle_mod
    g, mu, A, k = 1.4, 1e-2, 1e-6, 2 * np.pi
    errs = []
    for n in (32, 64, 128):
        xc, dx = C.centres(n, 0.0, 1.0)
        X, Y = np.meshgrid(xc, xc)
        s = np.sin(k * (X + Y))
        Q = C.prim_to_cons(np.ones_like(s), -A * s, A * s, np.ones_like(s), g)
        cfg = O.Config(n, n, dx, dx, g, mu, 0.72, (0, 0, 0, 0))
        R = O.residual(cfg, Q)
        ex_u, ex_v = -2 * mu * k * k * (-A * s), -2 * mu * k * k * (A * s)
        scale = 2 * mu * k * k * A
        errs.append(max(np.abs(R[1] - ex_u).max(), np.abs(R[2] - ex_v).max()) / scale)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 1.9).all() and (orders < 2.1).all(), (errs, orders)
    assert errs[-1] < 1e-4


def test_heat_conduction_fourth_order(oracle_mod):
    """Eq. visc-interface: with u = v = 0 and uniform p, a density wave is a
    stationary contact (no convective flux, HLLC keeps it exactly) and the
    energy residual is mu/(Pr (gamma-1)) T_xx with T = gamma p / rho."""
    O = oracle_mod
    g, mu, Pr, A = 1.4, 1e-2, 0.72, 1e-3
    errs = []
    for n in (32, 64, 128):
        xc, dx = C.centres(n, 0.0, 1.0)
        X, _ = np.meshgrid(xc, xc)
        k = 2 * np.pi
        rho = 1 + A * np.sin(k * X)
        z = np.zeros_like(rho)
        Q = C.prim_to_cons(rho, z, z, np.ones_like(rho), g)
        cfg = O.Config(n, n, dx, dx, g, mu, Pr, (0, 0, 0, 0))
        R = O.residual(cfg, Q)
        # T = g / rho; T_xx analytically
        rx = A * k * np.cos(k * X)
        rxx = -A * k * k * np.sin(k * X)
        Txx = g * (2 * rx * rx / rho ** 3 - rxx / rho ** 2)
        exact = mu / (Pr * (g - 1)) * Txx
        errs.append(np.abs(R[3] - exact).max() / np.abs(exact).max())
        assert np.abs(R[0]).max() < 1e-12 and np.abs(R[1]).max() < 1e-12
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 3.6).all(), (errs, orders)


def test_ghost_cells(oracle_mod):
    """Ghost-cell boundary conditions: periodic wraps, transmissive copies the
    edge cell, a no-slip wall mirrors with both velocities negated, a symmetry
    plane mirrors with the normal velocity negated."""
    O = oracle_mod
    G, nx, ny = O.G, 9, 8
    rng = np.random.default_rng(11)
    Qp = rng.uniform(0.5, 2.0, (4, ny + 2 * G, nx + 2 * G))
    I = lambda a: a[:, G:G + ny, G:G + nx]
    cfg = O.Config(nx, ny, 0.1, 0.1, 1.4, 0.0, 0.72, (0, 0, 2, 3))
    P = O.fill_ghosts_padded(cfg, Qp)
    assert np.array_equal(I(P), I(Qp))
    for k in range(G):
        # periodic in x, interior rows
        assert np.array_equal(P[:, G:G + ny, G - 1 - k], P[:, G:G + ny, G + nx - 1 - k])
        assert np.array_equal(P[:, G:G + ny, G + nx + k], P[:, G:G + ny, G + k])
        # south no-slip wall: mirror, both momenta negated (all columns)
        src, dst = P[:, G + k, :], P[:, G - 1 - k, :]
        assert np.array_equal(dst[[0, 3]], src[[0, 3]]) and np.array_equal(dst[[1, 2]], -src[[1, 2]])
        # north symmetry: mirror, normal (y) momentum negated
        src, dst = P[:, G + ny - 1 - k, :], P[:, G + ny + k, :]
        assert np.array_equal(dst[[0, 1, 3]], src[[0, 1, 3]]) and np.array_equal(dst[2], -src[2])
    cfg = O.Config(nx, ny, 0.1, 0.1, 1.4, 0.0, 0.72, (1, 1, 1, 1))
    P = O.fill_ghosts_padded(cfg, Qp)
    for k in range(G):
        assert np.array_equal(P[:, G:G + ny, k], P[:, G:G + ny, G])
        assert np.array_equal(P[:, k, :], P[:, G, :])


def test_max_wavespeed_closed_form(oracle_mod):
    """Sec. 2.5: dt = CFL / lambda; for a uniform state lambda is
    max((|u|+c)/dx, (|v|+c)/dy) and, with viscosity, at least 4 nu / dx^2."""
    O = oracle_mod
    c = C.free_stream(12, 10, state=(1.3, -0.7, 0.4, 2.1))
    cs = np.sqrt(1.4 * 2.1 / 1.3)
    lam = O.max_wavespeed(cfg_of(O, c), c.Q)
    assert abs(lam - max((0.7 + cs) / c.dx, (0.4 + cs) / c.dy)) < 1e-13 * lam
    c.mu = 5.0
    lam = O.max_wavespeed(cfg_of(O, c), c.Q)
    assert abs(lam - 4 * (5.0 / 1.3) / min(c.dx, c.dy) ** 2) < 1e-13 * lam


def test_fourth_order_member_truncation(oracle_mod):
    """Remark after Eq. grb: alpha = 4, beta = 0 (with Eq. fourth) is the
    fourth-order scheme: residual truncation order ~4 on the vortex."""
    O = oracle_mod
    errs = []
    for n in (64, 128, 256):
        c = C.isentropic_vortex(n)
        cfg = O.Config(n, n, c.dx, c.dy, 1.4, 0.0, 0.72, c.bc, 4)
        R = O.residual(cfg, c.Q)
        xc, _ = C.centres(n, 0.0, 10.0)
        X, Y = np.meshgrid(xc, xc)
        mask = np.hypot(X - 5, Y - 5) < 3
        errs.append(np.abs(R - _vortex_dqdt(X, Y))[:, mask].max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 3.6).all() and (orders < 4.6).all(), orders
