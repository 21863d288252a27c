"""Pins of the oracle's shock-stable HLLC (the HLLC-LM flux of Fleischmann,
Adami and Adams 2020, which Examples 7 and 8 of arXiv:2305.00762 use; reading
R24): an independent restatement in that work's signed, case-split form,
closed-form special cases, its limit to plain HLLC, grid invariants and the
grid-aligned shock instability it exists to suppress."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

G = 1.4
MA_LIM = 0.1


def _flux_and_cons(W):
    r, u, v, p = W
    E = p / (G - 1) + 0.5 * r * (u * u + v * v)
    return np.array([r * u, r * u * u + p, r * u * v, u * (E + p)]), np.array([r, r * u, r * v, E])


def _hllc_lm_signed(WL, WR):
    """HLLC-LM as Fleischmann et al. write it: upwind fluxes outside the fan,
    else 1/2(F_L+F_R) + 1/2[phi S_L (Q*_L - Q_L) + |S*| (Q*_L - Q*_R)
    + phi S_R (Q*_R - Q_R)] with signed S_L < 0 < S_R; star states from
    Toro's formula, Einfeldt/Roe bounds. Written without the oracle's |A|
    form."""
    FL, QL = _flux_and_cons(WL)
    FR, QR = _flux_and_cons(WR)
    rL, uL, vL, pL = WL
    rR, uR, vR, pR = WR
    cL, cR = np.sqrt(G * pL / rL), np.sqrt(G * pR / rR)
    w = np.sqrt(rR / rL)
    ub, vb = (uL + w * uR) / (1 + w), (vL + w * vR) / (1 + w)
    Hb = ((QL[3] + pL) / rL + w * (QR[3] + pR) / rR) / (1 + w)
    cb = np.sqrt((G - 1) * (Hb - 0.5 * (ub * ub + vb * vb)))
    SL, SR = min(uL - cL, ub - cb), max(uR + cR, ub + cb)
    if SL >= 0:
        return FL
    if SR <= 0:
        return FR
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(r, u, v, p, Q, S):
        k = r * (S - u) / (S - Ss)
        return k * np.array([1.0, Ss, v, Q[3] / r + (Ss - u) * (Ss + p / (r * (S - u)))])
    sL, sR = star(*WL, QL, SL), star(*WR, QR, SR)
    phi = np.sin(np.pi / 2 * min(1.0, max(abs(uL) / cL, abs(uR) / cR) / MA_LIM))
    return 0.5 * (FL + FR) + 0.5 * (phi * SL * (sL - QL) + abs(Ss) * (sL - sR) + phi * SR * (sR - QR))


def _pair(rng, ustd):
    return np.array([rng.uniform(0.1, 3), rng.normal() * ustd, rng.normal(), rng.uniform(0.05, 3)])


def test_hllc_lm_equals_signed_form(oracle_mod):
    """Random state pairs with face-normal Mach numbers spread over 0..0.3
    (phi < 1 on most of them) and over the supersonic range."""
    rng = np.random.default_rng(24)
    below = 0
    for k in range(4000):
        ustd = 0.05 if k % 2 == 0 else 2.0
        WL, WR = _pair(rng, ustd), _pair(rng, ustd)
        FL, _ = _flux_and_cons(WL)
        FR, _ = _flux_and_cons(WR)
        got = oracle_mod.hllc(G, WL, WR, FL, FR, lm=True)
        ref = _hllc_lm_signed(WL, WR)
        scale = 1 + np.abs(FL).max() + np.abs(FR).max()
        assert np.abs(got - ref).max() < 1e-12 * scale
        ma = max(abs(WL[1]) / np.sqrt(G * WL[3] / WL[0]), abs(WR[1]) / np.sqrt(G * WR[3] / WR[0]))
        below += ma < MA_LIM
    assert below > 1000


def test_hllc_lm_is_hllc_at_or_above_the_mach_limit(oracle_mod):
    """phi = 1 once either side's normal Mach number reaches Ma_lim: the
    flux is plain HLLC bit for bit; just below the limit it is continuous."""
    rng = np.random.default_rng(25)
    for _ in range(500):
        WL, WR = _pair(rng, 2.0), _pair(rng, 2.0)
        cL = np.sqrt(G * WL[3] / WL[0])
        WL[1] = np.sign(WL[1] or 1.0) * max(abs(WL[1]), MA_LIM * cL * 1.0000001)
        FL, _ = _flux_and_cons(WL)
        FR, _ = _flux_and_cons(WR)
        assert np.array_equal(oracle_mod.hllc(G, WL, WR, FL, FR, lm=True), oracle_mod.hllc(G, WL, WR, FL, FR))
    WL, WR = np.array([1.0, 0.0, 0.1, 1.0]), np.array([0.8, 0.0, -0.2, 0.7])
    for side in (WL, WR):
        side[1] = MA_LIM * np.sqrt(G * side[3] / side[0]) * (1 - 1e-4)  # phi = 1 - 1.2e-8
    FL, _ = _flux_and_cons(WL)
    FR, _ = _flux_and_cons(WR)
    a, b = oracle_mod.hllc(G, WL, WR, FL, FR, lm=True), oracle_mod.hllc(G, WL, WR, FL, FR)
    assert np.abs(a - b).max() < 1e-7 and not np.array_equal(a, b)


def test_hllc_lm_special_cases(oracle_mod):
    """Stationary contact: Ma = 0 and S* = 0, so the flux is (0, p, 0, 0)
    exactly. Equal states: the physical flux. A pressure jump at rest with
    equal densities: phi = 0 removes the acoustic dissipation, so the mass
    flux is the |S*| term alone, smaller than plain HLLC's."""
    WL, WR = np.array([2.0, 0.0, 0.3, 1.0]), np.array([0.5, 0.0, -0.7, 1.0])
    FL, _ = _flux_and_cons(WL)
    FR, _ = _flux_and_cons(WR)
    assert np.array_equal(oracle_mod.hllc(G, WL, WR, FL, FR, lm=True), np.array([0.0, 1.0, 0.0, 0.0]))
    for u in (0.0, 0.02, 0.5, -3.0):
        W = np.array([1.3, u, -0.2, 0.9])
        F, _ = _flux_and_cons(W)
        assert np.abs(oracle_mod.hllc(G, W, W, F, F, lm=True) - F).max() < 1e-14
    WL, WR = np.array([1.0, 0.0, 0.0, 1.2]), np.array([1.0, 0.0, 0.0, 0.8])
    FL, _ = _flux_and_cons(WL)
    FR, _ = _flux_and_cons(WR)
    lm, plain = oracle_mod.hllc(G, WL, WR, FL, FR, lm=True), oracle_mod.hllc(G, WL, WR, FL, FR)
    assert abs(lm[0]) < abs(plain[0])
    assert np.abs(lm - _hllc_lm_signed(WL, WR)).max() < 1e-14


def _cfg(O, case, riemann):
    return O.Config(case.nx, case.ny, case.dx, case.dy, case.gamma, case.mu, case.Pr, case.bc, 7,
                    riemann=riemann)


def test_hllc_lm_grid_invariants(oracle_mod):
    """A uniform state stays exact, and Eq. deriv still telescopes on a
    periodic grid (seeded rough low-Mach data with pressure jumps, so that
    phi < 1 changes the flux and the detector flags faces)."""
    O = oracle_mod
    for bc in ((0, 0, 0, 0), (1, 1, 1, 1)):
        c = C.free_stream(23, 17, bc=bc)
        assert np.abs(O.residual(_cfg(O, c, 1), c.Q)).max() <= 1e-13
    rng = np.random.default_rng(7)
    ny, nx = 36, 40
    r, p = rng.uniform(0.5, 1.5, (ny, nx)), rng.uniform(0.5, 1.5, (ny, nx))
    u, v = rng.normal(0, 0.02, (ny, nx)), rng.normal(0, 0.02, (ny, nx))
    Q = np.ascontiguousarray(C.prim_to_cons(r, u, v, p, G))
    c = O.Config(nx, ny, 1.0 / nx, 1.0 / ny, G, 0.0, 0.72, (0, 0, 0, 0), 7, riemann=1)
    R, sx, sy = O.residual(c, Q, want_flags=True)
    c.riemann = 0
    R0 = O.residual(c, Q)
    assert (sx == 0).sum() > 0 and np.abs(R - R0).max() > 1e-2 * np.abs(R0).max()
    for m in range(4):
        assert abs(R[m].sum()) <= 1e-13 * np.abs(R[m]).sum()


def test_hllc_lm_suppresses_odd_even_decoupling(oracle_mod):
    """The reason Examples 7 and 8 switch solvers (Quirk's odd-even
    decoupling problem): behind a grid-aligned Mach 6 shock, plain HLLC
    amplifies 1e-6 density noise into O(1e-2) row-to-row density differences
    within 200 steps, HLLC-LM keeps them two orders smaller."""
    O = oracle_mod
    case = C.odd_even_shock(160, 16, mach=6.0, seed=94)
    dev = {}
    for rm in (0, 1):
        c = _cfg(O, case, rm)
        q = case.Q
        for _ in range(200):
            q, rc = O.rk3_step(c, q, 0.5 / O.max_wavespeed(c, q))
            assert rc == 0
        dev[rm] = np.abs(q[0] - q[0].mean(axis=0, keepdims=True)).max()
    assert dev[0] > 1e-2
    assert dev[1] < 2e-3 and dev[1] < dev[0] / 20


def test_riemann_flag_is_checked(oracle_mod):
    O = oracle_mod
    c = C.free_stream(16, 16)
    with pytest.raises(RuntimeError):
        O.residual(_cfg(O, c, 2), c.Q)


def test_odd_even_shock_is_a_rankine_hugoniot_shock():
    """The generator's states: in the frame moving at the shock speed, mass,
    momentum and energy fluxes agree across the jump (to roundoff), and the
    pre-shock Mach number relative to the shock is the requested one."""
    c = C.odd_even_shock(64, 4, mach=6.0, noise=0.0)
    Q = c.Q
    us = c.meta["shock_speed"]

    def fluxes(j):
        r, mu, E = Q[0, 0, j], Q[1, 0, j], Q[3, 0, j]
        u = mu / r
        p = (G - 1) * (E - 0.5 * r * u * u)
        w = u - us
        return np.array([r * w, r * w * w + p, w * (E - r * u * us + 0.5 * r * us * us + p)]), r, p, w
    f2, r2, p2, _ = fluxes(0)       # behind the shock
    f1, r1, p1, w1 = fluxes(63)     # gas at rest ahead of it
    assert np.allclose(f1, f2, rtol=1e-13, atol=1e-12 * np.abs(f1).max())
    assert abs(-w1 / np.sqrt(G * p1 / r1) - 6.0) < 1e-12
