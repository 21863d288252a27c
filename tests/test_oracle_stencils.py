"""Pins of the oracle's one-dimensional building blocks against what the paper
and the mathematics fix (never against the oracle's own formulas retyped).

Sections and equations refer to arXiv:2305.00762.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Eq. six ----
def test_grad6_exact_for_degree6(oracle_mod):
    """Eq. six is a sixth-order central difference: exact (times dx) for every
    polynomial of degree <= 6, wrong for degree 7."""
    x = np.arange(-3, 4) * 0.37 + 1.3
    for deg in range(0, 8):
        c = _rng(deg).normal(size=deg + 1)
        exact = 0.37 * P.polyval(1.3, P.polyder(c)) if deg > 0 else 0.0
        got = oracle_mod.grad6(P.polyval(x, c))
        scale = 1 + np.abs(P.polyval(x, c)).max()
        if deg <= 6:
            assert abs(got - exact) < 1e-13 * scale
        else:
            assert abs(got - exact) > 1e-8 * scale


# ---------------------------------------------------------------- Eq. grb ----
def test_grb_equals_alpha_beta_family(oracle_mod):
    """Eq. grb is Eq. lingrb with the second derivative of Eqs. how-second,
    good_6tth-order_scheme_flux and alpha-beta at alpha = 38/7, beta = 3/190."""
    rng = _rng(1)
    for _ in range(200):
        phi, dphi = rng.normal(size=5), rng.normal(size=5)
        a = oracle_mod.grb_left(phi, dphi)
        b = oracle_mod.grb_alphabeta_left(phi, dphi, 38.0 / 7.0, 3.0 / 190.0)
        assert abs(a - b) < 1e-13 * (1 + abs(a))


def test_grb_left_matches_grb_sec(oracle_mod):
    """Eq. grb-sec gives dx^2 Phi''_j; with Eq. lingrb it must reproduce Eq. grb."""
    rng = _rng(2)
    for _ in range(200):
        ph, dp = rng.normal(size=5), rng.normal(size=5)
        # indices: 0..4 = j-2..j+2
        d2 = (60 * dp[1] - 60 * dp[3] - 362 * ph[2] + 178 * ph[1] + 3 * ph[0]
              + 178 * ph[3] + 3 * ph[4]) / 70.0
        ref = ph[2] + dp[2] / 2 + d2 / 12
        assert abs(oracle_mod.grb_left(ph, dp) - ref) < 1e-13 * (1 + abs(ref))


def test_grb_right_is_mirror_of_left(oracle_mod):
    """Eq. grb's right formula is its left formula mirrored about the face."""
    rng = _rng(3)
    for _ in range(100):
        ph, dp = rng.normal(size=5), rng.normal(size=5)   # j-1..j+3
        a = oracle_mod.grb_right(ph, dp)
        b = oracle_mod.grb_left(ph[::-1], -dp[::-1])
        assert abs(a - b) < 1e-13 * (1 + abs(a))


def _modified_wavenumber(oracle_mod, w, left):
    """Phi_k = exp(i w k), dx = 1: D(w) = Phi^L_{1/2} - Phi^L_{-1/2}."""
    k = np.arange(-6, 7)
    out = 0j
    for part, fac in ((np.cos, 1.0), (np.sin, 1j)):
        phi = part(w * k)
        dphi = {j: oracle_mod.grad6(phi[j + 3:j + 10]) for j in range(-3, 4)}

        def L(j):
            return left(phi[j + 4:j + 9], [dphi[i] for i in range(j - 2, j + 3)])
        out += fac * (L(0) - L(-1))
    return out


def test_fourier_leading_error_is_printed_one(oracle_mod):
    """Sec. 2.2: for linear advection the differenced left value behaves as
    dx (i + dx^7/280 - i dx^8/360 - dx^9/560 + ...) with k = 1, i.e. the
    seventh-order upwind scheme of alpha = 38/7, beta = 3/190."""
    w = 0.1
    d = _modified_wavenumber(oracle_mod, w, oracle_mod.grb_left) - 1j * w
    assert abs(d.real / w ** 8 * 280 - 1) < 0.01
    assert abs(d.imag / w ** 9 * 360 + 1) < 0.01
    assert abs((d.real - w ** 8 / 280) / w ** 10 * 560 + 1) < 0.02


def test_fourth_order_member(oracle_mod):
    """Remark after Eq. grb: alpha = 4, beta = 0 gives a fourth-order scheme
    (dispersion error ~ w^5), and Eq. fourth is its flux form."""
    left4 = lambda p, dp: oracle_mod.grb_alphabeta_left(p, dp, 4.0, 0.0)
    e1 = abs(_modified_wavenumber(oracle_mod, 0.1, left4) - 0.1j)
    e2 = abs(_modified_wavenumber(oracle_mod, 0.05, left4) - 0.05j)
    assert 4.6 < np.log2(e1 / e2) < 5.4
    rng = _rng(4)
    for _ in range(100):
        f = rng.normal(size=9)  # f_{j-4..j+4}
        d = [oracle_mod.grad6(f[i - 3:i + 4]) for i in range(3, 6)]  # j-1..j+1
        ref = oracle_mod.grb_alphabeta_left(f[2:7], [0.0] + d + [0.0], 4.0, 0.0)
        assert abs(oracle_mod.flux_recon4_left(f) - ref) < 1e-12 * (1 + abs(ref))


# ---------------------------------------------------- Eq. flux-full/right ----
def test_flux_recon_is_grb_of_cell_fluxes(oracle_mod):
    """Sec. 2.4: Eq. flux-full is Eq. grb with the sixth-order gradients of the
    cell fluxes substituted; Eq. flux-right is its mirror."""
    rng = _rng(5)
    for _ in range(200):
        f = rng.normal(size=10)  # f_{j-4..j+5}
        d = [oracle_mod.grad6(f[i - 3:i + 4]) for i in range(3, 7)]  # j-1..j+2
        ref_l = oracle_mod.grb_left(f[2:7], [0.0, d[0], d[1], d[2], 0.0])
        got_l = oracle_mod.flux_recon_left(f[0:9])
        assert abs(got_l - ref_l) < 1e-12 * (1 + abs(ref_l))
        ref_r = oracle_mod.grb_right(f[3:8], [0.0, d[1], d[2], d[3], 0.0])
        got_r = oracle_mod.flux_recon_right(f[1:10])
        assert abs(got_r - ref_r) < 1e-12 * (1 + abs(ref_r))


def test_flux_recon_differenced_exact_to_degree7(oracle_mod):
    """The differenced F(f_L) is a 7th-order derivative: exact for x^m,
    m <= 7 (and the L/R average exact for m <= 8); not for m = 9."""
    h = 0.21
    xs = 0.4 + h * np.arange(-5, 6)   # cells j-5..j+5, j at index 5
    for m in range(0, 10):
        f = xs ** m
        fl_p = oracle_mod.flux_recon_left(f[1:10])    # face j+1/2: f_{j-4..j+4}
        fl_m = oracle_mod.flux_recon_left(f[0:9])     # face j-1/2
        fr_p = oracle_mod.flux_recon_right(f[2:11])   # face j+1/2: f_{j-3..j+5}
        fr_m = oracle_mod.flux_recon_right(f[1:10])
        exact = m * 0.4 ** (m - 1) if m else 0.0
        up = (fl_p - fl_m) / h
        avg = 0.5 * ((fl_p + fr_p) - (fl_m + fr_m)) / h
        if m <= 7:
            assert abs(up - exact) < 1e-11
        else:
            assert abs(up - exact) > 1e-9
        if m <= 8:
            assert abs(avg - exact) < 1e-11
        else:
            assert abs(avg - exact) > 1e-9


# ---------------------------------------------------------- Eq. detector ----
def test_psi_hand_cases(oracle_mod):
    """Eq. detector with the printed epsilon: uniform and linear data give 1,
    a step gives ~0, and psi is symmetric under reflection."""
    assert oracle_mod.psi([2.0] * 5) == 1.0
    assert abs(oracle_mod.psi([1.0, 1.5, 2.0, 2.5, 3.0]) - 1.0) < 1e-15
    assert oracle_mod.psi([1.0, 1.0, 1.0, 5.0, 5.0]) < 1e-6
    rng = _rng(6)
    for _ in range(50):
        r = rng.uniform(0.1, 2.0, 5)
        assert abs(oracle_mod.psi(r) - oracle_mod.psi(r[::-1])) < 1e-15
    # a = 0, b > 0 gives eps / (b^2 + eps): eps = 0.45/0.55 * 1e-6
    b = 1e-3
    eps = 0.9 * 0.5 / (1 - 0.9 * 0.5) * 1e-6
    assert abs(oracle_mod.psi([1, 1, 1, 1 + b, 1 + 2 * b]) - eps / (b * b + eps)) < 1e-12


# -------------------------------------------------------- Eq. mp-procedure ----
def test_meg7_no_new_extrema_at_a_step(oracle_mod):
    """Sec. 2.3: across a jump between two constant states the MP-limited left
    value stays inside the two states, while the linear GRB value (Eq. grb,
    with the gradients of Eq. six) overshoots for many step positions."""
    rng = _rng(7)
    k = np.arange(-5, 6)   # cells j-5..j+5, j = 0
    overshoot_linear = 0
    for _ in range(3000):
        a, b = rng.normal(size=2) * 3
        f = np.where(k >= rng.integers(-3, 5), b, a)
        d = np.array([oracle_mod.grad6(f[i - 3:i + 4]) for i in range(3, 8)])
        lo, hi = min(a, b), max(a, b)
        v = oracle_mod.meg7_left(f[3:8], d)
        assert lo - 1e-12 <= v <= hi + 1e-12
        g = oracle_mod.grb_left(f[3:8], d)
        overshoot_linear += not (lo - 1e-12 <= g <= hi + 1e-12)
    assert overshoot_linear > 500


def test_meg7_smooth_data_keeps_linear_value(oracle_mod):
    """On smooth monotone data the MP condition (Eq. mp5Condition) holds and
    MEG7 returns the GRB value unchanged."""
    h = 0.05
    for x0 in np.linspace(0.2, 1.2, 11):
        x = x0 + h * np.arange(-5, 6)
        f = np.sin(x)
        d = np.array([oracle_mod.grad6(f[i - 3:i + 4]) for i in range(3, 8)])
        ph = f[3:8]
        assert oracle_mod.meg7_left(ph, d) == oracle_mod.grb_left(ph, d)


def test_meg7_right_mirrors_left(oracle_mod):
    rng = _rng(8)
    for _ in range(200):
        ph, dp = rng.normal(size=5), rng.normal(size=5)
        assert oracle_mod.meg7_right(ph, dp) == oracle_mod.meg7_left(ph[::-1], -dp[::-1])


# ------------------------------------------------------------------ HLLC ----
def _euler_flux(g, W):
    r, u, v, p = W
    E = p / (g - 1) + 0.5 * r * (u * u + v * v)
    return np.array([r * u, r * u * u + p, r * u * v, u * (E + p)]), np.array([r, r * u, r * v, E])


def _hllc_branch(g, WL, WR):
    """Textbook branch-form HLLC (Toro, Riemann Solvers, Sec. 10.4) with the
    Einfeldt/Roe wave-speed bounds; written independently of the oracle."""
    FL, QL = _euler_flux(g, WL)
    FR, QR = _euler_flux(g, WR)
    rL, uL, vL, pL = WL
    rR, uR, vR, pR = WR
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    w = np.sqrt(rR / rL)
    ub = (uL + w * uR) / (1 + w)
    vb = (vL + w * vR) / (1 + w)
    HL, HR = (QL[3] + pL) / rL, (QR[3] + pR) / rR
    Hb = (HL + w * HR) / (1 + w)
    cb = np.sqrt((g - 1) * (Hb - 0.5 * (ub * ub + vb * vb)))
    SL, SR = min(uL - cL, ub - cb), max(uR + cR, ub + cb)
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(r, u, v, p, Q, S):
        k = r * (S - u) / (S - Ss)
        return k * np.array([1.0, Ss, v, Q[3] / r + (Ss - u) * (Ss + p / (r * (S - u)))])
    if SL >= 0:
        return FL, 0
    if Ss >= 0:
        return FL + SL * (star(*WL, QL, SL) - QL), 1
    if SR >= 0:
        return FR + SR * (star(*WR, QR, SR) - QR), 2
    return FR, 3


def test_hllc_abs_form_equals_branch_form(oracle_mod):
    """Eq. Riemann_revisit's |A| form equals textbook HLLC when F_L = F(Q_L),
    F_R = F(Q_R), over random state pairs that hit all four branches."""
    rng = _rng(9)
    g = 1.4
    hit = set()
    for _ in range(4000):
        WL = np.array([rng.uniform(0.1, 3), rng.normal() * 2, rng.normal(), rng.uniform(0.05, 3)])
        WR = np.array([rng.uniform(0.1, 3), rng.normal() * 2, rng.normal(), rng.uniform(0.05, 3)])
        FL, _ = _euler_flux(g, WL)
        FR, _ = _euler_flux(g, WR)
        got = oracle_mod.hllc(g, WL, WR, FL, FR)
        ref, branch = _hllc_branch(g, WL, WR)
        scale = 1 + np.abs(FL).max() + np.abs(FR).max()
        assert np.abs(got - ref).max() < 1e-12 * scale
        hit.add(branch)
    assert hit == {0, 1, 2, 3}


def test_hllc_stationary_contact_and_consistency(oracle_mod):
    g = 1.4
    WL, WR = np.array([2.0, 0.0, 0.3, 1.0]), np.array([0.5, 0.0, -0.7, 1.0])
    FL, _ = _euler_flux(g, WL)
    FR, _ = _euler_flux(g, WR)
    assert np.array_equal(oracle_mod.hllc(g, WL, WR, FL, FR), np.array([0.0, 1.0, 0.0, 0.0]))
    W = np.array([1.3, 0.4, -0.2, 0.9])
    F, _ = _euler_flux(g, W)
    assert np.abs(oracle_mod.hllc(g, W, W, F, F) - F).max() < 1e-15


# ------------------------------------- MP bounds: closed forms (Sec. 2.3) ----
# Each case makes one bound of Eq. mp-procedure the binding one, so that the
# limited left value at j+1/2 equals a value fixed by that bound alone.
# phi, dphi: Phi_{j-2..j+2} and the dx-scaled Phi'_{j-2..j+2}. The curvatures
# d_k of Eq. mp-procedure are noted beside each case; the gradients are chosen
# so that the minmod in MD (of d_j, d_{j+1}) or in LC (of d_j, d_{j-1}) is
# decided by one named curvature, while the other pairing would give 0. In
# every case the GRB value lies beyond the binding bound, so the MP test
# (Eq. mp5Condition) fails and the limiter returns that bound.
MP_BOUND_CASES = {
    # Gentle rise Phi_j - Phi_{j-1} = 0.01 then a steep one: the upper limit
    # UL = Phi_j + xi (Phi_j - Phi_{j-1}), xi = 7 (Eq. alpha), binds.
    # d_{j-1} = -0.48, d_j = 17.96: LC = Phi_j + 0.005 stays below UL.
    "UL": ([1.0, 1.0, 1.01, 10.0, 19.0], [0.0, 0.0, 1.0, 0.0, 0.0], 1.01 + 7 * 0.01),
    # Steep rise onto a flat top (Phi_j = Phi_{j+1} = 4): the median bound
    # MD = (Phi_j + Phi_{j+1})/2 - minmod(d_j, d_{j+1})/2 binds.
    # d_{j-1} = 7, d_j = -1, d_{j+1} = -2: MD = 4 + 1/2.
    "MD_dj": ([0.0, 0.0, 4.0, 4.0, 4.0], [0.0, 14.0, 2.0, 0.0, 6.0], 4.5),
    # d_{j-1} = 7, d_j = -2, d_{j+1} = -1: MD = 4 + 1/2 again, now set by d_{j+1}.
    "MD_djp1": ([0.0, 0.0, 4.0, 4.0, 4.0], [0.0, 12.0, 2.0, 0.0, 4.0], 4.5),
    # Fall of 1 into a steep drop: the large-curvature bound
    # LC = Phi_j + (Phi_j - Phi_{j-1})/2 + 4/3 minmod(d_j, d_{j-1}) binds.
    # d_{j-1} = -6, d_j = -7, d_{j+1} = 13: LC = 1 - 1/2 - 8.
    "LC_djm1": ([-4.0, 2.0, 1.0, -10.0, -10.0], [-2.0, 0.0, -18.0, -26.0, 0.0], -7.5),
    # d_{j-1} = -7, d_j = -6, d_{j+1} = 13: LC = -7.5 again, set by d_j.
    "LC_dj": ([-4.0, 2.0, 1.0, -10.0, -10.0], [-4.0, 0.0, -18.0, -28.0, 0.0], -7.5),
}


@pytest.mark.parametrize("name", sorted(MP_BOUND_CASES))
@pytest.mark.parametrize("sign", [1.0, -1.0], ids=["upper", "lower"])
def test_mp_bounds_closed_forms(oracle_mod, name, sign):
    """The MD, UL and LC bounds of Eq. mp-procedure, one at a time. The
    procedure is odd (minmod is odd; min and max swap under negation), so the
    negated data test the other side (Phi^min instead of Phi^max) with the
    negated expected value. Also checks that the MP test fails (the limiter
    runs) and that the right value of the mirrored stencil is the same."""
    phi, dphi, expect = MP_BOUND_CASES[name]
    phi, dphi, expect = sign * np.array(phi), sign * np.array(dphi), sign * expect
    grb = oracle_mod.grb_left(phi, dphi)
    pj, pjm1, pjp1 = phi[2], phi[1], phi[3]
    a, b = pjp1 - pj, 7.0 * (pj - pjm1)
    pmp = pj + (0.0 if a * b <= 0 else (min(a, b) if a > 0 else max(a, b)))
    assert (grb - pj) * (grb - pmp) > 1e-40          # the limiter runs
    got = oracle_mod.meg7_left(phi, dphi)
    assert abs(got - expect) <= 1e-14 * (1 + abs(expect)), (got, expect, grb)
    assert oracle_mod.meg7_right(phi[::-1], -dphi[::-1]) == got


@pytest.mark.parametrize("offset", np.linspace(-0.45, 0.45, 19))
def test_mp_smooth_extremum_keeps_grb(oracle_mod, offset):
    """Sec. 2.3 adopts the MP bounds of Suresh and Huynh so that smooth
    extrema are not clipped. A cosine sampled at 24 cells per wavelength
    with its maximum near the face j+1/2: where the maximum lies between
    cells j and j+1, the GRB value lies above both of them, so Eq.
    mp5Condition fails and the limiter runs, yet
    the curvature-aware bounds MD and LC admit the GRB value and MEG7
    returns it unchanged. A monotonicity bound [min, max](Phi_j, Phi_{j+1})
    would have clipped it."""
    h = 2 * np.pi / 24
    x = (np.arange(-5, 6) - 0.5 - offset) * h   # cells j-5..j+5; peak at j+1/2+offset
    f = np.cos(x)
    d = np.array([oracle_mod.grad6(f[i - 3:i + 4]) for i in range(3, 8)])
    ph = f[3:8]
    grb = oracle_mod.grb_left(ph, d)
    pj = ph[2]
    a, b = ph[3] - pj, 7.0 * (pj - ph[1])
    pmp = pj + (0.0 if a * b <= 0 else (min(a, b) if a > 0 else max(a, b)))
    assert oracle_mod.meg7_left(ph, d) == grb
    if abs(offset) < 0.3:   # the maximum lies between cells j and j+1
        assert (grb - pj) * (grb - pmp) > 1e-40      # the limiter runs
        assert grb > max(ph[2], ph[3])               # a plain monotone bound would clip


# ----------------------- characteristic projection (reading R2, Sec. 2.3) ----
def _prim_jacobian(w, g=1.4):
    """A = (dQ/dU)^-1 dF/dU of the Euler x-flux F(Q(U)) in primitive variables
    U = (rho, u, v, p), both factors by complex-step differentiation."""
    def Q_of(U):
        r, u, v, p = U
        return np.array([r, r * u, r * v, p / (g - 1) + 0.5 * r * (u * u + v * v)])

    def F_of(U):
        r, u, v, p = U
        E = p / (g - 1) + 0.5 * r * (u * u + v * v)
        return np.array([r * u, r * u * u + p, r * u * v, u * (E + p)])
    dQ = np.zeros((4, 4))
    dF = np.zeros((4, 4))
    for k in range(4):
        U = np.array(w, complex)
        U[k] += 1e-30j
        dQ[:, k] = np.imag(Q_of(U)) / 1e-30
        dF[:, k] = np.imag(F_of(U)) / 1e-30
    return np.linalg.solve(dQ, dF)


def test_prim_eigenvectors_diagonalise_the_primitive_jacobian(oracle_mod):
    """The matrices the MEG7-prim face projection uses (reading R2): L R = I
    and L A R = diag(u - c, u, u, u + c), in that field order, with A the
    primitive-variable Jacobian of the Euler x-flux. A sign slip in l1/l4 or
    r1/r4 swapped consistently with L keeps L R = I but breaks this."""
    rng = _rng(11)
    for _ in range(20):
        w = np.array([rng.uniform(0.2, 3), rng.normal(), rng.normal(), rng.uniform(0.1, 3)])
        L, R = oracle_mod.prim_eigenvectors(1.4, w)
        assert np.abs(L @ R - np.eye(4)).max() < 1e-13
        A = _prim_jacobian(w)
        c = np.sqrt(1.4 * w[3] / w[0])
        D = L @ A @ R
        lam = np.array([w[1] - c, w[1], w[1], w[1] + c])
        assert np.abs(D - np.diag(lam)).max() < 1e-12 * (1 + np.abs(lam).max())
