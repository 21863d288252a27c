"""Example 2: the Sod and Lax shock tubes (N = 200, t = 0.2 and 0.14) against
the exact Riemann solution: small density L1 error that falls with N, over-
and undershoots within 1% of the exact solution's density range (Lax's
initial density jump, 0.055, is far smaller than that range, 0.96, so the
bound is taken on the range), MEG7-prim and MEG7-cons."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .exact_riemann import sample


def run(O, case, cons):
    cfg = O.Config(case.nx, case.ny, case.dx, case.dy, case.gamma, 0.0, 0.72, case.bc, 7, cons)
    Q, t, _ = O.run(cfg, case.Q, case.t_end, 0.5)
    return Q


@pytest.mark.parametrize("which", ["sod", "lax"])
@pytest.mark.parametrize("cons", [0, 1], ids=["prim", "cons"])
def test_shock_tube_vs_exact(oracle_mod, which, cons):
    O = oracle_mod
    left, right, t_end = C.SOD if which == "sod" else C.LAX
    errs = []
    for n in (200, 400):
        c = C.shock_tube(n, left, right, t_end)
        Q = run(O, c, cons)
        rho = Q[0]
        assert np.abs(rho - rho[0]).max() < 1e-12      # stays one-dimensional
        xc, _ = C.centres(n, 0.0, 1.0)
        ex = sample(left, right, (xc - 0.5) / t_end)
        errs.append(np.abs(rho[0] - ex[0]).mean())
        if n == 200:
            span = ex[0].max() - ex[0].min()     # density range of the exact solution
            assert rho[0].max() <= ex[0].max() + 0.01 * span
            assert rho[0].min() >= ex[0].min() - 0.01 * span
    assert errs[0] < (0.006 if which == "sod" else 0.02), errs
    assert errs[1] < 0.75 * errs[0], errs


@pytest.mark.parametrize("which", ["sod", "lax"])
def test_exact_solution_conserves(which):
    """The sampled exact solution itself: mass, momentum and energy on [0,1]
    change only by the boundary fluxes (no wave reaches x = 0 or 1), and the
    Sod star state is the textbook p* = 0.30313, u* = 0.92745."""
    from .exact_riemann import star_state
    g = 1.4
    left, right, t = C.SOD if which == "sod" else C.LAX
    x = (np.arange(400000) + 0.5) / 400000
    r, u, p = sample(left, right, (x - 0.5) / t, g)
    U = np.stack([r, r * u, p / (g - 1) + 0.5 * r * u * u])

    def flux(W):
        rr, uu, pp = W
        E = pp / (g - 1) + 0.5 * rr * uu * uu
        return np.array([rr * uu, rr * uu * uu + pp, uu * (E + pp)])

    U0 = 0.5 * (np.array([left[0], left[0] * left[1], left[2] / (g - 1) + 0.5 * left[0] * left[1] ** 2])
                + np.array([right[0], right[0] * right[1], right[2] / (g - 1) + 0.5 * right[0] * right[1] ** 2]))
    expect = U0 + t * (flux(left) - flux(right))
    assert np.allclose(U.mean(axis=1), expect, rtol=0, atol=2e-5)
    if which == "sod":
        ps, us = star_state(left, right, g)
        assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5
