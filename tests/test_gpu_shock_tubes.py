"""Example 2 (Sod, Lax shock tubes on N = 200 strips) and Example 9 (the 2D
Riemann problem at the paper's 400^2 grid to t = 0.8) on the CUDA path: the
strips against the oracle run and the exact Riemann solution, the 2D run
through its mirror symmetry about x = y, positivity and the end time."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .exact_riemann import sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_2305_00762_gb300 import build, gbr
    build.build()
    O.build()
    gbr.load()
    return torch, O, gbr


def run_gpu(gbr, c, t_end, cfl=0.5, **kw):
    """Advance to t_end with dt = min(cfl / lambda, t_end - t), as the oracle's
    run does; lambda and dt stay on the device."""
    s = gbr.Solver.for_case(c, **kw)
    s.set_state(c.Q)
    steps = 0
    while True:
        t = s.time()
        if t >= t_end * (1 - 1e-14):
            break
        s.step_cfl(cfl, t_end - t)
        steps += 1
    Q = s.get_state()
    t = s.time()
    s.close()
    return Q, t, steps


@pytest.mark.parametrize("which", ["sod", "lax"])
@pytest.mark.parametrize("cons", [False, True], ids=["prim", "cons"])
def test_shock_tube(env, which, cons):
    torch, O, gbr = env
    left, right, t_end = C.SOD if which == "sod" else C.LAX
    c = C.shock_tube(200, left, right, t_end)
    Q, t, steps = run_gpu(gbr, c, t_end, cons=cons)
    assert abs(t - t_end) < 1e-14
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, 0.0, 0.72, c.bc, 7, int(cons))
    Qo, to, so = O.run(cfg, c.Q, t_end, 0.5)
    assert so == steps
    scale = np.abs(Qo).reshape(4, -1).max(axis=1)
    scale[1:3] = scale[1:3].max()
    err = (np.abs(Q - Qo).reshape(4, -1).max(axis=1) / scale).max()
    print(f"{which} {'cons' if cons else 'prim'}: {steps} steps, max rel diff to oracle {err:.2e}")
    # a few hundred steps of switching limiter and detector: rounding
    # differences grow from 1e-16 per step to at most ~1e-9
    assert err < 1e-8
    assert np.abs(Q - Q[:, :1]).max() == 0.0                # rows identical
    xc, _ = C.centres(200, 0.0, 1.0)
    ex = sample(left, right, (xc - 0.5) / t_end)
    l1 = np.abs(Q[0, 0] - ex[0]).mean()
    assert l1 < (0.006 if which == "sod" else 0.02), l1


@pytest.mark.parametrize("precision,cons", [(64, False), (32, False), (64, True)],
                         ids=["fp64-prim", "fp32-prim", "fp64-cons"])
def test_riemann_2d_paper_grid(env, precision, cons):
    """400^2 to t = 0.8: the initial data are mirror-symmetric about x = y
    (rho(x,y) = rho(y,x), u(x,y) = v(y,x)); x and y faces share one code
    path and the per-cell x and y work rounds alike, so the solution keeps
    that symmetry to the last bit, through 1700 steps of a flow whose slip
    lines amplify any asymmetry."""
    torch, O, gbr = env
    c = C.riemann_2d(400)
    Q, t, steps = run_gpu(gbr, c, 0.8, precision=precision, cons=cons)
    assert abs(t - 0.8) < 1e-13
    assert np.all(np.isfinite(Q)) and Q[0].min() > 0
    p = 0.4 * (Q[3] - 0.5 * (Q[1] ** 2 + Q[2] ** 2) / Q[0])
    assert p.min() > 0
    asym = max(np.abs(Q[0] - Q[0].T).max() / Q[0].max(),
               np.abs(Q[1] - Q[2].T).max() / np.abs(Q[1]).max(),
               np.abs(Q[3] - Q[3].T).max() / Q[3].max())
    print(f"riemann400 fp{precision} {'cons' if cons else 'prim'}: {steps} steps, asymmetry {asym:.2e}, rho in [{Q[0].min():.4f}, {Q[0].max():.4f}]")
    assert asym == 0.0
    # density stays near the range of the four initial states (Example 9)
    assert 0.05 < Q[0].min() and Q[0].max() < 2.0
