"""Custom boundary sides on the CUDA path (fixed inflow states, kinds split
at a point that moves with time): Examples 7 (2D shock-entropy wave) and 8
(double Mach reflection) against the oracle, step by step with the moving
north side seen at each RK stage's time, and the double Mach reflection at
the paper's 1024 x 256 grid to t = 0.2."""
import dataclasses

import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .parity import assert_residual_close, assert_state_close, tie_faces_ok

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


def cfg_of(O, c, t=0.0, cons=0):
    return O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc, 7, cons, t=t, sides=c.meta["sides"])


CASES = [("dmr64x16", lambda: C.double_mach(64, 16)), ("dmr70x19", lambda: C.double_mach(70, 19)),
         ("se100x20", lambda: C.shock_entropy_2d(100, 20))]


@pytest.mark.parametrize("name,make", CASES, ids=[x[0] for x in CASES])
@pytest.mark.parametrize("cons", [0, 1], ids=["prim", "cons"])
def test_custom_sides_parity(env, name, make, cons):
    """Residual and flags at t = 0, then 6 RK3 steps (dt from the oracle's
    wavespeed) with the boundary time advancing; then a resumed run
    (gbr_set_time) from the oracle's state at that time."""
    torch, O, gbr = env
    c = make()
    s = gbr.Solver.for_case(c, cons=bool(cons))
    s.record_flags(True)
    s.set_state(c.Q)
    cfg = cfg_of(O, c, 0.0, cons)
    R = s.residual()
    sx, sy = s.flags()
    Ro, sxo, syo = O.residual(cfg, c.Q, want_flags=True)
    excl = tie_faces_ok(O, cfg, c.Q, sx, sxo, sy, syo)
    assert_residual_close(R, Ro, c.Q, c, exclude=excl, what=f"{name} residual")
    Q, t = c.Q.copy(), 0.0
    for k in range(6):
        dt = 0.5 / O.max_wavespeed(cfg, Q)
        s.step(dt)
        Q, rc = O.rk3_step(dataclasses.replace(cfg, t=t), Q, dt)
        assert rc == 0
        t += dt
    assert abs(s.time() - t) < 1e-15
    assert_state_close(s.get_state(), Q, tol=1e-11, what=f"{name} after 6 steps")
    s.set_state(Q)          # resume from the oracle's state at time t
    s.set_time(t)
    dt = 0.5 / O.max_wavespeed(cfg, Q)
    s.step(dt)
    Qo, rc = O.rk3_step(dataclasses.replace(cfg, t=t), Q, dt)
    assert_state_close(s.get_state(), Qo, what=f"{name} resumed step")
    s.close()


@pytest.mark.parametrize("cons,riemann", [(False, 0), (True, 0), (False, 1), (True, 1)],
                         ids=["prim", "cons", "prim-lm", "cons-lm"])
def test_double_mach_paper_grid(env, cons, riemann):
    """1024 x 256 to t = 0.2 (Example 8, with HLLC and with the shock-stable
    HLLC-LM the example names): positive throughout, and the incident shock,
    away from the wall, within two cells of its exact position
    x_s(y, t) = 1/6 + (y + 20 t)/sqrt(3) on rows y in [0.6, 0.95]."""
    torch, O, gbr = env
    import time
    c = C.double_mach(1024, 256)
    s = gbr.Solver.for_case(c, cons=cons, riemann=riemann)
    s.set_state(c.Q)
    steps = 0
    t0 = time.perf_counter()
    while True:
        t = s.time()
        if t >= 0.2 * (1 - 1e-14):
            break
        s.step_cfl(0.5, 0.2 - t)
        steps += 1
    Q = s.get_state()
    wall = time.perf_counter() - t0
    s.close()
    assert abs(t - 0.2) < 1e-13
    p = 0.4 * (Q[3] - 0.5 * (Q[1] ** 2 + Q[2] ** 2) / Q[0])
    assert np.all(np.isfinite(Q)) and Q[0].min() > 0 and p.min() > 0
    yc = (np.arange(c.ny) + 0.5) * c.dy
    xc = (np.arange(c.nx) + 0.5) * c.dx
    rows = np.nonzero((yc > 0.6) & (yc < 0.95))[0]
    for i in rows:
        j = np.nonzero(Q[0, i] < 0.5 * (8.0 + 1.4))[0][0]
        xs = 1.0 / 6.0 + (yc[i] + 20.0 * 0.2) / np.sqrt(3.0)
        assert abs(xc[j] - xs) < 2 * c.dx, (yc[i], xc[j], xs)
    print(f"double Mach {'cons' if cons else 'prim'}{'-lm' if riemann else ''} 1024x256 to t=0.2: {steps} steps, {wall:.2f} s "
          f"(host loop with a time read per step), rho in [{Q[0].min():.3f}, {Q[0].max():.3f}]")


def test_checkpoint_resume_is_bitwise(env, tmp_path):
    """Ten CFL steps of the double Mach reflection in one run, against five
    steps, a checkpoint file, a new solver resumed from it and five more
    steps: identical to the last bit (state and time)."""
    torch, O, gbr = env
    from paper_2305_00762_gb300 import checkpoint
    c = C.double_mach(96, 24)
    a = gbr.Solver.for_case(c, cons=True)
    a.set_state(c.Q)
    for _ in range(10):
        a.step_cfl(0.5)
    Qa, ta = a.get_state(), a.time()
    a.close()
    b = gbr.Solver.for_case(c, cons=True)
    b.set_state(c.Q)
    for _ in range(5):
        b.step_cfl(0.5)
    path = str(tmp_path / "dmr.npz")
    checkpoint.save(b, path, step=5)
    b.close()
    r, step = checkpoint.resume(path)
    assert step == 5
    for _ in range(5):
        r.step_cfl(0.5)
    assert np.array_equal(r.get_state(), Qa) and r.time() == ta
    r.close()
