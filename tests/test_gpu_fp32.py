"""FP32 form: stencil, reconstruction and flux arithmetic in FP32, stage
accumulation and positivity in FP64. Its error is stated against the FP64
oracle: density L1 error relative to the oracle's density L1 norm must stay
below 1e-5 over many steps, on smooth and on discontinuous data."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

pytestmark = pytest.mark.gpu

L1_TOL = 1e-5


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


def l1_rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("name,make,steps", [
    ("vortex64", lambda: C.isentropic_vortex(64), 100),
    ("riemann256", lambda: C.riemann_2d(256), 60),
    ("vst128x64", lambda: C.viscous_shock_tube(128, 64), 40),
    ("kh128", lambda: C.kelvin_helmholtz(128, np.random.default_rng(2)), 60),
], ids=lambda x: x if isinstance(x, str) else "")
def test_fp32_density_l1_vs_oracle(env, name, make, steps):
    torch, O, gbr = env
    c = make()
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)
    s = gbr.Solver.for_case(c, precision=32)
    s.set_state(c.Q)
    Q = c.Q.copy()
    for _ in range(steps):
        dt = 0.8 * c.cfl / O.max_wavespeed(cfg, Q)   # same dt on both sides
        s.step(dt)
        Q, rc = O.rk3_step(cfg, Q, dt)
        assert rc == 0
    Qg = s.get_state()
    err = l1_rel(Qg[0], Q[0])
    print(f"{name}: FP32 density L1 rel error after {steps} steps = {err:.3e}")
    assert err <= L1_TOL, err
    assert err > 0.0        # it really ran in FP32
    s.close()
