"""One grid split along y into slabs on one GPU (LocalSlabs): halo rows
copied between the slab contexts' buffers before every RK stage (Eq. rk) and
the wavespeed reduced across slabs after every step (Sec. 2.5) reproduce the
single-grid run bit for bit, which the other tests tie to the oracle. The
same bookkeeping drives one slab per GPU (DistSlab), whose exchange is
tested on the CPU with gloo ranks (tests/test_slab_gloo.py)."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00762_gb300 import build, gbr
    from paper_2305_00762_gb300 import slab as S
    build.build()
    gbr.load()
    return torch, gbr, S


CASES = [("riemann", lambda: C.riemann_2d(96, 70), 2),
         ("riemann", lambda: C.riemann_2d(96, 70), 3),
         ("vortex", lambda: C.isentropic_vortex(48, 50), 2),
         ("vortex", lambda: C.isentropic_vortex(48, 50), 4),
         ("vst", lambda: C.viscous_shock_tube(64, 40), 2),
         ("kh", lambda: C.kelvin_helmholtz(40, np.random.default_rng(3), ny=56), 3)]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name,make,n", CASES, ids=[f"{a}-{c}" for a, _, c in CASES])
def test_slabs_reproduce_single_grid(env, name, make, n, precision):
    torch, gbr, S = env
    c = make()
    cfl = getattr(c, "cfl", 0.5) or 0.5
    single = gbr.Solver.for_case(c, precision=precision)
    single.set_state(c.Q)
    slabs = S.LocalSlabs(c, n, precision=precision)
    slabs.set_state(c.Q)
    for _ in range(4):
        single.step_cfl(cfl)
        slabs.step_cfl(cfl)
    dt = 0.3 / single.max_wavespeed()
    single.step(dt)
    slabs.step(dt)
    assert np.array_equal(slabs.get_state(), single.get_state())
    assert slabs.time() == single.time()
    single.close()
    slabs.close()


def test_stage_order_and_halo_arguments_checked(env):
    torch, gbr, S = env
    c = C.riemann_2d(40, 36)
    slabs = S.LocalSlabs(c, 2)
    slabs.set_state(c.Q)
    s0 = slabs.solvers[0]
    with pytest.raises(gbr.GbrError):
        s0.step_stage(1)                     # a step starts with stage 0
    buf = torch.empty((4, 6, c.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(gbr.GbrError):
        s0.halo_copy(S.SOUTH, 1, buf)        # the first slab's south side is the grid's own
    s0.step_stage(0, 1e-4)
    with pytest.raises(gbr.GbrError):
        s0.step(1e-4)                        # no full step while one runs stage by stage
    s0.step_stage(1)
    s0.step_stage(2)
    s0.step(1e-4)
    slabs.close()
