"""gbr_step_static: the RK3 step for callers that cannot allocate device
memory at run time (a host application that owns all device memory through
its own pool, a real-time loop that must not enter the driver's allocator, a
process near its memory limit). It must give the same result as gbr_step,
which works on buffers allocated by gbr_create, on consecutive calls that
share its static scratch array. This file is collected last so that a failure
here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .parity import TOL64, assert_state_close

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
    return torch, gbr, O


@pytest.mark.parametrize("make", [lambda: C.isentropic_vortex(64),
                                  lambda: C.viscous_shock_tube(48, 40),
                                  lambda: C.riemann_2d(256)],
                         ids=["vortex64", "vst48x40", "riemann256"])
def test_static_step_matches_gbr_step_twice(env, make):
    """Two calls in a row (the second reuses the array the first left
    behind) and one in place: bit for bit the states gbr_step produces from
    its own cudaMalloc'ed buffers (the same kernels on the same inputs), and
    within 1e-12 of the oracle's RK3 step (Eq. rk) at the same dt."""
    torch, gbr, O = env
    c = make()
    ref = gbr.Solver.for_case(c)
    ref.set_state(c.Q)
    dt = 0.4 / ref.max_wavespeed()
    q0 = torch.from_numpy(c.Q).cuda()
    q1 = torch.empty_like(q0)
    q2 = torch.empty_like(q0)
    stream = torch.cuda.current_stream().cuda_stream
    args = (c.nx, c.ny, c.gamma, c.mu, c.Pr, c.bc, c.dx, c.dy, dt)
    assert gbr.gbr_step_static(q0, q1, *args, stream=stream) == gbr.GBR_OK
    assert gbr.gbr_step_static(q1, q2, *args, stream=stream) == gbr.GBR_OK
    ref.step(dt)
    r1 = ref.get_state()
    ref.step(dt)
    r2 = ref.get_state()
    assert np.array_equal(q1.cpu().numpy(), r1), "first static step differs from gbr_step"
    assert np.array_equal(q2.cpu().numpy(), r2), "second static step differs from gbr_step"
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)
    o1, rc1 = O.rk3_step(cfg, c.Q, dt)
    o2, rc2 = O.rk3_step(cfg, o1, dt)
    assert rc1 == 0 and rc2 == 0
    assert_state_close(q1.cpu().numpy(), o1, TOL64, what="first static step vs oracle")
    assert_state_close(q2.cpu().numpy(), o2, TOL64 * 2, what="second static step vs oracle")
    # in place
    q3 = q0.clone()
    assert gbr.gbr_step_static(q3, q3, *args, stream=stream) == gbr.GBR_OK
    assert np.array_equal(q3.cpu().numpy(), r1), "in-place static step differs from gbr_step"
    ref.close()


def test_static_step_allocates_no_device_memory(env):
    """After a warm-up call (which loads the library's code onto the device),
    further calls leave the device's free memory unchanged."""
    torch, gbr, _ = env
    c = C.riemann_2d(128)
    q0 = torch.from_numpy(c.Q).cuda()
    q1 = torch.empty_like(q0)
    stream = torch.cuda.current_stream().cuda_stream
    args = (c.nx, c.ny, c.gamma, c.mu, c.Pr, c.bc, c.dx, c.dy, 1e-4)
    assert gbr.gbr_step_static(q0, q1, *args, stream=stream) == gbr.GBR_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert gbr.gbr_step_static(q0, q1, *args, stream=stream) == gbr.GBR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_step_rejects_grids_beyond_capacity(env):
    torch, gbr, _ = env
    assert gbr.static_scratch_doubles(256, 256) <= gbr.GBR_STATIC_SCRATCH_DOUBLES
    assert gbr.static_scratch_doubles(300, 300) > gbr.GBR_STATIC_SCRATCH_DOUBLES
    c = C.riemann_2d(300)
    q = torch.from_numpy(c.Q).cuda()
    with pytest.raises(ValueError):
        gbr.gbr_step_static(q, q, c.nx, c.ny, c.gamma, c.mu, c.Pr, c.bc, c.dx, c.dy, 1e-4)
    # the C entry point itself refuses too, before touching anything
    b = gbr.gbr_bc(*c.bc, c.dx, c.dy)
    before = q.clone()
    rc = gbr.load().gbr_step_static(q.data_ptr(), q.data_ptr(), c.nx, c.ny, c.gamma, c.mu, c.Pr,
                                    ctypes.byref(b), 1e-4, None)
    assert rc == gbr.GBR_ERR_ARG
    assert torch.equal(q, before)


def test_static_step_reports_nonphysical(env):
    torch, gbr, _ = env
    c = C.riemann_2d(32)
    Q = c.Q.copy()
    Q[3, 10, 10] = 0.5 * (Q[1, 10, 10] ** 2 + Q[2, 10, 10] ** 2) / Q[0, 10, 10] - 0.05
    q = torch.from_numpy(Q).cuda()
    out = torch.empty_like(q)
    args = (c.nx, c.ny, c.gamma, c.mu, c.Pr, c.bc, c.dx, c.dy, 1e-4)
    assert gbr.gbr_step_static(q, out, *args, allow=(gbr.GBR_ERR_NONPHYSICAL,)) == gbr.GBR_ERR_NONPHYSICAL
    # the next call starts from a cleared error word
    good = torch.from_numpy(c.Q).cuda()
    assert gbr.gbr_step_static(good, out, *args) == gbr.GBR_OK
