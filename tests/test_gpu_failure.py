"""Failure detection without a GPU fault: the stage kernels' tile staging
waits on an mbarrier with an iteration limit. The test hook
GBR_OPT_STALL_TEST makes every CTA wait for bytes its copy never delivers:
the wait gives up, the kernel returns, the call reports GBR_ERR_TIMEOUT, and
the context stays usable (gbr_set_state clears the error)."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .parity import assert_residual_close

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


@pytest.mark.parametrize("precision", [64, 32])
def test_staging_wait_gives_up_and_context_recovers(env, precision):
    torch, O, gbr = env
    c = C.isentropic_vortex(32)
    s = gbr.Solver.for_case(c, precision=precision)
    s.set_state(c.Q)
    gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_STALL_TEST, 1)
    with pytest.raises(gbr.GbrError) as e:
        s.residual()
    assert e.value.status == gbr.GBR_ERR_TIMEOUT
    s.step(1e-3)  # asynchronous; the next synchronising call reports it
    assert s.sync(allow=(gbr.GBR_ERR_TIMEOUT,)) == gbr.GBR_ERR_TIMEOUT
    gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_STALL_TEST, 0)
    s.set_state(c.Q)
    assert s.sync() == gbr.GBR_OK
    R = s.residual()
    Ro, _, _ = O.residual(O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc), c.Q, want_flags=True)
    if precision == 64:
        assert_residual_close(R, Ro, c.Q, c, what="residual after recovery")
    else:
        assert np.abs(R - Ro).max() < 1e-4 * np.abs(Ro).max()
    s.close()


@pytest.mark.parametrize("mode", [1, 2], ids=["decision_pass", "fused"])
def test_tensor_core_wait_gives_up_and_context_recovers(env, mode):
    """The learned sensor waits, bounded, for its tcgen05 MMAs (in the
    decision pass, mode 1, or inside the stage kernel, mode 2); with
    GBR_OPT_STALL_TEST = 2 the first MMA batch is withheld, the wait gives
    up, the CTA frees its tensor memory and the call reports
    GBR_ERR_TIMEOUT; nothing faults and the context keeps working."""
    torch, O, gbr = env
    from paper_2305_00762_gb300 import sensor_train
    w = sensor_train.load_weights()
    c = C.isentropic_vortex(32)
    s = gbr.Solver.for_case(c, precision=32)
    s.set_state(c.Q)
    s.set_sensor(w)
    gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_SENSOR, mode)
    R0 = s.residual()
    gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_STALL_TEST, 2)
    with pytest.raises(gbr.GbrError) as e:
        s.residual()
    assert e.value.status == gbr.GBR_ERR_TIMEOUT
    gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_STALL_TEST, 0)
    s.set_state(c.Q)
    assert s.sync() == gbr.GBR_OK
    assert np.array_equal(s.residual(), R0)   # the same decisions as before the stall
    s.close()
