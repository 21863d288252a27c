"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs, element by element (FP64: 1e-12 relative per field;
detector flags identical except at psi ties)."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C

from .parity import (TOL64, assert_residual_close, assert_state_close, field_errors,
                     residual_scales, state_scales, tie_faces_ok)

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


def cfg_of(O, c):
    return O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)


SMALL = [
    ("vortex64", lambda: C.isentropic_vortex(64)),
    ("vortex_ragged", lambda: C.isentropic_vortex(50, 37)),
    ("riemann96", lambda: C.riemann_2d(96)),
    ("riemann_ragged", lambda: C.riemann_2d(70, 45)),
    ("vst64x32", lambda: C.viscous_shock_tube(64, 32)),
    ("vst_ragged", lambda: C.viscous_shock_tube(45, 29)),
    ("kh48", lambda: C.kelvin_helmholtz(48, np.random.default_rng(5))),
    ("tiny6", lambda: C.riemann_2d(6, 7)),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_residual_and_flags(env, name, make):
    torch, O, gbr = env
    c = make()
    s = gbr.Solver.for_case(c)
    s.record_flags(True)
    s.set_state(c.Q)
    R = s.residual()
    sx, sy = s.flags()
    Ro, sxo, syo = O.residual(cfg_of(O, c), c.Q, want_flags=True)
    excl = tie_faces_ok(O, cfg_of(O, c), c.Q, sx, sxo, sy, syo)
    assert_residual_close(R, Ro, c.Q, c, exclude=excl, what=f"{name} residual")
    s.close()


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_one_rk3_step(env, name, make):
    torch, O, gbr = env
    c = make()
    s = gbr.Solver.for_case(c)
    s.set_state(c.Q)
    lam = s.max_wavespeed()
    lam_o = O.max_wavespeed(cfg_of(O, c), c.Q)
    assert abs(lam - lam_o) <= 1e-14 * lam_o
    dt = c.cfl / lam_o
    s.step(dt)
    Q1 = s.get_state()
    Qo, rc = O.rk3_step(cfg_of(O, c), c.Q, dt)
    assert rc == 0
    assert_state_close(Q1, Qo, what=f"{name} step")
    lam1 = s.max_wavespeed()
    assert abs(lam1 - O.max_wavespeed(cfg_of(O, c), Qo)) <= 1e-12 * lam1
    s.close()


def test_vortex_100_stages(env):
    """Config 1: 64^2 vortex, 100 RK stages at CFL 0.5 through the
    device-side dt path; every step matches the oracle."""
    torch, O, gbr = env
    c = C.isentropic_vortex(64)
    cfg = cfg_of(O, c)
    s = gbr.Solver.for_case(c)
    s.set_state(c.Q)
    Q = c.Q.copy()
    worst = 0.0
    for k in range(34):   # 34 steps = 102 stages
        dt = 0.5 / O.max_wavespeed(cfg, Q)
        s.step_cfl(0.5)
        Q, rc = O.rk3_step(cfg, Q, dt)
        assert rc == 0
        if k % 11 == 10 or k == 33:
            worst = max(worst, max(field_errors(s.get_state(), Q, scales=state_scales(Q))))
    assert worst <= TOL64 * 10, worst   # 34 steps of roundoff growth
    t = s.time()
    assert t > 0
    s.close()


def test_device_buffers_and_streams(env):
    """Device tensors in and out (on_device = 1) on a torch stream."""
    torch, O, gbr = env
    c = C.riemann_2d(64, 48)
    st = torch.cuda.Stream()
    s = gbr.Solver.for_case(c, stream=st.cuda_stream)
    Qd = torch.from_numpy(c.Q).cuda()
    with torch.cuda.stream(st):
        s.set_state(Qd)
        Rd = torch.empty_like(Qd)
        gbr.gbr_residual(s.ctx, Rd, c.nx, c.ny)
        s.step(1e-4)
        Qout = torch.empty_like(Qd)
        gbr.gbr_get_state(s.ctx, Qout, c.nx, c.ny)
    st.synchronize()
    Ro = O.residual(cfg_of(O, c), c.Q)
    assert_residual_close(Rd.cpu().numpy(), Ro, c.Q, c, what="device residual")
    Qo, _ = O.rk3_step(cfg_of(O, c), c.Q, 1e-4)
    assert_state_close(Qout.cpu().numpy(), Qo, what="device step")
    s.close()


def test_checkpoint_resume_bitwise(env):
    """get_state / set_state round trip: a resumed run is bitwise identical."""
    torch, O, gbr = env
    c = C.kelvin_helmholtz(64, np.random.default_rng(1))
    a = gbr.Solver.for_case(c)
    a.set_state(c.Q)
    for _ in range(3):
        a.step_cfl(0.5)
    mid = a.get_state()
    b = gbr.Solver.for_case(c)
    b.set_state(mid)
    for _ in range(3):
        a.step(1e-3)
        b.step(1e-3)
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_nonphysical_state_reported(env):
    """A negative-pressure cell makes the next synchronising call report
    GBR_ERR_NONPHYSICAL (no trap, the context stays usable)."""
    torch, O, gbr = env
    c = C.riemann_2d(32)
    Q = c.Q.copy()
    Q[3, 10, 10] = 0.5 * (Q[1, 10, 10] ** 2 + Q[2, 10, 10] ** 2) / Q[0, 10, 10] - 0.05
    s = gbr.Solver.for_case(c)
    s.set_state(Q)
    s.step(1e-4)
    assert s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,)) == gbr.GBR_ERR_NONPHYSICAL
    s.set_state(c.Q)          # a fresh state clears the error word
    s.step(1e-4)
    assert s.sync() == gbr.GBR_OK
    s.close()


def test_full_size_riemann_1024(env):
    """Config 2 at full size (1024^2, transmissive), in the launch
    configuration the benchmark times: whole-grid residual parity and one
    RK3 step."""
    torch, O, gbr = env
    c = C.riemann_2d(1024)
    cfg = cfg_of(O, c)
    s = gbr.Solver.for_case(c)
    s.record_flags(True)
    s.set_state(c.Q)
    R = s.residual()
    sx, sy = s.flags()
    Ro, sxo, syo = O.residual(cfg, c.Q, want_flags=True)
    excl = tie_faces_ok(O, cfg, c.Q, sx, sxo, sy, syo)
    assert_residual_close(R, Ro, c.Q, c, exclude=excl, what="riemann1024 residual")
    dt = 0.5 / O.max_wavespeed(cfg, c.Q)
    s.step(dt)
    Qo, rc = O.rk3_step(cfg, c.Q, dt)
    assert rc == 0
    assert_state_close(s.get_state(), Qo, what="riemann1024 step")
    s.close()


def _sample_mask(Q, rng, n=4000):
    """Boundary cells, random cells, and random cells within 8 cells of a
    jump of the initial density (where the residual is non-zero)."""
    ny, nx = Q.shape[1:]
    m = np.zeros((ny, nx), np.uint8)
    m[rng.integers(0, ny, n), rng.integers(0, nx, n)] = 1
    jump = np.zeros((ny, nx), bool)
    jump[:, 1:] |= Q[0][:, 1:] != Q[0][:, :-1]
    jump[1:, :] |= Q[0][1:, :] != Q[0][:-1, :]
    near = np.zeros_like(jump)
    for d in range(-8, 9):
        near |= np.roll(jump, d, axis=0) | np.roll(jump, d, axis=1)
    ii, jj = np.nonzero(near)
    pick = rng.choice(len(ii), size=min(n, len(ii)), replace=False)
    m[ii[pick], jj[pick]] = 1
    m[0, :] = 1
    m[-1, :] = 1
    m[:, 0] = 1
    m[:, -1] = 1
    return m


FULL = {"riemann4096": lambda: C.riemann_2d(4096),
        "vst2048x1024": lambda: C.viscous_shock_tube(2048, 1024),
        "riemann8192x6144": lambda: C.riemann_2d(8192, 6144)}


@pytest.mark.parametrize("which", list(FULL))
def test_full_size_sampled(env, which):
    """Configs 3 and 4 at full size, and a 8192 x 6144 grid (50 M cells,
    padded planes of 50.5 M doubles: index arithmetic far past the benchmark's
    sizes, ragged in y): the residual at sampled cells (all boundary cells
    plus random interior ones), computed one by one by the oracle from the
    same state."""
    torch, O, gbr = env
    c = FULL[which]()
    cfg = cfg_of(O, c)
    s = gbr.Solver.for_case(c)
    s.set_state(c.Q)
    R = s.residual()
    mask = _sample_mask(c.Q, np.random.default_rng(7))
    Ro = O.residual(cfg, c.Q, mask=mask)
    sel = mask.astype(bool)
    sc = residual_scales(c.Q, c.dx, c.dy, c.gamma)
    sc = [max(sc[m], np.abs(Ro[m][sel]).max()) for m in range(4)]
    errs = [np.abs(R[m][sel] - Ro[m][sel]).max() / sc[m] for m in range(4)]
    assert max(np.abs(Ro[m][sel]).max() for m in range(4)) > 0   # samples hit the discontinuities
    assert max(errs) <= TOL64, errs
    s.close()


@pytest.mark.parametrize("name,make", [("vortex64", lambda: C.isentropic_vortex(64)),
                                       ("riemann70x45", lambda: C.riemann_2d(70, 45)),
                                       ("vst45x29", lambda: C.viscous_shock_tube(45, 29))],
                         ids=["vortex64", "riemann70x45", "vst45x29"])
def test_fourth_order_member(env, name, make):
    """GBR_OPT_ORDER = 4 (alpha = 4, beta = 0, Eq. fourth) against the oracle
    with order = 4: residual and one RK3 step."""
    torch, O, gbr = env
    c = make()
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc, 4)
    s = gbr.Solver.for_case(c, order=4)
    s.set_state(c.Q)
    assert_residual_close(s.residual(), O.residual(cfg, c.Q), c.Q, c, what=f"{name} order-4 residual")
    dt = c.cfl / O.max_wavespeed(cfg, c.Q)
    s.step(dt)
    Qo, rc = O.rk3_step(cfg, c.Q, dt)
    assert rc == 0
    assert_state_close(s.get_state(), Qo, what=f"{name} order-4 step")
    s.close()


CONS_CASES = [("vortex64", lambda: C.isentropic_vortex(64)),
              ("riemann70x45", lambda: C.riemann_2d(70, 45)),
              ("kh48", lambda: C.kelvin_helmholtz(48, np.random.default_rng(5))),
              ("vst45x29", lambda: C.viscous_shock_tube(45, 29))]


@pytest.mark.parametrize("name,make", CONS_CASES, ids=[x[0] for x in CONS_CASES])
def test_meg7_cons(env, name, make):
    """GBR_OPT_VARIABLES = 1 (MEG7-cons) against the oracle with cons = 1:
    residual and flags, then two RK3 steps."""
    torch, O, gbr = env
    c = make()
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc, 7, 1)
    s = gbr.Solver.for_case(c, cons=True)
    s.record_flags(True)
    s.set_state(c.Q)
    R = s.residual()
    sx, sy = s.flags()
    Ro, sxo, syo = O.residual(cfg, c.Q, want_flags=True)
    excl = tie_faces_ok(O, cfg, c.Q, sx, sxo, sy, syo)
    assert_residual_close(R, Ro, c.Q, c, exclude=excl, what=f"{name} cons residual")
    Q = c.Q.copy()
    for _ in range(2):
        dt = c.cfl / O.max_wavespeed(cfg, Q)
        s.step(dt)
        Q, rc = O.rk3_step(cfg, Q, dt)
        assert rc == 0
    assert_state_close(s.get_state(), Q, what=f"{name} cons steps")
    s.close()


def test_viscous_shock_tube_time_step(env):
    """Config 3 at full size (2048 x 1024), where the viscous bound of Sec.
    2.5 decides dt: 100 steps at the paper's CFL 0.2 stay physical (t grows
    by 100 viscous-limited steps); at CFL 0.5 the alpha-damping heat
    conduction is beyond TVD-RK3's stability interval and the state turns
    non-physical within 60 steps, which the positivity check reports
    (GBR_ERR_NONPHYSICAL, no fault) rather than a silent blow-up."""
    torch, O, gbr = env
    c = C.viscous_shock_tube(2048, 1024)
    assert c.cfl == 0.2
    s = gbr.Solver.for_case(c)
    s.set_state(c.Q)
    lam0 = s.max_wavespeed()
    assert lam0 > 3 * 2048 * 1.0              # viscous bound 4 nu/dx^2 dominates (|u| + c)/dx ~ 2048
    for _ in range(100):
        s.step_cfl(c.cfl)
    assert s.sync() == gbr.GBR_OK
    Q = s.get_state()
    p = 0.4 * (Q[3] - 0.5 * (Q[1] ** 2 + Q[2] ** 2) / Q[0])
    assert np.all(np.isfinite(Q)) and Q[0].min() > 0 and p.min() > 0
    assert 0.5 * 100 * c.cfl / lam0 < s.time() < 1.5 * 100 * c.cfl / lam0
    s.close()
    s = gbr.Solver.for_case(c)
    s.set_state(c.Q)
    for _ in range(60):
        s.step_cfl(0.5)
    assert s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,)) == gbr.GBR_ERR_NONPHYSICAL
    s.close()


def _rough_low_mach(n, seed):
    """Seeded cell-to-cell random rho, p in [0.5, 1.5] and u, v ~ N(0, 0.02)
    on the periodic unit square: low-Mach jumps on every face (the
    shock-stable flux's phi < 1 everywhere, the detector flagging many
    faces)."""
    rng = np.random.default_rng(seed)
    r, p = rng.uniform(0.5, 1.5, (n, n)), rng.uniform(0.5, 1.5, (n, n))
    u, v = rng.normal(0, 0.02, (n, n)), rng.normal(0, 0.02, (n, n))
    Q = np.ascontiguousarray(C.prim_to_cons(r, u, v, p, 1.4))
    return C.Case("rough_low_mach", Q, 1.0 / n, 1.0 / n, 1.4, 0.0, 0.72, (C.BC_PERIODIC,) * 4)


VARIANTS = {"cons_riemann1024": (lambda: C.riemann_2d(1024), {"cons": True}, {"cons": 1}),
            "order4_riemann1024": (lambda: C.riemann_2d(1024), {"order": 4}, {"order": 4}),
            "hllc_lm_rough1024": (lambda: _rough_low_mach(1024, 21), {"riemann": 1}, {"riemann": 1})}


@pytest.mark.parametrize("which", list(VARIANTS))
def test_full_size_variants_sampled(env, which):
    """The scheme variants the benchmark times on 1024^2 grids (MEG7-cons,
    the fourth-order member, the shock-stable HLLC-LM), in its launch
    configuration: the residual at sampled cells (every boundary cell plus
    random interior ones near the jumps) against the oracle's, computed one
    by one from the same state."""
    torch, O, gbr = env
    make, kw, okw = VARIANTS[which]
    c = make()
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc, okw.get("order", 7), okw.get("cons", 0),
                   riemann=okw.get("riemann", 0))
    s = gbr.Solver.for_case(c, **kw)
    s.set_state(c.Q)
    R = s.residual()
    mask = _sample_mask(c.Q, np.random.default_rng(8))
    Ro = O.residual(cfg, c.Q, mask=mask)
    sel = mask.astype(bool)
    sc = residual_scales(c.Q, c.dx, c.dy, c.gamma)
    sc = [max(sc[m], np.abs(Ro[m][sel]).max()) for m in range(4)]
    errs = [np.abs(R[m][sel] - Ro[m][sel]).max() / sc[m] for m in range(4)]
    assert max(np.abs(Ro[m][sel]).max() for m in range(4)) > 0
    assert max(errs) <= TOL64, errs
    s.close()
