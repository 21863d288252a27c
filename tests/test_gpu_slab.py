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


def _dist_rank(rank, ws, port, name, steps, out):
    """One rank of a DistSlab run: all ranks share GPU 0 and talk over gloo
    (halo rows and the wavespeed through pinned host buffers); no kernel
    waits on another process."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_2305_00762_gb300 import gbr
    from paper_2305_00762_gb300 import slab as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    gbr.load()
    c = dict(DIST_CASES)[name]()
    sl = S.DistSlab(c, rank, ws, transport="host")
    sl.set_state(np.ascontiguousarray(c.Q[:, sl.i0:sl.i1, :]))
    for _ in range(steps):
        sl.step_cfl(0.5)
    out[rank] = (sl.get_state(), sl.time())
    sl.close()
    dist.destroy_process_group()


DIST_CASES = [("riemann96x70", lambda: C.riemann_2d(96, 70)),
              ("vortex48x50", lambda: C.isentropic_vortex(48, 50))]


@pytest.mark.parametrize("name,ws", [("riemann96x70", 2), ("riemann96x70", 3), ("vortex48x50", 2)])
def test_dist_slabs_reproduce_single_grid(env, name, ws):
    """DistSlab, the one-slab-per-rank driver the benchmark runs under
    torchrun, here as ws processes sharing one GPU (gloo, host transport):
    five CFL steps with halo messages before every stage and the wavespeed
    max all-reduced after every step give the single-grid state bit for bit
    (periodic in y: the first and last slabs exchange across the seam)."""
    torch, gbr, S = env
    import socket
    import torch.multiprocessing as mp
    c = dict(DIST_CASES)[name]()
    single = gbr.Solver.for_case(c)
    single.set_state(c.Q)
    for _ in range(5):
        single.step_cfl(0.5)
    ref, t_ref = single.get_state(), single.time()
    single.close()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    with mp.get_context("spawn").Manager() as m:  # no fork after CUDA or threads start
        out = m.dict()
        mp.spawn(_dist_rank, args=(ws, port, name, 5, out), nprocs=ws, join=True)
        parts = [out[r] for r in range(ws)]
    assert np.array_equal(np.concatenate([p[0] for p in parts], axis=1), ref)
    assert all(p[1] == t_ref for p in parts)


def _bench_rank(rank, ws, port, out):
    import contextlib
    import io
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import bench
    from paper_2305_00762_gb300 import cases, gbr
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    gbr.load()
    sys.argv = ["bench.py", "--gpus", str(ws), "--n", "256", "--steps", "2", "--warmup", "1", "--t-window", "0.02"]
    args = bench.parse()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_slabs(args, torch, gbr, cases, dist, rank, ws, 0)
    out[rank] = buf.getvalue()


def test_bench_slab_mode_runs(env):
    """The benchmark's multi-GPU mode (the grid split into y-slabs, one per
    rank) end to end, as two processes sharing one GPU over gloo: a
    functional check of the JSON line, not a measurement."""
    torch, gbr, S = env
    import json
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    with mp.get_context("spawn").Manager() as m:  # no fork after CUDA or threads start
        out = m.dict()
        mp.spawn(_bench_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] == ""                      # only rank 0 prints
    line = json.loads(res[0].strip().splitlines()[-1])
    assert line["n_gpus"] == 2 and line["scaling"] == "strong" and line["status"] == "ok"
    assert line["value"] > 0 and line["e2e"]["value"] > 0 and line["gpu_launches"] > 0
    assert line["config"]["parallelism"] == "y-slabs x2"
