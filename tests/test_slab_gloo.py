"""The y-slab decomposition of one grid (Eq. deriv reaches six cells, so each
slab needs six rows of each neighbour per stage) on the CPU: the bookkeeping
(row ranges, boundary kinds at slab edges, neighbours, message order) and the
halo exchange itself, run as gloo ranks. Each rank receives its neighbours'
six boundary rows through the same exchange() the GPU driver uses, evaluates
the oracle's residual on its rows plus the received ones, and keeps its own
rows; gathered, they must equal the single-grid residual bit for bit (the
received rows are exact copies, and every face is computed from the same
data in the same order)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2305_00762_gb300 import cases as C  # noqa: E402
from paper_2305_00762_gb300 import slab as S  # noqa: E402

PERIODIC, TRANSMISSIVE, WALL, SYMMETRY, HALO = 0, 1, 2, 3, 6


def test_slab_rows_cover_the_grid():
    for ny, n in ((36, 2), (37, 3), (64, 5), (48, 8), (6, 1)):
        rows = S.slab_rows(ny, n)
        assert rows[0][0] == 0 and rows[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        h = [i1 - i0 for i0, i1 in rows]
        assert max(h) - min(h) <= 1 and min(h) >= 6
    with pytest.raises(ValueError):
        S.slab_rows(35, 6)          # a slab of fewer than six rows


def test_slab_boundary_kinds_and_neighbours():
    bc = (TRANSMISSIVE, WALL, WALL, SYMMETRY)
    assert S.slab_bc(bc, 0, 1) == bc
    assert S.slab_bc(bc, 0, 3) == (TRANSMISSIVE, WALL, WALL, HALO)
    assert S.slab_bc(bc, 1, 3) == (TRANSMISSIVE, WALL, HALO, HALO)
    assert S.slab_bc(bc, 2, 3) == (TRANSMISSIVE, WALL, HALO, SYMMETRY)
    per = (PERIODIC,) * 4
    assert S.slab_bc(per, 0, 2) == (PERIODIC, PERIODIC, HALO, HALO)
    assert S.slab_bc(per, 0, 1) == per
    assert S.neighbours(0, 3, False) == (None, 1)
    assert S.neighbours(2, 3, False) == (1, None)
    assert S.neighbours(0, 3, True) == (2, 1)
    assert S.neighbours(0, 2, True) == (1, 1)
    assert S.neighbours(0, 1, True) == (None, None)


def test_message_plan_pairs_match():
    """Between any two ranks, the k-th message one sends is the k-th one the
    other receives, and it lands on the side facing the sender."""
    for n in (2, 3, 4):
        for periodic in (False, True):
            plans = [S.message_plan(r, n, periodic) for r in range(n)]
            for a in range(n):
                for b in range(n):
                    sends = [side for op, peer, side in plans[a] if op == "send" and peer == b]
                    recvs = [side for op, peer, side in plans[b] if op == "recv" and peer == a]
                    assert len(sends) == len(recvs)
                    for s_side, r_side in zip(sends, recvs):
                        # a's south rows go to the neighbour below, into its north ghosts
                        assert r_side == (S.NORTH if s_side == S.SOUTH else S.SOUTH)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _make(name):
    if name == "riemann":
        return C.riemann_2d(40, 37)
    if name == "vortex":
        return C.isentropic_vortex(32, 36)
    return C.viscous_shock_tube(36, 38)


def _rank(rank, ws, port, name, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    from paper_2305_00762_gb300 import slab as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    c = _make(name)
    periodic = int(c.bc[2]) == PERIODIC
    i0, i1 = S.slab_rows(c.ny, ws)[rank]
    sides = S.slab_bc(c.bc, rank, ws)
    plan = S.message_plan(rank, ws, periodic)
    Q = c.Q[:, i0:i1, :]
    send = {S.SOUTH: torch.from_numpy(np.ascontiguousarray(Q[:, :6, :])),
            S.NORTH: torch.from_numpy(np.ascontiguousarray(Q[:, -6:, :]))}
    recv = {side: torch.empty((4, 6, c.nx), dtype=torch.float64) for side in (S.SOUTH, S.NORTH)}
    S.exchange(plan, send, recv)
    # rows: [received south halo] + own + [received north halo]; a halo
    # side's fake ghost rows beyond the received rows are never read by the
    # own rows' stencils (six cells reach)
    parts, lo = [], 0
    if sides[2] == HALO:
        parts.append(recv[S.SOUTH].numpy())
        lo = 6
    parts.append(Q)
    if sides[3] == HALO:
        parts.append(recv[S.NORTH].numpy())
    ext = np.ascontiguousarray(np.concatenate(parts, axis=1))
    bc = tuple(TRANSMISSIVE if k == HALO else k for k in sides)
    cfg = O.Config(c.nx, ext.shape[1], c.dx, c.dy, c.gamma, c.mu, c.Pr, bc)
    R = O.residual(cfg, ext)[:, lo:lo + (i1 - i0), :]
    out[rank] = R
    dist.destroy_process_group()


@pytest.mark.parametrize("name,ws", [("riemann", 2), ("riemann", 3), ("vortex", 2), ("vortex", 3),
                                     ("vst", 2)])
def test_halo_exchange_reproduces_single_grid_residual(oracle_mod, name, ws):
    c = _make(name)
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork after CUDA or threads start
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, name, out), nprocs=ws, join=True)
        parts = [out[r] for r in range(ws)]
    O = oracle_mod
    R = O.residual(O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc), c.Q)
    assert np.array_equal(np.concatenate(parts, axis=1), R)
