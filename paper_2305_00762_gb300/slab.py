"""One grid split along y into slabs, one solver context per slab.

Eq. deriv's residual at a cell reaches six cells in each direction (the LC
bound of Eq. mp-procedure uses d_{j-1}, hence Phi'_{j-2}, hence Phi_{j-5}; the
face adds one), so a slab needs six rows of each neighbour before every
Runge-Kutta stage (Eq. rk), and the CFL step of Sec. 2.5 needs the largest
wavespeed over all slabs once per step. Everything else is local. The slabs'
south / north sides inside the grid (and every side of a grid periodic in y)
are GBR_BC_HALO sides whose ghost rows the caller writes; the library fills
their west / east ghost cells and runs the unchanged stage kernels, so the
slabs reproduce the single-grid step bit for bit.

This module holds the bookkeeping (row ranges, boundary kinds at slab edges,
neighbours, the order of the halo messages) and two drivers:
LocalSlabs (all slabs in one process, on one device: halo copies between the
contexts' buffers) and DistSlab (one slab per torch.distributed rank: the
halos travel by point-to-point messages, the wavespeed by a max all-reduce).
Marshalling only: every step of the path runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import gbr

GHOST = 6
SOUTH, NORTH = 2, 3


def slab_rows(ny: int, n: int):
    """Row ranges [i0, i1) of n slabs of an ny-row grid; the first ny % n
    slabs get one row more. Every slab needs at least six rows, so that a
    halo comes from one neighbour."""
    if n < 1 or ny < n * GHOST:
        raise ValueError(f"{ny} rows cannot make {n} slabs of at least {GHOST} rows")
    base, extra = divmod(ny, n)
    out, i0 = [], 0
    for r in range(n):
        h = base + (1 if r < extra else 0)
        out.append((i0, i0 + h))
        i0 += h
    return out


def slab_bc(bc, rank: int, n: int):
    """Boundary kinds (west, east, south, north) of slab `rank` of n: a slab
    edge inside the grid is a halo side, and so is every slab edge of a grid
    periodic in y (split in n >= 2); the grid's own south / north kinds stay
    on the first / last slab otherwise."""
    w, e, s, nn = (int(k) for k in bc)
    if n == 1:
        return (w, e, s, nn)
    periodic = s == gbr.GBR_BC_PERIODIC
    south = gbr.GBR_BC_HALO if (rank > 0 or periodic) else s
    north = gbr.GBR_BC_HALO if (rank < n - 1 or periodic) else nn
    return (w, e, south, north)


def neighbours(rank: int, n: int, periodic: bool):
    """(south, north) neighbour ranks of slab `rank`, None at a grid edge."""
    if n == 1:
        return None, None
    south = rank - 1 if rank > 0 else (n - 1 if periodic else None)
    north = rank + 1 if rank < n - 1 else (0 if periodic else None)
    return south, north


def message_plan(rank: int, n: int, periodic: bool):
    """The halo messages of one stage, in the order a rank posts them:
    (op, peer, side) with op 'send' (the six rows next to `side` go to the
    neighbour there) or 'recv' (the neighbour on `side` fills the ghost rows
    beyond it). Sends go south then north, receives come from north then
    south: between two ranks the k-th send of one then matches the k-th
    receive of the other, also when they are each other's south and north
    neighbour (two slabs of a periodic grid)."""
    south, north = neighbours(rank, n, periodic)
    plan = []
    if south is not None:
        plan.append(("send", south, SOUTH))
    if north is not None:
        plan.append(("send", north, NORTH))
    if north is not None:
        plan.append(("recv", north, NORTH))
    if south is not None:
        plan.append(("recv", south, SOUTH))
    return plan


def exchange(plan, send, recv, group=None):
    """Post the plan's messages with torch.distributed (batched
    point-to-point, so no rank blocks on the order of another) and wait:
    send[side] and recv[side] are contiguous tensors [4][6][nx] on the
    group's device (CPU tensors with gloo, CUDA tensors with NCCL)."""
    import torch.distributed as dist
    ops = []
    for op, peer, side in plan:
        if op == "send":
            ops.append(dist.P2POp(dist.isend, send[side], peer, group))
        else:
            ops.append(dist.P2POp(dist.irecv, recv[side], peer, group))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


class LocalSlabs:
    """n slabs of one grid in one process, on the current device: before
    each stage every halo side receives its neighbour's rows by device
    copies (through one staging buffer), and after each step the
    wavespeeds are reduced by gbr_lambda_max."""

    def __init__(self, case, n, **solver_kw):
        import torch
        self.case, self.n = case, n
        self.rows = slab_rows(case.ny, n)
        self.periodic = int(case.bc[2]) == gbr.GBR_BC_PERIODIC
        self.solvers = [gbr.Solver(case.nx, i1 - i0, case.dx, case.dy, case.gamma, case.mu, case.Pr,
                                   slab_bc(case.bc, r, n), **solver_kw)
                        for r, (i0, i1) in enumerate(self.rows)]
        self.buf = torch.empty((4, GHOST, case.nx), dtype=torch.float64, device="cuda")

    def set_state(self, Q):
        for s, (i0, i1) in zip(self.solvers, self.rows):
            s.set_state(np.ascontiguousarray(Q[:, i0:i1, :]))
        gbr.lambda_max(self.solvers)

    def get_state(self):
        return np.concatenate([s.get_state() for s in self.solvers], axis=1)

    def _exchange(self):
        for r, s in enumerate(self.solvers):
            south, north = neighbours(r, self.n, self.periodic)
            if south is not None:
                self.solvers[south].halo_copy(NORTH, 0, self.buf)
                s.halo_copy(SOUTH, 1, self.buf)
            if north is not None:
                self.solvers[north].halo_copy(SOUTH, 0, self.buf)
                s.halo_copy(NORTH, 1, self.buf)

    def _step(self, dt, cfl, dt_max):
        for k in range(3):
            self._exchange()
            for s in self.solvers:
                s.step_stage(k, dt, cfl, dt_max)
        gbr.lambda_max(self.solvers)

    def step(self, dt):
        self._step(float(dt), 0.0, 0.0)

    def step_cfl(self, cfl, dt_max=1e300):
        self._step(0.0, float(cfl), float(dt_max))

    def time(self):
        return self.solvers[0].time()

    def close(self):
        for s in self.solvers:
            s.close()


class _DeviceWord:
    """A device address seen by torch as a one-element int64 tensor."""

    def __init__(self, ptr):
        self.__cuda_array_interface__ = {"shape": (1,), "typestr": "<i8", "data": (int(ptr), False),
                                         "version": 2}


class DistSlab:
    """Slab `rank` of a grid split over the ranks of a torch.distributed
    group (one slab per rank and GPU). The halo rows travel as contiguous
    [4][6][nx] buffers by batched point-to-point messages, the wavespeed
    words by a MAX all-reduce of their int64 view (the bits of non-negative
    doubles order as the values). transport "device" (NCCL): the buffers
    are device memory and the context works on torch's current stream,
    which the collectives follow. transport "host" (any backend, e.g. gloo):
    the buffers are pinned host memory filled and drained by synchronous
    copies, and the wavespeed word goes through the host."""

    def __init__(self, case, rank, world, group=None, transport="device", **solver_kw):
        import torch
        if transport not in ("device", "host"):
            raise ValueError(f"unknown transport {transport!r}")
        self.case, self.rank, self.world, self.group = case, rank, world, group
        self.transport = transport
        self.rows = slab_rows(case.ny, world)
        self.periodic = int(case.bc[2]) == gbr.GBR_BC_PERIODIC
        i0, i1 = self.rows[rank]
        self.i0, self.i1 = i0, i1
        solver_kw.setdefault("stream", torch.cuda.current_stream().cuda_stream)
        self.solver = gbr.Solver(case.nx, i1 - i0, case.dx, case.dy, case.gamma, case.mu, case.Pr,
                                 slab_bc(case.bc, rank, world), **solver_kw)
        self.plan = message_plan(rank, world, self.periodic)
        shape = (4, GHOST, case.nx)
        if transport == "device":
            alloc = lambda: torch.empty(shape, dtype=torch.float64, device="cuda")
        else:
            alloc = lambda: torch.empty(shape, dtype=torch.float64).pin_memory()
        self.send = {side: alloc() for side in (SOUTH, NORTH)}
        self.recv = {side: alloc() for side in (SOUTH, NORTH)}

    def set_state(self, Q_local):
        self.solver.set_state(Q_local)
        self._reduce_lambda()

    def _reduce_lambda(self):
        import torch
        import torch.distributed as dist
        w = torch.as_tensor(_DeviceWord(self.solver.lambda_word()), device="cuda")
        if self.transport == "device":
            dist.all_reduce(w, op=dist.ReduceOp.MAX, group=self.group)
            return
        h = w.cpu()  # synchronising copy (stream-ordered after the step)
        dist.all_reduce(h, op=dist.ReduceOp.MAX, group=self.group)
        w.copy_(h)
        torch.cuda.current_stream().synchronize()

    def _exchange(self):
        for op, _, side in self.plan:
            if op == "send":
                self.solver.halo_copy(side, 0, self.send[side])
        exchange(self.plan, self.send, self.recv, self.group)
        for op, _, side in self.plan:
            if op == "recv":
                self.solver.halo_copy(side, 1, self.recv[side])

    def _step(self, dt, cfl, dt_max):
        for k in range(3):
            self._exchange()
            self.solver.step_stage(k, dt, cfl, dt_max)
        self._reduce_lambda()

    def step(self, dt):
        self._step(float(dt), 0.0, 0.0)

    def step_cfl(self, cfl, dt_max=1e300):
        self._step(0.0, float(cfl), float(dt_max))

    def get_state(self):
        """This slab's rows of the state ([4][i1 - i0][nx], host)."""
        return self.solver.get_state()

    def time(self):
        return self.solver.time()

    def close(self):
        self.solver.close()
