"""Checkpoint files of a solver and bitwise-exact resumption.

A checkpoint is a numpy .npz file: the state Q ([4][ny][nx] float64, the
conservative cell values), the simulated time and step count, and a header
with everything gbr_create and the options need (grid, cell sizes, gamma,
mu, Pr, boundary kinds and custom sides, precision, order, variables).
Resuming creates a solver from the header, sets the state and the time
(gbr_set_state, gbr_set_time): the continued run is bitwise the run that was
never interrupted.
"""
from __future__ import annotations

import json

import numpy as np

from . import gbr


def save(solver: "gbr.Solver", path: str, step: int = 0) -> None:
    header = dict(solver.params, sides=solver.sides, time=solver.time(), step=int(step), format=1)
    np.savez(path, Q=solver.get_state(), header=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8))


def load(path: str):
    """(Q, header dict) of a checkpoint file."""
    with np.load(path) as f:
        header = json.loads(bytes(f["header"]).decode())
        return f["Q"].copy(), header


def resume(path: str, stream=None) -> tuple:
    """A solver positioned at the checkpoint, and the checkpoint's step count."""
    Q, h = load(path)
    s = gbr.Solver(h["nx"], h["ny"], h["dx"], h["dy"], h["gamma"], h["mu"], h["Pr"], tuple(h["bc"]),
                   precision=h["precision"], stream=stream, order=h["order"], cons=h["cons"],
                   riemann=h.get("riemann", 0))
    for k, sd in enumerate(h["sides"]):
        if sd is not None:
            s.set_side(k, *sd)
    s.set_state(Q)
    s.set_time(h["time"])
    return s, h["step"]
