"""Train the learned discontinuity sensor on the flags the density detector
(arXiv:2305.00762, Sec. 2.4, Eq. detector) produces on this solver's own runs.

Data: snapshots of seeded 2D four-quadrant Riemann problems with random
states (rho in [0.1, 2], p in [0.02, 2], |u|, |v| <= 1.5, split point in
[0.35, 0.65]^2) and of isentropic vortices of strength in [1, 5], run with the
FP32 form. Every interior cell of a snapshot is one sample: its 5 x 5 stencil
features (BF16) and a soft target derived from the plain detector,
1 / (1 + exp((psi_min - 0.5) / 0.02)) with psi_min = min(psi_x, psi_y) in FP64
(the hard label is psi_min < 0.5), all written on the device by
gbr_sensor_dataset. A cell near the detector threshold thus has a target
inside the fallback band [0.3, 0.7], where the plain detector decides; the
network is confident only where the detector's decision is clear. Training
runs in the library's hand-written kernels (gbr_sensor_train). Agreement with
the plain detector is scored on held-out snapshots through gbr_sensor_eval.

    python -m paper_2305_00762_gb300.sensor_train [--samples 20000000] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import cases, gbr

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "sensor_weights.json")
SEED = 2305


def random_quadrant(n, rng):
    xc, dx = cases.centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(xc, xc)
    sx, sy = rng.uniform(0.35, 0.65, 2)
    prim = np.zeros((4, n, n))
    for right in (False, True):
        for top in (False, True):
            m = ((X > sx) == right) & ((Y > sy) == top)
            st = (rng.uniform(0.1, 2.0), rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5), rng.uniform(0.02, 2.0))
            for k in range(4):
                prim[k][m] = st[k]
    Q = cases.prim_to_cons(*prim, 1.4)
    return cases.Case("random_quadrant", np.ascontiguousarray(Q), dx, dx, 1.4, 0.0, 0.72,
                      (cases.BC_TRANSMISSIVE,) * 4, 0.0, 0.5)


def init_weights(rng):
    """He-normal hidden layers, small output layer, output bias at the label
    prior (about 5% discontinuity cells)."""
    W1 = rng.normal(0, np.sqrt(2 / 50), (50, 32))
    W2 = rng.normal(0, np.sqrt(2 / 32), (32, 32))
    w3 = rng.normal(0, np.sqrt(1 / 32), 32)
    w = np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), w3, [np.log(0.05 / 0.95)]])
    assert w.size == gbr.GBR_SENSOR_PARAMS
    return w.astype(np.float32)


# Snapshot schedule of every run: after about 8, 32, 96 and 224 steps (each
# jittered), so that early, developing and developed flows are all sampled.
SCHEDULE = (8, 24, 64, 128)


def snapshots(torch, rng, n, count, cfl=0.5):
    """Yield a solver positioned at successive snapshots of seeded runs."""
    made = 0
    while made < count:
        if made % 4 == 3:
            c = cases.isentropic_vortex(n, eps=float(rng.uniform(1, 5)))
        else:
            c = random_quadrant(n, rng)
        s = gbr.Solver.for_case(c, precision=32)
        s.set_state(torch.from_numpy(c.Q).cuda())
        for k in range(4):
            for _ in range(int(rng.integers(SCHEDULE[k] // 2, SCHEDULE[k] * 3 // 2))):
                s.step_cfl(cfl)
            if s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,)) != gbr.GBR_OK:
                break
            yield s
            made += 1
            if made >= count:
                break
        s.close()


def dataset(torch, rng, samples, n=512):
    """Features, soft targets (units of 1/255) and plain-detector labels."""
    feats, targets, labels = [], [], []
    per = n * n
    for s in snapshots(torch, rng, n, (samples + per - 1) // per):
        f = torch.empty((per, 64), dtype=torch.bfloat16, device="cuda")
        t = torch.empty(per, dtype=torch.uint8, device="cuda")
        y = torch.empty(per, dtype=torch.uint8, device="cuda")
        gbr.gbr_sensor_dataset(s.ctx, f, y, t)
        feats.append(f)
        targets.append(t)
        labels.append(y)
    torch.cuda.synchronize()
    return torch.cat(feats)[:samples], torch.cat(targets)[:samples], torch.cat(labels)[:samples]


def agreement(torch, rng, w, count=8, n=512):
    """Decision agreement with the plain detector on held-out snapshots."""
    stats = {"cells": 0, "unsure": 0, "agree_confident": 0, "false_smooth": 0, "false_trouble": 0,
             "trouble": 0}
    for s in snapshots(torch, rng, n, count):
        y = torch.empty(n * n, dtype=torch.uint8, device="cuda")
        gbr.gbr_sensor_dataset(s.ctx, None, y)
        gbr.gbr_set_sensor_weights(s.ctx, w)
        p = torch.from_numpy(s.sensor_eval()).reshape(-1).cuda()
        y = y.bool()
        sure_t, sure_s = p > 0.7, p < 0.3
        stats["cells"] += n * n
        stats["trouble"] += int(y.sum())
        stats["unsure"] += int((~sure_t & ~sure_s).sum())
        stats["agree_confident"] += int((sure_t & y).sum() + (sure_s & ~y).sum())
        stats["false_smooth"] += int((sure_s & y).sum())
        stats["false_trouble"] += int((sure_t & ~y).sum())
    conf = stats["cells"] - stats["unsure"]
    stats["confident_agreement"] = stats["agree_confident"] / max(conf, 1)
    stats["unsure_fraction"] = stats["unsure"] / stats["cells"]
    return stats


# Fractions of the steps and learning-rate multipliers of the training phases
# (Adam restarts at each phase).
LR_SCHEDULE = ((0.6, 1.0), (0.25, 0.25), (0.15, 1.0 / 16.0))


def train(samples=20_000_000, epochs=256.0, batch=8192, lr=2e-3, pos_weight=1.0, seed=SEED, out=DEFAULT_WEIGHTS,
          verbose=True):
    import torch
    rng = np.random.default_rng(seed)
    t0 = time.time()
    X, tgt, y = dataset(torch, rng, samples)
    t1 = time.time()
    steps = max(1, int(epochs * X.shape[0] / batch))
    w = init_weights(rng)
    losses = []
    for k, (frac, scale) in enumerate(LR_SCHEDULE):  # step-wise learning-rate decay
        n = max(1, int(round(frac * steps)))
        w, loss = gbr.gbr_sensor_train(X, tgt, n, batch, lr * scale, pos_weight, seed + k, w)
        losses.append(loss)
    loss = np.concatenate(losses)
    steps = int(loss.size)
    t2 = time.time()
    held = agreement(torch, np.random.default_rng(seed + 1), w)
    info = {"seed": seed, "samples": int(X.shape[0]), "label_fraction": float(y.float().mean()),
            "steps": steps, "batch": batch, "lr": lr, "pos_weight": pos_weight,
            "loss_first": float(loss[: max(1, steps // 50)].mean() / batch),
            "loss_last": float(loss[-max(1, steps // 50):].mean() / batch),
            "data_s": t1 - t0, "train_s": t2 - t1, "held_out": held}
    if verbose:
        print(json.dumps(info, indent=1))
    if out:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        with open(out, "w") as f:
            json.dump({"info": info, "weights": [float(v) for v in w]}, f)
    return w, info


def load_weights(path=DEFAULT_WEIGHTS):
    with open(path) as f:
        return np.asarray(json.load(f)["weights"], dtype=np.float32)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=20_000_000)
    ap.add_argument("--epochs", type=float, default=256.0)
    ap.add_argument("--pos-weight", type=float, default=1.0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args()
    from . import build
    build.build()
    train(a.samples, a.epochs, pos_weight=a.pos_weight, out=a.out)
