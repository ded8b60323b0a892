"""Trains the LBM surrogate with the library's kernels and writes its weights.

Training data: `--rollouts` plain-LBM runs on an N^3 lattice (tau = 0.55,
inlet speed 0.05 in a random direction within 30 degrees of +x, random
leaf-cluster obstacle), each sampled at a random time in [t_lo, t_hi) for the
change of the coarse velocity over the next 20 steps. Training: Adam with a
cosine learning-rate decay over `--steps` steps. The result goes to
weights/surrogate_lbm{N}.npy (FP32, the library's parameter packing).

    python -m paper_2603_09668_gb300.train_surrogate --N 128 --rollouts 512 --steps 6000

--inlet-features trains on features relative to each rollout's inlet
velocity (surr_set_inlet); without it the reference velocity is zero, as
SurrogateLBM assumes by default.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import binding as B
from . import build as _build
from . import surrogate as S


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--rollouts", type=int, default=512)
    ap.add_argument("--t-lo", type=int, default=1000)
    ap.add_argument("--t-hi", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--per-rollout", type=int, default=1)
    ap.add_argument("--inlet-features", action="store_true")
    ap.add_argument("--turn-frac", type=float, default=0.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    _build.build_library()
    torch.cuda.set_device(0)
    t0 = time.time()
    xs, ys = S.generate_pairs(a.N, a.rollouts, a.t_lo, a.t_hi, seed=a.seed,
                              per_rollout=a.per_rollout, inlet_features=a.inlet_features,
                              turn_frac=a.turn_frac)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    surr = B.Surrogate(a.N // 2)
    surr.set_params(S.init_params(S.layer_slices(), seed=a.seed))
    t0 = time.time()
    hist = S.train(surr, xs, ys, a.steps, lr=a.lr, seed=a.seed, log_every=max(1, a.steps // 20))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    p = surr.params().cpu().numpy()
    out = a.out or S.weights_path(a.N)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    np.save(out, p)
    print(json.dumps({"weights": out, "args": vars(a), "rollouts": a.rollouts, "steps": a.steps,
                      "data_s": t_data, "train_s": t_train, "loss": hist}))


if __name__ == "__main__":
    main()
