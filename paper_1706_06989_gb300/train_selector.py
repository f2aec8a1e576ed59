"""Trains the learned pair selector and writes its parameters.

Run on a GPU from the repository root:

    python -m paper_1706_06989_gb300.train_selector [--steps 3000] [--out PATH]

Training data are the method's own accepted pairs: the Plummer spheres of
N = 2,000 and N = 1,048,576 (seed 0) walked at opening angles 0.35 ... 0.85,
each pair labelled with the error of its torque-corrected order-3 expansion
against the direct sum over its bodies (fmm_selector_samples).  The network
is trained by the library's own kernels (fmm_selector_train: tensor-core
forward and backward passes, Adam).  The output file holds the FP32
parameters and the acceptance setting they were evaluated with (relative
rule, band (0.45, 0.75], min_work 256, log10 target -3.25); the benchmark's
4M-body comparison and the selector tests load it through
selector.trained_params().
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import fmm, ics, selector

SETTING = {"rule": "relative", "theta_lo": 0.45, "theta_max": 0.75, "min_work": 256, "log10_target": -3.25}
THETAS = (0.35, 0.425, 0.5, 0.575, 0.65, 0.75, 0.85)


def main():
    import torch
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--out", default=selector.PARAMS_PATH)
    a = p.parse_args()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    s = fmm.FMM(theta=0.5, n_crit=25, variant="TC", precision="fp64")
    feats, labs = [], []
    for b, per in ((ics.plummer(2000, seed=0), 200_000), (ics.plummer(1 << 20, seed=0), 1_400_000)):
        x, y, z, m = (torch.from_numpy(v).to(dev) for v in (b.x, b.y, b.z, b.m))
        f, l = selector.pair_samples(s, x, y, z, m, thetas=THETAS, per_theta=per, seed=3)
        feats.append(f)
        labs.append(l)
    X, Y = torch.cat(feats), torch.cat(labs)
    params, losses = selector.train(s, X, Y, steps=a.steps, batch=8192, lr=2e-3, seed=4)
    s.close()
    meta = dict(SETTING, samples=int(X.shape[0]), steps=a.steps, batch=8192, lr=2e-3, seed=4,
                thetas=list(THETAS), loss_first=float(np.mean(losses[:20])), loss_last=float(np.mean(losses[-50:])),
                seconds=time.perf_counter() - t0)
    np.savez(a.out, params=params.astype(np.float32), meta=json.dumps(meta))
    print(json.dumps({"wrote": os.path.relpath(a.out), **meta}))


if __name__ == "__main__":
    main()
