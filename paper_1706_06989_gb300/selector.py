"""Learned pair selector: training data taken from the method's own accepted
pairs, and the network's training, through the C ABI.

Every numerical step (features, labels, forward, backward, Adam) runs in the
library's kernels; this module only chooses which pairs to label, how the
features are normalised and the initial weights.

Labels are the method's own errors: for a cell pair (A, B) accepted at some
opening angle, per side the rms over its bodies of the difference between the
torque-corrected order-3 M2L acceleration and the direct A<->B sum, in units
of the partner's monopole field M/|r|^2; the label is log10 of the larger
side (see fmm_selector_samples).

Scale invariance.  A label does not change when every mass is multiplied by
one factor, or every length by another (the error and the monopole field
scale alike).  Two features carry an absolute scale, log10 |r| and log10 M,
so systems of other N or other units would ask the network about masses and
lengths it never saw.  Training therefore adds, for every sample, a copy
whose log10 |r| is shifted by one random amount and whose two log10 M are
shifted by another (same label): the network learns the invariance.
"""
from __future__ import annotations

import json
import os

import numpy as np

NPARAMS = 8977
H, F = 64, 8
PARAMS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_params.npz")


def trained_params(path: str = PARAMS_PATH):
    """The committed trained network and its acceptance setting (written by
    train_selector.py), as a dict with keys params, rule, theta_lo,
    theta_max, min_work, log10_target; None if the file is absent."""
    if not os.path.exists(path):
        return None
    with np.load(path) as f:
        params = np.asarray(f["params"], dtype=np.float32)
        meta = json.loads(str(f["meta"]))
    if params.shape != (NPARAMS,):
        raise ValueError(f"{path}: expected {NPARAMS} parameters, found {params.shape}")
    return dict(meta, params=params)


def init_params(feat: np.ndarray, seed: int = 0) -> np.ndarray:
    """Feature normalisation from samples, weights by a seeded He-style draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(NPARAMS, dtype=np.float32)
    o = 0

    def put(a):
        nonlocal o
        p[o:o + a.size] = a.ravel()
        o += a.size

    put(rng.normal(0, np.sqrt(2.0 / F), (H, F)))
    put(np.zeros(H))
    put(rng.normal(0, np.sqrt(2.0 / H), (H, H)))
    put(np.zeros(H))
    put(rng.normal(0, np.sqrt(2.0 / H), (H, H)))
    put(np.zeros(H))
    put(rng.normal(0, np.sqrt(1.0 / H), H))
    put(np.zeros(1))
    f = np.asarray(feat, dtype=np.float64)
    mean = f.mean(0)
    std = f.std(0)
    put(mean)
    put(1.0 / np.where(std > 1e-6, std, 1.0))
    assert o == NPARAMS
    return p


def pair_samples(solver, x, y, z, m, thetas=(0.3, 0.5, 0.7, 1.0), per_theta: int = 200_000,
                 max_work: float = 1e8, seed: int = 0):
    """Features and labels of pairs accepted at the given opening angles.

    solver: an fmm.FMM (order 3, selector disabled); x, y, z, m: device
    tensors.  At most per_theta pairs per angle, drawn (seeded) among those
    whose label costs at most max_work body pairs (a label sums at most 128
    targets per side over every body of the partner).  Returns (feat [K, 8],
    label [K]) on the device.
    """
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    feats, labs = [], []
    for th in thetas:
        solver.set_opts(theta=th)
        solver.solve(x, y, z, m)
        m2l, _, _ = solver.export_lists()
        cnt = solver.export_tree(geometry=False)["count"].to(torch.int64)
        na, nb = cnt[m2l[:, 0].long()], cnt[m2l[:, 1].long()]
        work = (na.clamp(max=128) * nb + nb.clamp(max=128) * na).cpu().numpy()
        ok = np.nonzero(work <= max_work)[0]
        if ok.size == 0:
            continue
        pick = np.sort(rng.choice(ok, size=min(per_theta, ok.size), replace=False))
        pairs = m2l[torch.as_tensor(pick, device=m2l.device)].contiguous()
        # the tree of the last solve is current: fmm_selector_samples needs it
        f, l = solver.selector_samples(pairs, labels=True)
        feats.append(f)
        labs.append(l)
    return torch.cat(feats), torch.cat(labs)


LOG_R_SHIFT = (-2.0, 2.0)  # range of the random log10 length factor
LOG_M_SHIFT = (-3.0, 1.0)  # range of the random log10 mass factor


def augment_scales(feat, label, seed: int = 0):
    """The samples plus one copy of each under a random change of length and
    mass units (features 0 and 3, 4 shifted; labels unchanged)."""
    import torch
    g = torch.Generator(device=feat.device)
    g.manual_seed(seed)
    k = feat.shape[0]
    dr = torch.empty(k, device=feat.device).uniform_(*LOG_R_SHIFT, generator=g)
    dm = torch.empty(k, device=feat.device).uniform_(*LOG_M_SHIFT, generator=g)
    aug = feat.clone()
    aug[:, 0] += dr
    aug[:, 3] += dm
    aug[:, 4] += dm
    return torch.cat([feat, aug]).contiguous(), torch.cat([label, label]).contiguous()


def train(solver, feat, label, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
          params: np.ndarray | None = None, scale_augment: bool = True):
    """Trains the network; returns (params as numpy float32, losses)."""
    import torch
    if scale_augment:
        feat, label = augment_scales(feat, label, seed)
    p0 = init_params(feat.cpu().numpy(), seed) if params is None else params
    dev = torch.as_tensor(p0, device=feat.device).contiguous()
    losses, _ = solver.selector_train(dev, feat, label, batch=batch, steps=steps, lr=lr, seed=seed)
    return dev.cpu().numpy(), losses
