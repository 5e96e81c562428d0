"""Training the learned block-diagonal Lanczos preconditioner on the GPU.

Neighbourhoods come from seeded synthetic configurations (hard spheres at
several volume fractions and fractal gels); their features, structure
tensors and local inverse-square-root targets are produced by libpse
kernels, and the network is fitted by libpse's forward/backward/Adam
kernels.  Everything here is orchestration of C-ABI calls.
"""
from __future__ import annotations

import numpy as np

from . import Sampler, pse_precond_loss_grad, pse_precond_train, workloads

# (kind, N, phi, seed): hard spheres of the dilute and dense sampling
# workloads plus gels; 1e5 neighbourhoods in total by default.
DEFAULT_SETS = [("hs", 30000, 0.1, 101), ("hs", 30000, 0.2, 102), ("hs", 20000, 0.4, 103),
                ("gel", 20000, 0.1, 104)]


def init_theta(seed=0, nparam=450):
    """Same initialisation as the reference network: scaled normal weights, zero biases, small output layer."""
    rng = np.random.default_rng(seed)
    shapes = [(16, 8), (16,), (16, 16), (16,), (2, 16), (2,)]
    parts = []
    for shp in shapes:
        if len(shp) == 2:
            parts.append((rng.standard_normal(shp) / np.sqrt(shp[1])).ravel())
        else:
            parts.append(np.zeros(shp))
    th = np.concatenate(parts).astype(np.float32)
    th[-34:] *= 0.1
    assert th.size == nparam
    return th


def build_dataset(xi=0.5, tol=1e-3, sets=DEFAULT_SETS, a=1.0):
    """Features, structure tensors and targets (torch CUDA float32) of all neighbourhoods."""
    import torch
    feats, tens, tgts = [], [], []
    s0 = None
    for kind, N, phi, seed in sets:
        pos, L, _ = workloads.make(kind, N, phi, seed, a)
        s = Sampler(L, a, xi=xi, tol=tol)
        d = torch.from_numpy(pos).cuda()
        f, t = s.precond_features(d)
        g = s.precond_targets(d)
        torch.cuda.synchronize()
        feats.append(f)
        tens.append(t)
        tgts.append(g)
        s0 = s.precond_s0
        s.close()
    return torch.cat(feats), torch.cat(tens), torch.cat(tgts), s0


def train(xi=0.5, tol=1e-3, sets=DEFAULT_SETS, steps=1500, lr=3e-3, seed=0):
    """Returns (theta as numpy float32, info dict with loss history)."""
    import torch
    feat, tens, tgt, s0 = build_dataset(xi, tol, sets)
    theta = torch.from_numpy(init_theta(seed)).cuda()
    loss0, _ = pse_precond_loss_grad(feat, tens, tgt, theta, s0)
    hist = pse_precond_train(feat, tens, tgt, theta, s0, steps, lr)
    loss1, _ = pse_precond_loss_grad(feat, tens, tgt, theta, s0)
    # the analytic self block s0 I as a reference point
    eye = torch.zeros_like(tgt)
    eye[:, :3] = s0
    d = tgt - eye
    base = float(((d[:, :3] ** 2).sum(1) + 2 * (d[:, 3:] ** 2).sum(1)).mean().item() / s0 ** 2)
    info = {"n_samples": int(feat.shape[0]), "s0": s0, "loss_init": float(loss0.item()),
            "loss_final": float(loss1.item()), "loss_self_block": base, "steps": steps, "lr": lr,
            "loss_hist": hist.cpu().numpy()}
    return theta.cpu().numpy(), info
