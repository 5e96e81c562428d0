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
# held-out configurations (other seeds) on which the trained network must
# earn its place: the mean Lanczos count with it against without it
HELDOUT_SETS = [("hs", 20000, 0.1, 201), ("hs", 20000, 0.3, 202), ("gel", 20000, 0.1, 203)]


def init_theta(seed=0, nparam=450):
    """Initial weights: scaled normal weights, zero biases, a small output layer (S starts near s0 I)."""
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


def iteration_gain(theta, xi=0.5, tol=1e-3, sets=HELDOUT_SETS, samples=3, seed=77, a=1.0):
    """Mean Lanczos iterations to reach tol (the same stop rule) without and
    with the network, over `samples` samples of each held-out configuration."""
    import torch
    jp, jl = [], []
    for kind, N, phi, cseed in sets:
        pos, L, _ = workloads.make(kind, N, phi, cseed, a)
        d = torch.from_numpy(pos).cuda()
        out = torch.empty_like(d)
        for th, acc in ((None, jp), (theta, jl)):
            s = Sampler(L, a, xi=xi, tol=tol)
            if th is not None:
                s.precond_set_weights(th)
            for k in range(samples):
                s.sample(d, seed, k, out=out)
                acc.append(s.stats()["lanczos_iters"])
            s.close()
    return {"iters_plain": float(np.mean(jp)), "iters_learned": float(np.mean(jl)),
            "gain": float(np.mean(jp) - np.mean(jl))}


def train_or_fallback(xi=0.5, tol=1e-3, min_gain=1.0, **kw):
    """Train the network, then keep it only if it cuts the mean Lanczos count
    on the held-out configurations by at least `min_gain` iterations.  When
    it does not, the preconditioner falls back to P = I (theta None: no
    inference kernel, no block products in the matvec), so the learned form
    never costs time without saving iterations.  Returns (theta or None, info);
    info["theta"] holds the trained weights either way."""
    theta, info = train(xi=xi, tol=tol, **kw)
    gain = iteration_gain(theta, xi, tol)
    info.update(gain)
    info["theta"] = theta
    info["min_gain"] = min_gain
    info["fallback"] = gain["gain"] < min_gain
    return (None if info["fallback"] else theta), info
