"""Learned block-diagonal preconditioner: FP64 reference of the network (oracle side).

Not in the paper: the real-space Lanczos of Sec. II B 1 may run on
P M_r P^T for any invertible block-diagonal P, the sample P^{-1} (P M_r P^T)^{1/2} z
keeps covariance M_r exactly, and only the iteration count changes.

Block (rotation-equivariant, SPD by construction):
    S_i = s0 exp(a_i) (I + tanh(b_i) T_i / (1 + tr T_i)),   T_i = sum_j w(r_ij) rr_ij
with w(r) = exp(-((r - 2a)/a)^2) over the neighbours j within r_cut, s0 the
inverse square root of the self mobility; a = b = 0 gives the analytic
self-mobility block s0 I.  (a_i, b_i) come from a 8 -> 16 -> 16 -> 2 tanh
MLP on rotation-invariant features of i's neighbourhood:
    f = [tr T, tr T^2, det T, n(r<2.5a), n(r<3.5a), n(r<4.5a), n(r<r_cut), mean 2a/r] / scales
(n(.) smooth counts sum_j sigmoid(4 (r_c' - r)/a)).
Training target: the diagonal 3x3 block of (M_loc)^{-1/2}, M_loc being M_r
restricted to i and its neighbours within r_loc = 3a (at most K = 16
nearest, ties by index), pair blocks truncated at r_cut as in the sampler.
Parameter vector layout: W1 (16x8), b1 (16), W2 (16x16), b2 (16), W3 (2x16), b3 (2).
"""
from __future__ import annotations

import numpy as np

from . import ewald, pse, rpy

D_IN, H = 8, 16
SHAPES = [("W1", (H, D_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (2, H)), ("b3", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
FEAT_SCALE = np.array([4.0, 8.0, 16.0, 4.0, 8.0, 16.0, 32.0, 1.0])


def unpack(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    th = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            th.append((rng.standard_normal(shp) * (1.0 / np.sqrt(shp[1]))).ravel())
        else:
            th.append(np.zeros(shp).ravel())
    th = np.concatenate(th)
    th[-2 * H - 2:] *= 0.1  # small output layer: S starts near s0 I
    return th


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def features(pos, plan):
    """(N, 8) invariant features and (N, 3, 3) structure tensors T_i."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    a = plan.a
    i, j, d = pse.pair_list(pos, plan.L, plan.r_cut)
    ii = np.concatenate([i, j])
    dd = np.concatenate([d, -d])
    r = np.linalg.norm(dd, axis=1)
    rh = dd / r[:, None]
    w = np.exp(-(((r - 2 * a) / a) ** 2))
    T = np.zeros((N, 3, 3))
    np.add.at(T, ii, w[:, None, None] * rh[:, :, None] * rh[:, None, :])
    trT = np.trace(T, axis1=1, axis2=2)
    trT2 = np.einsum("nab,nba->n", T, T)
    det = np.linalg.det(T)
    f = np.zeros((N, D_IN))
    f[:, 0], f[:, 1], f[:, 2] = trT, trT2, det
    for col, rc in ((3, 2.5 * a), (4, 3.5 * a), (5, 4.5 * a), (6, plan.r_cut)):
        f[:, col] = np.bincount(ii, weights=_sigmoid(4 * (rc - r) / a), minlength=N)
    cnt = np.bincount(ii, minlength=N)
    f[:, 7] = np.bincount(ii, weights=2 * a / r, minlength=N) / np.maximum(cnt, 1)
    return f / FEAT_SCALE, T


def forward(theta, feat, T, s0):
    """S (N,3,3) and the cache for backward."""
    p = unpack(theta)
    z1 = feat @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    o = h2 @ p["W3"].T + p["b3"]
    av, bv = o[:, 0], o[:, 1]
    trT = np.trace(T, axis1=1, axis2=2)
    Tn = T / (1 + trT)[:, None, None]
    tb = np.tanh(bv)
    S = s0 * np.exp(av)[:, None, None] * (np.eye(3)[None] + tb[:, None, None] * Tn)
    return S, dict(p=p, feat=feat, h1=h1, h2=h2, av=av, tb=tb, Tn=Tn, s0=s0)


def loss(theta, feat, T, target, s0):
    """mean_i ||S_i - target_i||_F^2 / s0^2."""
    S, _ = forward(theta, feat, T, s0)
    return float(np.mean(np.sum((S - target) ** 2, axis=(1, 2))) / s0 ** 2)


def loss_grad(theta, feat, T, target, s0):
    """Loss and its gradient w.r.t. the parameter vector (backpropagation)."""
    S, c = forward(theta, feat, T, s0)
    n = feat.shape[0]
    p = c["p"]
    dS = 2.0 * (S - target) / (n * s0 ** 2)  # dL/dS
    E = np.exp(c["av"])
    base = np.eye(3)[None] + c["tb"][:, None, None] * c["Tn"]
    # S = s0 E base  -> dL/da = sum dS * S ; dL/db = sum dS * s0 E (1 - tb^2) Tn
    da = np.sum(dS * S, axis=(1, 2))
    db = np.sum(dS * (s0 * E * (1 - c["tb"] ** 2))[:, None, None] * c["Tn"], axis=(1, 2))
    do = np.stack([da, db], axis=1)
    gW3 = do.T @ c["h2"]
    gb3 = do.sum(axis=0)
    dh2 = do @ p["W3"]
    dz2 = dh2 * (1 - c["h2"] ** 2)
    gW2 = dz2.T @ c["h1"]
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (1 - c["h1"] ** 2)
    gW1 = dz1.T @ c["feat"]
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    L = float(np.mean(np.sum((S - target) ** 2, axis=(1, 2))) / s0 ** 2)
    return L, g


def local_targets(pos, plan, r_loc=3.0, K=16, idx=None):
    """[(M_loc)^{-1/2}]_ii for each particle (or those in idx): eigendecomposition."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    L = plan.L
    sel = np.arange(N) if idx is None else np.asarray(idx)
    out = np.zeros((sel.size, 3, 3))
    for n, i in enumerate(sel):
        d = pos - pos[i]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=1)
        r[i] = np.inf
        nb = np.lexsort((np.arange(N), r))  # by distance, ties by index
        nb = nb[r[nb] < r_loc * plan.a][:K]
        loc_pos = np.concatenate([[pos[i]], pos[i] + d[nb]])
        Mloc = _real_block_matrix(loc_pos, plan)
        lam, Q = np.linalg.eigh(Mloc)
        Mih = (Q * lam ** -0.5) @ Q.T
        out[n] = Mih[:3, :3]
    return out


def _real_block_matrix(p, plan):
    """Dense M_r (eq. Mreal, App. A) of a few particles, no periodic images."""
    m = p.shape[0]
    M = np.zeros((3 * m, 3 * m))
    s = rpy.self_real(plan.xi, plan.a) / (6 * np.pi * plan.a)
    for a_ in range(m):
        M[3 * a_:3 * a_ + 3, 3 * a_:3 * a_ + 3] = s * np.eye(3)
        for b_ in range(a_ + 1, m):
            d = p[a_] - p[b_]
            r = np.linalg.norm(d)
            if r >= plan.r_cut:
                continue
            F, G = rpy.fg(r, plan.xi, plan.a)
            rh = d / r
            blk = (F * (np.eye(3) - np.outer(rh, rh)) + G * np.outer(rh, rh)) / (6 * np.pi * plan.a)
            M[3 * a_:3 * a_ + 3, 3 * b_:3 * b_ + 3] = blk
            M[3 * b_:3 * b_ + 3, 3 * a_:3 * a_ + 3] = blk
    return M
