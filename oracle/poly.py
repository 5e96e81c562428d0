"""Polydisperse suspensions: the size-dependent shape factor of Sec. V (FP64 oracle).

Test infrastructure: only tests/, the smoke check and the benchmark's CPU leg
use this module.

Sec. V notes that polydispersity enters the positively split Ewald sum by
making the shape factor size dependent: the pair mobility of spheres of radii
a_i and a_j is the k-integral of eq. pairmobility with sinc(k a_i) sinc(k a_j)
in place of sinc^2(k a), and the split with H(k, xi) stays positive on both
sides (H and 1 - H are non-negative, and sum_k c_k phi_i(k) conj(phi_j(k)) with
phi_i = sinc(k a_i) exp(i k.x_i) is a Gram matrix).  Written out (eta = 1):

  M_ij   = int d^3k/(2 pi)^3 sinc(k a_i) sinc(k a_j)/k^2 (I - kk) exp(i k.r)
         = the free-space RPY tensor of two unequal spheres (Zuk, Wajnryb,
           Mizerski & Szymczak, J. Fluid Mech. 741, R5 (2014)),
  M^w_ij = (1/V) sum_{k != 0} H(k, xi) sinc(k a_i) sinc(k a_j)/k^2 (I - kk) exp(i k.r_ij),
  M^r_ij = M_ij - [the same k-integral with weight H]   (summed over images).

The second form of M^r is exact because the continuous k-integral with
weight 1 (eq. pairmobility's) is the free-space tensor; its H-weighted part
decays like a Gaussian in k, so plain Gauss-Legendre quadrature on
[0, 16 xi] evaluates it to rounding.  For a_i = a_j this is the App. A pair
(checked against the closed form in the tests).

Scalars here are in mobility units: block = F (I - rr) + G rr (no 6 pi a).

Wave sample: the noise dW2 and the Gaussian spreading are those of the
monodisperse path; species s (radius a_s) gets its own velocity grid, the
mode scale of oracle.pse.wave_scale evaluated with a = a_s, and its particles
interpolate from it, so Cov(u_i, u_j) carries sinc(k a_i) sinc(k a_j).
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

from . import ewald, pse, rpy


# ----------------------------------------------------------------------------- pair scalars

def rpy_free(r, ai, aj):
    """Free-space RPY tensor of spheres of radii ai, aj as (F, G), block = F (I - rr) + G rr.

    r > ai + aj:           A = (1 + (ai^2 + aj^2)/3r^2)/(8 pi r),  B = (1 - (ai^2 + aj^2)/r^2)/(8 pi r)
    |ai - aj| < r <= ai+aj: A = (16 r^3 (ai + aj) - ((ai - aj)^2 + 3 r^2)^2)/(32 r^3) / (6 pi ai aj),
                            B = 3 ((ai - aj)^2 - r^2)^2/(32 r^3) / (6 pi ai aj)
    r <= |ai - aj|:         A = 1/(6 pi max(ai, aj)), B = 0
    and F = A, G = A + B.
    """
    r = np.asarray(r, dtype=np.float64)
    ai = np.broadcast_to(np.asarray(ai, dtype=np.float64), r.shape)
    aj = np.broadcast_to(np.asarray(aj, dtype=np.float64), r.shape)
    s2 = ai * ai + aj * aj
    far = r > ai + aj
    inner = r <= np.abs(ai - aj)
    rs = np.where(r > 0, r, 1.0)
    A_far = (1 + s2 / (3 * rs * rs)) / (8 * np.pi * rs)
    B_far = (1 - s2 / (rs * rs)) / (8 * np.pi * rs)
    d2 = (ai - aj) ** 2
    A_mid = (16 * rs ** 3 * (ai + aj) - (d2 + 3 * rs * rs) ** 2) / (32 * rs ** 3) / (6 * np.pi * ai * aj)
    B_mid = 3 * (d2 - rs * rs) ** 2 / (32 * rs ** 3) / (6 * np.pi * ai * aj)
    A_in = 1.0 / (6 * np.pi * np.maximum(ai, aj))
    A = np.where(far, A_far, np.where(inner, A_in, A_mid))
    B = np.where(far, B_far, np.where(inner, 0.0, B_mid))
    return A, A + B


def _sinc(x):
    xs = np.where(x != 0, x, 1.0)
    return np.where(x != 0, np.sin(xs) / xs, 1.0)


@functools.lru_cache(maxsize=8)
def _leggauss(nq):
    return np.polynomial.legendre.leggauss(nq)


def wave_free(r, xi, ai, aj, nq=400):
    """The H-weighted continuous k-integral (F, G), mobility units:
    F = (1/2pi^2) int H sinc(k ai) sinc(k aj) kF(kr) dk, G = (1/pi^2) int ... kG(kr) dk,
    with the radial kernels of eqs. int1/int2; Gauss-Legendre on [0, 16 xi]."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    ai = np.broadcast_to(np.asarray(ai, dtype=np.float64), r.shape)
    aj = np.broadcast_to(np.asarray(aj, dtype=np.float64), r.shape)
    kmax = 16.0 * xi
    t, w = _leggauss(nq)
    k = 0.5 * kmax * (t + 1.0)
    w = 0.5 * kmax * w
    base = rpy._H(k, xi)[None, :] * w[None, :] * _sinc(np.outer(ai, k)) * _sinc(np.outer(aj, k))
    kF, kG = rpy._kernels(np.outer(r, k))
    return (kF * base).sum(axis=1) / (2 * np.pi ** 2), (kG * base).sum(axis=1) / (np.pi ** 2)


def fg(r, xi, ai, aj):
    """Real-space pair scalars (F, G) in mobility units, r >= 0 (r = 0 of one
    sphere with itself, ai = aj, is the self term)."""
    Fr, Gr = rpy_free(r, ai, aj)
    Fw, Gw = wave_free(r, xi, ai, aj)
    return Fr - Fw, Gr - Gw


def self_real(xi, a):
    """Self block s I of a sphere of radius a: free-space 1/(6 pi a) less the H-weighted integral at r = 0."""
    F, _ = fg(np.zeros(1), xi, a, a)
    return float(F[0])


# ----------------------------------------------------------------------------- dense Ewald sum

def mobility_real_dense(pos, radii, L, xi, rc):
    """Grand M^r (3N x 3N) of spheres with radii[i]: every image within r_cut, self blocks on the diagonal."""
    pos = np.asarray(pos, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    N = pos.shape[0]
    Mr = np.zeros((N, 3, N, 3))
    n_img = int(math.ceil(rc / L))
    rng = np.arange(-n_img, n_img + 1)
    R = np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T * L
    d0 = pos[:, None, :] - pos[None, :, :]
    d0 -= L * np.round(d0 / L)
    same = np.eye(N, dtype=bool)
    for Rv in R:
        d = d0 + Rv
        r = np.linalg.norm(d, axis=2)
        mask = (r < rc) & ~(same & (r == 0))
        if not mask.any():
            continue
        ii, jj = np.nonzero(mask)
        F, G = fg(r[ii, jj], xi, radii[ii], radii[jj])
        rh = ewald.unit(d[ii, jj])
        outer = rh[:, :, None] * rh[:, None, :]
        Mr[ii, :, jj, :] += F[:, None, None] * (np.eye(3)[None] - outer) + G[:, None, None] * outer
    selfs = {a: self_real(xi, a) for a in np.unique(radii)}
    for i in range(N):
        Mr[i, :, i, :] += selfs[radii[i]] * np.eye(3)
    return Mr.reshape(3 * N, 3 * N)


def mobility_wave_dense(pos, radii, L, xi, kvec, chunk=4096):
    """Grand M^w (3N x 3N): direct k-sum with sinc(k a_i) sinc(k a_j) H / (V k^2) (I - kk)."""
    pos = np.asarray(pos, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    N = pos.shape[0]
    Mw = np.zeros((3, 3, N, N))
    for s in range(0, kvec.shape[0], chunk):
        k = kvec[s:s + chunk]
        kk = np.linalg.norm(k, axis=1)
        c2 = ewald.H(kk, xi) / (L ** 3 * kk * kk)
        kh = k / kk[:, None]
        ph = np.exp(1j * pos @ k.T) * _sinc(np.outer(radii, kk))
        for p in range(3):
            for q in range(p, 3):
                proj = (1.0 if p == q else 0.0) - kh[:, p] * kh[:, q]
                blk = ((ph * (c2 * proj)[None, :]) @ ph.conj().T).real
                Mw[p, q] += blk
                if q != p:
                    Mw[q, p] += blk
    return Mw.transpose(2, 0, 3, 1).reshape(3 * N, 3 * N)


def mobility_dense(pos, radii, L, xi, tol=1e-12):
    """M = M^w + M^r, both truncated at `tol` (k_cut from the smallest radius)."""
    rc = ewald.r_cut(xi, tol)
    kc = ewald.k_cut(xi, tol, float(np.min(radii)))
    Mr = mobility_real_dense(pos, radii, L, xi, rc)
    Mw = mobility_wave_dense(pos, radii, L, xi, ewald.modes_sphere(kc, L))
    return Mr + Mw, Mr, Mw


# ----------------------------------------------------------------------------- PSE sample

def plan(L, radii, xi, tol, M=None, P=None):
    """The monodisperse plan (Sec. II C) with a = the smallest species radius:
    its wave cutoff bound is the strictest."""
    return ewald.plan(L, float(np.min(radii)), xi, tol, M=M, P=P)


class RealOperator:
    """Sparse polydisperse M^r as a matvec on (N, 3) arrays (pairs within r_cut, nearest image)."""

    def __init__(self, pos, radii, plan_):
        pos = np.asarray(pos, dtype=np.float64)
        radii = np.asarray(radii, dtype=np.float64)
        self.N = pos.shape[0]
        i, j, d = pse.pair_list(pos, plan_.L, plan_.r_cut)
        r = np.linalg.norm(d, axis=1)
        F, G = fg(r, plan_.xi, radii[i], radii[j]) if r.size else (r, r)
        self.i, self.j = i, j
        self.rh = ewald.unit(d) if r.size else d
        self.F, self.GmF = F, G - F
        uniq = np.unique(radii)
        self.self_ = np.array([self_real(plan_.xi, a) for a in uniq])[np.searchsorted(uniq, radii)]

    def __call__(self, v):
        v = np.asarray(v, dtype=np.float64).reshape(self.N, 3)
        out = self.self_[:, None] * v
        if self.i.size:
            i, j, rh = self.i, self.j, self.rh
            bj = self.F[:, None] * v[j] + (self.GmF * np.einsum("kd,kd->k", rh, v[j]))[:, None] * rh
            bi = self.F[:, None] * v[i] + (self.GmF * np.einsum("kd,kd->k", rh, v[i]))[:, None] * rh
            for c in range(3):
                out[:, c] += np.bincount(i, weights=bj[:, c], minlength=self.N)
                out[:, c] += np.bincount(j, weights=bi[:, c], minlength=self.N)
        return out


def real_sample(pos, radii, plan_, seed, sample, n_iter=None, system=0):
    """M^r^{1/2} z1 by the Lanczos of Sec. II B 1 on the polydisperse M^r."""
    pos = np.asarray(pos, dtype=np.float64)
    z = pse.real_noise(pos.shape[0], seed, sample, system)
    return pse.lanczos_sqrt(RealOperator(pos, radii, plan_), z, tol=plan_.tol, n_iter=n_iter)


def wave_sample_grid(pos, species, species_radii, plan_, seed, sample, system=0):
    """Gridded M^w^{1/2} dW2 with the same noise for every species; species s
    interpolates from the grid scaled with its own shape factor sinc(k a_s)."""
    pos = np.asarray(pos, dtype=np.float64)
    species = np.asarray(species)
    out = np.zeros((pos.shape[0], 3))
    for s, a in enumerate(species_radii):
        sel = np.nonzero(species == s)[0]
        if sel.size == 0:
            continue
        v, _ = pse.wave_grid_velocity(dataclasses.replace(plan_, a=float(a)), seed, sample, system)
        out[sel] = pse.interpolate(v, pos[sel], plan_)
    return out


def wave_covariance_grid(pos, species, species_radii, plan_):
    """Exact covariance (3N x 3N) of the gridded polydisperse wave sampler: the
    monodisperse mode sum with sc(k; a_i) sc(k; a_j) in place of sc(k)^2."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    k = ewald.modes_cube(plan_.M, plan_.L)
    kk = np.linalg.norm(k, axis=1)
    rad = np.asarray(species_radii, dtype=np.float64)[np.asarray(species)]
    c = 2 * plan_.xi ** 2 / plan_.eta
    phi = np.full((N, k.shape[0]), (c / np.pi) ** 1.5 * plan_.h ** 3, dtype=np.complex128)
    for d in range(3):
        i0, s = pse.support_start(pos[:, d], plan_)
        nodes = i0[:, None] + np.arange(plan_.P)[None, :]
        w = np.exp(-c * ((s[:, None] - nodes) * plan_.h) ** 2)
        phi *= (w[:, :, None] * np.exp(1j * (nodes * plan_.h)[:, :, None] * k[None, None, :, d])).sum(axis=1)
    phi *= np.stack([pse.wave_scale(kk, dataclasses.replace(plan_, a=float(a))) for a in rad])
    kh = k / kk[:, None]
    C = np.zeros((3, 3, N, N))
    for p in range(3):
        for q in range(3):
            proj = (1.0 if p == q else 0.0) - kh[:, p] * kh[:, q]
            C[p, q] = ((phi * proj[None, :]) @ phi.conj().T).real
    return C.transpose(2, 0, 3, 1).reshape(3 * N, 3 * N)
