"""Positively split Ewald sum of the periodic RPY mobility (FP64, dense).

Sec. II A (eqs. pairmobility, Mwave, Mreal) and Sec. II C (error bounds).
Units: eta = 1; positions in a periodic cube of side L; V = L^3.

Functions
---------
H(k, xi)                    Hasimoto splitting function (Sec. II A)
r_cut(xi, tol)              eps_R ~ exp(-xi^2 r_cut^2)            (Sec. II C)
k_cut(xi, tol, a)           smallest k with the eq. errbound closed-form bound <= tol
quadrature_P_m(tol)         smallest integer P with min_m eps_q(P, m) <= tol  (Sec. II C)
grid_size(k_cut, L, P)      smallest 2,3,5,7-smooth M with pi M / L >= k_cut
plan(L, a, xi, tol)         all of the above plus the Gaussian shape eta_g
mobility_real_dense(...)    grand M^(r): blocks (F(I-rr)+Grr)/(6 pi a), all images
mobility_wave_dense(...)    grand M^(w): direct k-sum of eq. Mwave over a mode set
mobility_dense(...)         M = M^(w) + M^(r)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import rpy


def H(k, xi):
    """H(k, xi) = (1 + k^2/4xi^2) exp(-k^2/4xi^2)  (Sec. II A, below eq. green)."""
    q = np.asarray(k, dtype=np.float64) ** 2 / (4.0 * xi * xi)
    return (1.0 + q) * np.exp(-q)


def r_cut(xi, tol):
    """Real-space cutoff from eps_R ~ exp(-xi^2 r_cut^2) = tol (Sec. II A/C)."""
    return math.sqrt(math.log(1.0 / tol)) / xi


def kcut_bound(k, xi, a=1.0):
    """eq. errbound's closed-form upper bound on the wave truncation error."""
    return (4.0 / k * math.exp(-k * k / (4 * xi * xi))
            - math.sqrt(math.pi) / xi * math.erfc(k / (2 * xi))) / (2 * math.pi * a)


def k_cut(xi, tol, a=1.0):
    """Smallest k_cut with kcut_bound(k_cut) <= tol (bisection, the bound decreases in k)."""
    lo, hi = 1e-6, 1.0
    while kcut_bound(hi, xi, a) > tol:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if kcut_bound(mid, xi, a) > tol:
            lo = mid
        else:
            hi = mid
    return hi


def quadrature_error(P, m):
    """eps_q ~ exp(-pi^2 P^2 / 2 m^2) + erfc(m / sqrt 2)  (Sec. II C)."""
    return math.exp(-math.pi ** 2 * P * P / (2 * m * m)) + math.erfc(m / math.sqrt(2.0))


def best_m(P):
    """Minimiser over m of quadrature_error(P, m): root of its m-derivative.

    d/dm = exp(-c/m^2) 2c/m^3 - sqrt(2/pi) exp(-m^2/2),  c = pi^2 P^2 / 2;
    negative at m = 0.5, positive at m = 2P; bisection to machine precision.
    """
    c = math.pi ** 2 * P * P / 2.0

    def d(m):
        return math.exp(-c / (m * m)) * 2 * c / m ** 3 - math.sqrt(2 / math.pi) * math.exp(-m * m / 2)

    lo, hi = 0.5, 2.0 * P
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if d(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def quadrature_P_m(tol, P_min=3):
    """Smallest integer P (>= P_min) whose best m gives eps_q <= tol."""
    P = P_min
    while quadrature_error(P, best_m(P)) > tol:
        P += 1
    return P, best_m(P)


def _smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def grid_size(kc, L, P):
    """Smallest 2,3,5,7-smooth M with Nyquist pi M / L >= k_cut and M >= P + 1."""
    M = max(int(math.ceil(kc * L / math.pi - 1e-9)), P + 1, 4)
    while not _smooth(M):
        M += 1
    return M


@dataclass
class Plan:
    L: float
    a: float
    xi: float
    tol: float
    r_cut: float
    k_cut: float
    P: int
    m: float
    M: int
    h: float
    eta: float  # Gaussian shape: sigma^2 = eta / (4 xi^2)


def plan(L, a, xi, tol, M=None, P=None):
    """PSE parameters from (L, a, xi, tol): r_cut, k_cut, P, m, grid M, eta_g.

    Reading of Sec. II B/C: the Gaussian is truncated at m standard
    deviations on a P-point support, so its half-width P h / 2 = m sigma,
    with sigma^2 = eta / (4 xi^2), giving eta = (P h xi / m)^2.  eta must be
    <= 1 so that the mode scaling exp(-(1-eta) k^2 / 8 xi^2) never grows; the
    grid is enlarged until it is.
    """
    rc = r_cut(xi, tol)
    kc = k_cut(xi, tol, a)
    if P is None:
        P, m = quadrature_P_m(tol)
    else:
        m = best_m(P)
    if M is None:
        M = grid_size(kc, L, P)
        while (P * (L / M) * xi / m) ** 2 > 1.0:
            M += 1
            while not _smooth(M):
                M += 1
    h = L / M
    eta = (P * h * xi / m) ** 2
    return Plan(L=L, a=a, xi=xi, tol=tol, r_cut=rc, k_cut=kc, P=P, m=m, M=M, h=h, eta=eta)


def unit(rvec):
    """Unit vectors of rows of rvec; 0 for a zero row.  At r = 0 the App. A
    scalars meet (F(0) = G(0), eq. self), so the block F (I - rr) + G rr is
    F I whatever direction is used."""
    r = np.linalg.norm(rvec, axis=1)
    return np.divide(rvec, r[:, None], out=np.zeros_like(rvec), where=r[:, None] > 0)


def _block(rvec, F, G, a):
    """Pair blocks (F (I - rr) + G rr) / (6 pi a) for rows of rvec (K, 3)."""
    rh = unit(rvec)
    outer = rh[:, :, None] * rh[:, None, :]
    eye = np.eye(3)[None]
    return (F[:, None, None] * (eye - outer) + G[:, None, None] * outer) / (6 * np.pi * a)


def mobility_real_dense(pos, L, a, xi, rc):
    """Grand real-space mobility M^(r) (3N x 3N), eq. Mreal with App. A scalars.

    Sums every periodic image R with |x_i - x_j + R| < r_cut (so r_cut may
    exceed L/2); the diagonal block adds the self term of eq. self.
    """
    pos = np.asarray(pos, dtype=np.float64)
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
        # every image pair inside r_cut except a particle with itself at R = 0
        # (the self term below); distinct particles at r = 0 keep the r -> 0 block
        mask = (r < rc) & ~(same & (r == 0))
        if not mask.any():
            continue
        ii, jj = np.nonzero(mask)
        F, G = rpy.fg(r[ii, jj], xi, a)
        Mr[ii, :, jj, :] += _block(d[ii, jj], F, G, a)
    s = rpy.self_real(xi, a) / (6 * np.pi * a)
    for i in range(N):
        Mr[i, :, i, :] += s * np.eye(3)
    return Mr.reshape(3 * N, 3 * N)


def modes_cube(M, L):
    """Wave vectors of an M^3 grid's modes: integer triples in (-M/2, M/2)^3.

    k = 0 is excluded (eq. green) and so is any Nyquist index (n = M/2 for
    even M), whose mode is its own conjugate partner; returns (K, 3) k.
    """
    n = np.arange(M)
    n = np.where(n > M // 2, n - M, n)
    if M % 2 == 0:
        n = n[n != M // 2]
    grid = np.array(np.meshgrid(n, n, n, indexing="ij")).reshape(3, -1).T
    grid = grid[np.any(grid != 0, axis=1)]
    return grid * (2 * np.pi / L)


def modes_sphere(kmax, L):
    """All k = 2 pi n / L, n integer, 0 < |k| <= kmax."""
    nmax = int(math.floor(kmax * L / (2 * np.pi))) + 1
    n = np.arange(-nmax, nmax + 1)
    grid = np.array(np.meshgrid(n, n, n, indexing="ij")).reshape(3, -1).T
    k = grid * (2 * np.pi / L)
    kk = np.linalg.norm(k, axis=1)
    return k[(kk > 0) & (kk <= kmax)]


def wave_coeff2(k, a, xi, L):
    """c_k^2 = sinc^2(ka) H(k, xi) / (V k^2): the scalar of eq. Mwave (eta = 1)."""
    kk = np.linalg.norm(k, axis=1)
    ka = kk * a
    sinc = np.sin(ka) / ka
    return sinc * sinc * H(kk, xi) / (L ** 3 * kk * kk)


def mobility_wave_dense(pos, L, a, xi, kvec, chunk=4096):
    """Grand wave-space mobility M^(w) (3N x 3N), eq. Mwave, direct k-sum.

    M^(w)_ij = sum_k c_k^2 cos(k.(x_i - x_j)) (I - kk) over the given modes.
    """
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    Mw = np.zeros((3, 3, N, N))
    for s in range(0, kvec.shape[0], chunk):
        k = kvec[s:s + chunk]
        c2 = wave_coeff2(k, a, xi, L)
        kh = k / np.linalg.norm(k, axis=1)[:, None]
        ph = np.exp(1j * pos @ k.T)  # (N, K)
        for p in range(3):
            for q in range(p, 3):
                proj = (1.0 if p == q else 0.0) - kh[:, p] * kh[:, q]
                blk = ((ph * (c2 * proj)[None, :]) @ ph.conj().T).real
                Mw[p, q] += blk
                if q != p:
                    Mw[q, p] += blk
    return Mw.transpose(2, 0, 3, 1).reshape(3 * N, 3 * N)


def mobility_dense(pos, L, a, xi, tol=1e-12):
    """M = M^(w) + M^(r) with both truncations at `tol` (Sec. II A)."""
    rc = r_cut(xi, tol)
    kc = k_cut(xi, tol, a)
    Mr = mobility_real_dense(pos, L, a, xi, rc)
    Mw = mobility_wave_dense(pos, L, a, xi, modes_sphere(kc, L))
    return Mr + Mw, Mr, Mw
