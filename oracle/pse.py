"""PSE Brownian sample u = M_r^{1/2} z1 + M_w^{1/2} dW2 (FP64 CPU oracle).

Sec. II B of the paper: eq. split draws the sample as the sum of two
independent parts.

Real part (Sec. II B 1): Krylov / Lanczos approximation of M_r^{1/2} z1
(Chow & Saad): V_j, T_j from j Lanczos steps on A = M_r started at
z1/||z1||; x_j = ||z1|| V_j T_j^{1/2} e_1; stop at the first j with
||x_j - x_{j-1}|| / ||x_j|| < tol.  With a block-diagonal preconditioner P
the iteration runs on P M_r P^T and the result is P^{-1} x_j.

Wave part (Sec. II B 2): M_w^{1/2} = sigma^{1/2} S^T F^dagger B^{1/2}
applied to complex Hermitian noise.  Written out on a grid of M^3 nodes,
spacing h, sigma = h^3, Gaussian g(r) = (2xi^2/(pi eta))^{3/2} exp(-2 xi^2 r^2 / eta)
with Fourier transform ghat(k) = exp(-eta k^2 / 8 xi^2):
    vhat(k) = V^{-1/2} sinc(ka)/k sqrt(1 + k^2/4xi^2) exp(-(1-eta) k^2/8xi^2)
              (I - kk) dW2(k)
    v(x_g)  = sum_k vhat(k) exp(i k . x_g)                 (inverse DFT, unnormalised)
    u_i     = h^3 sum_{P^3 nodes g near x_i} g(x_i - x_g) v(x_g)
so that u_i = sum_k exp(i k.x_i) c_k (I - kk) dW2(k) up to the quadrature
error, with c_k^2 = sinc^2(ka) H(k, xi) / (V k^2), the scalar of eq. Mwave.
``wave_sample_direct`` evaluates that last sum exactly (a non-uniform DFT).

Noise: dW2(k) = (g1 + i g2)/sqrt 2 per component on one representative of
each {k, -k} pair, its partner gets the conjugate (Sec. II B 2's conjugacy
condition); k = 0 and Nyquist modes are zero.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from . import ewald, philox, rpy


# ----------------------------------------------------------------------------- noise

def real_noise(N, seed, sample, system=0):
    """z1 (N, 3): Philox stream 2*system, element = particle index (caller order)."""
    z = philox.normals4(np.arange(N, dtype=np.uint64), 2 * system, seed, sample)
    return z[:, :3].copy()


def _signed(M):
    n = np.arange(M)
    return np.where(n > M // 2, n - M, n)


def wave_noise_full(M, seed, sample, system=0):
    """dW2 on the full M^3 spectrum, shape (3, M, M, M) complex, Hermitian.

    The representative of {k, -k} is the mode whose half-spectrum index has
    nz > 0, or nz = 0 and (ny > 0 or (ny = 0 and nx > 0)); its linear id
    q = (ix*M + iy)*(M//2 + 1) + iz (ix, iy, iz its unsigned indices) keys
    two Philox blocks 2q and 2q+1 (six normals).
    """
    s = _signed(M)
    nx, ny, nz = np.meshgrid(s, s, s, indexing="ij")
    rep = (nz > 0) | ((nz == 0) & ((ny > 0) | ((ny == 0) & (nx > 0))))
    nyq = np.zeros_like(rep)
    if M % 2 == 0:
        h = M // 2
        nyq = (nx == h) | (ny == h) | (nz == h)
    rep &= ~nyq
    ix, iy, iz = np.nonzero(rep)
    q = ((ix.astype(np.uint64) * M + iy) * (M // 2 + 1) + iz).astype(np.uint64)
    a = philox.normals4(2 * q, 2 * system + 1, seed, sample)
    b = philox.normals4(2 * q + 1, 2 * system + 1, seed, sample)
    w = np.zeros((3, M, M, M), dtype=np.complex128)
    inv = 1.0 / math.sqrt(2.0)
    vals = np.stack([(a[:, 0] + 1j * a[:, 1]), (a[:, 2] + 1j * a[:, 3]), (b[:, 0] + 1j * b[:, 1])]) * inv
    w[:, ix, iy, iz] = vals
    jx, jy, jz = (-nx[ix, iy, iz]) % M, (-ny[ix, iy, iz]) % M, (-nz[ix, iy, iz]) % M
    w[:, jx, jy, jz] = vals.conj()
    return w


def wave_vectors_full(M, L):
    s = _signed(M) * (2 * np.pi / L)
    kx, ky, kz = np.meshgrid(s, s, s, indexing="ij")
    return kx, ky, kz


def _project(kx, ky, kz, w):
    """(I - kk) w per mode; k = 0 entries returned unchanged (they are zero)."""
    k2 = kx * kx + ky * ky + kz * kz
    k2s = np.where(k2 > 0, k2, 1.0)
    dot = (kx * w[0] + ky * w[1] + kz * w[2]) / k2s
    return np.stack([w[0] - kx * dot, w[1] - ky * dot, w[2] - kz * dot])


# ----------------------------------------------------------------------------- wave part

def wave_scale(k, plan):
    """V^{-1/2} sinc(ka)/k sqrt(1 + k^2/4xi^2) exp(-(1-eta) k^2/8xi^2); 0 at k = 0."""
    a, xi, eta, V = plan.a, plan.xi, plan.eta, plan.L ** 3
    ks = np.where(k > 0, k, 1.0)
    sinc = np.sin(ks * a) / (ks * a)
    out = (sinc / ks) * np.sqrt(1 + ks * ks / (4 * xi * xi)) * np.exp(-(1 - eta) * ks * ks / (8 * xi * xi))
    return np.where(k > 0, out / math.sqrt(V), 0.0)


def wave_grid_velocity(plan, seed, sample, system=0):
    """v(x_g) on the M^3 grid, shape (3, M, M, M) float64 (and its max |imag|)."""
    M = plan.M
    w = wave_noise_full(M, seed, sample, system)
    kx, ky, kz = wave_vectors_full(M, plan.L)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    vhat = _project(kx, ky, kz, w) * wave_scale(k, plan)[None]
    v = np.fft.ifftn(vhat, axes=(1, 2, 3)) * float(M) ** 3
    return v.real, float(np.abs(v.imag).max())


def support_start(x, plan):
    """First node index of each particle's P-point support along one axis.

    i0 = floor(x/h - P/2) + 1, so the P nodes i0 .. i0+P-1 are the ones
    within P h / 2 of x.  Decided in float64 from the float32-exact x.
    """
    s = np.asarray(x, dtype=np.float64) * plan.M / plan.L
    return np.floor(s - plan.P / 2.0).astype(np.int64) + 1, s


def interpolate(vgrid, pos, plan):
    """u_i = h^3 sum over the P^3 support of g(x_i - x_g) v(x_g)   (S^dagger = sigma S^T)."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    M, P, h = plan.M, plan.P, plan.h
    c = 2 * plan.xi ** 2 / plan.eta
    norm = (c / np.pi) ** 1.5 * h ** 3
    out = np.zeros((N, 3))
    idx = []
    wts = []
    for d in range(3):
        i0, s = support_start(pos[:, d], plan)
        off = np.arange(P)
        nodes = i0[:, None] + off[None, :]
        dist = (s[:, None] - nodes) * h
        wts.append(np.exp(-c * dist * dist))
        idx.append(np.mod(nodes, M))
    for p in range(P):
        for q in range(P):
            wxy = wts[0][:, p] * wts[1][:, q]
            for r in range(P):
                wgt = wxy * wts[2][:, r]
                gx, gy, gz = idx[0][:, p], idx[1][:, q], idx[2][:, r]
                out += (wgt[:, None] * vgrid[:, gx, gy, gz].T)
    return out * norm


def wave_sample_grid(pos, plan, seed, sample, system=0):
    """Gridded wave-space sample M_w^{1/2} dW2 at the particles (N, 3)."""
    v, _ = wave_grid_velocity(plan, seed, sample, system)
    return interpolate(v, pos, plan)


def wave_sample_direct(pos, plan, seed, sample, system=0, chunk=8192):
    """Exact non-uniform sum u_i = sum_k exp(i k.x_i) c_k (I - kk) dW2(k), same modes/noise."""
    pos = np.asarray(pos, dtype=np.float64)
    M = plan.M
    w = wave_noise_full(M, seed, sample, system)
    kx, ky, kz = wave_vectors_full(M, plan.L)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    ghat = np.exp(-plan.eta * k * k / (8 * plan.xi ** 2))
    coef = _project(kx, ky, kz, w) * (wave_scale(k, plan) * ghat)[None]
    sel = np.nonzero(k.ravel() > 0)[0]
    kv = np.stack([kx.ravel()[sel], ky.ravel()[sel], kz.ravel()[sel]], axis=1)
    cf = coef.reshape(3, -1)[:, sel]
    out = np.zeros((pos.shape[0], 3), dtype=np.complex128)
    for s in range(0, kv.shape[0], chunk):
        ph = np.exp(1j * pos @ kv[s:s + chunk].T)
        out += ph @ cf[:, s:s + chunk].T
    return out.real


def wave_covariance_grid(pos, plan):
    """Exact covariance (3N x 3N) of the gridded wave sampler, mode by mode.

    u is linear in dW2, so Cov(u)_ij = sum_k |vscale_k|^2 (I - kk) phi_i(k) conj(phi_j(k))
    with phi_i(k) = h^3 sum_{support of i} g(x_i - x_g) exp(i k.x_g), the
    interpolation of one unit mode.  Compared with eq. Mwave this measures
    the NUFFT's quadrature + aliasing + truncation error without sampling.
    """
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    k = ewald.modes_cube(plan.M, plan.L)
    kk = np.linalg.norm(k, axis=1)
    vs2 = wave_scale(kk, plan) ** 2
    c = 2 * plan.xi ** 2 / plan.eta
    phi = np.full((N, k.shape[0]), (c / np.pi) ** 1.5 * plan.h ** 3, dtype=np.complex128)
    for d in range(3):
        i0, s = support_start(pos[:, d], plan)
        nodes = i0[:, None] + np.arange(plan.P)[None, :]
        w = np.exp(-c * ((s[:, None] - nodes) * plan.h) ** 2)
        phi *= (w[:, :, None] * np.exp(1j * (nodes * plan.h)[:, :, None] * k[None, None, :, d])).sum(axis=1)
    kh = k / kk[:, None]
    C = np.zeros((3, 3, N, N))
    for p in range(3):
        for q in range(3):
            proj = (1.0 if p == q else 0.0) - kh[:, p] * kh[:, q]
            C[p, q] = ((phi * (vs2 * proj)[None, :]) @ phi.conj().T).real
    return C.transpose(2, 0, 3, 1).reshape(3 * N, 3 * N)


# ----------------------------------------------------------------------------- spreading, M_w F and grid noise

def nyquist_mask(M):
    """(M, M, M) bool: modes with an index at the Nyquist frequency of an even grid."""
    if M % 2:
        return np.zeros((M, M, M), dtype=bool)
    h = M // 2
    i = np.arange(M) == h
    return i[:, None, None] | i[None, :, None] | i[None, None, :]


def spread(F, pos, plan):
    """Grid force density s(x_g) = sum_i g(x_g - x_i) F_i, shape (3, M, M, M).

    The spreading operator S of Sec. II B 2 on the same P^3 support and
    Gaussian g as ``interpolate`` (S^dagger = h^3 S^T).
    """
    pos = np.asarray(pos, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 3)
    M, P, h = plan.M, plan.P, plan.h
    c = 2 * plan.xi ** 2 / plan.eta
    norm = (c / np.pi) ** 1.5
    grid = np.zeros((3, M, M, M))
    idx, wts = [], []
    for d in range(3):
        i0, s = support_start(pos[:, d], plan)
        nodes = i0[:, None] + np.arange(P)[None, :]
        dist = (s[:, None] - nodes) * h
        wts.append(np.exp(-c * dist * dist))
        idx.append(np.mod(nodes, M))
    for p in range(P):
        for q in range(P):
            for r in range(P):
                wgt = wts[0][:, p] * wts[1][:, q] * wts[2][:, r]
                at = (idx[0][:, p], idx[1][:, q], idx[2][:, r])
                for d in range(3):
                    np.add.at(grid[d], at, wgt * F[:, d])
    return grid * norm


def wave_apply_grid(F, pos, plan):
    """Gridded wave-space product M_w F (N, 3): spread, forward DFT, the mode
    factor h^3 B(k) (I - kk) with B(k)/V = wave_scale(k)^2 (so that with
    ghat^2 it is c_k^2 of eq. Mwave), k = 0 and Nyquist dropped, inverse DFT
    (unnormalised), interpolation.  The deterministic wave path of Sec. III."""
    M = plan.M
    shat = np.fft.fftn(spread(F, pos, plan), axes=(1, 2, 3))
    kx, ky, kz = wave_vectors_full(M, plan.L)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    fac = plan.h ** 3 * wave_scale(k, plan) ** 2
    fac[nyquist_mask(M)] = 0.0
    vhat = _project(kx, ky, kz, shat) * fac[None]
    v = np.fft.ifftn(vhat, axes=(1, 2, 3)) * float(M) ** 3
    return interpolate(v.real, pos, plan)


def mobility_apply(F, pos, plan, op=None):
    """M F = M_r F (sparse, eq. Mreal) + gridded M_w F (N, 3)."""
    A = RealOperator(np.asarray(pos, dtype=np.float64), plan) if op is None else op
    return A(F) + wave_apply_grid(F, pos, plan)


def grid_noise(M, seed, sample, system=0):
    """White noise W(x_g) ~ N(0, 1) per node and component, shape (3, M, M, M).

    Node id g = (ix*M + iy)*M + iz keys one Philox block on the wave stream
    2*system + 1; its first three normals are the x, y, z components.
    """
    g = np.arange(M ** 3, dtype=np.uint64)
    n = philox.normals4(g, 2 * system + 1, seed, sample)
    return np.ascontiguousarray(n[:, :3].T).reshape(3, M, M, M)


def wave_sample_gridnoise(pos, plan, seed, sample, system=0, W=None):
    """Wave-space sample drawn from white noise on the grid instead of in k-space.

    What(k) = M^{-3/2} sum_g W(x_g) exp(-i k.x_g) has, on every mode pair
    {k, -k} off Nyquist, the law of dW2(k) (real and imaginary parts of
    variance 1/2, conjugate partners), so scaling it exactly as in the
    k-space path (wave_scale(k) (I - kk), k = 0 and Nyquist dropped) gives a
    sample with the same covariance as ``wave_sample_grid`` (the fluctuating
    hydrodynamics remark of Sec. II B 2).  ``W`` overrides the drawn noise.
    """
    M = plan.M
    if W is None:
        W = grid_noise(M, seed, sample, system)
    What = np.fft.fftn(np.asarray(W, dtype=np.float64), axes=(1, 2, 3)) / float(M) ** 1.5
    kx, ky, kz = wave_vectors_full(M, plan.L)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    fac = wave_scale(k, plan)
    fac[nyquist_mask(M)] = 0.0
    vhat = _project(kx, ky, kz, What) * fac[None]
    v = np.fft.ifftn(vhat, axes=(1, 2, 3)) * float(M) ** 3
    return interpolate(v.real, pos, plan)


def sample_with_forces(pos, F, plan, seed, sample, c_det=1.0, c_noise=1.0, n_iter=None, system=0):
    """c_det M F + c_noise M^{1/2} z (N, 3): the deterministic and Brownian parts
    of one Euler-Maruyama displacement (Sec. III: the wave parts share one
    inverse FFT).  Returns (out, j_lanczos)."""
    pos = np.asarray(pos, dtype=np.float64)
    A = RealOperator(pos, plan)
    out = np.zeros((pos.shape[0], 3))
    j = 0
    if c_det != 0.0:
        out += c_det * mobility_apply(F, pos, plan, op=A)
    if c_noise != 0.0:
        ur, j, _ = real_sample(pos, plan, seed, sample, n_iter=n_iter, system=system, op=A)
        out += c_noise * (ur + wave_sample_grid(pos, plan, seed, sample, system))
    return out, j


# ----------------------------------------------------------------------------- Brownian dynamics

def repulsion_forces(pos, L, a, k_rep):
    """Harmonic overlap repulsion F_i = k_rep sum_j (2a - r_ij) rhat_ij over the
    pairs closer than 2a (minimum image), rhat_ij pointing from j to i."""
    pos = np.asarray(pos, dtype=np.float64)
    F = np.zeros_like(pos)
    i, j, d = pair_list(pos, L, 2 * a * (1 - 1e-12))
    if i.size:
        r = np.linalg.norm(d, axis=1)
        f = (k_rep * (2 * a - r) / r)[:, None] * d
        np.add.at(F, i, f)
        np.add.at(F, j, -f)
    return F


def bd_step(pos, plan, seed, step, dt, kT, k_rep, f_ext=None, n_iter=None, system=0):
    """One Euler-Maruyama step of Brownian dynamics (Sec. II B, eq. langevin, div M = 0 in a periodic box):
    x + dt M F + sqrt(2 kT dt) M^{1/2} z, F = overlap repulsion (+ f_ext), the
    noise of (seed, step); the new positions are wrapped into [0, L).
    Returns (new positions, displacement, j_lanczos)."""
    pos = np.asarray(pos, dtype=np.float64)
    F = repulsion_forces(pos, plan.L, plan.a, k_rep)
    if f_ext is not None:
        F = F + np.asarray(f_ext, dtype=np.float64).reshape(-1, 3)
    dx, j = sample_with_forces(pos, F, plan, seed, step, c_det=dt, c_noise=math.sqrt(2 * kT * dt),
                               n_iter=n_iter, system=system)
    return np.mod(pos + dx, plan.L), dx, j


# ----------------------------------------------------------------------------- real part

def pair_list(pos, L, rc):
    """All pairs i < j with minimum-image distance < r_cut (requires r_cut < L/2)."""
    if rc >= L / 2:
        raise ValueError("pair_list needs r_cut < L/2; use ewald.mobility_real_dense")
    p = np.mod(np.asarray(pos, dtype=np.float64), L)
    p[p >= L] = 0.0
    tree = cKDTree(p, boxsize=L)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3))
    i, j = pairs[:, 0], pairs[:, 1]
    d = p[i] - p[j]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    keep = r < rc
    return i[keep], j[keep], d[keep]


class RealOperator:
    """Sparse M_r (eq. Mreal, App. A) as a matvec on (N, 3) arrays."""

    def __init__(self, pos, plan, pairs=None):
        self.N = pos.shape[0]
        a, xi = plan.a, plan.xi
        i, j, d = pair_list(pos, plan.L, plan.r_cut) if pairs is None else pairs
        r = np.linalg.norm(d, axis=1)
        F, G = rpy.fg(r, xi, a)
        self.i, self.j = i, j
        self.rh = ewald.unit(d) if r.size else d
        self.F = F / (6 * np.pi * a)
        self.GmF = (G - F) / (6 * np.pi * a)
        self.self_ = rpy.self_real(xi, a) / (6 * np.pi * a)

    def __call__(self, v):
        v = np.asarray(v, dtype=np.float64).reshape(self.N, 3)
        out = self.self_ * v
        if self.i.size:
            i, j, rh = self.i, self.j, self.rh
            # block B = F I + (G - F) rr, symmetric and the same for (i,j) and (j,i)
            bj = self.F[:, None] * v[j] + (self.GmF * np.einsum("kd,kd->k", rh, v[j]))[:, None] * rh
            bi = self.F[:, None] * v[i] + (self.GmF * np.einsum("kd,kd->k", rh, v[i]))[:, None] * rh
            for d in range(3):
                out[:, d] += np.bincount(i, weights=bj[:, d], minlength=self.N)
                out[:, d] += np.bincount(j, weights=bi[:, d], minlength=self.N)
        return out


def real_rows(pos, plan, rows, v):
    """Rows `rows` of M_r v (eq. Mreal with the App. A scalars, eq. self on the
    diagonal), evaluated one particle at a time from its neighbours within
    r_cut (minimum image): the near-field product at sampled particles of a
    system too large for the full pair list.  Returns (len(rows), 3)."""
    pos = np.asarray(pos, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    L, a, xi = plan.L, plan.a, plan.xi
    p = np.mod(pos, L)
    p[p >= L] = 0.0
    tree = cKDTree(p, boxsize=L)
    s = rpy.self_real(xi, a) / (6 * np.pi * a)
    out = np.zeros((len(rows), 3))
    for n, i in enumerate(rows):
        nb = np.asarray(tree.query_ball_point(p[i], plan.r_cut), dtype=np.int64)
        nb = nb[nb != i]
        d = p[i] - p[nb]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=1)
        keep = r < plan.r_cut
        nb, d, r = nb[keep], d[keep], r[keep]
        acc = s * v[i]
        if nb.size:
            F, G = rpy.fg(r, xi, a)
            rh = ewald.unit(d)
            vj = v[nb]
            dot = np.einsum("kd,kd->k", rh, vj)
            acc = acc + ((F[:, None] * vj + ((G - F) * dot)[:, None] * rh) / (6 * np.pi * a)).sum(axis=0)
        out[n] = acc
    return out


def sqrt_tridiag_e1(alpha, beta):
    """T^{1/2} e_1 for the symmetric tridiagonal T (diag alpha, off-diag beta)."""
    j = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: j - 1], 1) + np.diag(beta[: j - 1], -1)
    lam, Q = np.linalg.eigh(T)
    if lam.min() < 0:
        raise FloatingPointError("Lanczos T not positive definite")
    return Q @ (np.sqrt(lam) * Q[0, :])


def lanczos_sqrt(apply_A, z, tol=1e-3, n_iter=None, max_iter=100):
    """x ~ A^{1/2} z by Lanczos (Chow & Saad), FP64, no reorthogonalisation.

    Steps: v_1 = z/||z||; w = A v_j - beta_{j-1} v_{j-1}; alpha_j = <w, v_j>;
    w -= alpha_j v_j; beta_j = ||w||; v_{j+1} = w / beta_j.
    x_j = ||z|| V_j T_j^{1/2} e_1.  With n_iter given, exactly n_iter steps
    are taken; otherwise the first j >= 2 with ||x_j - x_{j-1}||/||x_j|| < tol.
    Returns (x, j, history of relative changes).
    """
    shape = z.shape
    z = np.asarray(z, dtype=np.float64).ravel()
    nz = np.linalg.norm(z)
    V = [z / nz]
    alpha, beta = [], []
    v_prev = np.zeros_like(z)
    b_prev = 0.0
    x_prev = None
    hist = []
    limit = n_iter if n_iter is not None else max_iter
    x = None
    for j in range(1, limit + 1):
        w = apply_A(V[-1].reshape(shape)).ravel() - b_prev * v_prev
        a_j = float(w @ V[-1])
        w = w - a_j * V[-1]
        b_j = float(np.linalg.norm(w))
        alpha.append(a_j)
        beta.append(b_j)
        y = sqrt_tridiag_e1(np.array(alpha), np.array(beta))
        x = nz * (np.array(V).T @ y)
        if x_prev is not None:
            rel = np.linalg.norm(x - x_prev) / np.linalg.norm(x)
            hist.append(rel)
            if n_iter is None and rel < tol:
                return x.reshape(shape), j, hist
        x_prev = x
        v_prev = V[-1]
        b_prev = b_j
        if b_j == 0.0:
            break
        V.append(w / b_j)
    return x.reshape(shape), j, hist


def real_sample(pos, plan, seed, sample, n_iter=None, lanczos_tol=None, precond=None, system=0,
                op=None):
    """M_r^{1/2} z1 by Lanczos; with `precond` = (S (N,3,3) SPD blocks), P^{-1} (P M_r P)^{1/2} z1."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    z = real_noise(N, seed, sample, system)
    A = RealOperator(pos, plan) if op is None else op
    tol = plan.tol if lanczos_tol is None else lanczos_tol
    if precond is None:
        x, j, hist = lanczos_sqrt(A, z, tol=tol, n_iter=n_iter)
        return x, j, hist
    S = np.asarray(precond, dtype=np.float64)

    def PAP(v):
        return np.einsum("nab,nb->na", S, A(np.einsum("nab,nb->na", S, v)))

    x, j, hist = lanczos_sqrt(PAP, z, tol=tol, n_iter=n_iter)
    return np.linalg.solve(S, x[..., None])[..., 0], j, hist


def full_sample(pos, plan, seed, sample, n_iter=None, lanczos_tol=None, system=0, max_iter=100):
    """The comparison method of Sec. IV (Fig. timing, Fig. RelLanc): Lanczos
    applied to the whole mobility, M^{1/2} z by the same Chow & Saad
    iteration and stop rule as the real part, every step one product
    M q = M_r q + gridded M_w q (``mobility_apply``, the M F of Sec. III).
    z is the real-space noise z1 of (seed, sample, system).
    Returns (x (N, 3), j, history of relative changes)."""
    pos = np.asarray(pos, dtype=np.float64)
    A = RealOperator(pos, plan)
    z = real_noise(pos.shape[0], seed, sample, system)
    tol = plan.tol if lanczos_tol is None else lanczos_tol
    return lanczos_sqrt(lambda v: mobility_apply(v, pos, plan, op=A), z, tol=tol, n_iter=n_iter,
                        max_iter=max_iter)
