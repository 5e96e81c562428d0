"""Pins of the oracle's PSE sample (Sec. II B) against facts that do not depend on it."""
import math

import numpy as np
import pytest

from oracle import ewald, pse, rpy

SEED = 20240601


def _hs(N, phi, seed):
    from paper_1611_09322_gb300 import workloads
    p, L, _ = workloads.hard_spheres(N, phi, seed)
    return p.astype(np.float64), L


def test_gridded_wave_covariance_within_tolerance():
    """Sec. II C: with r_cut, k_cut, P, m and the grid chosen from tol, the gridded
    wave operator's exact covariance reproduces eq. Mwave (all k, converged) to
    O(tol) relative to the Stokes mobility; the error falls with tol.  The
    paper's bounds are order-of-magnitude ("~"): the measured constant is 5-13,
    almost all of it on the self term (modes aliased near the grid's Nyquist)."""
    pos, L = _hs(64, 0.1, 3)
    Mw = ewald.mobility_wave_dense(pos, L, 1.0, 0.5, ewald.modes_sphere(ewald.k_cut(0.5, 1e-14), L))
    errs = []
    for tol in (1e-3, 1e-4, 1e-5):
        plan = ewald.plan(L, 1.0, 0.5, tol)
        Cg = pse.wave_covariance_grid(pos, plan)
        err = np.abs(Cg - Mw).max() * 6 * math.pi
        assert err < 20 * tol
        errs.append(err)
    assert errs[0] > 5 * errs[1] > 25 * errs[2]


def test_covariance_formula_matches_direct_sum_statistics():
    """The gridded sample with the same noise as the exact non-uniform k-sum differs
    from it by the aliased near-Nyquist modes, ~sqrt(covariance error)."""
    pos, L = _hs(64, 0.1, 3)
    plan = ewald.plan(L, 1.0, 0.5, 1e-5)
    ug = pse.wave_sample_grid(pos, plan, SEED, 0)
    ud = pse.wave_sample_direct(pos, plan, SEED, 0)
    err = np.linalg.norm(ug - ud) / np.linalg.norm(ud)
    assert err < 10 * math.sqrt(plan.tol)


def test_grid_velocity_is_real():
    """Hermitian noise (dW2(-k) = conj dW2(k)) gives a real velocity field."""
    pos, L = _hs(64, 0.1, 3)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    v, imag = pse.wave_grid_velocity(plan, SEED, 1)
    assert imag < 1e-12 * np.abs(v).max()


@pytest.mark.parametrize("M", [9, 10])
def test_wave_noise_conjugacy_and_variance(M):
    w = pse.wave_noise_full(M, SEED, 3)
    idx = (-np.arange(M)) % M
    assert np.allclose(w, w[:, idx][:, :, idx][:, :, :, idx].conj())
    assert w[:, 0, 0, 0].sum() == 0
    if M % 2 == 0:
        assert np.all(w[:, M // 2] == 0) and np.all(w[:, :, :, M // 2] == 0)
    nz = np.abs(w[w != 0]) ** 2
    assert abs(nz.mean() - 1) < 5 * math.sqrt(1 / nz.size)


def test_sparse_operator_matches_dense():
    """The pair-list matvec is the same M^(r) as the dense all-image assembly."""
    pos, L = _hs(64, 0.2, 5)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    op = pse.RealOperator(pos, plan)
    Md = ewald.mobility_real_dense(pos, L, 1.0, 0.5, plan.r_cut)
    v = np.random.default_rng(0).standard_normal((64, 3))
    assert np.abs(op(v).ravel() - Md @ v.ravel()).max() < 1e-14


def test_lanczos_converges_to_dense_square_root():
    """Lanczos at tight tolerance = M_r^{1/2} z from the dense eigendecomposition."""
    pos, L = _hs(64, 0.1, 7)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    Md = ewald.mobility_real_dense(pos, L, 1.0, 0.5, plan.r_cut)
    lam, Q = np.linalg.eigh(Md)
    z = pse.real_noise(64, SEED, 0)
    exact = Q @ (np.sqrt(lam) * (Q.T @ z.ravel()))
    x, j, _ = pse.lanczos_sqrt(pse.RealOperator(pos, plan), z, tol=1e-10)
    assert np.linalg.norm(x.ravel() - exact) / np.linalg.norm(exact) < 1e-8
    x3, j3, _ = pse.lanczos_sqrt(pse.RealOperator(pos, plan), z, tol=1e-3)
    assert np.linalg.norm(x3.ravel() - exact) / np.linalg.norm(exact) < 1e-3
    assert 2 <= j3 < j


def test_preconditioned_sample_is_exact_transform():
    """With block-diagonal P: P^{-1} (P M_r P)^{1/2} z, computed densely."""
    pos, L = _hs(32, 0.1, 9)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((32, 3, 3)) * 0.2
    S = np.einsum("nab,ncb->nac", A, A) + np.eye(3)[None] * 2.0
    y, j, _ = pse.real_sample(pos, plan, SEED, 0, lanczos_tol=1e-11, precond=S)
    Md = ewald.mobility_real_dense(pos, L, 1.0, 0.5, plan.r_cut)
    Pm = np.zeros((96, 96))
    for n in range(32):
        Pm[3 * n:3 * n + 3, 3 * n:3 * n + 3] = S[n]
    lam, Q = np.linalg.eigh(Pm @ Md @ Pm)
    z = pse.real_noise(32, SEED, 0).ravel()
    exact = np.linalg.solve(Pm, Q @ (np.sqrt(lam) * (Q.T @ z)))
    assert np.linalg.norm(y.ravel() - exact) / np.linalg.norm(exact) < 1e-8


def test_sample_covariance_is_the_mobility():
    """eq. split: Cov(u_real + u_wave) = M_r + M_w = M (whitened statistics, 4 sigma)."""
    N, n = 32, 1500
    pos, L = _hs(N, 0.1, 11)
    plan = ewald.plan(L, 1.0, 0.7, 1e-4)
    op = pse.RealOperator(pos, plan)
    Mr = ewald.mobility_real_dense(pos, L, 1.0, plan.xi, plan.r_cut)
    Mw = ewald.mobility_wave_dense(pos, L, 1.0, plan.xi, ewald.modes_cube(plan.M, L))
    Lc = np.linalg.cholesky(Mr + Mw)
    rng = np.random.default_rng(0)
    q = rng.standard_normal((20, 3 * N))
    qMq = np.einsum("ki,ij,kj->k", q, Mr + Mw, q)
    white = np.empty(n)
    proj = np.empty((n, 20))
    for s in range(n):
        ur, _, _ = pse.real_sample(pos, plan, SEED, s, op=op, lanczos_tol=1e-8)
        uw = pse.wave_sample_grid(pos, plan, SEED, s)
        u = (ur + uw).ravel()
        white[s] = np.sum(np.linalg.solve(Lc, u) ** 2) / (3 * N)
        proj[s] = q @ u
    assert abs(white.mean() - 1) < 4 * math.sqrt(2 / (3 * N * n))
    ratio = proj.var(axis=0) / qMq
    assert np.all(np.abs(ratio - 1) < 4 * math.sqrt(2 / n))


def test_real_rows_match_the_dense_real_mobility():
    """Row-at-a-time M_r v (for sampled particles of large systems) = rows of the
    dense eq. Mreal matrix (all images)."""
    pos, L = _hs(200, 0.3, 8)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    Mr = ewald.mobility_real_dense(pos, L, 1.0, 0.5, plan.r_cut)
    v = np.random.default_rng(3).standard_normal((200, 3))
    rows = np.array([0, 7, 50, 199])
    got = pse.real_rows(pos, plan, rows, v)
    ref = (Mr @ v.ravel()).reshape(200, 3)[rows]
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_coincident_particles_take_the_r_to_zero_limit():
    """Distinct particles at the same position (the degenerate overlap of App. B):
    the pair block is the r -> 0 limit F(0) I of App. A (F(0) = G(0), eq. self),
    so M_r is continuous as two particles merge; it stays positive
    semi-definite (two coincident spheres act as one, one zero mode); the
    sparse operator and the row-by-row product agree with the dense matrix."""
    L, xi = 20.0, 0.5
    plan = ewald.plan(L, 1.0, xi, 1e-3)
    base = np.array([[3.0, 4.0, 5.0], [3.0, 4.0, 5.0], [6.2, 4.1, 5.3], [10.0, 10.0, 10.0]])
    M0 = ewald.mobility_real_dense(base, L, 1.0, xi, plan.r_cut)
    for eps in (1e-3, 1e-5):
        moved = base.copy()
        moved[1, 0] += eps
        Me = ewald.mobility_real_dense(moved, L, 1.0, xi, plan.r_cut)
        assert np.abs(Me - M0).max() <= 10 * eps * np.abs(M0).max()
    # the pair block of the coincident particles is F(0) I = the self term
    s = rpy.self_real(xi, 1.0) / (6 * math.pi)
    assert np.allclose(M0[0:3, 3:6], s * np.eye(3), rtol=1e-12, atol=0)
    w = np.linalg.eigvalsh(M0)
    assert w.min() >= -1e-12 * w.max() and np.sum(np.abs(w) < 1e-10 * w.max()) == 3
    op = pse.RealOperator(base, plan)
    v = np.random.default_rng(3).standard_normal((4, 3))
    ref = (M0 @ v.ravel()).reshape(4, 3)
    assert np.allclose(op(v), ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(pse.real_rows(base, plan, np.arange(4), v), ref, rtol=1e-12, atol=1e-14)
