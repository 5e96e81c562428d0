"""Pins of the oracle's spreading, deterministic M F and grid-noise wave sample
(Sec. II B 2, Sec. III) against facts that do not depend on those functions."""
import math

import numpy as np
import pytest

from oracle import ewald, pse


def _hs(N, phi, seed):
    from paper_1611_09322_gb300 import workloads
    p, L, _ = workloads.hard_spheres(N, phi, seed)
    return p.astype(np.float64), L


def test_spreading_is_the_adjoint_of_interpolation():
    """S^dagger = h^3 S^T (Sec. II B 2): <h^3 S F, v> = <F, S^dagger v> for any F, v."""
    pos, L = _hs(40, 0.1, 5)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    rng = np.random.default_rng(1)
    F = rng.standard_normal((40, 3))
    v = rng.standard_normal((3, plan.M, plan.M, plan.M))
    lhs = plan.h ** 3 * np.sum(pse.spread(F, pos, plan) * v)
    rhs = np.sum(F * pse.interpolate(v, pos, plan))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300) * 1e2


def test_spreading_conserves_force_within_the_quadrature_bound():
    """The P-point truncated Gaussian sums to 1 on the grid up to the per-axis error
    exp(-pi^2 P^2 / 2m^2) + erfc(m / sqrt 2) <= tol of Sec. II C, so h^3 sum_g S F = sum F
    to 3 tol per particle, for every position relative to the grid."""
    rng = np.random.default_rng(2)
    for tol in (1e-3, 1e-5):
        L = 20.0
        plan = ewald.plan(L, 1.0, 0.5, tol)
        pos = rng.uniform(0, L, (50, 3))
        for i in range(5):
            F = np.zeros((50, 3))
            F[i] = [1.0, -2.0, 0.5]
            tot = pse.spread(F, pos, plan).reshape(3, -1).sum(axis=1) * plan.h ** 3
            assert np.abs(tot - F[i]).max() <= 3 * tol * np.abs(F[i]).max()


def test_wave_apply_matrix_is_the_gridded_covariance():
    """The deterministic gridded operator and the gridded sampler use the same
    mode factor B(k) = V wave_scale(k)^2: the matrix of F -> M_w F equals the
    exact covariance of the wave sample mode by mode (pinned to eq. Mwave in
    test_oracle_pse), for odd and even grids."""
    pos, L = _hs(12, 0.1, 7)
    for M in (None, 10):
        plan = ewald.plan(L, 1.0, 0.5, 1e-3, M=M)
        N = pos.shape[0]
        A = np.zeros((3 * N, 3 * N))
        for c in range(3 * N):
            F = np.zeros(3 * N)
            F[c] = 1.0
            A[:, c] = pse.wave_apply_grid(F.reshape(N, 3), pos, plan).ravel()
        C = pse.wave_covariance_grid(pos, plan)
        assert np.abs(A - C).max() <= 1e-12 * np.abs(C).max()
        assert np.abs(A - A.T).max() <= 1e-12 * np.abs(C).max()


def test_wave_apply_matches_the_ewald_sum():
    """M_w F from the grid vs the direct k-sum of eq. Mwave (converged): the error
    relative to the Stokes velocity scale stays O(tol) and falls with tol."""
    pos, L = _hs(64, 0.1, 3)
    Mw = ewald.mobility_wave_dense(pos, L, 1.0, 0.5, ewald.modes_sphere(ewald.k_cut(0.5, 1e-14), L))
    F = np.random.default_rng(4).standard_normal((64, 3))
    ref = (Mw @ F.ravel()).reshape(64, 3)
    errs = []
    for tol in (1e-3, 1e-4, 1e-5):
        plan = ewald.plan(L, 1.0, 0.5, tol)
        u = pse.wave_apply_grid(F, pos, plan)
        err = np.abs(u - ref).max() * 6 * math.pi / np.abs(F).max()
        assert err < 20 * tol
        errs.append(err)
    assert errs[0] > errs[1] > errs[2] and errs[0] > 20 * errs[2]


def test_mobility_apply_matches_dense_ewald_rpy():
    """M F = M_r F + M_w F vs the dense Ewald-summed RPY mobility (all images,
    tol 1e-12): O(tol) relative to the Stokes scale, at two tolerances."""
    pos, L = _hs(64, 0.1, 3)
    Mfull, _, _ = ewald.mobility_dense(pos, L, 1.0, 0.5, tol=1e-12)
    F = np.random.default_rng(5).standard_normal((64, 3))
    ref = (Mfull @ F.ravel()).reshape(64, 3)
    for tol in (1e-3, 1e-5):
        plan = ewald.plan(L, 1.0, 0.5, tol)
        assert plan.r_cut < L / 2
        u = pse.mobility_apply(F, pos, plan)
        assert np.abs(u - ref).max() * 6 * math.pi / np.abs(F).max() < 20 * tol


@pytest.mark.parametrize("M", [8, 9])
def test_grid_noise_sample_has_the_kspace_covariance(M):
    """White grid noise -> DFT -> the k-space scaling gives the same covariance as
    drawing dW2 in k-space: the linear map W -> u has A A^T equal to the exact
    covariance of the k-space sampler (mode by mode), for even and odd grids."""
    pos, L = _hs(6, 0.1, 9)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3, M=M)
    assert plan.eta <= 1.0
    n = 3 * M ** 3
    A = np.zeros((3 * pos.shape[0], n))
    for c in range(n):
        W = np.zeros(n)
        W[c] = 1.0
        A[:, c] = pse.wave_sample_gridnoise(pos, plan, 0, 0, W=W.reshape(3, M, M, M)).ravel()
    C = pse.wave_covariance_grid(pos, plan)
    assert np.abs(A @ A.T - C).max() <= 1e-11 * np.abs(C).max()


def test_grid_noise_is_standard_normal_and_uncorrelated():
    W = pse.grid_noise(24, 11, 3)
    n = W[0].size
    assert abs(W.mean()) < 4 / math.sqrt(3 * n)
    assert abs(W.var() - 1) < 4 * math.sqrt(2 / (3 * n))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        assert abs(np.mean(W[a] * W[b])) < 4 / math.sqrt(n)
    assert not np.array_equal(W, pse.grid_noise(24, 11, 4))


def test_sample_with_forces_without_noise_is_the_mobility_product():
    pos, L = _hs(80, 0.2, 13)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    F = np.random.default_rng(6).standard_normal((80, 3))
    out, j = pse.sample_with_forces(pos, F, plan, 1, 2, c_det=2.5, c_noise=0.0)
    assert j == 0
    assert np.allclose(out, 2.5 * pse.mobility_apply(F, pos, plan), rtol=1e-13, atol=1e-15)


def test_repulsion_forces_pair_and_momentum():
    """Two overlapping spheres: equal and opposite forces along the line of
    centres, magnitude k (2a - r); a many-body packing: sum of forces 0, and a
    pair just outside contact feels nothing; across the periodic boundary."""
    L = 20.0
    pos = np.array([[0.5, 5.0, 5.0], [19.7, 5.3, 5.0]])  # separated by 0.8, 0.3 through the boundary
    F = pse.repulsion_forces(pos, L, 1.0, 10.0)
    d = np.array([0.5 - (19.7 - 20.0), 5.0 - 5.3, 0.0])
    r = np.linalg.norm(d)
    assert np.allclose(F[0], 10.0 * (2 - r) * d / r, rtol=1e-14)
    assert np.allclose(F[1], -F[0], rtol=1e-14)
    far = pse.repulsion_forces(np.array([[1.0, 1.0, 1.0], [3.0001, 1.0, 1.0]]), L, 1.0, 10.0)
    assert np.all(far == 0)
    rng = np.random.default_rng(3)
    many = rng.uniform(0, L, (300, 3))
    Fm = pse.repulsion_forces(many, L, 1.0, 5.0)
    assert np.abs(Fm.sum(axis=0)).max() < 1e-10 * np.abs(Fm).max()


def test_bd_step_without_noise_is_the_mobility_product():
    pos, L = _hs(200, 0.3, 21)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    new, dx, j = pse.bd_step(pos, plan, 1, 2, dt=1e-3, kT=0.0, k_rep=100.0)
    F = pse.repulsion_forces(pos, L, 1.0, 100.0)
    assert j == 0
    assert np.allclose(dx, 1e-3 * pse.mobility_apply(F, pos, plan), rtol=1e-12, atol=1e-16)
    assert np.allclose(new, np.mod(pos + dx, L))


def test_full_mobility_lanczos_converges_to_the_square_root_of_the_gridded_mobility():
    """The full-mobility Lanczos of Sec. IV: with a tight stop rule its result
    is A^{1/2} z for the matrix A of the M F product it applies (built column
    by column from unit forces, symmetric and positive definite), computed by
    a dense eigendecomposition; and A itself is the dense Ewald-summed RPY
    mobility to within the method's tolerance (20 tol of the Stokes scale
    1/(6 pi a), eq. Mwave + eq. Mreal)."""
    N = 40
    pos, L = _hs(N, 0.1, 21)
    plan = ewald.plan(L, 1.0, 0.5, 1e-3)
    A = np.stack([pse.mobility_apply(e.reshape(N, 3), pos, plan).ravel() for e in np.eye(3 * N)], axis=1)
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    lam, Q = np.linalg.eigh(0.5 * (A + A.T))
    assert lam.min() > 0
    z = pse.real_noise(N, 3, 4).ravel()
    exact = Q @ (np.sqrt(lam) * (Q.T @ z))
    x, j, _ = pse.full_sample(pos, plan, 3, 4, lanczos_tol=1e-11)
    assert np.linalg.norm(x.ravel() - exact) < 1e-8 * np.linalg.norm(exact)
    x4, j4, _ = pse.full_sample(pos, plan, 3, 4, n_iter=4)
    assert j4 == 4 and np.linalg.norm(x4.ravel() - exact) > 1e-6 * np.linalg.norm(exact)
    Md, _, _ = ewald.mobility_dense(pos, L, 1.0, 0.5, tol=1e-12)
    assert np.abs(A - Md).max() * 6 * math.pi < 20 * 1e-3
