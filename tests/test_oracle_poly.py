"""Pins of the polydisperse oracle (the size-dependent shape factor of Sec. V)
against facts that do not depend on it: the k-integral definition of the pair
mobility, the paper's equal-radius case (App. A, eq. self), the
xi-independence of the Ewald sum, Hasimoto's periodic self-mobility, and
positivity of both parts."""
import math

import numpy as np
import pytest

from oracle import ewald, poly, pse, rpy


def _k_integral(r, ai, aj, weight_h=None, dps=20):
    """The pair mobility as the k-integral of eq. pairmobility with shape factors
    sinc(k ai) sinc(k aj) (weight 1, or 1 - H(k, xi) when weight_h = xi), by
    mpmath oscillatory quadrature: (F, G) in mobility units."""
    import mpmath as mp
    mp.mp.dps = dps
    r, ai, aj = mp.mpf(r), mp.mpf(ai), mp.mpf(aj)

    def s(k, a):
        return mp.sin(k * a) / (k * a) if k != 0 else mp.mpf(1)

    def w(k):
        if weight_h is None:
            return mp.mpf(1)
        q = k * k / (4 * mp.mpf(weight_h) ** 2)
        return 1 - (1 + q) * mp.exp(-q)

    def kF(k):
        x = k * r
        return mp.mpf(2) / 3 if x < mp.mpf("1e-6") else (x * mp.cos(x) + (x * x - 1) * mp.sin(x)) / x ** 3

    def kG(k):
        x = k * r
        return mp.mpf(1) / 3 if x < mp.mpf("1e-6") else (mp.sin(x) - x * mp.cos(x)) / x ** 3

    per = 2 * mp.pi / (r + ai + aj)
    Fi = mp.quadosc(lambda k: w(k) * s(k, ai) * s(k, aj) * kF(k), [0, mp.inf], period=per)
    Gi = mp.quadosc(lambda k: w(k) * s(k, ai) * s(k, aj) * kG(k), [0, mp.inf], period=per)
    return float(Fi / (2 * mp.pi ** 2)), float(Gi / mp.pi ** 2)


@pytest.mark.parametrize("r,ai,aj", [(3.0, 1.0, 0.5), (1.2, 1.0, 0.5), (0.3, 1.0, 0.5), (2.0, 1.0, 2.0),
                                     (5.0, 0.7, 1.9), (2.6, 1.3, 1.3)])
def test_free_space_tensor_is_the_k_integral(r, ai, aj):
    """Unequal-sphere RPY (far, overlapping and enclosed branches) = the
    shape-factor k-integral with weight 1."""
    F, G = poly.rpy_free(np.array([r]), ai, aj)
    Fi, Gi = _k_integral(r, ai, aj)
    assert abs(F[0] - Fi) < 1e-12 and abs(G[0] - Gi) < 1e-12


@pytest.mark.parametrize("r,ai,aj,xi", [(3.0, 1.0, 0.5, 0.5), (1.2, 1.0, 0.5, 0.7), (4.5, 0.6, 1.4, 0.4)])
def test_real_space_scalars_are_the_complementary_k_integral(r, ai, aj, xi):
    """F, G of M^r = the k-integral with weight 1 - H(k, xi) (eqs. int1/int2
    with the size-dependent shape factor)."""
    F, G = poly.fg(np.array([r]), xi, ai, aj)
    Fi, Gi = _k_integral(r, ai, aj, weight_h=xi)
    assert abs(F[0] - Fi) < 1e-11 and abs(G[0] - Gi) < 1e-11


def test_equal_radii_reduce_to_appendix_a():
    """a_i = a_j = a gives the App. A closed forms (times 1/(6 pi a)) and eq. self."""
    for a, xi in ((1.0, 0.5), (0.7, 0.8), (1.5, 0.3)):
        r = np.linspace(0.05, 6.0, 300) * a
        F, G = poly.fg(r, xi, a, a)
        Fc, Gc = rpy.fg(r, xi, a)
        assert np.abs(F * 6 * np.pi * a - Fc).max() < 1e-12
        assert np.abs(G * 6 * np.pi * a - Gc).max() < 1e-12
        assert abs(poly.self_real(xi, a) * 6 * np.pi * a - rpy.self_real(xi, a)) < 1e-13


def test_scalars_symmetric_in_the_radii():
    r = np.linspace(0.1, 5.0, 50)
    F1, G1 = poly.fg(r, 0.5, 0.6, 1.7)
    F2, G2 = poly.fg(r, 0.5, 1.7, 0.6)
    assert np.allclose(F1, F2, rtol=1e-13, atol=1e-17) and np.allclose(G1, G2, rtol=1e-13, atol=1e-17)


def _bidisperse(N, phi, seed, radii=(1.0, 0.5)):
    """Random non-overlapping spheres of two sizes (half each) in a periodic cube."""
    rng = np.random.default_rng(seed)
    species = np.arange(N) % 2
    rad = np.asarray(radii)[species]
    L = (np.sum(4 / 3 * np.pi * rad ** 3) / phi) ** (1 / 3)
    pos = np.zeros((N, 3))
    for i in range(N):
        while True:
            x = rng.uniform(0, L, 3)
            d = pos[:i] - x
            d -= L * np.round(d / L)
            if i == 0 or np.all(np.linalg.norm(d, axis=1) >= rad[:i] + rad[i]):
                pos[i] = x
                break
    return pos, species, rad, L


def test_ewald_sum_is_independent_of_xi():
    """M^r + M^w does not depend on the splitting (Sec. II A) for unequal spheres."""
    pos, species, rad, L = _bidisperse(16, 0.15, 1)
    # the truncation estimates of Sec. II C carry polynomial prefactors and
    # ignore the 2a shift of the real-space decay: truncate far below 1e-10
    # and keep xi a_max <= 0.9
    Ms = [poly.mobility_dense(pos, rad, L, xi, tol=1e-15)[0] for xi in (0.5, 0.7, 0.9)]
    assert np.abs(Ms[0] - Ms[1]).max() < 1e-10 * np.abs(Ms[0]).max()
    assert np.abs(Ms[0] - Ms[2]).max() < 1e-10 * np.abs(Ms[0]).max()


@pytest.mark.parametrize("a", [1.0, 0.5, 1.7])
def test_periodic_self_mobility_of_each_size(a):
    """One sphere of radius a in a box of side L: 6 pi a M_self = 1 - 2.837297 a/L + (4 pi/3)(a/L)^3 (Hasimoto)."""
    L = 40.0 * a
    M, _, _ = poly.mobility_dense(np.zeros((1, 3)), np.array([a]), L, 0.5 / a)
    ref = 1 - 2.837297 * a / L + 4 * np.pi / 3 * (a / L) ** 3
    assert abs(M[0, 0] * 6 * np.pi * a - ref) < 2e-6


def test_both_parts_positive_definite_with_overlaps():
    pos, species, rad, L = _bidisperse(14, 0.15, 2)
    pos[1] = pos[0] + np.array([0.9, 0.0, 0.0])   # overlapping unequal pair
    pos[3] = pos[2] + np.array([0.2, 0.1, 0.0])   # small sphere nearly inside the big one
    _, Mr, Mw = poly.mobility_dense(pos, rad, L, 0.7)
    assert np.linalg.eigvalsh(Mr).min() > 0 and np.linalg.eigvalsh(Mw).min() > -1e-14


def test_gridded_wave_covariance_matches_the_ewald_sum():
    """The gridded polydisperse wave sampler's exact covariance is the eq. Mwave
    sum with sinc(k a_i) sinc(k a_j), within the method's 20 tol of the
    smallest sphere's Stokes scale 1/(6 pi a_min)."""
    pos, species, rad, L = _bidisperse(12, 0.1, 3)
    for tol in (1e-3, 1e-4):
        p = poly.plan(L, (1.0, 0.5), 0.6, tol)
        C = poly.wave_covariance_grid(pos, species, (1.0, 0.5), p)
        kc = ewald.k_cut(0.6, 1e-12, 0.5)
        Mw = poly.mobility_wave_dense(pos, rad, L, 0.6, ewald.modes_sphere(kc, L))
        assert np.abs(C - Mw).max() * 6 * np.pi * 0.5 < 20 * tol


def test_lanczos_real_part_converges_to_the_dense_square_root():
    pos, species, rad, L = _bidisperse(60, 0.1, 4)
    p = poly.plan(L, (1.0, 0.5), 0.6, 1e-3)
    assert p.r_cut < L / 2
    Mr = poly.mobility_real_dense(pos, rad, L, 0.6, p.r_cut)
    lam, Q = np.linalg.eigh(Mr)
    z = pse.real_noise(60, 9, 2).ravel()
    exact = Q @ (np.sqrt(lam) * (Q.T @ z))
    x, j, _ = poly.real_sample(pos, rad, dataclasses_replace(p, tol=1e-12), 9, 2)
    assert np.linalg.norm(x.ravel() - exact) < 1e-9 * np.linalg.norm(exact)


def dataclasses_replace(p, **kw):
    import dataclasses
    return dataclasses.replace(p, **kw)
