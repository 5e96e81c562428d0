"""Pins of the oracle's Ewald-split mobility (Sec. II A, App. B) and parameters (Sec. II C)."""
import math
import os

import numpy as np
import pytest

from oracle import ewald, rpy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hasimoto_C():
    with open(os.path.join(GOLDEN, "hasimoto.txt")) as f:
        for line in f:
            if line.startswith("C "):
                return float(line.split()[1])


@pytest.mark.parametrize("L,a,xi", [(10.0, 1.0, 0.4), (20.0, 1.0, 0.7), (40.0, 1.0, 0.5), (30.0, 1.5, 0.35)])
def test_single_particle_hasimoto(L, a, xi):
    """Periodic self-mobility = 1 - C a/L + (4pi/3)(a/L)^3 + O((a/L)^6) (Hasimoto)."""
    C = _hasimoto_C()
    M, _, _ = ewald.mobility_dense(np.zeros((1, 3)), L, a, xi, tol=1e-13)
    val = M[0, 0] * 6 * math.pi * a
    expect = 1 - C * a / L + 4 * math.pi / 3 * (a / L) ** 3
    assert abs(val - expect) < 2e-9 + 2 * (a / L) ** 6
    assert abs(M[0, 1]) < 1e-12 and abs(M[0, 0] - M[1, 1]) < 1e-12


def _config(seed, N=10, L=9.0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0, L, (N, 3))
    p[1] = p[0] + np.array([0.6, 0.2, -0.1])  # an overlapping pair (r < 2a)
    p[2] = p[0] + np.array([2.0, 0.0, 0.0])  # exact contact
    return np.mod(p, L), L


def test_split_is_xi_independent():
    """M^(r)(xi) + M^(w)(xi) is the same periodic RPY mobility for every xi (Sec. II A)."""
    p, L = _config(1)
    # the truncation estimates of Sec. II C carry polynomial prefactors: truncate far below 1e-10
    Ms = [ewald.mobility_dense(p, L, 1.0, xi, tol=1e-15)[0] for xi in (0.3, 0.5, 0.8)]
    scale = np.abs(Ms[0]).max()
    assert np.abs(Ms[0] - Ms[1]).max() < 1e-10 * scale
    assert np.abs(Ms[0] - Ms[2]).max() < 1e-10 * scale


@pytest.mark.parametrize("xi", [0.3, 0.5, 1.0])
def test_both_parts_spd_with_overlaps(xi):
    """App. B: M^(r) and M^(w) are each symmetric positive (semi)definite, overlaps included."""
    p, L = _config(2)
    _, Mr, Mw = ewald.mobility_dense(p, L, 1.0, xi, tol=1e-12)
    for M in (Mr, Mw):
        assert np.abs(M - M.T).max() < 1e-13
    assert np.linalg.eigvalsh(Mr).min() > 0
    assert np.linalg.eigvalsh(Mw).min() > -1e-13


def test_beenakker_splitting_violates_bound():
    """Sec. II A: Hasimoto's H stays in [0, 1]; Beenakker's H_B exceeds 1."""
    k = np.linspace(0, 20, 2001)
    xi = 0.5
    Hh = ewald.H(k, xi)
    q = k * k / (4 * xi * xi)
    HB = (1 + q + 2 * q * q) * np.exp(-q)
    assert Hh.min() >= 0 and Hh.max() <= 1 + 1e-15
    assert HB.max() > 1.0


def test_pair_tends_to_free_rpy():
    """A pair in a large box: M_12 - M_RPY(r) equals the self shift M_11 - 1/(6 pi a)
    to O(r^2/L^3) (the periodic correction is uniform at leading order)."""
    L = 80.0
    for r in (1.5, 3.0, 5.0):
        p = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        M, _, _ = ewald.mobility_dense(p, L, 1.0, 0.5, tol=1e-12)
        F, G = rpy.rpy_free_fg(r)
        rpy_blk = np.diag([G, F, F]) / (6 * math.pi)
        shift = M[0, 0] - 1 / (6 * math.pi)
        diff = M[0:3, 3:6] - rpy_blk
        assert np.abs(diff - shift * np.eye(3)).max() < 3 * r * r / L ** 3


def test_parameters_match_bounds():
    """Sec. II C bounds: r_cut, k_cut (eq. errbound), P and m (eps_q), grid resolves k_cut."""
    xi, tol = 0.5, 1e-3
    p = ewald.plan(34.7, 1.0, xi, tol)
    assert abs(math.exp(-(xi * p.r_cut) ** 2) - tol) < 1e-15
    assert ewald.kcut_bound(p.k_cut, xi) <= tol < ewald.kcut_bound(p.k_cut * 0.999, xi)
    assert p.P == 5 and ewald.quadrature_error(p.P, p.m) <= tol
    assert ewald.quadrature_error(4, ewald.best_m(4)) > tol
    for mm in (p.m * 0.95, p.m * 1.05):
        assert ewald.quadrature_error(5, mm) > ewald.quadrature_error(5, p.m)
    assert math.pi * p.M / p.L >= p.k_cut and p.M == 25
    assert 0 < p.eta <= 1
    p5 = ewald.plan(382.3, 1.0, xi, 1e-5)
    assert p5.P == 8 and p5.M == 375


def test_kcut_bound_is_an_upper_bound():
    """eq. errbound: the closed form bounds (2a/pi) int_kc^inf sinc^2 H dk from above."""
    from scipy.integrate import quad
    xi, a = 0.5, 1.0
    for kc in (1.5, 2.24, 3.0):
        s2 = lambda k: (math.sin(k * a) / (k * a)) ** 2 * ewald.H(k, xi)
        exact = 2 * a / math.pi * quad(s2, kc, 60, limit=400)[0]
        assert exact <= ewald.kcut_bound(kc, xi, a)
        assert exact > 0.01 * ewald.kcut_bound(kc, xi, a)  # and not vacuous


def test_modes_cube_excludes_zero_and_nyquist():
    k = ewald.modes_cube(8, 2 * math.pi)
    n = np.rint(k).astype(int)
    assert not np.any(np.all(n == 0, axis=1))
    assert np.abs(n).max() == 3 and k.shape[0] == 7 ** 3 - 1
    k = ewald.modes_cube(7, 2 * math.pi)
    assert k.shape[0] == 7 ** 3 - 1
