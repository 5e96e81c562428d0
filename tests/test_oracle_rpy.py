"""Pins of the oracle's real-space RPY scalars (Appendix A) to facts fixed by the paper."""
import math
import os

import numpy as np
import pytest

from oracle import rpy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _quad_cases():
    rows = []
    with open(os.path.join(GOLDEN, "fg_quadrature.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            r, xi, a, F, G = map(float, line.split())
            rows.append((r, xi, a, F, G))
    return rows


@pytest.mark.parametrize("r,xi,a,F,G", _quad_cases())
def test_closed_form_matches_integrals(r, xi, a, F, G):
    """Appendix A closed forms = direct quadrature of eqs. int1/int2 (stored by the golden script)."""
    Fc, Gc = rpy.fg_closed(r, xi, a)
    assert abs(Fc - F) < 2e-12 and abs(Gc - G) < 2e-12


def test_quadrature_live_one_point():
    """One live mpmath quadrature so the golden file cannot silently drift from eqs. int1/int2."""
    pytest.importorskip("mpmath")
    F, G = rpy.fg_integral(1.7, 0.45, 1.0, dps=20)
    Fc, Gc = rpy.fg_closed(1.7, 0.45, 1.0)
    assert abs(F - Fc) < 1e-10 and abs(G - Gc) < 1e-10


@pytest.mark.parametrize("xi,a", [(0.5, 1.0), (0.3, 1.0), (0.7, 1.4)])
def test_continuous_at_contact(xi, a):
    """Cases 1 and 2 of Appendix A meet at r = 2a."""
    lo = rpy.fg_closed(2 * a * (1 - 1e-10), xi, a)
    hi = rpy.fg_closed(2 * a * (1 + 1e-10), xi, a)
    assert abs(lo[0] - hi[0]) < 1e-8 and abs(lo[1] - hi[1]) < 1e-8


@pytest.mark.parametrize("xi,a", [(0.5, 1.0), (0.3, 1.0), (1.0, 1.0), (0.6, 2.0)])
def test_r_to_zero_is_self_term(xi, a):
    """F(r->0) = G(r->0) = eq. self (Appendix A case 3)."""
    s = rpy.self_real(xi, a)
    F, G = rpy.fg(1e-7 * a, xi, a)
    assert abs(F - s) < 1e-6 and abs(G - s) < 1e-6
    F0, G0 = rpy.fg(0.0, xi, a)
    assert F0 == s and G0 == s


@pytest.mark.parametrize("r", [0.05, 0.15, 0.19, 0.21, 0.3])
def test_small_r_branch_agrees_with_closed_form(r):
    """The r < R_SMALL evaluation (RPY minus Gaussian wave part) is the same function."""
    xi = 0.5
    Fc, Gc = rpy.fg_closed(r, xi)
    Fr, Gr = rpy.rpy_free_fg(r)
    Fw, Gw = rpy.fg_wave_free(np.array([r]), xi)
    tol = 1e-9 if r > 0.1 else 1e-7  # closed form itself loses digits below 0.1a
    assert abs(Fc - (Fr - Fw[0])) < tol and abs(Gc - (Gr - Gw[0])) < tol


@pytest.mark.parametrize("r", [0.7, 1.5, 2.0, 2.5, 4.0, 7.0])
def test_xi_to_zero_is_free_space_rpy(r):
    """xi -> 0: M^(r) -> free-space RPY (eq. RPY_free_space) minus the k->0 wave
    part (1/(2 pi^2))(2/3) int H dk * 6 pi a = 3 xi a / sqrt(pi) on both F and G.
    xi = 3e-3 keeps the O(xi^2) remainder below 1e-6 while the closed form's
    own 1/xi^4 cancellation stays below it too; the bound
    allows the O(r^2 xi^3) next term."""
    xi = 3e-3
    F, G = rpy.fg(r, xi)
    Fr, Gr = rpy.rpy_free_fg(r)
    shift = 3 * xi / math.sqrt(math.pi)
    # next term of the k-expansion is O(r^2 xi^3)
    bound = 3e-7 + 5e-8 * r * r
    assert abs(F - (Fr - shift)) < bound
    assert abs(G - (Gr - shift)) < bound


def test_self_term_limits():
    """eq. self: xi -> 0 gives the Stokes drag 1 (minus 3 xi a/sqrt pi); xi -> inf gives 0."""
    assert abs(rpy.self_real(1e-4) - (1 - 3e-4 / math.sqrt(math.pi))) < 1e-7
    assert rpy.self_real(50.0) < 1e-2


def test_free_rpy_branches_meet():
    """eq. RPY_free_space is continuous (and C^1) at r = 2a."""
    F1, G1 = rpy.rpy_free_fg(2 - 1e-9)
    F2, G2 = rpy.rpy_free_fg(2 + 1e-9)
    assert abs(F1 - F2) < 1e-8 and abs(G1 - G2) < 1e-8
    assert abs(F1 - 7 / 16) < 1e-8 and abs(G1 - 5 / 8) < 1e-8


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_real_part_decays_at_cutoff(tol):
    """eps_R ~ exp(-xi^2 r_cut^2): the scalars are O(tol) at r_cut."""
    from oracle import ewald
    xi = 0.5
    rc = ewald.r_cut(xi, tol)
    F, G = rpy.fg(rc, xi)
    assert abs(F) < 5 * tol and abs(G) < 5 * tol
    F2, G2 = rpy.fg(2 * rc, xi)
    assert abs(F2) < tol ** 3 and abs(G2) < tol ** 3
