"""Real-space RPY scalar functions of the positively split Ewald sum (FP64).

Conventions: viscosity eta = 1.  The dimensionless scalars F(r), G(r) are
those of Appendix A, i.e. 6*pi*eta*a * M^(r)_ij = F (I - rr) + G rr, so the
real-space pair block is ``(F (I - rr) + G rr) / (6 pi a)``.

Functions
---------
fg_closed(r, xi, a)      Appendix A, case 1 (r > 2a) and case 2 (r <= 2a)
self_real(xi, a)         Appendix A, case 3 (eq. self): F(r->0) = G(r->0)
fg(r, xi, a)             closed form, with the r -> 0 region evaluated as
                         free-space RPY minus the Gaussian-damped wave part
                         (the same integral, split as in eq. pairmobility)
fg_integral(r, xi, a)    eqs. int1 / int2 by direct quadrature (mpmath; pins)
rpy_free_fg(r, a)        eq. RPY_free_space written as (F, G) scalars
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

SQRT_PI = np.sqrt(np.pi)

# Below this separation (in units of a) the closed form of Appendix A loses
# more than ~5 digits to cancellation between its 1/(r^3 xi^4) terms; there
# fg() evaluates the same function through the decomposition
# F = F_RPY - F_wave (the k-integral of eq. pairmobility with weight H).
R_SMALL = 0.2


def fg_closed(r, xi, a=1.0):
    """F(r), G(r) of Appendix A (cases 1 and 2), dimensionless.

    6*pi*eta*a*M^(r) = F (I - rr) + G rr.  Case 1 (r > 2a) has f0 = g0 = 0;
    case 2 (r <= 2a) adds the overlap polynomials f0, g0.  All other
    coefficients are shared by the two cases.
    """
    r = np.asarray(r, dtype=np.float64)
    x2 = xi * xi
    x3 = x2 * xi
    x4 = x2 * x2
    r2 = r * r
    r3 = r2 * r
    e1 = np.exp(-r2 * x2)
    e2 = np.exp(-((r - 2 * a) ** 2) * x2)
    e3 = np.exp(-((r + 2 * a) ** 2) * x2)
    c4 = erfc(r * xi)
    c5 = erfc((r - 2 * a) * xi)
    c6 = erfc((r + 2 * a) * xi)

    f1 = (18 * r2 * x2 + 3) / (64 * SQRT_PI * a * r2 * x3)
    f2 = (2 * x2 * (2 * a - r) * (4 * a * a + 4 * a * r + 9 * r2) - 2 * a - 3 * r) / (
        128 * SQRT_PI * a * r3 * x3)
    f3 = (-2 * x2 * (2 * a + r) * (4 * a * a - 4 * a * r + 9 * r2) + 2 * a - 3 * r) / (
        128 * SQRT_PI * a * r3 * x3)
    f4 = (3 - 36 * r2 * r2 * x4) / (128 * a * r3 * x4)
    f5 = (4 * x4 * (r - 2 * a) ** 2 * (4 * a * a + 4 * a * r + 9 * r2) - 3) / (256 * a * r3 * x4)
    f6 = (4 * x4 * (2 * a + r) ** 2 * (4 * a * a - 4 * a * r + 9 * r2) - 3) / (256 * a * r3 * x4)

    g1 = (6 * r2 * x2 - 3) / (32 * SQRT_PI * a * r2 * x3)
    g2 = (-2 * x2 * (r - 2 * a) ** 2 * (2 * a + 3 * r) + 2 * a + 3 * r) / (64 * SQRT_PI * a * r3 * x3)
    g3 = (2 * x2 * (2 * a + r) ** 2 * (2 * a - 3 * r) - 2 * a + 3 * r) / (64 * SQRT_PI * a * r3 * x3)
    g4 = -3 * (4 * r2 * r2 * x4 + 1) / (64 * a * r3 * x4)
    g5 = (3 - 4 * x4 * (2 * a - r) ** 3 * (2 * a + 3 * r)) / (128 * a * r3 * x4)
    g6 = (3 - 4 * x4 * (2 * a - 3 * r) * (2 * a + r) ** 3) / (128 * a * r3 * x4)

    overlap = r <= 2 * a
    f0 = np.where(overlap, -((r - 2 * a) ** 2) * (4 * a * a + 4 * a * r + 9 * r2) / (32 * a * r3), 0.0)
    g0 = np.where(overlap, (2 * a - r) ** 3 * (2 * a + 3 * r) / (16 * a * r3), 0.0)

    F = f0 + f1 * e1 + f2 * e2 + f3 * e3 + f4 * c4 + f5 * c5 + f6 * c6
    G = g0 + g1 * e1 + g2 * e2 + g3 * e3 + g4 * c4 + g5 * c5 + g6 * c6
    return F, G


def self_real(xi, a=1.0):
    """Appendix A, case 3 (eq. self): 6 pi a M^(r)_ii = s I, returns s."""
    return (1.0 - np.exp(-4 * a * a * xi * xi) + 4 * SQRT_PI * a * xi * erfc(2 * a * xi)) / (
        4 * SQRT_PI * xi * a)


def rpy_free_fg(r, a=1.0):
    """eq. RPY_free_space as scalars: 6 pi a M_RPY = F (I - rr) + G rr.

    r > 2a : A I + B rr with A = 3a/4r + a^3/2r^3, B = 3a/4r - 3a^3/2r^3
    r <= 2a: A = 1 - 9r/32a, B = 3r/32a.  Then F = A, G = A + B.
    """
    r = np.asarray(r, dtype=np.float64)
    far = r > 2 * a
    rs = np.where(far, r, 1.0)
    A_far = 0.75 * a / rs + 0.5 * a ** 3 / rs ** 3
    B_far = 0.75 * a / rs - 1.5 * a ** 3 / rs ** 3
    A_near = 1.0 - 9.0 * r / (32.0 * a)
    B_near = 3.0 * r / (32.0 * a)
    A = np.where(far, A_far, A_near)
    B = np.where(far, B_far, B_near)
    return A, A + B


def _kernels(x):
    """Radial kernels of eqs. int1/int2 at x = k r, stable as x -> 0.

    kF(x) = (x cos x + (x^2 - 1) sin x) / x^3   -> 2/3 - 2x^2/15 + x^4/140
    kG(x) = (sin x - x cos x) / x^3             -> 1/3 - x^2/30 + x^4/840
    """
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 2e-2
    xs = np.where(small, 1.0, x)
    kF = (xs * np.cos(xs) + (xs * xs - 1) * np.sin(xs)) / xs ** 3
    kG = (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    x2 = x * x
    kF_s = 2.0 / 3.0 - 2.0 * x2 / 15.0 + x2 * x2 / 140.0
    kG_s = 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0
    return np.where(small, kF_s, kF), np.where(small, kG_s, kG)


def _H(k, xi):
    """Hasimoto splitting function H(k, xi) = (1 + k^2/4xi^2) exp(-k^2/4xi^2)."""
    q = k * k / (4 * xi * xi)
    return (1 + q) * np.exp(-q)


def fg_wave_free(r, xi, a=1.0, nq=400):
    """Free-space (continuous-k) wave part of eq. pairmobility, as F, G scalars.

    The integrals of eqs. int1/int2 with weight H(k, xi) instead of 1 - H,
    times 6 pi a.  H decays like a Gaussian, so Gauss-Legendre quadrature on
    k in [0, 16 xi] is exact to rounding.  Used only for r < R_SMALL, where
    F = F_RPY - F_wave avoids the cancellation of the closed form.
    """
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    kmax = 16.0 * xi
    t, w = np.polynomial.legendre.leggauss(nq)
    k = 0.5 * kmax * (t + 1.0)
    w = 0.5 * kmax * w
    ka = k * a
    sinc2 = np.where(ka > 0, (np.sin(ka) / np.where(ka > 0, ka, 1.0)) ** 2, 1.0)
    base = _H(k, xi) * sinc2 * w
    kF, kG = _kernels(np.outer(r, k))
    F = (kF * base).sum(axis=1) / (2 * np.pi ** 2) * 6 * np.pi * a
    G = (kG * base).sum(axis=1) / (np.pi ** 2) * 6 * np.pi * a
    return F, G


def fg(r, xi, a=1.0):
    """F(r), G(r) for any r >= 0 (dimensionless, Appendix A normalisation).

    r >= R_SMALL*a : Appendix A closed form (cases 1/2).
    0 < r < R_SMALL*a: free-space RPY (eq. RPY_free_space, overlap branch)
        minus the free-space wave part; this is the same function because
        the full k-integral of eq. pairmobility is the free-space RPY tensor
        and eqs. int1/int2 carry the complementary weight 1 - H.
    r == 0: eq. self.
    """
    r = np.asarray(r, dtype=np.float64)
    scalar = r.ndim == 0
    r = np.atleast_1d(r)
    F = np.empty_like(r)
    G = np.empty_like(r)
    big = r >= R_SMALL * a
    if big.any():
        F[big], G[big] = fg_closed(r[big], xi, a)
    small = (~big) & (r > 0)
    if small.any():
        Fr, Gr = rpy_free_fg(r[small], a)
        Fw, Gw = fg_wave_free(r[small], xi, a)
        F[small] = Fr - Fw
        G[small] = Gr - Gw
    zero = r == 0
    if zero.any():
        F[zero] = self_real(xi, a)
        G[zero] = self_real(xi, a)
    if scalar:
        return F[0], G[0]
    return F, G


def fg_integral(r, xi, a=1.0, dps=30):
    """eqs. int1 / int2 evaluated by mpmath quadrature, times 6 pi a.

    F = (1/2pi^2) int_0^inf (1 - H) sinc^2(ka) kF(kr) dk
    G = (1/pi^2)  int_0^inf (1 - H) sinc^2(ka) kG(kr) dk
    The oscillatory, algebraically decaying integrand is integrated panel by
    panel between multiples of pi/(r + 2a) and summed with mpmath's
    nsum-style Richardson extrapolation (quadosc).  Slow: pins only.
    """
    import mpmath as mp
    mp.mp.dps = dps
    r = mp.mpf(r)
    xi = mp.mpf(xi)
    a = mp.mpf(a)

    def Hm(k):
        q = k * k / (4 * xi * xi)
        return (1 + q) * mp.exp(-q)

    def sinc2(k):
        return (mp.sin(k * a) / (k * a)) ** 2 if k != 0 else mp.mpf(1)

    def kF(k):
        x = k * r
        if x < mp.mpf('1e-6'):
            return mp.mpf(2) / 3
        return (x * mp.cos(x) + (x * x - 1) * mp.sin(x)) / x ** 3

    def kG(k):
        x = k * r
        if x < mp.mpf('1e-6'):
            return mp.mpf(1) / 3
        return (mp.sin(x) - x * mp.cos(x)) / x ** 3

    period = 2 * mp.pi / (r + 2 * a)
    Fi = mp.quadosc(lambda k: (1 - Hm(k)) * sinc2(k) * kF(k), [0, mp.inf], period=period)
    Gi = mp.quadosc(lambda k: (1 - Hm(k)) * sinc2(k) * kG(k), [0, mp.inf], period=period)
    F = Fi / (2 * mp.pi ** 2) * 6 * mp.pi * a
    G = Gi / (mp.pi ** 2) * 6 * mp.pi * a
    return float(F), float(G)
