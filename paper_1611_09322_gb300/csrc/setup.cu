// Host-side FP64 setup: Sec. II C parameter planning and the tabulated
// real-space scalars F(r), G(r) of Appendix A.
#include <math.h>
#include <string.h>

#include <vector>

#include "pse_internal.cuh"

namespace pse {

static const double kPi = 3.14159265358979323846;

static void fg_closed(double r, double xi, double a, double *F, double *G) { fg_closed_hd(r, xi, a, F, G); }

// Appendix A, case 3 (eq. self), dimensionless.
double self_real(double xi, double a) {
    return (1.0 - exp(-4 * a * a * xi * xi) + 4 * sqrt(kPi) * a * xi * erfc(2 * a * xi)) / (4 * sqrt(kPi) * xi * a);
}

// Near r = 0 the closed form cancels catastrophically (terms ~ 1/(r^3 xi^4)).
// There F = F_RPY - F_w: the free-space RPY tensor (overlap branch of
// eq. RPY_free_space) minus the k-integral of eqs. int1/int2 taken with the
// weight H instead of 1 - H.  H decays like a Gaussian, so composite Simpson
// on [0, 16 xi] converges to rounding.
static void fg_small(double r, double xi, double a, double *F, double *G) {
    const int n = 8192;  // even
    const double kmax = 16.0 * xi, hk = kmax / n;
    double sF = 0.0, sG = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double k = i * hk;
        const double q = k * k / (4 * xi * xi);
        const double Hk = (1 + q) * exp(-q);
        const double ka = k * a;
        const double s2 = (ka > 0) ? (sin(ka) / ka) * (sin(ka) / ka) : 1.0;
        const double x = k * r;
        double kF, kG;
        if (x < 1e-2) {
            const double x2 = x * x;
            kF = 2.0 / 3.0 - 2.0 * x2 / 15.0 + x2 * x2 / 140.0;
            kG = 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0;
        } else {
            kF = (x * cos(x) + (x * x - 1) * sin(x)) / (x * x * x);
            kG = (sin(x) - x * cos(x)) / (x * x * x);
        }
        const double wgt = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        sF += wgt * Hk * s2 * kF;
        sG += wgt * Hk * s2 * kG;
    }
    sF *= hk / 3.0;
    sG *= hk / 3.0;
    const double Fw = sF / (2 * kPi * kPi) * 6 * kPi * a;
    const double Gw = sG / (kPi * kPi) * 6 * kPi * a;
    const double A = 1.0 - 9.0 * r / (32.0 * a), B = 3.0 * r / (32.0 * a);
    *F = A - Fw;
    *G = A + B - Gw;
}

// F, G at one separation (the same branches as the tables below).
void fg_at(double r, double xi, double a, double *F, double *G) {
    if (r <= 0.0) {
        *F = *G = self_real(xi, a);
    } else if (r < 0.2 * a) {
        fg_small(r, xi, a, F, G);
    } else {
        fg_closed(r, xi, a, F, G);
    }
}

void build_fg_table(double r_cut, double xi, double a, int n, double *F, double *G) {
    const double dr = r_cut / (n - 1);
    for (int i = 0; i < n; ++i) {
        const double r = i * dr;
        if (i == 0) {
            F[i] = G[i] = self_real(xi, a);
        } else if (r < 0.2 * a) {
            fg_small(r, xi, a, &F[i], &G[i]);
        } else {
            fg_closed(r, xi, a, &F[i], &G[i]);
        }
    }
}

// ------------------------------------------------------------------ polydisperse pairs
// The size-dependent shape factor of Sec. V: spheres of radii ai, aj carry
// sinc(k ai) sinc(k aj) where equal spheres carry sinc^2(k a).  With weight 1
// the k-integral of eq. pairmobility is the free-space RPY tensor of two
// unequal spheres (Zuk, Wajnryb, Mizerski & Szymczak, J. Fluid Mech. 741,
// R5, 2014); the real-space part (weight 1 - H) is that tensor minus the
// H-weighted integral, which decays like a Gaussian in k and is evaluated by
// Gauss-Legendre quadrature on [0, 16 xi].  Scalars in mobility units:
// block = F (I - rr) + G rr.

// Free-space RPY of spheres ai, aj at separation r > 0 as (F, G).
static void rpy_pair(double r, double ai, double aj, double *F, double *G) {
    const double s2 = ai * ai + aj * aj, d = ai - aj;
    double A, B;
    if (r > ai + aj) {
        A = (1 + s2 / (3 * r * r)) / (8 * kPi * r);
        B = (1 - s2 / (r * r)) / (8 * kPi * r);
    } else if (r > fabs(d)) {
        const double t = d * d + 3 * r * r, u = d * d - r * r;
        A = (16 * r * r * r * (ai + aj) - t * t) / (32 * r * r * r) / (6 * kPi * ai * aj);
        B = 3 * u * u / (32 * r * r * r) / (6 * kPi * ai * aj);
    } else {
        A = 1.0 / (6 * kPi * (ai > aj ? ai : aj));
        B = 0.0;
    }
    *F = A;
    *G = A + B;
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on P_n from
// the usual Chebyshev-like initial guesses.
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
    }
}

// Quadrature of the H-weighted integral for one (xi, ai, aj).
struct PolyQuad {
    std::vector<double> k, base;
    PolyQuad(double xi, double ai, double aj) {
        const int nq = 400;
        std::vector<double> t(nq), wq(nq);
        gauss_legendre(nq, t.data(), wq.data());
        k.resize(nq);
        base.resize(nq);
        const double kmax = 16.0 * xi;
        for (int q = 0; q < nq; ++q) {
            k[q] = 0.5 * kmax * (t[q] + 1.0);
            const double kk = k[q], h = kk * kk / (4 * xi * xi);
            const double si = kk * ai > 0 ? sin(kk * ai) / (kk * ai) : 1.0;
            const double sj = kk * aj > 0 ? sin(kk * aj) / (kk * aj) : 1.0;
            base[q] = 0.5 * kmax * wq[q] * (1 + h) * exp(-h) * si * sj;
        }
    }
    void at(double r, double ai, double aj, double *F, double *G) const {
        double sF = 0.0, sG = 0.0;
        for (size_t q = 0; q < k.size(); ++q) {
            const double x = k[q] * r;
            double kF, kG;
            if (x < 2e-2) {
                const double x2 = x * x;
                kF = 2.0 / 3.0 - 2.0 * x2 / 15.0 + x2 * x2 / 140.0;
                kG = 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0;
            } else {
                kF = (x * cos(x) + (x * x - 1) * sin(x)) / (x * x * x);
                kG = (sin(x) - x * cos(x)) / (x * x * x);
            }
            sF += base[q] * kF;
            sG += base[q] * kG;
        }
        double Fr, Gr;
        if (r > 0) {
            rpy_pair(r, ai, aj, &Fr, &Gr);
        } else {  // r -> 0: 1/(6 pi max(ai, aj)) I
            Fr = Gr = 1.0 / (6 * kPi * (ai > aj ? ai : aj));
        }
        *F = Fr - sF / (2 * kPi * kPi);
        *G = Gr - sG / (kPi * kPi);
    }
};

void build_fg_table_poly(double r_cut, double xi, double ai, double aj, int n, double *F, double *G) {
    const PolyQuad pq(xi, ai, aj);
    const double dr = r_cut / (n - 1);
    for (int i = 0; i < n; ++i) pq.at(i * dr, ai, aj, &F[i], &G[i]);
}

double self_poly(double xi, double a) {
    double F, G;
    PolyQuad(xi, a, a).at(0.0, a, a, &F, &G);
    return F;
}

// ------------------------------------------------------------------ Sec. II C parameters
static double kcut_bound(double k, double xi, double a) {
    return (4.0 / k * exp(-k * k / (4 * xi * xi)) - sqrt(kPi) / xi * erfc(k / (2 * xi))) / (2 * kPi * a);
}

static double quad_err(int P, double m) {
    return exp(-kPi * kPi * P * P / (2 * m * m)) + erfc(m / sqrt(2.0));
}

// Minimiser over m of quad_err(P, m): bisection on the sign of its derivative.
static double best_m(int P) {
    const double c = kPi * kPi * P * P / 2.0;
    double lo = 0.5, hi = 2.0 * P;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (lo + hi);
        const double d = exp(-c / (m * m)) * 2 * c / (m * m * m) - sqrt(2 / kPi) * exp(-m * m / 2);
        if (d < 0) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
}

static int smooth2357(int n) {
    const int p[4] = {2, 3, 5, 7};
    for (int i = 0; i < 4; ++i) while (n % p[i] == 0) n /= p[i];
    return n == 1;
}

}  // namespace pse

using namespace pse;

extern "C" pse_status pse_plan(double L, double a, const pse_params *p, pse_plan_info *out) {
    if (!p || !out) return PSE_EINVAL;
    if (!(L > 0) || !(a > 0) || !isfinite(L) || !isfinite(a)) return PSE_EINVAL;
    const double tol = p->tol;
    if (!(tol > 0) || tol > 0.1) return PSE_EINVAL;
    const double xi = (p->xi > 0) ? p->xi : 0.5 / a;
    if (!isfinite(xi)) return PSE_EINVAL;
    if (p->precision != PSE_FP32 && p->precision != PSE_FP64) return PSE_EINVAL;
    memset(out, 0, sizeof(*out));
    out->L = L;
    out->a = a;
    out->xi = xi;
    out->tol = tol;
    out->precision = p->precision;
    out->r_cut = sqrt(log(1.0 / tol)) / xi;
    if (out->r_cut >= 0.5 * L) return PSE_EINVAL;
    // k_cut: bisection on the decreasing eq. errbound bound
    double lo = 1e-6, hi = 1.0;
    while (kcut_bound(hi, xi, a) > tol) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (kcut_bound(mid, xi, a) > tol) lo = mid; else hi = mid;
    }
    out->k_cut = hi;
    int P;
    if (p->support_P > 0) {
        P = p->support_P;
    } else {
        P = 3;
        while (quad_err(P, best_m(P)) > tol) ++P;
    }
    out->P = P;
    out->m = best_m(P);
    int M;
    if (p->grid_M > 0) {
        M = p->grid_M;
    } else {
        M = (int)ceil(out->k_cut * L / kPi - 1e-9);
        if (M < P + 1) M = P + 1;
        if (M < 4) M = 4;
        while (!smooth2357(M)) ++M;
        while (pow(P * (L / M) * xi / out->m, 2) > 1.0) {
            ++M;
            while (!smooth2357(M)) ++M;
        }
    }
    if (M < P + 1 || M > 2048) return PSE_EINVAL;
    out->M = M;
    out->h = L / M;
    out->eta = pow(P * out->h * xi / out->m, 2);
    if (out->eta > 1.0 + 1e-12 && p->grid_M > 0) return PSE_EINVAL;
    // neighbour-search cells: side >= r_cut with a 1e-4 margin for float binning
    int nc = (int)floor(L / (out->r_cut * (1.0 + 1e-4)));
    if (nc < 2) nc = 2;
    if (nc > 1024) nc = 1024;
    out->ncell = nc;
    out->self_mobility = self_real(xi, a) / (6 * kPi * a);
    return PSE_OK;
}

extern "C" pse_status pse_real_scalars(double xi, double a, int64_t n, const double *r, double *F, double *G) {
    if (!(xi > 0) || !(a > 0) || n < 0 || (n > 0 && (!r || !F || !G))) return PSE_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        if (!(r[i] >= 0) || !isfinite(r[i])) return PSE_EINVAL;
        if (r[i] == 0.0) {
            F[i] = G[i] = self_real(xi, a);
        } else if (r[i] < 0.2 * a) {
            fg_small(r[i], xi, a, &F[i], &G[i]);
        } else {
            fg_closed(r[i], xi, a, &F[i], &G[i]);
        }
    }
    return PSE_OK;
}

extern "C" pse_status pse_real_scalars_poly(double xi, double ai, double aj, int64_t n, const double *r, double *F,
                                            double *G) {
    if (!(xi > 0) || !(ai > 0) || !(aj > 0) || n < 0 || (n > 0 && (!r || !F || !G))) return PSE_EINVAL;
    const PolyQuad pq(xi, ai, aj);
    for (int64_t i = 0; i < n; ++i) {
        if (!(r[i] >= 0) || !isfinite(r[i])) return PSE_EINVAL;
        pq.at(r[i], ai, aj, &F[i], &G[i]);
    }
    return PSE_OK;
}

// Sec. II C, eqs. work and xistar with the constants calibrated at xi0: the
// xi-dependent work is T_R (xi0/xi)^d_f + T_W (xi/xi0)^3 (neighbours within
// r_cut ~ 1/xi grow as r_cut^d_f; Fourier modes ~ k_cut^3 ~ xi^3, the FFT's
// logarithm and n_iter held at their xi0 values), whose stationary point is
// xi* = xi0 (d_f T_R / (3 T_W))^(1/(d_f + 3)).
extern "C" pse_status pse_xi_model(double xi0, double t_real, double t_wave, double d_f, double *xi_star) {
    if (!xi_star) return PSE_EINVAL;
    if (!(xi0 > 0) || !(t_real > 0) || !(t_wave > 0) || !isfinite(xi0) || !isfinite(t_real) || !isfinite(t_wave))
        return PSE_EINVAL;
    if (!(d_f >= 1.0 && d_f <= 3.0)) return PSE_EINVAL;
    *xi_star = xi0 * pow(d_f * t_real / (3.0 * t_wave), 1.0 / (d_f + 3.0));
    return PSE_OK;
}

extern "C" const char *pse_strerror(pse_status s) {
    switch (s) {
        case PSE_OK: return "ok";
        case PSE_EINVAL: return "invalid argument";
        case PSE_ENOMEM: return "out of memory or capacity exceeded";
        case PSE_ECUDA: return "CUDA runtime error";
        case PSE_ECUFFT: return "cuFFT error";
        case PSE_ENOTCONVERGED: return "Lanczos iteration did not converge within max_iter";
        case PSE_ENOTSUPPORTED: return "operation not supported for this context";
        case PSE_ENOTREADY: return "required state (e.g. preconditioner weights) not set";
    }
    return "unknown status";
}
