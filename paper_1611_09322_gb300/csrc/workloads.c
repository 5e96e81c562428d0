/*
 * Seeded synthetic particle configurations in a periodic cube.
 *
 * This module holds no PSE arithmetic: it only places spheres.  Both the
 * CUDA path (via bench.py) and the test oracle draw their inputs from it.
 *
 *   wl_rsa      random sequential addition of non-overlapping spheres
 *   wl_rsa_poly the same for spheres of unequal radii
 *   wl_relax    harmonic overlap relaxation (gradient descent) of spheres
 *   wl_cca_gel  fractal clusters built by tunable-dimension cluster-cluster
 *               aggregation (monomer contact at 2a), packed into the box
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014), which is
 * independent of the Philox streams the sampler itself uses.
 * Plain C99, no platform intrinsics: identical results on x86-64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t rng_next(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_normal(rng_t *r) {
    double u = rng_u01(r), v = rng_u01(r);
    if (u < 1e-300) u = 1e-300;
    return sqrt(-2.0 * log(u)) * cos(2.0 * M_PI * v);
}

static double wrap(double x, double L) {
    x = fmod(x, L);
    if (x < 0) x += L;
    if (x >= L) x -= L;
    return x;
}
static double mind(double d, double L) { return d - L * floor(d / L + 0.5); }

/* ------------------------------------------------------------------ cell grid */
typedef struct {
    int nc;          /* cells per side */
    double cs;       /* cell side */
    int64_t *head;   /* nc^3 */
    int64_t *next;   /* capacity */
} grid_t;

static int grid_init(grid_t *g, double L, double min_side, int64_t cap) {
    g->nc = (int)floor(L / min_side);
    if (g->nc < 1) g->nc = 1;
    if (g->nc > 512) g->nc = 512;
    g->cs = L / g->nc;
    int64_t n3 = (int64_t)g->nc * g->nc * g->nc;
    g->head = (int64_t *)malloc(sizeof(int64_t) * n3);
    g->next = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    if (!g->head || !g->next) return -1;
    for (int64_t i = 0; i < n3; ++i) g->head[i] = -1;
    return 0;
}
static void grid_free(grid_t *g) { free(g->head); free(g->next); }
static int cell_of(const grid_t *g, double x) {
    int c = (int)floor(x / g->cs);
    if (c < 0) c = 0;
    if (c >= g->nc) c = g->nc - 1;
    return c;
}
static int64_t cell_id(const grid_t *g, int cx, int cy, int cz) {
    int n = g->nc;
    cx = ((cx % n) + n) % n; cy = ((cy % n) + n) % n; cz = ((cz % n) + n) % n;
    return ((int64_t)cx * n + cy) * n + cz;
}
static void grid_insert(grid_t *g, const double *p, int64_t i) {
    int64_t c = cell_id(g, cell_of(g, p[0]), cell_of(g, p[1]), cell_of(g, p[2]));
    g->next[i] = g->head[c];
    g->head[c] = i;
}
/* 1 if any stored point lies closer than dmin to q (skipping index `skip`). */
static int grid_overlaps(const grid_t *g, const double *pos, const double *q, double dmin, double L,
                         int64_t skip) {
    int cx = cell_of(g, q[0]), cy = cell_of(g, q[1]), cz = cell_of(g, q[2]);
    int span = g->nc >= 3 ? 1 : 0;
    double d2min = dmin * dmin;
    for (int dx = -span; dx <= span; ++dx)
        for (int dy = -span; dy <= span; ++dy)
            for (int dz = -span; dz <= span; ++dz) {
                int64_t c = cell_id(g, cx + dx, cy + dy, cz + dz);
                if (g->nc < 3 && (dx || dy || dz)) continue;
                for (int64_t j = g->head[c]; j >= 0; j = g->next[j]) {
                    if (j == skip) continue;
                    double ex = mind(q[0] - pos[3 * j], L), ey = mind(q[1] - pos[3 * j + 1], L),
                           ez = mind(q[2] - pos[3 * j + 2], L);
                    if (ex * ex + ey * ey + ez * ez < d2min) return 1;
                }
            }
    return 0;
}

/*
 * Random sequential addition: up to max_trials uniform proposals, each kept
 * if no earlier sphere is within `diameter`.  Returns the number placed
 * (== N on success).  out: N x 3 doubles in [0, L).
 */
int64_t wl_rsa(int64_t N, double L, double diameter, uint64_t seed, int64_t max_trials, double *out) {
    grid_t g;
    if (grid_init(&g, L, diameter, N) != 0) return -1;
    rng_t r = {seed * 0x2545F4914F6CDD1DULL + 1};
    int64_t n = 0;
    for (int64_t t = 0; t < max_trials && n < N; ++t) {
        double q[3] = {rng_u01(&r) * L, rng_u01(&r) * L, rng_u01(&r) * L};
        if (grid_overlaps(&g, out, q, diameter, L, -1)) continue;
        out[3 * n] = q[0]; out[3 * n + 1] = q[1]; out[3 * n + 2] = q[2];
        grid_insert(&g, out + 3 * n, n);
        ++n;
    }
    grid_free(&g);
    return n;
}

/*
 * Harmonic overlap relaxation: E = sum_{r_ij < d} (d - r_ij)^2 / 2, steepest
 * descent x_i += step * sum_j (d - r_ij) rhat_ij, for up to `steps` steps or
 * until the largest overlap is below `stop_overlap`.  Returns the final
 * largest overlap d - r_ij (0 if none).
 */
/*
 * Random sequential addition of spheres with radii[i]: a proposal for
 * sphere n is kept if it overlaps no earlier sphere (distance >= r_n + r_j).
 * Spheres are placed in the given order (largest first packs best).
 * rmax bounds every radius.  Returns the number placed.
 */
int64_t wl_rsa_poly(int64_t N, double L, const double *radii, double rmax, uint64_t seed, int64_t max_trials,
                    double *out) {
    grid_t g;
    if (grid_init(&g, L, 2.0 * rmax, N) != 0) return -1;
    rng_t r = {seed * 0x2545F4914F6CDD1DULL + 7};
    int64_t n = 0;
    for (int64_t t = 0; t < max_trials && n < N; ++t) {
        double q[3] = {rng_u01(&r) * L, rng_u01(&r) * L, rng_u01(&r) * L};
        int cx = cell_of(&g, q[0]), cy = cell_of(&g, q[1]), cz = cell_of(&g, q[2]);
        int span = g.nc >= 3 ? 1 : 0, hit = 0;
        for (int dx = -span; dx <= span && !hit; ++dx)
            for (int dy = -span; dy <= span && !hit; ++dy)
                for (int dz = -span; dz <= span && !hit; ++dz) {
                    if (g.nc < 3 && (dx || dy || dz)) continue;
                    for (int64_t j = g.head[cell_id(&g, cx + dx, cy + dy, cz + dz)]; j >= 0; j = g.next[j]) {
                        double ex = mind(q[0] - out[3 * j], L), ey = mind(q[1] - out[3 * j + 1], L),
                               ez = mind(q[2] - out[3 * j + 2], L), dm = radii[n] + radii[j];
                        if (ex * ex + ey * ey + ez * ez < dm * dm) { hit = 1; break; }
                    }
                }
        if (hit) continue;
        out[3 * n] = q[0]; out[3 * n + 1] = q[1]; out[3 * n + 2] = q[2];
        grid_insert(&g, out + 3 * n, n);
        ++n;
    }
    grid_free(&g);
    return n;
}

double wl_relax(int64_t N, double L, double diameter, int64_t steps, double step, double stop_overlap,
                double *pos) {
    double *f = (double *)malloc(sizeof(double) * 3 * N);
    if (!f) return -1.0;
    double worst = 0.0;
    for (int64_t s = 0; s <= steps; ++s) {
        grid_t g;
        if (grid_init(&g, L, diameter, N) != 0) { free(f); return -1.0; }
        for (int64_t i = 0; i < N; ++i) grid_insert(&g, pos + 3 * i, i);
        memset(f, 0, sizeof(double) * 3 * N);
        worst = 0.0;
        int span = g.nc >= 3 ? 1 : 0;
        for (int64_t i = 0; i < N; ++i) {
            const double *q = pos + 3 * i;
            int cx = cell_of(&g, q[0]), cy = cell_of(&g, q[1]), cz = cell_of(&g, q[2]);
            for (int dx = -span; dx <= span; ++dx)
                for (int dy = -span; dy <= span; ++dy)
                    for (int dz = -span; dz <= span; ++dz) {
                        if (g.nc < 3 && (dx || dy || dz)) continue;
                        int64_t c = cell_id(&g, cx + dx, cy + dy, cz + dz);
                        for (int64_t j = g.head[c]; j >= 0; j = g.next[j]) {
                            if (j == i) continue;
                            double ex = mind(q[0] - pos[3 * j], L), ey = mind(q[1] - pos[3 * j + 1], L),
                                   ez = mind(q[2] - pos[3 * j + 2], L);
                            double r2 = ex * ex + ey * ey + ez * ez;
                            if (r2 >= diameter * diameter || r2 == 0.0) continue;
                            double rr = sqrt(r2), ov = diameter - rr;
                            if (ov > worst) worst = ov;
                            f[3 * i] += ov * ex / rr; f[3 * i + 1] += ov * ey / rr; f[3 * i + 2] += ov * ez / rr;
                        }
                    }
        }
        grid_free(&g);
        if (worst < stop_overlap || s == steps) break;
        for (int64_t i = 0; i < 3 * N; ++i) pos[i] = wrap(pos[i] + step * f[i], L);
    }
    free(f);
    return worst;
}

/* ------------------------------------------------------------------ tunable-dimension CCA */
typedef struct { int64_t n; double *p; double rg2; } cluster_t;

static void centre(cluster_t *c) {
    double m[3] = {0, 0, 0};
    for (int64_t i = 0; i < c->n; ++i) for (int d = 0; d < 3; ++d) m[d] += c->p[3 * i + d];
    for (int d = 0; d < 3; ++d) m[d] /= (double)c->n;
    double s = 0;
    for (int64_t i = 0; i < c->n; ++i)
        for (int d = 0; d < 3; ++d) { c->p[3 * i + d] -= m[d]; s += c->p[3 * i + d] * c->p[3 * i + d]; }
    c->rg2 = s / (double)c->n;
}

static void random_rotation(rng_t *r, double R[9]) {
    /* uniform rotation from a normalised random quaternion */
    double q0 = rng_normal(r), q1 = rng_normal(r), q2 = rng_normal(r), q3 = rng_normal(r);
    double n = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    q0 /= n; q1 /= n; q2 /= n; q3 /= n;
    R[0] = 1 - 2 * (q2 * q2 + q3 * q3); R[1] = 2 * (q1 * q2 - q0 * q3); R[2] = 2 * (q1 * q3 + q0 * q2);
    R[3] = 2 * (q1 * q2 + q0 * q3); R[4] = 1 - 2 * (q1 * q1 + q3 * q3); R[5] = 2 * (q2 * q3 - q0 * q1);
    R[6] = 2 * (q1 * q3 - q0 * q2); R[7] = 2 * (q2 * q3 + q0 * q1); R[8] = 1 - 2 * (q1 * q1 + q2 * q2);
}

/*
 * Merge B into A: B (randomly rotated) approaches A's centre of mass along a
 * random direction n and stops at first monomer contact (distance 2a).  The
 * target centre distance Gamma makes the merged cluster obey
 * R_g = a (N / kf)^(1/df), from N R_g^2 = N1 Rg1^2 + N2 Rg2^2 + (N1 N2 / N) Gamma^2.
 * Of up to 400 random (rotation, direction) tries, the contact whose centre
 * distance is closest to Gamma is kept (the first within 0.05 a ends the
 * search); small clusters cannot always reach Gamma exactly.
 */
static int cca_merge(cluster_t *A, cluster_t *B, double a, double df, double kf, rng_t *r, double *scratch,
                     double *best) {
    int64_t N1 = A->n, N2 = B->n, N = N1 + N2;
    double rg = a * pow((double)N / kf, 1.0 / df);
    double G2 = ((double)N / ((double)N1 * (double)N2)) * (N * rg * rg - N1 * A->rg2 - N2 * B->rg2);
    double Gam = G2 > 0 ? sqrt(G2) : 2 * a;
    double dd = 4 * a * a;
    double best_err = 1e300;
    for (int attempt = 0; attempt < 400; ++attempt) {
        double R[9], n[3];
        random_rotation(r, R);
        double nn;
        do {
            n[0] = rng_normal(r); n[1] = rng_normal(r); n[2] = rng_normal(r);
            nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        } while (nn < 1e-12);
        n[0] /= nn; n[1] /= nn; n[2] /= nn;
        for (int64_t j = 0; j < N2; ++j) {
            const double *q = B->p + 3 * j;
            for (int d = 0; d < 3; ++d) scratch[3 * j + d] = R[3 * d] * q[0] + R[3 * d + 1] * q[1] + R[3 * d + 2] * q[2];
        }
        /* B's monomers at q_j + t n; contact with p_i where |p_i - q_j - t n| = 2a.
           The first contact coming in from t = +inf is the largest root. */
        double tstar = -1e300;
        for (int64_t i = 0; i < N1; ++i) {
            const double *p = A->p + 3 * i;
            for (int64_t j = 0; j < N2; ++j) {
                double w0 = p[0] - scratch[3 * j], w1 = p[1] - scratch[3 * j + 1], w2 = p[2] - scratch[3 * j + 2];
                double b = w0 * n[0] + w1 * n[1] + w2 * n[2];
                double c = w0 * w0 + w1 * w1 + w2 * w2 - dd;
                double disc = b * b - c;
                if (disc < 0) continue;
                double t = b + sqrt(disc);
                if (t > tstar) tstar = t;
            }
        }
        if (tstar < -1e299) continue;
        double err = fabs(tstar - Gam);
        if (err < best_err) {
            best_err = err;
            for (int64_t j = 0; j < N2; ++j)
                for (int d = 0; d < 3; ++d) best[3 * j + d] = scratch[3 * j + d] + tstar * n[d];
        }
        if (err < 0.05 * a) break;
    }
    if (best_err > 1e299) return 1;
    double *np_ = (double *)realloc(A->p, sizeof(double) * 3 * N);
    if (!np_) return -1;
    A->p = np_;
    memcpy(A->p + 3 * N1, best, sizeof(double) * 3 * N2);
    A->n = N;
    centre(A);
    return 0;
}

/*
 * Fractal gel stand-in: clusters of up to `csize` monomers (a power of two,
 * capped so that a cluster's extent 4 R_g stays below L/2) are grown by
 * hierarchical tunable-dimension cluster-cluster aggregation (target df,
 * prefactor kf, contact at 2a), then each cluster is dropped into the
 * periodic box at a random position and orientation, retried while any of
 * its monomers would overlap an earlier one; after 200 failed tries the
 * cluster size is halved for the rest of the box.  The last cluster is
 * truncated to reach exactly N.  Returns the number placed.
 */
int64_t wl_cca_gel(int64_t N, double L, double a, double df, double kf, int64_t csize, uint64_t seed,
                   double *out) {
    if (csize < 1) csize = 1;
    rng_t r = {seed * 0x9E3779B97F4A7C15ULL + 7};
    grid_t g;
    if (grid_init(&g, L, 2 * a, N) != 0) return -1;
    double *scratch = (double *)malloc(sizeof(double) * 3 * (csize + 1));
    double *best = (double *)malloc(sizeof(double) * 3 * (csize + 1));
    cluster_t *lvl = (cluster_t *)malloc(sizeof(cluster_t) * csize);
    if (!scratch || !lvl || !best) { grid_free(&g); free(scratch); free(best); free(lvl); return -1; }
    /* clusters must fit the box: extent ~ 4 R_g = 4 a (n/kf)^(1/df) <= L/2 */
    int64_t cmax = 1;
    while (cmax * 2 <= csize && 4.0 * a * pow((double)(cmax * 2) / kf, 1.0 / df) <= 0.5 * L) cmax *= 2;
    int64_t cs = cmax;
    int64_t placed = 0;
    int64_t fails = 0;
    while (placed < N) {
        /* grow one cluster of cs monomers */
        int64_t m = cs;
        for (int64_t i = 0; i < m; ++i) {
            lvl[i].n = 1;
            lvl[i].p = (double *)calloc(3, sizeof(double));
            lvl[i].rg2 = 0.0;
        }
        int ok = 1;
        while (m > 1 && ok) {
            int64_t k = 0;
            for (int64_t i = 0; i + 1 < m; i += 2) {
                int rc = cca_merge(&lvl[i], &lvl[i + 1], a, df, kf, &r, scratch, best);
                if (rc < 0) { ok = 0; break; }
                free(lvl[i + 1].p);
                lvl[k++] = lvl[i];
            }
            if (m % 2 == 1) lvl[k++] = lvl[m - 1];
            m = k;
        }
        cluster_t *c = &lvl[0];
        /* place */
        int64_t take = c->n < N - placed ? c->n : N - placed;
        int done = 0;
        for (int attempt = 0; attempt < 200 && !done; ++attempt) {
            double R[9], t[3] = {rng_u01(&r) * L, rng_u01(&r) * L, rng_u01(&r) * L};
            random_rotation(&r, R);
            int clash = 0;
            for (int64_t j = 0; j < take && !clash; ++j) {
                const double *q = c->p + 3 * j;
                double w[3];
                for (int d = 0; d < 3; ++d)
                    w[d] = wrap(t[d] + R[3 * d] * q[0] + R[3 * d + 1] * q[1] + R[3 * d + 2] * q[2], L);
                memcpy(scratch + 3 * j, w, sizeof(w));
                if (grid_overlaps(&g, out, w, 2 * a * 0.999999, L, -1)) clash = 1;
                /* also against monomers of this cluster already mapped (self-overlap via periodic wrap) */
                for (int64_t k2 = 0; k2 < j && !clash; ++k2) {
                    double ex = mind(w[0] - scratch[3 * k2], L), ey = mind(w[1] - scratch[3 * k2 + 1], L),
                           ez = mind(w[2] - scratch[3 * k2 + 2], L);
                    if (ex * ex + ey * ey + ez * ez < 4 * a * a * 0.999998) clash = 1;
                }
            }
            if (clash) continue;
            for (int64_t j = 0; j < take; ++j) {
                memcpy(out + 3 * (placed + j), scratch + 3 * j, 3 * sizeof(double));
                grid_insert(&g, out + 3 * (placed + j), placed + j);
            }
            placed += take;
            done = 1;
        }
        free(c->p);
        if (!done) {
            /* crowded box: smaller clusters from now on (size 1 is plain RSA) */
            if (cs > 1) cs /= 2;
            else if (++fails > 1000000) break;
        }
    }
    free(scratch);
    free(best);
    free(lvl);
    grid_free(&g);
    return placed;
}
