/*
 * pse.h -- C ABI of the GB300 Positively Split Ewald (PSE) Brownian sampler.
 *
 * Method: A. M. Fiore, F. Balboa Usabiaga, A. Donev, J. W. Swan, "Rapid
 * sampling of stochastic displacements in Brownian dynamics simulations",
 * J. Chem. Phys. 146, 124116 (2017), arXiv:1611.09322.
 *
 * A sample is u = M_r^{1/2} z1 + M_w^{1/2} dW2 (Sec. II B, eq. split), whose
 * covariance is the periodic Ewald-summed RPY mobility M = M_r + M_w
 * (Sec. II A, eqs. pairmobility, Mwave, Mreal).  The caller multiplies u by
 * sqrt(2 kT dt) (eq. langevin).  Units: viscosity eta = 1.
 *
 * Conventions for every entry point
 *   - Positions are float32 (or float64 for the *_f64 calls), AoS x,y,z per
 *     particle, 3N values, in a periodic cube of side L; values outside
 *     [0, L) are wrapped.  Outputs are 3N values in the caller's order.
 *   - Pointers named d_* are device pointers on the context's device; h_*
 *     are host pointers.  The caller owns positions and outputs; the context
 *     owns every internal buffer, cuFFT plan and CUDA graph.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it unless stated otherwise.
 *   - (seed, sample_index) fully determine the noise: z1 and dW2 are drawn
 *     from Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *     (element, stream, sample_index), so a sample is reproducible.
 *   - Errors are returned as pse_status, never by exit/abort.  A context is
 *     not thread-safe; use one per host thread.
 */
#ifndef PSE_H
#define PSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSE_OK = 0,
    PSE_EINVAL = 1,          /* invalid argument (box, radius, tol, N, pointer, sizes) */
    PSE_ENOMEM = 2,          /* device or host allocation failed / capacity exceeded */
    PSE_ECUDA = 3,           /* a CUDA runtime call failed */
    PSE_ECUFFT = 4,          /* a cuFFT call failed */
    PSE_ENOTCONVERGED = 5,   /* Lanczos hit max_iter; output holds the last iterate */
    PSE_ENOTSUPPORTED = 6,   /* call not available for this context (e.g. precision) */
    PSE_ENOTREADY = 7        /* required state missing (e.g. preconditioner weights) */
} pse_status;

enum { PSE_FP32 = 0, PSE_FP64 = 1 };

/* Creation parameters.  Zero-initialise and set what you need. */
typedef struct {
    double tol;          /* relative tolerance of the Ewald truncations, the NUFFT
                            quadrature and the Lanczos iteration, in (0, 0.1]   */
    double xi;           /* splitting parameter; <= 0 selects 0.5 / a           */
    int precision;       /* PSE_FP32: grid, FFT, matvec in float32 with float64
                            Lanczos scalars; PSE_FP64: everything in float64    */
    int max_iter;        /* Lanczos cap, 1..64; 0 selects 64                    */
    int fixed_iter;      /* > 0: exactly this many Lanczos steps, no test        */
    int grid_M;          /* > 0: override the FFT grid size (per side)          */
    int support_P;       /* > 0: override the Gaussian support (points per side) */
    int use_precond;     /* 1: block-diagonal learned preconditioner (weights
                            set by pse_precond_set_weights), 0: none            */
    double lanczos_tol;  /* <= 0: same as tol                                    */
    int use_graph;       /* >= 0 (default): one CUDA graph per sample with a
                            device-side Lanczos loop; -1: plain stream launches
                            with a host-side loop (one sync per iteration)      */
    int autotune;        /* bit 0: time cuFFT C2R for every 2,3,5,7-smooth grid
                            size in [M, 1.12 M] at creation and keep the fastest
                            (a finer grid only lowers the NUFFT error); needs
                            the GPU at pse_create_ex.  0: the Sec. II C grid.
                            bit 1: time every spreading tile shape at the first
                            forces call and keep the fastest.
                            bit 2: time every near-field matvec launch shape
                            at the first sample and keep the fastest.
                            bit 3: once the grid is fixed (planned, tuned or
                            given), raise xi to the largest value whose
                            Sec. II C plan fits that grid: the wave part
                            costs the same, r_cut and the near-field work
                            shrink (pse_get_plan reports the xi used).      */
    int system;          /* Philox stream index of this system (streams 2*system
                            and 2*system + 1): independent noise for systems
                            sampled side by side; 0 by default                 */
    int wave_noise;      /* 0 (default): dW2 drawn in k-space (Sec. II B 2);
                            1: white noise drawn on the M^3 grid and taken to
                            k-space by a forward FFT -- same covariance, other
                            samples (the fluctuating-hydrodynamics form)       */
    int spread_tile;     /* 0 (default): spreading tile chosen automatically
                            (largest that fits shared memory, or timed with
                            autotune bit 1); 1, 2 or 4: tiles of that many
                            cells per side (PSE_ENOTSUPPORTED at the first
                            forces call if it does not fit shared memory)      */
    int matvec_shape;    /* 0 (default): near-field matvec with 2 threads x 4
                            gathers per particle in blocks of 1024 threads
                            (FP32; 4 x 4 in blocks of 128 in FP64), or timed
                            with autotune bit 2;
                            1..10 force threads x gathers, block size: 4x4
                            128, 8x2 128, 16x1 128, 4x2 128, 4x4 1024, 4x4
                            512, 8x2 1024, 4x2 1024, 1x4 1024, 2x4 1024;
                            11: brick-tiled (each 4x4x4-cell brick's
                            neighbourhood staged in shared memory; FP32
                            without the preconditioner, else shape 5);
                            12: list-free (one thread per particle walks
                            its 27 stencil cells on every product; the
                            sample builds no neighbour list and reports
                            n_pairs 0; FP32 monodisperse without the
                            preconditioner, else shape 1)                 */
    int interp_form;     /* FP32 wave interpolation: 0 (default) copies the
                            three velocity grids into one node-major float4
                            grid (16 M^3 bytes more) and reads one record per
                            support node, one warp per particle (P in 3..10);
                            1: reads the planar grids directly, 16 lanes per
                            particle                                           */
    int wave_fft;        /* FP32 sample path with k-space noise: 0 (default)
                            cuFFT C2R; 1: on grids M = 64 and 256, the noise
                            and the inverse FFT as three kernels of this
                            library (noise generated inside the first pass,
                            the last pass writing the node-major grid of the
                            interpolation; needs interp_form = 0), cuFFT on
                            other grids.  Alone the three passes take about
                            as long as noise + cuFFT + grid copy (417 vs 434 us
                            at M = 256); beside the near-field kernels of a
                            sample their shared memory costs those kernels
                            L1, so the default is cuFFT                        */
} pse_params;

/* Parameters derived from (L, a, xi, tol) by Sec. II C of the paper:
 *   r_cut:  exp(-xi^2 r_cut^2) = tol                        (real truncation)
 *   k_cut:  smallest k with the eq. errbound bound <= tol    (wave truncation)
 *   P, m:   smallest integer P with min_m exp(-pi^2 P^2/2m^2) + erfc(m/sqrt2) <= tol
 *   M:      smallest 2,3,5,7-smooth grid with pi M / L >= k_cut and eta <= 1
 *   eta:    Gaussian shape, sigma^2 = eta / (4 xi^2), eta = (P h xi / m)^2, h = L/M
 *   ncell:  cells per side of the neighbour search, cell side >= r_cut          */
typedef struct {
    double L, a, xi, tol, r_cut, k_cut, m, eta, h, self_mobility;
    int P, M, ncell, precision;
} pse_plan_info;

/* Statistics of the last completed pse_sample* call (read after the stream
 * has been synchronised; pse_get_stats synchronises it). */
typedef struct {
    int lanczos_iters;   /* j at which the Lanczos test passed (or the cap)     */
    int converged;       /* 1 if the test passed                               */
    double lanczos_rel_change; /* ||x_j - x_{j-1}|| / ||x_j|| at exit          */
    int64_t n_pairs;     /* directed near-field pairs within r_cut              */
    int overflow;        /* 1 if the neighbour list exceeded its capacity       */
    int matvec_shape;    /* matvec launch shape in use (1..12 as in pse_params)  */
    int reserved[4];
} pse_stats;

typedef struct pse_ctx pse_ctx;

/* ---------------------------------------------------------------- setup */

/* Host-only: derive the Sec. II C parameters without touching a GPU.
 * L > 0 (box side), a > 0 (sphere radius), p->tol in (0, 0.1].
 * Returns PSE_EINVAL on bad arguments or if r_cut >= L/2 (the near field
 * would need more than the nearest periodic image). */
pse_status pse_plan(double L, double a, const pse_params *p, pse_plan_info *out);

/* Host-only: the dimensionless real-space scalars of Appendix A at n
 * separations r[i] >= 0 (6 pi eta a M^(r) = F (I - rr) + G rr, eq. Mreal),
 * in float64 -- the values the device table is built from.  r = 0 gives the
 * self term of eq. self; 0 < r < 0.2a uses free-space RPY minus the
 * Gaussian-damped wave integral (the closed form cancels there).
 * xi > 0, a > 0; r, F, G: host arrays of n doubles (caller-owned). */
pse_status pse_real_scalars(double xi, double a, int64_t n, const double *r, double *F, double *G);

/* Host-only: real-space scalars of a polydisperse pair (Sec. V: the shape
 * factor sinc(k a_i) sinc(k a_j) in the k-integral of eq. pairmobility),
 * split by H(k, xi) as in eq. Mreal: M^(r)_ij = F (I - rr) + G rr in mobility
 * units (eta = 1, no 6 pi a factor).  Computed as the free-space RPY tensor
 * of two unequal spheres less the H-weighted k-integral (Gauss-Legendre on
 * [0, 16 xi]); r = 0 gives the r -> 0 limit (the self term when ai = aj).
 * xi, ai, aj > 0; r, F, G: host arrays of n doubles (caller-owned). */
pse_status pse_real_scalars_poly(double xi, double ai, double aj, int64_t n, const double *r, double *F,
                                 double *G);

/* Create a sampler for a cube of side L and spheres of radius a with the
 * default parameters (FP32, graph, max_iter 64) -- Sec. II.
 * Allocates device memory on the current device lazily, at the first
 * sample for a given N.  *out is NULL on failure. */
pse_status pse_create(pse_ctx **out, double L, double a, double xi, double tol);

/* As pse_create with explicit parameters. */
pse_status pse_create_ex(pse_ctx **out, double L, double a, const pse_params *p);

/* Release every device buffer, plan and graph of the context (synchronises
 * the device first).  NULL is accepted. */
void pse_destroy(pse_ctx *ctx);

pse_status pse_get_plan(const pse_ctx *ctx, pse_plan_info *out);

/* ---------------------------------------------------------------- choice of xi */

/* eq. xistar (Sec. II C) with the implementation constants C_R, C_W of
 * eq. work calibrated by two measured times at a splitting xi0 (host only,
 * no GPU):
 *   t_real: time of the xi-dependent real-space work at xi0 (neighbour list
 *           and near-field matvecs; the neighbour count within r_cut ~ 1/xi
 *           grows as r_cut^d_f),
 *   t_wave: time of the xi-dependent wave-space work at xi0 (k-space noise
 *           and FFT, ~ xi^3 Fourier modes),
 *   d_f:    fractal dimension of the suspension in [1, 3] (3: hard spheres).
 * The minimiser of t_real (xi0/xi)^d_f + t_wave (xi/xi0)^3 is
 *   *xi_star = xi0 (d_f t_real / (3 t_wave))^(1/(d_f + 3)),
 * n_iter and the FFT's logarithm held at their xi0 values.  PSE_EINVAL for
 * non-positive or non-finite times or xi0, or d_f outside [1, 3]. */
pse_status pse_xi_model(double xi0, double t_real, double t_wave, double d_f, double *xi_star);

#define PSE_XI_TRIALS 8
#define PSE_XI_GRIDS 64
/* Result of pse_tune_xi (times in ms of device time per sample). */
typedef struct {
    double xi_start;     /* p->xi (or 0.5 / a)                                  */
    double t_real, t_wave; /* xi-dependent stage times at xi_start, one staged
                            sample: neighbour list + matvecs; noise + FFT      */
    double xi_model;     /* pse_xi_model(xi_start, t_real, t_wave, d_f)          */
    double xi_best;      /* fastest trial (xi_start on ties)                     */
    double ms_start, ms_best;
    int M_best;          /* its grid: create the sampler with xi = xi_best and
                            grid_M = M_best                                     */
    int n_grids;         /* candidate grids whose FFT was timed                 */
    int n_tried;         /* trials below; trial 0 is the start context          */
    double xi_tried[PSE_XI_TRIALS];
    double ms_tried[PSE_XI_TRIALS]; /* -1: unusable (list overflow, no
                                       convergence within max_iter)            */
    double ms_pred[PSE_XI_TRIALS];  /* the prediction that selected the trial   */
    int iters_tried[PSE_XI_TRIALS]; /* Lanczos steps of the last timed sample   */
    int M_tried[PSE_XI_TRIALS];     /* FFT grid per side                        */
} pse_xi_tuning;

/* Choice of the splitting parameter for a configuration (Sec. II C: the work
 * of eq. work is minimised at xi*).
 *   1. Times `reps` FP32 samples (0 selects 5) of a context created with *p
 *      at xi_start and one staged sample, giving t_real and t_wave; predicts
 *      xi* with pse_xi_model.
 *   2. Candidate grids: the 2,3,5,7-smooth sizes that the plan gives between
 *      0.75 xi* and 1.35 xi* (at most PSE_XI_GRIDS).  On a fixed grid the wave
 *      part costs the same for every xi it admits while the real part shrinks
 *      as xi grows, so each grid is paired with the largest xi whose plan fits
 *      it (k_cut L / pi <= M, eta <= 1).  Each grid's cuFFT C2R is timed and
 *      its sample time predicted from the start context's stage times scaled
 *      by eq. work (real part ~ xi^-d_f, noise ~ M^3, FFT as timed).
 *   3. The best predictions are timed as whole samples (up to seven), and the
 *      fastest trial, the start context included, is reported.
 * Every trial context is destroyed before the next is made; d_pos (3N
 * float32, device, caller order) is only read.  Synchronises `stream`.
 * Create the sampler with xi = out->xi_best and grid_M = out->M_best.
 * PSE_ENOTSUPPORTED for FP64 parameters or use_precond = 1 (the network is
 * trained at one xi); errors of the start context are returned, those of the
 * other trials mark them unusable. */
pse_status pse_tune_xi(double L, double a, const pse_params *p, int64_t N, const float *d_pos, double d_f,
                       int reps, pse_xi_tuning *out, void *stream);

/* ---------------------------------------------------------------- sampling */

/* One PSE Brownian sample (Sec. II B, eq. split), FP32 context.
 *   N >= 1 particles; d_pos: 3N float32 (device); d_out: 3N float32
 *   (device, caller-owned, may not alias d_pos).
 * Real part: Lanczos on the sparse M_r (eq. Mreal, App. A) from a cell list,
 * stopped when ||x_j - x_{j-1}|| / ||x_j|| < lanczos_tol (Chow & Saad).
 * Wave part: Hermitian complex noise scaled per mode by eq. Mwave's
 * B^{1/2} and the Gaussian deconvolution, inverse FFT (cuFFT), Gaussian
 * interpolation at the particles (the Spectral-Ewald NUFFT of Sec. II B 2).
 * Returns once the work is queued; whether the Lanczos test passed is
 * reported by pse_get_stats (PSE_ENOTCONVERGED if the cap was hit, with the
 * last iterate written).  Synchronises the device only when N changed since
 * the previous call (buffers and the graph are then rebuilt). */
pse_status pse_sample(pse_ctx *ctx, int64_t N, const float *d_pos, uint64_t seed,
                      uint64_t sample_index, float *d_out, void *stream);

/* As pse_sample, also writing the two independent parts of eq. split:
 * d_real = M_r^{1/2} z1 and d_wave = M_w^{1/2} dW2 (each 3N float32, device;
 * either may be NULL).  d_out may be NULL too. */
pse_status pse_sample_parts(pse_ctx *ctx, int64_t N, const float *d_pos, uint64_t seed,
                            uint64_t sample_index, float *d_out, float *d_real, float *d_wave,
                            void *stream);

/* As pse_sample with HOST buffers: copies h_pos (3N float32) to the device,
 * samples, copies the result to h_out (3N float32) and synchronises `stream`.
 * Pinned host memory makes the copies asynchronous-capable. */
pse_status pse_sample_host(pse_ctx *ctx, int64_t N, const float *h_pos, uint64_t seed,
                           uint64_t sample_index, float *h_out, void *stream);

/* Pipelined form of pse_sample_host: returns without waiting.  The input
 * copy runs on a copy stream of the context and `stream` waits for it; the
 * result is copied back on a second copy stream once the sample on `stream`
 * is done.  Two staging buffer pairs alternate, so the copies of one call
 * overlap the sampling of its neighbours.  h_pos and h_out must stay valid
 * and untouched until pse_host_sync returns; h_out then holds the result.
 * Host memory should be pinned (pageable memory makes the copies
 * synchronous). */
pse_status pse_sample_host_async(pse_ctx *ctx, int64_t N, const float *h_pos, uint64_t seed,
                                 uint64_t sample_index, float *h_out, void *stream);

/* Waits for every copy issued by pse_sample_host_async (and so for their
 * samples). */
pse_status pse_host_sync(pse_ctx *ctx);

/* FP64 context (params.precision = PSE_FP64): positions, outputs and all
 * arithmetic in float64.  Same semantics as pse_sample_parts. */
pse_status pse_sample_f64(pse_ctx *ctx, int64_t N, const double *d_pos, uint64_t seed,
                          uint64_t sample_index, double *d_out, double *d_real, double *d_wave,
                          void *stream);

/* One Euler-Maruyama displacement's two parts in one call (Sec. III: the
 * deterministic and Brownian wave parts share one inverse FFT):
 *   d_out = c_det M F + c_noise M^{1/2} z,
 * M F = M_r F (sparse, eq. Mreal) + M_w F (spread F with the Gaussian, forward
 * FFT, per mode h^3 B(k) (I - kk) with B from eq. Mwave and the Gaussian
 * deconvolution, inverse FFT, interpolate), M^{1/2} z as in pse_sample with
 * the same (seed, sample_index) noise.  c_noise = 0 skips the Lanczos loop
 * and the noise (the deterministic product alone); for a Brownian step take
 * c_det = dt and c_noise = sqrt(2 kT dt).  d_pos, d_force, d_out: 3N float32
 * device arrays in the caller's order (d_out may not alias the inputs).
 * Contexts with wave_noise = 1 support only c_noise = 0 here
 * (PSE_ENOTSUPPORTED otherwise).  The spreading uses float atomics, so the
 * last bits of M F may differ from call to call. */
pse_status pse_sample_with_forces(pse_ctx *ctx, int64_t N, const float *d_pos, const float *d_force,
                                  uint64_t seed, uint64_t sample_index, double c_det, double c_noise,
                                  float *d_out, void *stream);

/* FP64 context form of pse_sample_with_forces (float64 arrays). */
pse_status pse_sample_with_forces_f64(pse_ctx *ctx, int64_t N, const double *d_pos, const double *d_force,
                                      uint64_t seed, uint64_t sample_index, double c_det, double c_noise,
                                      double *d_out, void *stream);

/* One Euler-Maruyama step of Brownian dynamics (Sec. II B, eq. langevin with
 * div M = 0 in a periodic box), positions updated in place:
 *   d_pos <- wrap(d_pos + dt M F + sqrt(2 kT dt) M^{1/2} z),
 * F_i = k_rep sum_j (2a - r_ij) rhat_ij over the pairs closer than 2a (a
 * harmonic overlap repulsion, computed from the neighbour list in the same
 * graph) plus d_fext (3N float32, device, caller order; NULL for none); the
 * noise is that of (seed, step).  kT = 0 gives the deterministic step.
 * dt, kT, k_rep >= 0.  One graph launch per step; the neighbour list and the
 * forces follow the positions of the step.  Contexts with wave_noise = 1
 * need kT = 0, and k_rep > 0 needs r_cut >= 2a so that the neighbour list
 * holds every contact (PSE_ENOTSUPPORTED otherwise); PSE_EINVAL for a
 * negative or non-finite dt, kT or k_rep. */
pse_status pse_bd_step(pse_ctx *ctx, int64_t N, float *d_pos, const float *d_fext, double dt, double kT,
                       double k_rep, uint64_t seed, uint64_t step, void *stream);

/* FP64 context form of pse_bd_step. */
pse_status pse_bd_step_f64(pse_ctx *ctx, int64_t N, double *d_pos, const double *d_fext, double dt, double kT,
                           double k_rep, uint64_t seed, uint64_t step, void *stream);

/* The comparison method of Sec. IV (Fig. timing, Fig. RelLanc): a Brownian
 * sample M^{1/2} z drawn by Lanczos applied to the WHOLE mobility M = M_r +
 * M_w, each iteration one product M q_j -- the near-field M_r q_j (eq.
 * Mreal) plus the gridded wave product M_w q_j (spread q_j, forward FFT, the
 * per-mode factor h^3 B(k) (I - kk) of eq. Mwave with the Gaussian
 * deconvolution, inverse FFT, interpolate: the M F of Sec. III) -- with the
 * Chow & Saad stop rule and the FP64 Lanczos scalars of pse_sample.  z is
 * the z1 of pse_sample for the same (seed, sample_index) and the context's
 * system index.  The paper reports that PSE sampling beats this method by
 * more than an order of magnitude, its iteration count growing with N.
 *   d_pos, d_out: 3N float32 device arrays in the caller's order (d_out may
 *   not alias d_pos).
 * The iteration count and whether the test passed are reported by
 * pse_get_stats (PSE_ENOTCONVERGED at the cap max_iter, with the last
 * iterate written).  The spreading uses float atomics, so the last bits may
 * differ from call to call.  Contexts with the learned preconditioner
 * installed return PSE_ENOTSUPPORTED (the method runs on M itself). */
pse_status pse_sample_full_lanczos(pse_ctx *ctx, int64_t N, const float *d_pos, uint64_t seed,
                                   uint64_t sample_index, float *d_out, void *stream);

/* FP64 context form of pse_sample_full_lanczos (float64 arrays). */
pse_status pse_sample_full_lanczos_f64(pse_ctx *ctx, int64_t N, const double *d_pos, uint64_t seed,
                                       uint64_t sample_index, double *d_out, void *stream);

/* The deterministic product d_out = M d_force alone (pse_sample_with_forces
 * with c_det = 1, c_noise = 0), FP32 context. */
pse_status pse_mobility_apply(pse_ctx *ctx, int64_t N, const float *d_pos, const float *d_force, float *d_out,
                              void *stream);

/* Near-field product d_out = M_r d_v (eq. Mreal with the App. A scalars and
 * the eq. self diagonal), FP32 context.  d_pos, d_v, d_out: 3N float32
 * device arrays in the caller's order. */
pse_status pse_real_matvec(pse_ctx *ctx, int64_t N, const float *d_pos, const float *d_v,
                           float *d_out, void *stream);

/* ---------------------------------------------------------------- polydisperse suspensions
 * Sec. V: polydispersity enters by making the shape factor size dependent.
 * Spheres of radii a_i, a_j carry sinc(k a_i) sinc(k a_j) where equal
 * spheres carry sinc^2(k a) in eq. pairmobility; the H(k, xi) split keeps
 * both parts positive.  Wave part: one noise dW2, one spectrum per species
 * scaled with that species' sinc(k a_s) (eq. Mwave's B^{1/2} otherwise
 * unchanged), one inverse FFT per species, each particle interpolated from
 * its species' grid -- the exact covariance sum_k sinc(k a_i) sinc(k a_j) ...
 * of the gridded sampler.  Real part: Lanczos on M_r with per-pair scalars
 * (pse_real_scalars_poly) tabulated per species pair and a per-species self
 * term.  Up to PSE_MAX_SPECIES radii; FP32 with FP64 Lanczos scalars.  The
 * Sec. II C parameters use the smallest radius (the strictest wave cutoff). */
#define PSE_MAX_SPECIES 4

/* Create a sampler for spheres of n_species radii (radii[0 .. n_species-1]
 * > 0) in a cube of side L.  p as for pse_create_ex; n_species >= 2 needs
 * precision FP32, wave_noise 0, wave_fft 0, interp_form 0, use_precond 0
 * and a Gaussian support P in 3..10 (PSE_ENOTSUPPORTED otherwise).  One
 * species is the monodisperse sampler at that radius.  Device memory: the
 * spectrum and grids once per species. */
pse_status pse_create_poly(pse_ctx **out, double L, int n_species, const double *radii, const pse_params *p);

/* Number of species (0 for a context made by pse_create[_ex]) and their radii
 * (host array of PSE_MAX_SPECIES doubles, may be NULL). */
pse_status pse_get_species(const pse_ctx *ctx, int *n_species, double *radii);

/* One polydisperse PSE sample (as pse_sample_parts): d_species holds the
 * species index of every particle (N int32, device, caller order; values
 * outside [0, n_species) are clamped into it).  d_out, d_real, d_wave: 3N
 * float32 device arrays or NULL (at least one).  The monodisperse entry
 * points, the forces, Brownian, full-mobility, profiling and
 * preconditioner calls return PSE_ENOTSUPPORTED for contexts with two or
 * more species. */
pse_status pse_sample_poly(pse_ctx *ctx, int64_t N, const float *d_pos, const int *d_species, uint64_t seed,
                           uint64_t sample_index, float *d_out, float *d_real, float *d_wave, void *stream);

/* Polydisperse near-field product d_out = M_r d_v (arguments as above). */
pse_status pse_real_matvec_poly(pse_ctx *ctx, int64_t N, const float *d_pos, const int *d_species,
                                const float *d_v, float *d_out, void *stream);

/* ---------------------------------------------------------------- learned preconditioner
 * Not in the paper.  The real-space Lanczos may run on S M_r S for any
 * invertible block-diagonal S; the sample S^{-1} (S M_r S)^{1/2} z1 keeps
 * covariance M_r exactly and only the iteration count changes.  Block i is
 *   S_i = s0 exp(a_i) (I + tanh(b_i) T_i / (1 + tr T_i)),
 *   T_i = sum_j exp(-((r_ij - 2a)/a)^2) rr_ij over the neighbours within r_cut,
 * SPD and rotation-equivariant; s0 = self_mobility^{-1/2}, so a = b = 0 is the
 * analytic self-mobility block.  (a_i, b_i) = MLP(f_i), 8 -> 16 -> 16 -> 2 with
 * tanh, f_i = invariant features of i's neighbourhood (tr T, tr T^2, det T,
 * smooth neighbour counts within 2.5a, 3.5a, 4.5a, r_cut, mean 2a/r; scaled).
 * Parameter vector (float32, PSE_PRECOND_NPARAM): W1 (16x8, row-major), b1,
 * W2 (16x16), b2, W3 (2x16), b3.  FP32 contexts only. */
#define PSE_PRECOND_NPARAM 450

/* Training inputs for positions d_pos (3N float32, device): d_feat (N x 8)
 * features and d_tens (N x 6: xx, yy, zz, xy, xz, yz) structure tensors, in
 * the caller's particle order (device arrays, caller-owned). */
pse_status pse_precond_features(pse_ctx *ctx, int64_t N, const float *d_pos, float *d_feat, float *d_tens,
                                void *stream);

/* Training targets: the diagonal 3x3 block of (M_loc)^{-1/2}, M_loc = M_r
 * restricted to particle i and its neighbours within 3a (the 16 nearest,
 * ties by caller index), by Newton-Schulz iteration in float32.  d_target:
 * N x 6 (xx, yy, zz, xy, xz, yz), caller order, device. */
pse_status pse_precond_targets(pse_ctx *ctx, int64_t N, const float *d_pos, float *d_target, void *stream);

/* Loss mean_i ||S_i - target_i||_F^2 / s0^2 over n samples and its gradient
 * d_grad (PSE_PRECOND_NPARAM floats) w.r.t. d_theta; *d_loss (device double).
 * All device arrays.  Gradients are summed with atomics (order-dependent
 * rounding). */
pse_status pse_precond_loss_grad(int64_t n, const float *d_feat, const float *d_tens, const float *d_target,
                                 const float *d_theta, float s0, float *d_grad, double *d_loss, void *stream);

/* `steps` full-batch Adam steps (lr, beta 0.9/0.999) on d_theta in place.
 * d_work: device scratch of 3 * PSE_PRECOND_NPARAM + 4 floats; d_loss_hist:
 * device array of `steps` doubles receiving the loss before each step (or
 * NULL). */
pse_status pse_precond_train(int64_t n, const float *d_feat, const float *d_tens, const float *d_target,
                             float *d_theta, float s0, int steps, float lr, float *d_work, double *d_loss_hist,
                             void *stream);

/* Install network weights (host array of PSE_PRECOND_NPARAM floats) and turn
 * the preconditioner on (h_theta = NULL turns it off).  Subsequent samples
 * run Lanczos on S M_r S and return S^{-1} x.  Rebuilds the sample graph. */
pse_status pse_precond_set_weights(pse_ctx *ctx, const float *h_theta, int nparam);

/* The blocks S_i the installed network assigns to positions d_pos: d_S is
 * N x 6 (xx, yy, zz, xy, xz, yz), caller order, device. */
pse_status pse_precond_blocks(pse_ctx *ctx, int64_t N, const float *d_pos, float *d_S, void *stream);

/* Stage indices of pse_profile_stages (the paper's Fig. gel split: real-space
 * matvecs, other Lanczos work, FFT + scaling + RNG, spreading/interpolation). */
enum {
    PSE_STAGE_CELLS = 0,      /* binning + cell scan                         */
    PSE_STAGE_SORT,           /* scatter into cell order + per-cell sort      */
    PSE_STAGE_REAL_NOISE,     /* z1 and ||z1||                                */
    PSE_STAGE_NEIGHBOURS,     /* neighbour count, scan, fill                  */
    PSE_STAGE_MATVEC,         /* M_r q_j, all iterations                      */
    PSE_STAGE_LANCZOS_UPDATE, /* three-term update + ||w||, all iterations    */
    PSE_STAGE_EIGEN,          /* FP64 T_j^{1/2} e_1 + stop test, all iterations */
    PSE_STAGE_FINAL,          /* x = V y, + wave part, caller order           */
    PSE_STAGE_WAVE_NOISE,     /* k-space noise and B^{1/2} scaling (fused
                                 path: with the first FFT pass)               */
    PSE_STAGE_FFT,            /* cuFFT C2R, three components (fused path:
                                 the second and third passes)                 */
    PSE_STAGE_INTERP,         /* Gaussian interpolation at the particles      */
    PSE_STAGE_GRID_COPY,      /* node-major copy of the velocity grid (FP32)  */
    PSE_NSTAGES
};

/* One FP32 sample (as pse_sample) run stage by stage with plain launches and
 * CUDA events between stages on `stream`; synchronises it.  ms[PSE_NSTAGES]
 * receives each stage's device time in milliseconds and launches[PSE_NSTAGES]
 * its number of kernel launches of this library (host arrays, caller-owned).
 * The output equals pse_sample's for the same arguments. */
pse_status pse_profile_stages(pse_ctx *ctx, int64_t N, const float *d_pos, uint64_t seed,
                              uint64_t sample_index, float *d_out, double *ms, int *launches,
                              void *stream);

/* Near-field product d_out = M_r d_v, like pse_real_matvec, for callers that
 * cannot allocate device memory: code that must not call cudaMalloc (or any
 * allocating library routine) because device memory is owned by someone else
 * -- an application's own memory pool, a plugin with a fixed footprint, a
 * real-time loop that may not block in the allocator.  The paper has no
 * counterpart; this is a deployment variant of pse_real_matvec.
 *   L, a, xi, tol: as for pse_create (xi <= 0 selects 0.5/a);
 *   d_pos, d_v, d_out: 3N float32 device arrays in the caller's order.
 * No context and no allocation: all scratch (cell list, sorted positions,
 * neighbour list, F/G table) lives in one static device array of about
 * 12 MB.  The module holding it is loaded on a device when it is first used
 * there (CUDA loads modules lazily by default), so the first call on each
 * device reserves the array, which then stays reserved until the process
 * exits; a caller with a fixed memory budget should make that first call
 * during its set-up.  Limits: N <= 16384, ncell^3 <= 32768 cells (box side up to about
 * 32 r_cut), at most 2,621,440 / N neighbours within r_cut per particle
 * (160 at N = 16384); beyond the first two it returns PSE_EINVAL before
 * launching anything, beyond the last PSE_ENOMEM after the run (the output
 * is then incomplete).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and fills the F/G table; make that first call
 * before any stream capture.  The table is rebuilt when (xi, a, r_cut)
 * change.  The array is shared by every call and keeps the last call's
 * contents (what must start at zero is cleared on each call); calls that
 * overlap on the GPU -- concurrent streams, threads or devices sharing a
 * context -- race on it, so serialise them.  The call synchronises `stream`
 * before returning. */
pse_status pse_real_matvec_noalloc(double L, double a, double xi, double tol, int64_t N,
                                   const float *d_pos, const float *d_v, float *d_out, void *stream);

/* ---------------------------------------------------------------- batched systems
 * Many independent periodic systems of uneven size sampled together (not in
 * the paper).  Each system has its own box, radius and parameters (its own
 * xi, cut-offs and grid); one pse_batch_sample is ONE CUDA graph launch whose
 * kernels each work for all systems at once (a block -> system table): cell
 * lists, neighbour lists, q_1, the wave noise and interpolation, and in the
 * device-side loop the near-field matvec, the Lanczos update and the FP64
 * eigen-solves; systems that converge drop out of the loop.  The inverse
 * FFTs run as one batched cuFFT call per grid size: each system's grid is
 * raised to the next size of a fixed list (16, 20, 24, 28, 32, 40, 48, ...,
 * a finer grid only lowers the NUFFT error), so systems share sizes.
 * System k draws its noise from Philox streams 2k and 2k + 1: its output
 * equals, to float rounding and with the same Lanczos J, that of a lone
 * context created with params.system = k and grid_M = its batch grid
 * (pse_batch_get_plan). */
typedef struct pse_batch pse_batch;

/* nsys >= 1 systems: L[k], a[k] and params p[k] (host arrays of nsys
 * entries).  p[k].system is set to k; p[k].grid_M, when set, is kept;
 * autotune bit 0 is ignored (the size classes replace it).  Interpolation
 * supports P <= 16 (PSE_ENOTSUPPORTED at the first sample otherwise).  FP32
 * only. */
pse_status pse_batch_create(pse_batch **out, int nsys, const double *L, const double *a, const pse_params *p);

/* The grid side a system (L, a, p) gets in a batch, `step` size classes
 * finer: its Sec. II C plan's grid (p->grid_M when set) raised to the next
 * class of the list above, then `step` classes further (the last class at
 * most; a plan beyond the last class keeps its own grid).  Setting
 * grid_M to the step-1 or step-2 grid with autotune bit 3 trades a larger
 * xi (shorter r_cut, fewer neighbour pairs) for a larger FFT.  Host only,
 * no GPU needed.  PSE_EINVAL on null pointers or step < 0; pse_plan's
 * status otherwise. */
pse_status pse_batch_grid(double L, double a, const pse_params *p, int step, int *M_out);

/* Sample all systems.  offsets: host array of nsys + 1 particle offsets
 * (offsets[0] = 0, system k owns particles offsets[k] .. offsets[k+1]-1,
 * each N_k >= 1); d_pos / d_out: 3 * offsets[nsys] float32 device arrays,
 * concatenated in system order.  The graph is rebuilt (with a device
 * synchronisation) when any N_k changes. */
pse_status pse_batch_sample(pse_batch *b, const int64_t *offsets, const float *d_pos, uint64_t seed,
                            uint64_t sample_index, float *d_out, void *stream);

/* Install (or with h_theta = NULL remove) learned-preconditioner weights in
 * system k (see pse_precond_set_weights); the batch graph is rebuilt. */
pse_status pse_batch_set_precond(pse_batch *b, int k, const float *h_theta, int nparam);

/* Statistics of system k after the last batch sample (synchronises). */
pse_status pse_batch_get_stats(pse_batch *b, int k, pse_stats *out);
pse_status pse_batch_get_plan(const pse_batch *b, int k, pse_plan_info *out);
void pse_batch_destroy(pse_batch *b);

/* Statistics of the last sample (synchronises the context's last stream). */
pse_status pse_get_stats(pse_ctx *ctx, pse_stats *out);

/* Static description of a status code. */
const char *pse_strerror(pse_status s);

#ifdef __cplusplus
}
#endif
#endif /* PSE_H */
