// Internal declarations shared by the CUDA translation units of libpse.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <stdint.h>

#include "pse.h"

#define PSE_MAXIT 64          // Lanczos cap (basis holds PSE_MAXIT + 2 vectors)
#define PSE_TABLE_N 4096      // entries of the F, G table on [0, r_cut]
#define PSE_TABLEC_N 1024     // entries of the compact table the Lanczos matvec stages in shared memory
#define PSE_TABLEC_A 256      // of which on [0, 2a): knots at 2a, where F and G have a kink
#define PSE_SCAN_ITEMS 4096   // elements per block of the device scan
#define PSE_SPECIES_SHIFT 28  // species index in bits 28-29 of a cell record's w (cell ids < 2^24)
#define PSE_CELL_MASK 0x0FFFFFFF
#define PSE_MAX_SCAN (PSE_SCAN_ITEMS * PSE_SCAN_ITEMS)

namespace pse {

// 16-byte (float) / 32-byte (double) aligned 4-vector.
template <typename T> struct alignas(4 * sizeof(T)) V4 { T x, y, z, w; };

// Cell ids are brick-major: cells are grouped in 4x4x4 bricks (bricks in
// x-major order, cells x-major inside a brick), so consecutive sorted
// particles fill compact 3-D regions.  The id space covers whole bricks
// (nb^3 * 64 slots, nb = ceil(ncell / 4)); slots past ncell stay empty.
#ifdef __CUDACC__
#define PSE_HD __host__ __device__
#else
#define PSE_HD
#endif
PSE_HD inline int bricks_per_side(int nc) { return (nc + 3) >> 2; }
PSE_HD inline int64_t cell_slots(int nc) {
    const int64_t nb = bricks_per_side(nc);
    return nb * nb * nb * 64;
}
PSE_HD inline int cell_id(int cx, int cy, int cz, int nb) {
    const int brick = ((cx >> 2) * nb + (cy >> 2)) * nb + (cz >> 2);
    return (brick << 6) | ((cx & 3) << 4) | ((cy & 3) << 2) | (cz & 3);
}
PSE_HD inline void cell_xyz(int id, int nb, int &cx, int &cy, int &cz) {
    const int brick = id >> 6, in = id & 63;
    const int bz = brick % nb, by = (brick / nb) % nb, bx = brick / (nb * nb);
    cx = (bx << 2) | (in >> 4);
    cy = (by << 2) | ((in >> 2) & 3);
    cz = (bz << 2) | (in & 3);
}

// Matvec record of one sorted particle: cell-local offsets and the current
// Lanczos vector side by side, so a neighbour gather is one 32-byte sector
// (float) instead of two.
template <typename T> struct alignas(8 * sizeof(T)) Rec { V4<T> l; V4<T> q; };

// Geometry of one periodic system, by value into kernels.
template <typename T> struct Geom {
    T L;          // box side
    T cs;         // cell side (>= r_cut)
    T cs_lo;      // cs - (T)cs in the next precision (compensation; 0 for double)
    T inv_cs;
    T rc2;        // r_cut^2
    T tab_inv_dr; // (PSE_TABLE_N - 1) / r_cut
    T self_m;     // self mobility of eq. self, divided by 6 pi a
    T a;          // sphere radius (FP64 path: closed-form F, G for r >= 0.2 a)
    T xi;         // splitting parameter
    int nc;       // cells per side
    int nb;       // bricks per side (4x4x4 cells each)
    int mv;       // matvec launch shape: threads x gathers per particle, threads per block
                  // (0: 4 x 4, 128; 1: 8 x 2, 128; 2: 16 x 1, 128; 3: 4 x 2, 128;
                  //  4: 4 x 4, 1024; 5: 4 x 4, 512; 6: 8 x 2, 1024; 7: 4 x 2, 1024;
                  //  8: 1 x 4, 1024; 9: 2 x 4, 1024; 10: brick-tiled, records staged in
                  //  shared memory, FP32 monodisperse without preconditioner;
                  //  11: list-free, one thread per particle walking its 27 stencil
                  //  cells, FP32 monodisperse without preconditioner)
    // compact table: PSE_TABLEC_A uniform knots on [0, tc_split), the rest
    // uniform on [tc_split, r_cut]; tc_split = min(2a, r_cut)
    T tc_split, tc_invA, tc_invB;
    // a pair whose float32 r^2 lies in [rc2_lo, rc2_hi) (within rounding of
    // r_cut^2; both rc2 in the FP64 path) is decided again in float64 from
    // the positions with the float64 r_cut^2 and box side
    T rc2_lo, rc2_hi;
    double rc2_d, L_d, invL_d;
    // polydisperse contexts (nspec >= 2): per-species self mobility; pair
    // (s, t) reads table block pair_index(s, t, nspec) of PSE_TABLE_N entries
    int nspec;
    T self_s[PSE_MAX_SPECIES];
};

// Block of the (unordered) species pair (s, t) in a polydisperse table.
PSE_HD inline int pair_index(int s, int t, int S) {
    const int i = s < t ? s : t, j = s < t ? t : s;
    return i * S - (i * (i - 1)) / 2 + (j - i);
}
#define PSE_MV_VARIANTS 11
#define PSE_MV_TILED 10
#define PSE_MV_NOLIST 11  // list-free matvec (not among the timed shapes)

#ifdef __CUDACC__
// The float64 r < r_cut decision for a pair whose float32 distance lies
// within rounding of r_cut: wrapped positions, nearest periodic image.
__device__ __forceinline__ bool pair_inside_f64(const V4<float> &a, const V4<float> &b, const Geom<float> &g) {
    double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y, dz = (double)a.z - (double)b.z;
    dx -= g.L_d * rint(dx * g.invL_d);
    dy -= g.L_d * rint(dy * g.invL_d);
    dz -= g.L_d * rint(dz * g.invL_d);
    return dx * dx + dy * dy + dz * dz < g.rc2_d;
}
#endif

// Wave-space parameters of one system.
template <typename T> struct WaveGeom {
    int M, P, Mh1;       // grid side, support, M/2 + 1
    T kscale;            // 2 pi / L
    T a;                 // sphere radius
    T inv4xi2;           // 1 / (4 xi^2)
    T decay;             // (1 - eta) / (8 xi^2)
    T inv_sqrtV;         // V^{-1/2}
    T gl_hi, gl_lo;      // M / L split in two (compensated product x * M / L)
    T ch2;               // 2 xi^2 h^2 / eta: Gaussian exponent per squared grid unit
    T norm;              // (2 xi^2 / (pi eta))^{3/2} h^3
    T inv_M15;           // M^{-3/2}: white grid noise -> dW2 normalisation
    const T *sc_tab;     // per n^2 = nx^2 + ny^2 + nz^2 <= 3 (M/2)^2: (sc(k), 1/|n|) pairs
    uint32_t dv_h1_m, dv_M_m;  // division of 32-bit mode ids by Mh1 and M: multipliers
    int dv_h1_l, dv_M_l;       // and shifts (Granlund-Montgomery, round-up form)
    int big;             // M^2 Mh1 >= 2^32: 64-bit mode ids
    const void *fft_tw;  // M/2 float2 e^{2 pi i k / M} (power-of-two grids, fused FFT path)
    int interp_lanes;    // lanes per particle in the interpolation (8, 16, 32; 0 = pick)
    int nspec;           // spectra / grids, one per species (1: monodisperse)
    int64_t sc_stride;   // entries of one species' block of sc_tab
};

// Per-sample arguments, read by the kernels from device memory so that one
// instantiated graph serves every call.
template <typename T> struct SampleArgs {
    const T *pos;   // 3N caller positions
    T *out;         // 3N or null
    T *real;        // 3N or null
    T *wave;        // 3N or null
    const T *vin;   // 3N caller vector (matvec input, or forces), or null
    uint64_t seed;
    uint64_t sample;
    double c_det;   // weight of M F (forces path)
    double c_noise; // weight of M^{1/2} z (1 for a plain sample)
    T *advance;     // Brownian step: positions advanced in place by out (3N), or null
    const T *fext;  // Brownian step: external force (3N) added to the repulsion, or null
    double k_rep;   // Brownian step: overlap repulsion stiffness
    const int *species;  // polydisperse contexts: species index per caller particle, or null
};

// Tiling of the spreading kernel: tiles of G^3 cells, each spread into a
// padded E^3 node block in shared memory, CP of the 3 components per pass.
struct SpreadTile {
    int G, E, CP, ntx;  // ntx = tiles per side
};

// Device-side state of the Lanczos iteration (one system).
struct LzState {
    double alpha[PSE_MAXIT + 2];
    double beta[PSE_MAXIT + 2];     // beta[0] = ||z1||
    double y[PSE_MAXIT + 2];        // T_j^{1/2} e_1 of the last checked j
    float coef[PSE_MAXIT + 2];      // beta0 * y_i / beta_{i-1}, i = 1..J (float for the final pass)
    float c_u, c_q, c_p;            // update coefficients of the current iteration
    int iter;                       // iteration the matvec/update kernels run next
    int jeig;                       // T_j the eigen kernel processes next
    int J;                          // accepted iteration count
    int converged;
    int cont;                       // loop continues (host-loop mode reads this)
    int active;                     // matvec/update/eigen still run; changes only between loop bodies
    double rel;                     // last ||y_j - y_{j-1}|| / ||y_j||
    unsigned int counter_mv, counter_up, counter_init;
    int overflow;                   // neighbour list capacity exceeded
    int pad_;
    unsigned long long n_pairs;     // directed pairs found by the neighbour search
};

// Appendix A, cases 1 and 2 (FP64): 6 pi eta a M^(r) = F (I - rr) + G rr.
// Used by the host table builder and by the FP64 device matvec.
#ifdef __CUDACC__
__host__ __device__
#endif
inline void fg_closed_hd(double r, double xi, double a, double *F, double *G) {
    const double sp = 1.7724538509055160273;  // sqrt(pi)
    const double x2 = xi * xi, x3 = x2 * xi, x4 = x2 * x2;
    const double r2 = r * r, r3 = r2 * r;
    const double rm = r - 2 * a, rp = r + 2 * a, am = 2 * a - r;
    const double e1 = exp(-r2 * x2), e2 = exp(-rm * rm * x2), e3 = exp(-rp * rp * x2);
    const double c4 = erfc(r * xi), c5 = erfc(rm * xi), c6 = erfc(rp * xi);
    const double A4 = 4 * a * a;
    const double f1 = (18 * r2 * x2 + 3) / (64 * sp * a * r2 * x3);
    const double f2 = (2 * x2 * am * (A4 + 4 * a * r + 9 * r2) - 2 * a - 3 * r) / (128 * sp * a * r3 * x3);
    const double f3 = (-2 * x2 * rp * (A4 - 4 * a * r + 9 * r2) + 2 * a - 3 * r) / (128 * sp * a * r3 * x3);
    const double f4 = (3 - 36 * r2 * r2 * x4) / (128 * a * r3 * x4);
    const double f5 = (4 * x4 * rm * rm * (A4 + 4 * a * r + 9 * r2) - 3) / (256 * a * r3 * x4);
    const double f6 = (4 * x4 * rp * rp * (A4 - 4 * a * r + 9 * r2) - 3) / (256 * a * r3 * x4);
    const double g1 = (6 * r2 * x2 - 3) / (32 * sp * a * r2 * x3);
    const double g2 = (-2 * x2 * rm * rm * (2 * a + 3 * r) + 2 * a + 3 * r) / (64 * sp * a * r3 * x3);
    const double g3 = (2 * x2 * rp * rp * (2 * a - 3 * r) - 2 * a + 3 * r) / (64 * sp * a * r3 * x3);
    const double g4 = -3 * (4 * r2 * r2 * x4 + 1) / (64 * a * r3 * x4);
    const double g5 = (3 - 4 * x4 * am * am * am * (2 * a + 3 * r)) / (128 * a * r3 * x4);
    const double g6 = (3 - 4 * x4 * (2 * a - 3 * r) * rp * rp * rp) / (128 * a * r3 * x4);
    double f0 = 0.0, g0 = 0.0;
    if (r <= 2 * a) {
        f0 = -rm * rm * (A4 + 4 * a * r + 9 * r2) / (32 * a * r3);
        g0 = am * am * am * (2 * a + 3 * r) / (16 * a * r3);
    }
    *F = f0 + f1 * e1 + f2 * e2 + f3 * e3 + f4 * c4 + f5 * c5 + f6 * c6;
    *G = g0 + g1 * e1 + g2 * e2 + g3 * e3 + g4 * c4 + g5 * c5 + g6 * c6;
}

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies,
// Weyl-bumped key between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Four N(0,1) from one Philox block: uniforms (2k+1) 2^-24 from the top 23
// bits (exact in float), Box-Muller with sincospi.
template <typename T> struct Normals4 { T v[4]; };

// Float path: the hardware log2 / sin / cos approximations (absolute error
// ~2^-21 on these ranges, far below the sampler's tolerance).
__device__ __forceinline__ void bm_pair(uint32_t xa, uint32_t xb, float &z0, float &z1) {
    const float ua = ((float)(xa >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
    const float ub = ((float)(xb >> 9) + 0.5f) * 1.1920928955078125e-07f;
    const float r = sqrtf(-2.0f * __logf(ua));
    float s, c;
    __sincosf(6.28318530717958648f * ub, &s, &c);
    z0 = r * c;
    z1 = r * s;
}
__device__ __forceinline__ void bm_pair(uint32_t xa, uint32_t xb, double &z0, double &z1) {
    const double ua = ((double)(xa >> 9) + 0.5) * 1.1920928955078125e-07;
    const double ub = ((double)(xb >> 9) + 0.5) * 1.1920928955078125e-07;
    const double r = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

template <typename T>
__device__ __forceinline__ Normals4<T> normals4(uint32_t element, uint32_t stream, uint64_t seed,
                                                 uint64_t sample) {
    const uint4 x = philox(make_uint4(element, stream, (uint32_t)sample, (uint32_t)(sample >> 32)),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    Normals4<T> n;
    bm_pair(x.x, x.y, n.v[0], n.v[1]);
    bm_pair(x.z, x.w, n.v[2], n.v[3]);
    return n;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of per-thread float partials: float inside each warp (the
// operands are float products), double across warps and blocks.  Result
// valid in all threads.
__device__ __forceinline__ double block_sum_fw(float v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_f(v);
    __syncthreads();
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024); result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Deterministic grid-wide sum: every block stores its partial, the last block
// to arrive (atomic ticket, no waiting) adds the partials in block order.
// Returns true in the last block, with *total valid in all its threads.
// bidx / nblk: this block's index among the nblk blocks reducing together
// (the launch's grid, or one system's share of a fused multi-system launch).
__device__ __forceinline__ bool grid_sum_last(double partial, double *partials, unsigned int *counter,
                                              double *sh, double *total, unsigned int bidx, unsigned int nblk) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        partials[bidx] = partial;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        s_last = (t == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc = 0.0;
    for (unsigned int b = threadIdx.x; b < nblk; b += blockDim.x) acc += __ldcg(partials + b);
    *total = block_sum(acc, sh);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}
__device__ __forceinline__ bool grid_sum_last(double partial, double *partials, unsigned int *counter,
                                              double *sh, double *total) {
    return grid_sum_last(partial, partials, counter, sh, total, blockIdx.x, gridDim.x);
}
#endif

// ------------------------------------------------------------------ host launchers
struct Buffers;  // defined in pse_api.cu

template <typename T> struct Dev {
    // sorted particle data
    V4<T> *pos_sorted;   // wrapped caller positions, w = original index (int bits)
    V4<T> *loc_sorted;   // offsets from the cell corner, w = cell id (int bits)
    int *cell_of;        // per caller particle
    int *slot;           // per caller particle
    int *perm;           // counting-sort slot -> caller index
    int *cell_count;     // ncell^3
    int *cell_start;     // ncell^3 + 1
    int *nbr_count;      // N: neighbours of each sorted particle
    int *nbr;            // ELL, column-major: entry k of particle s at nbr[k * N + s],
                         // (t << 6) | stencil code (2 bits per axis, offset + 1)
    int64_t nbr_cap;     // total entries; per-particle capacity = nbr_cap / N
    int4 *edge;          // pairs found within rounding of r_cut: (s, t, code, slot)
    int *edge_n;         // their count (cleared by the float64 decision kernel)
    int edge_cap;
    int *scan_sums;      // PSE_SCAN_ITEMS
    Rec<T> *rec;         // N: cell-local offsets + current q_j (matvec input)
    V4<T> *basis;        // (PSE_MAXIT + 2) * N, q_1 .. q_{J+1}
    float *pc;           // N x 16: preconditioner blocks S (0..5), S^{-1} (8..13), sorted order
    const float *pc_on;  // == pc while the learned preconditioner is active, else null
    float *pc_theta;     // network parameters (PSE_PRECOND_NPARAM)
    V4<T> *u;            // matvec output
    const V4<T> *mv_add; // added to every Lanczos matvec row (the wave product of the
                         // full-mobility Lanczos), or null
    V4<T> *uwave;        // wave part at sorted particles
    V4<T> *udet;         // M_r F at sorted particles (forces path)
    T *bd_force;         // 3N, caller order: forces of a Brownian step
    T *bd_dx;            // 3N, caller order: displacement of a Brownian step
    double *partials;    // per-block partial sums
    LzState *lz;
    V4<T> *table;        // PSE_TABLE_N: (F, G - F, dF, d(G-F)) / (6 pi a)
    V4<T> *table_c;      // PSE_TABLEC_N, same columns, on the two-segment knots
    void *spec;          // 3 * M * M * Mh1 complex
    T *grid;             // 3 * M^3 real
    V4<T> *grid4;        // M^3 node-major copy (x, y, z, 0) of grid for the interpolation (float)
    SampleArgs<T> *args;
};

// SM count of the current device (cached): persistent grids of the
// reducing kernels are sized from it.
int num_sms();

// cells / scan / neighbour list
template <typename T> void launch_bin(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d,
                                      cudaStream_t s);
void launch_scan(const int *in, int *out, int64_t n, int *sums, cudaStream_t s);
template <typename T> void launch_scatter(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d,
                                          cudaStream_t s);
template <typename T>
void launch_place(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_nbr(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s);

inline int nbr_k(int64_t N, int64_t cap) {
    const int64_t k = cap / (N > 0 ? N : 1);
    return (int)(k > 4096 ? 4096 : k);
}

// Lanczos
template <typename T> void launch_lz_init(int64_t N, const SampleArgs<T> *args, int system, const Dev<T> &d,
                                          cudaStream_t s);
template <typename T> void launch_lz_matvec(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_lz_update(int64_t N, int max_iter, const Dev<T> &d, cudaStream_t s);
void launch_lz_eig(LzState *lz, int max_iter, int fixed_iter, double tol, cudaGraphConditionalHandle h,
                   cudaStream_t s);
// batch loop condition: active_k = cont_k for every system, continue while any is active
void launch_batch_cond(LzState *const *lzs, int nsys, cudaGraphConditionalHandle h, cudaStream_t s,
                       int *any_out = nullptr);

// One system of a fused multi-system Lanczos step (FP32 contexts): its
// buffers, geometry, stop rule and the block ranges it owns in the fused
// matvec and update launches.
struct LzSys {
    int64_t N;
    int K;                       // ELL capacity per particle
    int blk_mv, nblk_mv;         // first block and block count in the fused matvec
    int blk_up, nblk_up;         // same in the fused update
    int max_iter, fixed_iter;
    double tol;
    Geom<float> g;
    Rec<float> *rec;
    const int *count;
    const int *nbr;
    const V4<float> *table;
    const V4<float> *table_c;    // compact table (staged in shared memory by the matvec)
    V4<float> *u;
    double *part_mv, *part_up;   // per-block partial sums of the matvec and the update
    LzState *lz;
    const float *pc;
    V4<float> *basis;
};
// the fused batch matvec: one thread per particle with 8 independent
// gathers, blocks of 512 (the batch's systems are denser than the lone
// headline's: 22 neighbours per particle against 12.5).  64 systems of
// 1e3-5e4 particles: 1.520 ms per batched sample against 1.656 for the lone
// default (2 x 4 in blocks of 1024), 1.529 for 1 x 4 in 512, 1.585 for 1 x 4
// in 1024 and 1.859 for 4 x 4 in 1024.
#define PSE_BATCH_MV_TPP 1
#define PSE_BATCH_MV_ILP 8
#define PSE_BATCH_MV_THREADS 512
#define PSE_NOLIST_THREADS 512  // threads per block of the list-free matvec

// One system of a batch for the fused prologue / epilogue kernels (FP32):
// sizes, geometry, buffers and, per fused kernel kind, the first block and
// block count it owns (block -> system tables map the other way).
enum { BK_ZERO = 0, BK_BIN, BK_SCATTER, BK_SORT, BK_NBR, BK_INIT, BK_NOISE, BK_INTERP, BK_FINAL, BK_PC, BK_COPY, PSE_BK };
#define PSE_BATCH_INTERP_G 16
struct BSys {
    int64_t N;
    int nc3;        // cell slots
    int system;     // Philox stream pair
    int K;          // ELL capacity per particle
    float pc_s0;    // self-mobility^{-1/2} (learned preconditioner)
    Geom<float> g;
    WaveGeom<float> w;
    Dev<float> d;
    int b0[PSE_BK], nb[PSE_BK];
};
void launch_batch_prologue_cells(const BSys *sys, int nsys, int *const *tab, const int *nblk, cudaStream_t s);
void launch_batch_nbr(const BSys *sys, int nsys, int *const *tab, const int *nblk, cudaStream_t s);
void launch_batch_init(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s);
void launch_batch_final(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s);
void launch_batch_noise(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s);
// P4 = the common support P (3..10) of node-major interpolation, 0 for the planar form
void launch_batch_interp(const BSys *sys, int *const *tab, const int *nblk, int P4, cudaStream_t s);
void launch_batch_pc_infer(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s);
void launch_lz_matvec_batch(const LzSys *sys, const int *blk2sys, int nblocks, cudaStream_t s);
void launch_lz_update_batch(const LzSys *sys, const int *blk2sys, int nblocks, cudaStream_t s);
void launch_lz_eig_batch(const LzSys *sys, int nsys, cudaStream_t s);
template <typename T> void launch_lz_final(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, bool with_wave,
                                           cudaStream_t s);
// plain matvec of a caller vector (sorted gather -> M_r -> scatter back)
template <typename T> void launch_matvec_caller(int64_t N, const SampleArgs<T> *args, Geom<T> g,
                                                const Dev<T> &d, cudaStream_t s);

// wave space
template <typename T> void launch_wave_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, void *spec,
                                             cudaStream_t s);
template <typename T> void launch_interp(int64_t N, WaveGeom<T> w, Geom<T> g, const Dev<T> &d, cudaStream_t s);
// fused k-space noise + three-pass C2R into the node-major grid (FP32,
// power-of-two M in 16..512); prepare once per M outside any capture
bool fused_fft_supported(int M);
cudaError_t fused_fft_prepare(int M);
// parts: bit 0 the noise + x pass, bit 1 the y pass, bit 2 the z pass
void launch_fused_fft(const WaveGeom<float> &w, const SampleArgs<float> *args, int system, const Dev<float> &d,
                      int parts, cudaStream_t s);
// resident blocks per SM of the FP32 4x4 matvec (its persistent grid is one wave of them)
int matvec_blocks_per_sm();
int update_blocks_per_sm();
void matvec_prepare();
// node-major copy of the velocity grid for the FP32 interpolation (no-op otherwise)
template <typename T> void launch_grid_copy(WaveGeom<T> w, const Dev<T> &d, cudaStream_t s);
enum { WAVE_MODE_DET = 0, WAVE_MODE_GRIDNOISE = 1 };
template <typename T>
void launch_wave_apply(WaveGeom<T> w, const SampleArgs<T> *args, int system, void *spec, int mode, int with_noise,
                       cudaStream_t s);
template <typename T>
void launch_grid_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, T *grid, cudaStream_t s);
size_t spread_smem_bytes(SpreadTile st, int P, size_t elem);
#define PSE_COVER 8  // tile blocks that may cover one grid node along one axis
// src: the vector to spread in sorted order (its q field), or null for the
// caller-order forces args->vin
template <typename T>
cudaError_t launch_spread(WaveGeom<T> w, Geom<T> g, SpreadTile st, const int *orig, const int2 *cover,
                          const int *cover_cnt, T *scratch, const Dev<T> &d, cudaStream_t s,
                          const Rec<T> *src = nullptr);
template <typename T> cudaError_t spread_prepare(size_t *max_dynamic);
template <typename T> void launch_matvec_sorted(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_gather_vec(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_det_final(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s);
template <typename T>
void launch_lz_final_forces(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_repulsion(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s);
template <typename T> void launch_advance(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s);

// learned preconditioner (float contexts)
void launch_pc_infer(int64_t N, Geom<float> g, const Dev<float> &d, const float *theta, float s0, float *pc,
                     cudaStream_t s);
void launch_pc_features(int64_t N, Geom<float> g, const Dev<float> &d, float *feat, float *tens, cudaStream_t s);
void launch_pc_targets(int64_t N, Geom<float> g, const Dev<float> &d, float *target, cudaStream_t s);
void launch_pc_blocks_caller(int64_t N, const Dev<float> &d, float *S, cudaStream_t s);

// symmetric 3x3 (xx, yy, zz, xy, xz, yz) times a vector
#ifdef __CUDACC__
__device__ __forceinline__ void sym3_apply(const float *M, float x, float y, float z, float &ox, float &oy,
                                           float &oz) {
    ox = M[0] * x + M[3] * y + M[4] * z;
    oy = M[3] * x + M[1] * y + M[5] * z;
    oz = M[4] * x + M[5] * y + M[2] * z;
}
#endif

// host-side setup (FP64 arithmetic)
void build_fg_table(double r_cut, double xi, double a, int n, double *F, double *G);
// Polydisperse pair (radii ai, aj): real-space scalars in mobility units on
// n uniform knots of [0, r_cut]; knot 0 holds the self term when ai = aj.
void build_fg_table_poly(double r_cut, double xi, double ai, double aj, int n, double *F, double *G);
double self_poly(double xi, double a);
void fg_at(double r, double xi, double a, double *F, double *G);
double self_real(double xi, double a);

}  // namespace pse
