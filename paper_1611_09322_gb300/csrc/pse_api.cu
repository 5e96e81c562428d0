// C ABI of libpse (include/pse.h): context, buffers, the per-sample CUDA
// graph and the entry points.
//
// One sample is one graph launch.  The graph forks after the cell sort:
//   real branch:  neighbour list -> WHILE { matvec -> update -> eig(T_j) }
//   wave branch:  k-space noise -> cuFFT C2R (x3) -> interpolation
// and joins in the final combination kernel.  The Lanczos loop runs on the
// device: after the matvec and update of step j, the eigen kernel (FP64, one
// warp) solves T_j, runs the stop test and sets the WHILE node's condition,
// so the host never waits inside a sample.  Per-call arguments (pointers,
// seed, sample index) live in a small device struct refreshed by one copy
// before launch.  The forces path (c_det M F + c_noise M^{1/2} z) adds M_r F
// on the real branch before the loop, and its wave branch spreads F, runs
// cuFFT R2C, applies the deterministic mode factor with the k-space noise
// fused in, then C2R and interpolation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "pse_internal.cuh"

using namespace pse;

struct pse_ctx {
    pse_params params;
    pse_plan_info plan;
    int device = 0;
    int max_iter = PSE_MAXIT;
    int64_t N = 0;       // size the per-N buffers and the graph were built for
    Dev<float> df{};
    Dev<double> dd{};
    Geom<float> gf{};
    Geom<double> gd{};
    WaveGeom<float> wf{};
    WaveGeom<double> wd{};
    int ncell3 = 0;
    cufftHandle fft = 0;
    bool fft_made = false;
    cudaStream_t s_main = nullptr, s_wave = nullptr, s_body = nullptr, s_init = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};  // fork of the wave branch; its join
    cudaEvent_t ev_init = nullptr;           // q_1 written beside the neighbour search
    cudaGraph_t graph[6] = {};            // per graph mode (GM_*)
    cudaGraphExec_t exec[6] = {};
    cudaGraphConditionalHandle cond[6] = {};
    cufftHandle fft_r2c = 0;                            // forward FFT (spreading / grid noise)
    bool r2c_made = false;
    bool fused_fft = false;                             // sample path: our noise + C2R kernels (FP32, M = 2^k)
    SpreadTile spread{};                                // spreading tile shape
    bool spread_ready = false, spread_tuned = false;
    size_t spread_smem_max = 0;                         // dynamic shared memory the spreading may use
    int *sp_orig = nullptr;                             // block origin of each tile index (ncell + 1)
    int2 *sp_cover = nullptr;                           // M * PSE_COVER (tile, offset) pairs
    int *sp_cnt = nullptr;                              // M: blocks covering each node
    void *sp_scratch = nullptr;                         // tile blocks of the two-phase spreading
    size_t sp_scratch_bytes = 0;
    bool sp_two_phase = false;
    bool mv_tuned = false;                              // matvec launch shape timed
    cudaStream_t last_stream = nullptr;
    void *stage_pos = nullptr, *stage_out = nullptr;  // device staging for the host-buffer call
    // pipelined host-buffer calls: two staging pairs, a copy stream, and per
    // pair the event of its input copy and of its sample
    void *stage_pos2 = nullptr, *stage_out2 = nullptr;
    cudaStream_t s_copy = nullptr, s_back = nullptr;  // input copies; result copies
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_back[2] = {nullptr, nullptr};
    bool host_used[2] = {false, false};
    int host_flip = 0;
    // per-call arguments go to the device from a ring of pinned host slots:
    // a copy from pageable memory would wait for the stream, so a call would
    // block until the previous sample is done
    unsigned char *args_ring = nullptr;
    cudaEvent_t ev_args[8] = {};
    bool args_used[8] = {};
    int args_slot = 0;
    std::vector<void *> per_n;                          // buffers freed when N changes
    std::vector<void *> per_ctx;                        // buffers freed at destroy
    bool pc_enabled = false;                            // learned preconditioner installed
    float pc_s0 = 0.f;                                  // self mobility^{-1/2}
    int nspec = 0;                                      // polydisperse: species radii (0: monodisperse)
    double radii[PSE_MAX_SPECIES] = {};
};

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) { return PSE_ECUDA; }        \
    } while (0)
#define CKF(call)                                           \
    do {                                                    \
        cufftResult r_ = (call);                            \
        if (r_ != CUFFT_SUCCESS) { return PSE_ECUFFT; }     \
    } while (0)

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr int PSE_ARGS_SLOTS = 8, PSE_ARGS_SLOT_BYTES = 256;
static_assert(sizeof(SampleArgs<double>) <= PSE_ARGS_SLOT_BYTES, "argument slot too small");
static_assert(PSE_ARGS_SLOTS == sizeof(pse_ctx::ev_args) / sizeof(cudaEvent_t), "argument ring size");

// Copy n bytes of per-call arguments to dst on s through the next pinned slot
// (waiting, on the host, only for that slot's copy of 8 calls ago).
cudaError_t push_args(pse_ctx *c, void *dst, const void *src, size_t n, cudaStream_t s);

template <typename T> Dev<T> &dev(pse_ctx *c);
template <> Dev<float> &dev<float>(pse_ctx *c) { return c->df; }
template <> Dev<double> &dev<double>(pse_ctx *c) { return c->dd; }
template <typename T> Geom<T> &geom(pse_ctx *c);
template <> Geom<float> &geom<float>(pse_ctx *c) { return c->gf; }
template <> Geom<double> &geom<double>(pse_ctx *c) { return c->gd; }
template <typename T> WaveGeom<T> &wgeom(pse_ctx *c);
template <> WaveGeom<float> &wgeom<float>(pse_ctx *c) { return c->wf; }
template <> WaveGeom<double> &wgeom<double>(pse_ctx *c) { return c->wd; }

pse_status alloc(std::vector<void *> &list, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return PSE_ENOMEM;
    }
    list.push_back(*p);
    return PSE_OK;
}

cudaError_t push_args(pse_ctx *c, void *dst, const void *src, size_t n, cudaStream_t s) {
    const int k = c->args_slot;
    c->args_slot = (k + 1) % PSE_ARGS_SLOTS;
    if (c->args_used[k]) {
        const cudaError_t e = cudaEventSynchronize(c->ev_args[k]);
        if (e != cudaSuccess) return e;
    }
    unsigned char *slot = c->args_ring + (size_t)k * PSE_ARGS_SLOT_BYTES;
    memcpy(slot, src, n);
    cudaError_t e = cudaMemcpyAsync(dst, slot, n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_args[k], s);
    c->args_used[k] = e == cudaSuccess;
    return e;
}

void free_list(std::vector<void *> &list) {
    for (void *p : list) cudaFree(p);
    list.clear();
}

// Graph modes: a plain sample; the forces path with and without noise; a
// Brownian step (overlap forces computed in the graph, positions advanced)
// with and without noise; Lanczos on the whole mobility (the comparison
// method of Sec. IV).
enum { GM_SAMPLE = 0, GM_FORCES_NOISE = 1, GM_FORCES = 2, GM_BD_NOISE = 3, GM_BD = 4, GM_FULL = 5, GM_COUNT = 6 };
static_assert(GM_COUNT == sizeof(pse_ctx::exec) / sizeof(cudaGraphExec_t), "graph mode table size");
static inline bool gm_noise(int m) { return m == GM_SAMPLE || m == GM_FORCES_NOISE || m == GM_BD_NOISE; }
static inline bool gm_bd(int m) { return m == GM_BD_NOISE || m == GM_BD; }

void drop_graph(pse_ctx *c) {
    for (int m = 0; m < GM_COUNT; ++m) {
        if (c->exec[m]) cudaGraphExecDestroy(c->exec[m]);
        if (c->graph[m]) cudaGraphDestroy(c->graph[m]);
        c->exec[m] = nullptr;
        c->graph[m] = nullptr;
    }
}

// Multiplier and shift for n / d, 32-bit n, d >= 2 (Granlund and Montgomery,
// PLDI 1994, round-up method): l = ceil(log2 d), m = 2^32 (2^l - d) / d + 1.
static void magic_div(uint32_t d, uint32_t *m, int *l) {
    int k = 0;
    while ((1ull << k) < d) ++k;
    *l = k;
    *m = (uint32_t)((((uint64_t)1 << 32) * ((1ull << k) - d)) / d + 1);
}

// Noise scale per n^2 = nx^2 + ny^2 + nz^2 (FP64): (sc(k), 1/|n|) with k =
// 2 pi |n| / L and sc(k) = V^{-1/2} sinc(ka)/k sqrt(1 + k^2/4xi^2)
// exp(-(1 - eta) k^2/8xi^2) (eq. Mwave, the Gaussian's share removed).
template <typename T> int64_t scale_table_len(const pse_plan_info &p) {
    const int h = p.M / 2;
    return 2 * (3ll * h * h + 1);
}
// a: the sphere radius of the shape factor (a species' radius in a
// polydisperse context); the table is appended to tab.
template <typename T> void build_scale_table(const pse_plan_info &p, double a, std::vector<T> &tab) {
    const int h = p.M / 2;
    const int64_t n = 3ll * h * h + 1;
    const size_t off = tab.size();
    tab.resize(off + 2 * n, T(0));
    T *out = tab.data() + off;
    const double ks = 2 * M_PI / p.L, inv_sqrtV = 1.0 / sqrt(p.L * p.L * p.L);
    for (int64_t n2 = 1; n2 < n; ++n2) {
        const double k = ks * sqrt((double)n2), ka = k * a, k2 = k * k;
        const double sc = inv_sqrtV * sin(ka) / (ka * k) * sqrt(1.0 + k2 / (4 * p.xi * p.xi)) *
                          exp(-(1 - p.eta) * k2 / (8 * p.xi * p.xi));
        out[2 * n2] = (T)sc;
        out[2 * n2 + 1] = (T)(1.0 / sqrt((double)n2));
    }
}

template <typename T> void fill_geom(pse_ctx *c) {
    const pse_plan_info &p = c->plan;
    Geom<T> g{};
    g.L = (T)p.L;
    const double cs = p.L / p.ncell;
    g.cs = (T)cs;
    g.cs_lo = (T)(cs - (double)(T)cs);
    g.inv_cs = (T)(p.ncell / p.L);
    g.rc2 = (T)(p.r_cut * p.r_cut);
    g.tab_inv_dr = (T)((PSE_TABLE_N - 1) / p.r_cut);
    const double split = 2 * p.a < p.r_cut ? 2 * p.a : p.r_cut;
    g.tc_split = (T)split;
    g.tc_invA = (T)(PSE_TABLEC_A / split);
    g.tc_invB = (T)((PSE_TABLEC_N - 1 - PSE_TABLEC_A) / (p.r_cut - split > 0 ? p.r_cut - split : 1.0));
    g.self_m = (T)p.self_mobility;
    g.a = (T)p.a;
    g.xi = (T)p.xi;
    g.nc = p.ncell;
    g.nb = bricks_per_side(p.ncell);
    // default launch shape: FP32 2 threads x 4 gathers per particle in blocks
    // of 1024 threads (one copy of the shared-memory table per SM leaves more
    // of it to the L1: 81 us per matvec at N = 1e6 against 86 for 4 x 4 and 95
    // for 4 x 4 in blocks of 128), FP64 4 x 4 in blocks of 128
    g.mv = c->params.matvec_shape > 0 ? c->params.matvec_shape - 1 : (sizeof(T) == 4 ? 9 : 0);
    g.rc2_d = p.r_cut * p.r_cut;
    g.L_d = p.L;
    g.invL_d = 1.0 / p.L;
    // the float path's band of float64 decisions at r_cut (none in FP64)
    g.rc2_lo = sizeof(T) == 4 ? (T)(g.rc2_d * (1.0 - 4e-6)) : g.rc2;
    g.rc2_hi = sizeof(T) == 4 ? (T)(g.rc2_d * (1.0 + 4e-6)) : g.rc2;
    g.nspec = c->nspec;
    for (int sp = 0; sp < c->nspec; ++sp) g.self_s[sp] = (T)self_poly(p.xi, c->radii[sp]);
    geom<T>(c) = g;
    WaveGeom<T> w{};
    w.M = p.M;
    w.P = p.P;
    w.Mh1 = p.M / 2 + 1;
    w.kscale = (T)(2 * M_PI / p.L);
    w.a = (T)p.a;
    w.inv4xi2 = (T)(1.0 / (4 * p.xi * p.xi));
    w.decay = (T)((1 - p.eta) / (8 * p.xi * p.xi));
    w.inv_sqrtV = (T)(1.0 / sqrt(p.L * p.L * p.L));
    const double gl = p.M / p.L;
    w.gl_hi = (T)gl;
    w.gl_lo = (T)(gl - (double)(T)gl);
    w.ch2 = (T)(2 * p.xi * p.xi * p.h * p.h / p.eta);
    w.norm = (T)(pow(2 * p.xi * p.xi / (M_PI * p.eta), 1.5) * p.h * p.h * p.h);
    w.inv_M15 = (T)pow((double)p.M, -1.5);
    const uint64_t nmodes = (uint64_t)p.M * p.M * (p.M / 2 + 1);
    w.big = nmodes >= (1ull << 32);
    magic_div((uint32_t)w.Mh1, &w.dv_h1_m, &w.dv_h1_l);
    magic_div((uint32_t)p.M, &w.dv_M_m, &w.dv_M_l);
    // 0: node-major grid copy + one warp per particle (FP32, P in 3..10)
    w.interp_lanes = (sizeof(T) == 4 && c->params.interp_form == 0 && p.P >= 3 && p.P <= 10) ? 0 : 16;
    w.nspec = c->nspec > 1 ? c->nspec : 1;
    w.sc_stride = scale_table_len<T>(p);
    wgeom<T>(c) = w;
}

// Per-context buffers: table, spectrum, grid, FFT plan, streams, events.
template <typename T> pse_status init_ctx(pse_ctx *c) {
    fill_geom<T>(c);
    matvec_prepare();

    Dev<T> &d = dev<T>(c);
    const pse_plan_info &p = c->plan;
    // F, G table in FP64, stored (F, G-F, dF, d(G-F)) / (6 pi a) in T; a
    // polydisperse context holds one block per species pair (mobility units)
    const int S = c->nspec > 1 ? c->nspec : 1, npair = c->nspec > 1 ? S * (S + 1) / 2 : 1;
    std::vector<V4<T>> tab((size_t)PSE_TABLE_N * npair);
    std::vector<double> F(PSE_TABLE_N), G(PSE_TABLE_N);
    for (int i0 = 0; i0 < S; ++i0)
        for (int j0 = i0; j0 < S; ++j0) {
            double s;
            if (c->nspec > 1) {
                build_fg_table_poly(p.r_cut, p.xi, c->radii[i0], c->radii[j0], PSE_TABLE_N, F.data(), G.data());
                s = 1.0;
            } else {
                build_fg_table(p.r_cut, p.xi, p.a, PSE_TABLE_N, F.data(), G.data());
                s = 1.0 / (6 * M_PI * p.a);
            }
            V4<T> *blk = tab.data() + (size_t)pair_index(i0, j0, S) * PSE_TABLE_N;
            for (int i = 0; i < PSE_TABLE_N; ++i) {
                const double f0 = F[i] * s, g0 = (G[i] - F[i]) * s;
                const double f1 = (i + 1 < PSE_TABLE_N) ? F[i + 1] * s : f0;
                const double g1 = (i + 1 < PSE_TABLE_N) ? (G[i + 1] - F[i + 1]) * s : g0;
                blk[i].x = (T)f0;
                blk[i].y = (T)g0;
                blk[i].z = (T)(f1 - f0);
                blk[i].w = (T)(g1 - g0);
            }
        }
    pse_status st;
    if ((st = alloc(c->per_ctx, (void **)&d.table, sizeof(V4<T>) * tab.size())) != PSE_OK) return st;
    CK(cudaMemcpy(d.table, tab.data(), sizeof(V4<T>) * tab.size(), cudaMemcpyHostToDevice));
    {  // compact two-segment table for the shared-memory matvec
        const double split = 2 * p.a < p.r_cut ? 2 * p.a : p.r_cut;
        const double dA = split / PSE_TABLEC_A;
        const double dB = (p.r_cut - split > 0 ? p.r_cut - split : 1.0) / (PSE_TABLEC_N - 1 - PSE_TABLEC_A);
        std::vector<double> Fc(PSE_TABLEC_N), Gc(PSE_TABLEC_N);
        for (int i = 0; i < PSE_TABLEC_N; ++i) {
            const double r = i <= PSE_TABLEC_A ? i * dA : split + (i - PSE_TABLEC_A) * dB;
            fg_at(r, p.xi, p.a, &Fc[i], &Gc[i]);
        }
        std::vector<V4<T>> tc(PSE_TABLEC_N);
        const double s = 1.0 / (6 * M_PI * p.a);
        for (int i = 0; i < PSE_TABLEC_N; ++i) {
            const double f0 = Fc[i] * s, g0 = (Gc[i] - Fc[i]) * s;
            const double f1 = (i + 1 < PSE_TABLEC_N) ? Fc[i + 1] * s : f0;
            const double g1 = (i + 1 < PSE_TABLEC_N) ? (Gc[i + 1] - Fc[i + 1]) * s : g0;
            tc[i].x = (T)f0;
            tc[i].y = (T)g0;
            tc[i].z = (T)(f1 - f0);
            tc[i].w = (T)(g1 - g0);
        }
        if ((st = alloc(c->per_ctx, (void **)&d.table_c, sizeof(V4<T>) * PSE_TABLEC_N)) != PSE_OK) return st;
        CK(cudaMemcpy(d.table_c, tc.data(), sizeof(V4<T>) * PSE_TABLEC_N, cudaMemcpyHostToDevice));
    }
    const int64_t M = p.M, plane = M * M * (M / 2 + 1);
    const size_t csize = sizeof(T) * 2;
    if ((st = alloc(c->per_ctx, &d.spec, csize * 3 * plane * S)) != PSE_OK) return st;
    if ((st = alloc(c->per_ctx, (void **)&d.grid, sizeof(T) * 3 * M * M * M * S)) != PSE_OK) return st;
    if constexpr (sizeof(T) == 4) {
        // power-of-two grids: the sample path's own inverse FFT (needs the
        // node-major grid of the interpolation)
        if (c->params.wave_fft == 1 && c->params.wave_noise == 0 && wgeom<T>(c).interp_lanes == 0 &&
            fused_fft_supported((int)M) && fused_fft_prepare((int)M) == cudaSuccess) {
            std::vector<float> tw(M);
            for (int64_t k = 0; k < M / 2; ++k) {
                tw[2 * k] = (float)cos(2 * M_PI * k / M);
                tw[2 * k + 1] = (float)sin(2 * M_PI * k / M);
            }
            float *d_tw = nullptr;
            if ((st = alloc(c->per_ctx, (void **)&d_tw, sizeof(float) * tw.size())) != PSE_OK) return st;
            CK(cudaMemcpy(d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice));
            wgeom<T>(c).fft_tw = d_tw;
            c->fused_fft = true;
        }
        cudaGetLastError();
    }
    {
        std::vector<T> sct;
        if (c->nspec > 1)
            for (int sp = 0; sp < S; ++sp) build_scale_table<T>(p, c->radii[sp], sct);
        else
            build_scale_table<T>(p, p.a, sct);
        T *d_sct = nullptr;
        if ((st = alloc(c->per_ctx, (void **)&d_sct, sizeof(T) * sct.size())) != PSE_OK) return st;
        CK(cudaMemcpy(d_sct, sct.data(), sizeof(T) * sct.size(), cudaMemcpyHostToDevice));
        wgeom<T>(c).sc_tab = d_sct;
    }
    if constexpr (sizeof(T) == 4)
        if (c->params.interp_form == 0 && p.P >= 3 && p.P <= 10 &&
            (st = alloc(c->per_ctx, (void **)&d.grid4, sizeof(V4<T>) * M * M * M * S)) != PSE_OK)
            return st;
    if ((st = alloc(c->per_ctx, (void **)&d.lz, sizeof(LzState))) != PSE_OK) return st;
    CK(cudaMemset(d.lz, 0, sizeof(LzState)));
    if ((st = alloc(c->per_ctx, (void **)&d.args, sizeof(SampleArgs<T>))) != PSE_OK) return st;
    if ((st = alloc(c->per_ctx, (void **)&d.scan_sums, sizeof(int) * PSE_SCAN_ITEMS)) != PSE_OK) return st;
    if ((st = alloc(c->per_ctx, (void **)&d.pc_theta, sizeof(float) * PSE_PRECOND_NPARAM)) != PSE_OK) return st;
    c->pc_s0 = (float)(1.0 / sqrt(p.self_mobility));
    int n[3] = {(int)M, (int)M, (int)M};
    CKF(cufftPlanMany(&c->fft, 3, n, nullptr, 1, (int)plane, nullptr, 1, (int)(M * M * M),
                      sizeof(T) == 4 ? CUFFT_C2R : CUFFT_Z2D, 3 * S));
    c->fft_made = true;
    // The real-space chain (cell list, neighbour list, Lanczos loop) is the
    // sample's critical path and its persistent kernels size their grids to
    // the whole GPU: its streams get the highest priority and the wave
    // branch the lowest, so that waiting wave blocks never take the SMs a
    // Lanczos step is about to use (graphs keep the captured priorities,
    // cudaGraphInstantiateFlagUseNodePriority): 1.336 -> 1.215 ms per sample
    // at N = 1e6, the same results bit for bit.
    int p_lo = 0, p_hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&p_lo, &p_hi));
    CK(cudaStreamCreateWithPriority(&c->s_main, cudaStreamNonBlocking, p_hi));
    CK(cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->s_back, cudaStreamNonBlocking));
    CK(cudaMallocHost((void **)&c->args_ring, (size_t)PSE_ARGS_SLOTS * PSE_ARGS_SLOT_BYTES));
    for (int k = 0; k < PSE_ARGS_SLOTS; ++k) CK(cudaEventCreateWithFlags(&c->ev_args[k], cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        CK(cudaEventCreateWithFlags(&c->ev_in[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_done[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_back[b], cudaEventDisableTiming));
    }
    CK(cudaStreamCreateWithPriority(&c->s_wave, cudaStreamNonBlocking, p_lo));
    CK(cudaStreamCreateWithPriority(&c->s_body, cudaStreamNonBlocking, p_hi));
    CK(cudaStreamCreateWithPriority(&c->s_init, cudaStreamNonBlocking, p_hi));
    CK(cudaEventCreateWithFlags(&c->ev_init, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) CK(cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming));
    return PSE_OK;
}

// Forward (R2C, batch 3) plan: grid -> spectrum, same layouts as the C2R plan.
template <typename T> pse_status ensure_r2c(pse_ctx *c) {
    if (c->r2c_made) return PSE_OK;
    const int M = c->plan.M;
    const int64_t plane = (int64_t)M * M * (M / 2 + 1);
    int n[3] = {M, M, M};
    CKF(cufftPlanMany(&c->fft_r2c, 3, n, nullptr, 1, M * M * M, nullptr, 1, (int)plane,
                      sizeof(T) == 4 ? CUFFT_R2C : CUFFT_D2Z, 3));
    c->r2c_made = true;
    return PSE_OK;
}

// Spreading tile: G^3 cells per CTA spread into a padded E^3 node block,
// E = ceil(G cs / h) + P + 2 (support of any particle of the tile, one node
// of margin each side), CP components per pass; the block must fit the
// dynamic shared memory a CTA may use (smem_max).
static bool spread_tile(const pse_plan_info &p, int G, int CP, size_t elem, size_t smem_max, SpreadTile *st) {
    const double cs = p.L / p.ncell;
    SpreadTile t;
    t.G = G;
    t.CP = CP;
    t.E = (int)ceil(G * cs / p.h) + p.P + 2;
    t.ntx = (p.ncell + G - 1) / G;
    if (spread_smem_bytes(t, p.P, elem) > smem_max) return false;
    *st = t;
    return true;
}

// Make tile t current: block origins of each tile index, the table of blocks
// covering each grid node and the scratch for the two-phase spreading (used
// when every node is covered by at most PSE_COVER blocks per axis and the
// scratch stays within 6 grids; otherwise the blocks are added with atomics).
template <typename T> pse_status set_spread_tile(pse_ctx *c, const SpreadTile &t) {
    const pse_plan_info &p = c->plan;
    const int M = p.M, ntx = t.ntx, E = t.E;
    const double cs = p.L / p.ncell;
    std::vector<int> orig(ntx);
    for (int k = 0; k < ntx; ++k) orig[k] = (int)floor(k * t.G * cs * M / p.L - 0.5 * p.P) + 1 - 1;
    std::vector<int2> cover((size_t)M * PSE_COVER, int2{0, 0});
    std::vector<int> cnt(M, 0);
    bool fits = true;
    for (int x = 0; x < M && fits; ++x)
        for (int k = 0; k < ntx && fits; ++k) {
            int l = (x - orig[k]) % M;
            if (l < 0) l += M;
            for (; l < E; l += M) {
                if (cnt[x] == PSE_COVER) { fits = false; break; }
                cover[(size_t)x * PSE_COVER + cnt[x]++] = int2{k, l};
            }
        }
    pse_status st;
    if (!c->sp_orig) {
        if ((st = alloc(c->per_ctx, (void **)&c->sp_orig, sizeof(int) * (p.ncell + 1))) != PSE_OK) return st;
        if ((st = alloc(c->per_ctx, (void **)&c->sp_cover, sizeof(int2) * M * PSE_COVER)) != PSE_OK) return st;
        if ((st = alloc(c->per_ctx, (void **)&c->sp_cnt, sizeof(int) * M)) != PSE_OK) return st;
    }
    CK(cudaMemcpy(c->sp_orig, orig.data(), sizeof(int) * ntx, cudaMemcpyHostToDevice));
    const size_t need = sizeof(T) * 3 * (size_t)ntx * ntx * ntx * (size_t)E * E * E;
    const size_t grid_bytes = sizeof(T) * 3 * (size_t)M * M * M;
    c->sp_two_phase = fits && need <= 6 * grid_bytes;
    if (c->sp_two_phase) {
        CK(cudaMemcpy(c->sp_cover, cover.data(), sizeof(int2) * M * PSE_COVER, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->sp_cnt, cnt.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
        if (need > c->sp_scratch_bytes) {
            if (c->sp_scratch) {
                cudaDeviceSynchronize();
                cudaFree(c->sp_scratch);
            }
            c->sp_scratch = nullptr;
            c->sp_scratch_bytes = 0;
            if (cudaMalloc(&c->sp_scratch, need) != cudaSuccess) {
                cudaGetLastError();
                c->sp_scratch = nullptr;
                c->sp_two_phase = false;
            } else {
                c->sp_scratch_bytes = need;
            }
        }
    }
    c->spread = t;
    drop_graph(c);
    return PSE_OK;
}

template <typename T>
cudaError_t run_spread(pse_ctx *c, const SpreadTile &t, cudaStream_t s, const Rec<T> *src = nullptr) {
    Dev<T> &d = dev<T>(c);
    const bool tp = c->sp_two_phase;
    return launch_spread<T>(wgeom<T>(c), geom<T>(c), t, c->sp_orig, tp ? c->sp_cover : nullptr,
                            tp ? c->sp_cnt : nullptr, tp ? (T *)c->sp_scratch : nullptr, d, s, src);
}

// Default: the largest tile that holds all three components, else the
// largest holding one; spread_tile = 1, 2, 4 forces that many cells per side.
template <typename T> pse_status choose_spread(pse_ctx *c) {
    if (c->spread_ready) return PSE_OK;
    CK(spread_prepare<T>(&c->spread_smem_max));
    const int Gs[3] = {4, 2, 1};
    const int want = c->params.spread_tile;
    bool ok = false;
    for (int CP : {3, 1}) {
        for (int G : Gs)
            if ((want == 0 || want == G) && spread_tile(c->plan, G, CP, sizeof(T), c->spread_smem_max, &c->spread)) {
                ok = true;
                break;
            }
        if (ok) break;
    }
    if (!ok) return PSE_ENOTSUPPORTED;
    pse_status st = set_spread_tile<T>(c, c->spread);
    if (st != PSE_OK) return st;
    c->spread_ready = true;
    return PSE_OK;
}

// Per-N buffers.
template <typename T> pse_status ensure(pse_ctx *c, int64_t N) {
    if (N == c->N) return PSE_OK;
    if (c->last_stream) cudaStreamSynchronize(c->last_stream);
    cudaDeviceSynchronize();
    drop_graph(c);
    free_list(c->per_n);
    c->N = 0;
    Dev<T> &d = dev<T>(c);
    const pse_plan_info &p = c->plan;
    const int64_t nc3 = cell_slots(p.ncell);
    c->ncell3 = (int)nc3;
    // list entries are (sorted index << 6) | stencil code, non-negative below 2^25 particles
    if (nc3 + 1 > PSE_MAX_SCAN || N + 1 > PSE_MAX_SCAN || N >= (1 << 25)) return PSE_EINVAL;
    // neighbour capacity: spheres of radius a within r_cut + a, at most a
    // close-packed fraction of that ball, plus slack for small overlaps
    const double rr = p.r_cut / p.a + 1.0;
    int64_t per = (int64_t)ceil(0.8 * rr * rr * rr) + 32;
    int64_t cap = N * per;
    if (cap > 0x7fffffffLL) cap = 0x7fffffffLL;
    d.nbr_cap = cap;
    pse_status st;
#define A(ptr, bytes) \
    if ((st = alloc(c->per_n, (void **)&(ptr), (bytes))) != PSE_OK) return st
    A(d.pos_sorted, sizeof(V4<T>) * N);
    A(d.loc_sorted, sizeof(V4<T>) * N);
    A(d.cell_of, sizeof(int) * N);
    A(d.slot, sizeof(int) * N);
    A(d.perm, sizeof(int) * N);
    A(d.cell_count, sizeof(int) * nc3);
    A(d.cell_start, sizeof(int) * (nc3 + 1));
    A(d.nbr_count, sizeof(int) * N);
    A(d.nbr, sizeof(int) * cap);
    d.edge_cap = (int)(4096 + N / 128);
    A(d.edge, sizeof(int4) * d.edge_cap);
    A(d.edge_n, sizeof(int));
    CK(cudaMemset(d.edge_n, 0, sizeof(int)));
    A(d.basis, sizeof(V4<T>) * N * (c->max_iter + 2));
    A(d.u, sizeof(V4<T>) * N);
    A(d.rec, sizeof(Rec<T>) * N);
    A(d.pc, sizeof(float) * 16 * N);
    d.pc_on = c->pc_enabled ? d.pc : nullptr;
    A(d.uwave, sizeof(V4<T>) * N);
    A(d.udet, sizeof(V4<T>) * N);
    A(d.bd_force, sizeof(T) * 3 * N);
    A(d.bd_dx, sizeof(T) * 3 * N);
    A(d.partials, sizeof(double) * (2 * num_sms() * 16 + 64));
    A(c->stage_pos, sizeof(T) * 3 * N);
    A(c->stage_out, sizeof(T) * 3 * N);
    A(c->stage_pos2, sizeof(T) * 3 * N);
    A(c->stage_out2, sizeof(T) * 3 * N);
    c->host_used[0] = c->host_used[1] = false;
#undef A
    c->N = N;
    return PSE_OK;
}

// Kernels before the fork: bin, scan, scatter, per-cell sort, q_1 = z1.
template <typename T> void pre(pse_ctx *c, int64_t N, cudaStream_t s) {
    Dev<T> &d = dev<T>(c);
    launch_bin<T>(N, d.args, geom<T>(c), d, s);
    launch_scatter<T>(N, d.args, geom<T>(c), d, s);
    launch_place<T>(N, d.args, geom<T>(c), d, s);
    cudaMemsetAsync(&d.lz->overflow, 0, sizeof(int), s);
    cudaMemsetAsync(&d.lz->n_pairs, 0, sizeof(unsigned long long), s);
}

// After the neighbour list: preconditioner blocks (if installed), then q_1 = z1.
template <typename T> void real_setup(pse_ctx *c, int64_t N, cudaStream_t s) {
    Dev<T> &d = dev<T>(c);
    if constexpr (sizeof(T) == 4) {
        if (c->pc_enabled) launch_pc_infer(N, c->gf, c->df, c->df.pc_theta, c->pc_s0, c->df.pc, s);
    }
    launch_lz_init<T>(N, d.args, c->params.system, d, s);
}

template <typename T> void interp(pse_ctx *c, int64_t N, cudaStream_t s) {
    launch_grid_copy<T>(wgeom<T>(c), dev<T>(c), s);
    launch_interp<T>(N, wgeom<T>(c), geom<T>(c), dev<T>(c), s);
}

// The wave branch on `s`.  `sorted` (may be null): an event the
// interpolation waits for -- the noise, the FFTs and the grid copy do not
// read the positions and may run before the cell list is done.
template <typename T>
pse_status wave_branch(pse_ctx *c, int64_t N, cudaStream_t s, int mode, cudaEvent_t sorted = nullptr) {
    Dev<T> &d = dev<T>(c);
    const WaveGeom<T> &w = wgeom<T>(c);
    if constexpr (sizeof(T) == 4) {
        if (mode == GM_SAMPLE && c->fused_fft) {
            launch_fused_fft(w, d.args, c->params.system, d, 7, s);
            if (sorted) cudaStreamWaitEvent(s, sorted, 0);
            launch_interp<T>(N, w, geom<T>(c), d, s);
            return PSE_OK;
        }
    }
    if (mode == GM_SAMPLE && c->params.wave_noise == 0) {
        launch_wave_noise<T>(w, d.args, c->params.system, d.spec, s);
    } else {
        const int64_t M3 = (int64_t)w.M * w.M * w.M;
        if (mode == GM_SAMPLE) {
            launch_grid_noise<T>(w, d.args, c->params.system, d.grid, s);
        } else {
            CK(cudaMemsetAsync(d.grid, 0, sizeof(T) * 3 * M3, s));
            CK(run_spread<T>(c, c->spread, s));
        }
        CKF(cufftSetStream(c->fft_r2c, s));
        if constexpr (sizeof(T) == 4) {
            CKF(cufftExecR2C(c->fft_r2c, (cufftReal *)d.grid, (cufftComplex *)d.spec));
        } else {
            CKF(cufftExecD2Z(c->fft_r2c, (cufftDoubleReal *)d.grid, (cufftDoubleComplex *)d.spec));
        }
        launch_wave_apply<T>(w, d.args, c->params.system, d.spec,
                             mode == GM_SAMPLE ? WAVE_MODE_GRIDNOISE : WAVE_MODE_DET, gm_noise(mode), s);
    }
    CKF(cufftSetStream(c->fft, s));
    if constexpr (sizeof(T) == 4) {
        CKF(cufftExecC2R(c->fft, (cufftComplex *)d.spec, (cufftReal *)d.grid));
    } else {
        CKF(cufftExecZ2D(c->fft, (cufftDoubleComplex *)d.spec, (cufftDoubleReal *)d.grid));
    }
    launch_grid_copy<T>(w, d, s);
    if (sorted) cudaStreamWaitEvent(s, sorted, 0);
    launch_interp<T>(N, w, geom<T>(c), d, s);
    return PSE_OK;
}

// Capture pieces of one sample.  The prologue runs on c->s_main (which must
// be capturing): cell list, wave branch forked onto c->s_wave, neighbour
// list, preconditioner blocks and q_1.  The loop body is one Lanczos step
// (matvec -> update -> eigen-solve of T_j, all on `sa`).  The
// epilogue joins the wave branch and writes the output.
// The list-free matvec (FP32 monodisperse sampling without preconditioner)
// needs no neighbour list: the sample then builds none.
template <typename T> bool nolist_sample(pse_ctx *c, int mode) {
    const Geom<T> &g = geom<T>(c);
    return sizeof(T) == 4 && mode == GM_SAMPLE && g.mv == PSE_MV_NOLIST && g.nspec <= 1 && !dev<T>(c).pc_on;
}

template <typename T> pse_status capture_pre(pse_ctx *c, int mode) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    cudaStream_t s = c->s_main;
    // a sample's wave branch forks before the cell list (its noise and FFTs
    // do not read the positions); the forces' branch spreads the sorted
    // forces and forks after it
    const bool early = mode == GM_SAMPLE;
    if (early) {
        cudaEventRecord(c->ev[1], s);
        cudaStreamWaitEvent(c->s_wave, c->ev[1], 0);
    }
    pre<T>(c, N, s);
    if (gm_bd(mode)) {  // the forces need the neighbour list before the wave branch spreads them
        launch_nbr<T>(N, geom<T>(c), d, s);
        launch_repulsion<T>(N, geom<T>(c), d, s);
    }
    cudaEventRecord(c->ev[0], s);
    if (!early) cudaStreamWaitEvent(c->s_wave, c->ev[0], 0);
    const pse_status wst = wave_branch<T>(c, N, c->s_wave, mode, early ? c->ev[0] : nullptr);
    cudaEventRecord(c->ev[1], c->s_wave);
    // a plain sample's q_1 = z1 needs only the sorted order: it is drawn beside
    // the neighbour search (which reads the offsets, not the records' q);
    // with the preconditioner it needs the blocks, which need the list
    const bool init_beside = mode == GM_SAMPLE && !c->pc_enabled;
    if (init_beside) {
        cudaStreamWaitEvent(c->s_init, c->ev[0], 0);
        launch_lz_init<T>(N, d.args, c->params.system, d, c->s_init);
        cudaEventRecord(c->ev_init, c->s_init);
    }
    if (!gm_bd(mode) && !nolist_sample<T>(c, mode)) launch_nbr<T>(N, geom<T>(c), d, s);
    if (mode != GM_SAMPLE) {  // M_r F into udet (the records are overwritten by q_1 next)
        launch_gather_vec<T>(N, d.args, d, s);
        launch_matvec_sorted<T>(N, geom<T>(c), d, s);
    }
    if (init_beside) cudaStreamWaitEvent(s, c->ev_init, 0);
    else if (gm_noise(mode)) real_setup<T>(c, N, s);
    return wst;
}

template <typename T>
void capture_body(pse_ctx *c, cudaStream_t sa, cudaGraphConditionalHandle h) {
    Dev<T> &d = dev<T>(c);
    const double ltol = c->params.lanczos_tol > 0 ? c->params.lanczos_tol : c->plan.tol;
    launch_lz_matvec<T>(c->N, geom<T>(c), d, sa);
    launch_lz_update<T>(c->N, c->max_iter, d, sa);
    launch_lz_eig(d.lz, c->max_iter, c->params.fixed_iter, ltol, h, sa);
}

template <typename T> void capture_post(pse_ctx *c, int mode) {
    Dev<T> &d = dev<T>(c);
    cudaStreamWaitEvent(c->s_main, c->ev[1], 0);
    if (mode == GM_SAMPLE) launch_lz_final<T>(c->N, d.args, d, true, c->s_main);
    else if (gm_noise(mode)) launch_lz_final_forces<T>(c->N, d.args, d, c->s_main);
    else launch_det_final<T>(c->N, d.args, d, c->s_main);
    if (gm_bd(mode)) launch_advance<T>(c->N, geom<T>(c), d, c->s_main);
}

// Insert a WHILE node (default condition 1) at the capture point of `s`;
// returns its handle and body graph, and makes `s` continue after it.
static cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle *h, cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    e = cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = *h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// One whole sample on c->s_main (capturing): prologue, a WHILE node whose
// body is one Lanczos step with the eigen kernel setting the condition, and
// the epilogue.
template <typename T> pse_status capture_sample(pse_ctx *c, int mode) {
    const pse_status wst = capture_pre<T>(c, mode);
    if (!gm_noise(mode)) {
        capture_post<T>(c, mode);
        return wst;
    }
    cudaGraph_t body = nullptr;
    cudaError_t e = add_while(c->s_main, &c->cond[mode], &body);
    if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(c->s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            capture_body<T>(c, c->s_body, c->cond[mode]);
            cudaGraph_t body_out = nullptr;
            e = cudaStreamEndCapture(c->s_body, &body_out);
        }
    }
    capture_post<T>(c, mode);
    if (wst != PSE_OK) return wst;
    return e == cudaSuccess ? PSE_OK : PSE_ECUDA;
}

// One step of Lanczos on the whole mobility M = M_r + M_w (Sec. IV's
// comparison method), on `s`: the wave product of the current vector q_j
// (spread from the matvec records, forward FFT, the deterministic mode
// factor of Sec. III, inverse FFT, interpolation into uwave), then the
// near-field matvec with uwave added to its rows (so alpha_j = q_j . M q_j),
// the three-term update and the eigen-solve with the stop test.
template <typename T> pse_status full_step(pse_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    const WaveGeom<T> &w = wgeom<T>(c);
    const int64_t M3 = (int64_t)w.M * w.M * w.M;
    const double ltol = c->params.lanczos_tol > 0 ? c->params.lanczos_tol : c->plan.tol;
    CK(cudaMemsetAsync(d.grid, 0, sizeof(T) * 3 * M3, s));
    CK(run_spread<T>(c, c->spread, s, d.rec));
    CKF(cufftSetStream(c->fft_r2c, s));
    if constexpr (sizeof(T) == 4) {
        CKF(cufftExecR2C(c->fft_r2c, (cufftReal *)d.grid, (cufftComplex *)d.spec));
    } else {
        CKF(cufftExecD2Z(c->fft_r2c, (cufftDoubleReal *)d.grid, (cufftDoubleComplex *)d.spec));
    }
    launch_wave_apply<T>(w, d.args, c->params.system, d.spec, WAVE_MODE_DET, 0, s);
    CKF(cufftSetStream(c->fft, s));
    if constexpr (sizeof(T) == 4) {
        CKF(cufftExecC2R(c->fft, (cufftComplex *)d.spec, (cufftReal *)d.grid));
    } else {
        CKF(cufftExecZ2D(c->fft, (cufftDoubleComplex *)d.spec, (cufftDoubleReal *)d.grid));
    }
    interp<T>(c, N, s);
    Dev<T> da = d;
    da.mv_add = d.uwave;
    launch_lz_matvec<T>(N, geom<T>(c), da, s);
    launch_lz_update<T>(N, c->max_iter, d, s);
    launch_lz_eig(d.lz, c->max_iter, c->params.fixed_iter, ltol, h, s);
    return PSE_OK;
}

// The full-mobility sample on c->s_main (capturing): cell and neighbour
// lists, q_1 = z1, a WHILE node whose body is one full_step, and the final
// combination x = ||z1|| V_J T_J^{1/2} e_1 in caller order.
template <typename T> pse_status capture_full(pse_ctx *c) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    cudaStream_t s = c->s_main;
    pre<T>(c, N, s);
    launch_nbr<T>(N, geom<T>(c), d, s);
    launch_lz_init<T>(N, d.args, c->params.system, d, s);
    cudaGraph_t body = nullptr;
    pse_status st = PSE_OK;
    cudaError_t e = add_while(s, &c->cond[GM_FULL], &body);
    if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(c->s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = full_step<T>(c, c->s_body, c->cond[GM_FULL]);
            cudaGraph_t body_out = nullptr;
            e = cudaStreamEndCapture(c->s_body, &body_out);
        }
    }
    launch_lz_final<T>(N, d.args, d, false, s);
    if (st != PSE_OK) return st;
    return e == cudaSuccess ? PSE_OK : PSE_ECUDA;
}

template <typename T> pse_status build_graph(pse_ctx *c, int mode) {
    cudaStream_t s = c->s_main;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const pse_status st = mode == GM_FULL ? capture_full<T>(c) : capture_sample<T>(c, mode);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (st != PSE_OK || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st != PSE_OK ? st : PSE_ECUDA;
    }
    c->graph[mode] = graph;
    if (cudaGraphInstantiate(&c->exec[mode], graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(c);
        return PSE_ECUDA;
    }
    return PSE_OK;
}

// Same kernels, launched directly with a host-side Lanczos loop (one
// synchronisation per iteration).  Used when use_graph = -1.
template <typename T> pse_status run_plain(pse_ctx *c, cudaStream_t s, int mode) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    const double ltol = c->params.lanczos_tol > 0 ? c->params.lanczos_tol : c->plan.tol;
    pre<T>(c, N, s);
    launch_nbr<T>(N, geom<T>(c), d, s);
    if (gm_bd(mode)) launch_repulsion<T>(N, geom<T>(c), d, s);
    pse_status st = wave_branch<T>(c, N, s, mode);
    if (st != PSE_OK) return st;
    if (mode != GM_SAMPLE) {
        launch_gather_vec<T>(N, d.args, d, s);
        launch_matvec_sorted<T>(N, geom<T>(c), d, s);
    }
    if (!gm_noise(mode)) {
        launch_det_final<T>(N, d.args, d, s);
        if (gm_bd(mode)) launch_advance<T>(N, geom<T>(c), d, s);
        return PSE_OK;
    }
    real_setup<T>(c, N, s);
    for (int it = 0; it < c->max_iter + 2; ++it) {
        launch_lz_matvec<T>(N, geom<T>(c), d, s);
        launch_lz_update<T>(N, c->max_iter, d, s);
        launch_lz_eig(d.lz, c->max_iter, c->params.fixed_iter, ltol, 0, s);
        int cont = 0;
        CK(cudaMemcpyAsync(&cont, &d.lz->cont, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!cont) break;
    }
    if (mode == GM_SAMPLE) launch_lz_final<T>(N, d.args, d, true, s);
    else launch_lz_final_forces<T>(N, d.args, d, s);
    if (gm_bd(mode)) launch_advance<T>(N, geom<T>(c), d, s);
    return PSE_OK;
}

// The full-mobility sample with plain launches and a host-side loop (one
// synchronisation per iteration): use_graph = -1.
template <typename T> pse_status run_full_plain(pse_ctx *c, cudaStream_t s) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    pre<T>(c, N, s);
    launch_nbr<T>(N, geom<T>(c), d, s);
    launch_lz_init<T>(N, d.args, c->params.system, d, s);
    for (int it = 0; it < c->max_iter + 2; ++it) {
        const pse_status st = full_step<T>(c, s, 0);
        if (st != PSE_OK) return st;
        int cont = 0;
        CK(cudaMemcpyAsync(&cont, &d.lz->cont, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!cont) break;
    }
    launch_lz_final<T>(N, d.args, d, false, s);
    return PSE_OK;
}

// Time each matvec launch shape (3 launches after one warm-up) on the
// current call's neighbour list and keep the fastest.  Needs d.args set.
template <typename T> pse_status tune_matvec(pse_ctx *c, cudaStream_t s) {
    const int64_t N = c->N;
    Dev<T> &d = dev<T>(c);
    pre<T>(c, N, s);
    launch_nbr<T>(N, geom<T>(c), d, s);
    real_setup<T>(c, N, s);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // two sweeps over the shapes, 8 timed launches each after 2 warm-ups; a
    // shape's time is its better sweep (robust to a slow first pass)
    float t[PSE_MV_VARIANTS];
    for (int v = 0; v < PSE_MV_VARIANTS; ++v) t[v] = 1e30f;
    Geom<T> g = geom<T>(c);
    for (int sweep = 0; sweep < 2; ++sweep)
        for (int v = 0; v < PSE_MV_VARIANTS; ++v) {
            g.mv = v;
            for (int rep = 0; rep < 10; ++rep) {
                if (rep == 2) cudaEventRecord(e0, s);
                launch_lz_matvec<T>(N, g, d, s);
            }
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess) continue;
            cudaEventElapsedTime(&ms, e0, e1);
            t[v] = ms < t[v] ? ms : t[v];
        }
    int keep = 0;
    for (int v = 1; v < PSE_MV_VARIANTS; ++v)
        if (t[v] < t[keep]) keep = v;
    geom<T>(c).mv = keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->mv_tuned = true;
    drop_graph(c);
    CK(cudaGetLastError());
    return PSE_OK;
}

template <typename T>
pse_status sample_impl(pse_ctx *c, int64_t N, const T *pos, uint64_t seed, uint64_t sample, T *out, T *real,
                       T *wave, cudaStream_t s, const int *species = nullptr) {
    if (!pos || N < 1) return PSE_EINVAL;
    if (!out && !real && !wave) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    pse_status st = ensure<T>(c, N);
    if (st != PSE_OK) return st;
    if (c->params.wave_noise == 1 && (st = ensure_r2c<T>(c)) != PSE_OK) return st;
    const bool use_graph = c->params.use_graph >= 0;
    if (use_graph && !c->exec[GM_SAMPLE]) {
        st = build_graph<T>(c, GM_SAMPLE);
        if (st != PSE_OK) return st;
    }
    SampleArgs<T> a{};
    a.pos = pos;
    a.out = out;
    a.real = real;
    a.wave = wave;
    a.vin = nullptr;
    a.seed = seed;
    a.sample = sample;
    a.c_det = 0.0;
    a.c_noise = 1.0;
    a.species = species;
    CK(push_args(c, dev<T>(c).args, &a, sizeof(a), s));
    if ((c->params.autotune & 4) && c->params.matvec_shape == 0 && !c->mv_tuned && c->nspec < 2) {
        if ((st = tune_matvec<T>(c, s)) != PSE_OK) return st;
        if (use_graph && (st = build_graph<T>(c, GM_SAMPLE)) != PSE_OK) return st;
    }
    if (use_graph) {
        CK(cudaGraphLaunch(c->exec[GM_SAMPLE], s));
    } else {
        st = run_plain<T>(c, s, GM_SAMPLE);
        if (st != PSE_OK) return st;
    }
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

template <typename T>
pse_status full_impl(pse_ctx *c, int64_t N, const T *pos, uint64_t seed, uint64_t sample, T *out, cudaStream_t s) {
    if (!pos || !out || N < 1) return PSE_EINVAL;
    if (c->pc_enabled) return PSE_ENOTSUPPORTED;  // the comparison method runs on M itself
    DeviceGuard guard(c->device);
    pse_status st = ensure<T>(c, N);
    if (st != PSE_OK) return st;
    if ((st = ensure_r2c<T>(c)) != PSE_OK) return st;
    if ((st = choose_spread<T>(c)) != PSE_OK) return st;
    SampleArgs<T> a{};
    a.pos = pos;
    a.out = out;
    a.seed = seed;
    a.sample = sample;
    a.c_det = 1.0;  // the mode factor of the wave product, unscaled
    a.c_noise = 0.0;
    CK(push_args(c, dev<T>(c).args, &a, sizeof(a), s));
    const bool use_graph = c->params.use_graph >= 0;
    if (use_graph && !c->exec[GM_FULL]) {
        st = build_graph<T>(c, GM_FULL);
        if (st != PSE_OK) return st;
    }
    if (use_graph) {
        CK(cudaGraphLaunch(c->exec[GM_FULL], s));
    } else {
        st = run_full_plain<T>(c, s);
        if (st != PSE_OK) return st;
    }
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

// Time every tile shape that fits (3 spreads each after one warm-up) on the
// cell list of the current call and keep the fastest.
template <typename T> pse_status tune_spread(pse_ctx *c, cudaStream_t s) {
    Dev<T> &d = dev<T>(c);
    const int64_t M3 = (int64_t)c->plan.M * c->plan.M * c->plan.M;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    SpreadTile keep = c->spread;
    for (int CP : {3, 1})
        for (int G : {4, 2, 1}) {
            SpreadTile t;
            if (!spread_tile(c->plan, G, CP, sizeof(T), c->spread_smem_max, &t)) continue;
            if (set_spread_tile<T>(c, t) != PSE_OK) continue;
            float ms = 0.f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                if (rep == 1) cudaEventRecord(e0, s);
                ok = cudaMemsetAsync(d.grid, 0, sizeof(T) * 3 * M3, s) == cudaSuccess &&
                     run_spread<T>(c, t, s) == cudaSuccess;
            }
            cudaEventRecord(e1, s);
            if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                keep = t;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    c->spread_tuned = true;
    return set_spread_tile<T>(c, keep);
}

template <typename T>
pse_status bd_impl(pse_ctx *c, int64_t N, T *pos, const T *fext, double dt, double kT, double k_rep, uint64_t seed,
                   uint64_t step, cudaStream_t s) {
    if (!pos || N < 1) return PSE_EINVAL;
    if (!(dt >= 0.0) || !(kT >= 0.0) || !(k_rep >= 0.0) || !isfinite(dt) || !isfinite(kT) || !isfinite(k_rep))
        return PSE_EINVAL;
    if (kT > 0.0 && c->params.wave_noise == 1) return PSE_ENOTSUPPORTED;
    if (k_rep > 0.0 && c->plan.r_cut < 2.0 * c->plan.a) return PSE_ENOTSUPPORTED;  // contacts beyond the list
    DeviceGuard guard(c->device);
    pse_status st = ensure<T>(c, N);
    if (st != PSE_OK) return st;
    if ((st = ensure_r2c<T>(c)) != PSE_OK) return st;
    if ((st = choose_spread<T>(c)) != PSE_OK) return st;
    const int mode = kT > 0.0 ? GM_BD_NOISE : GM_BD;
    Dev<T> &d = dev<T>(c);
    SampleArgs<T> a{};
    a.pos = pos;
    a.out = d.bd_dx;
    a.vin = d.bd_force;
    a.advance = pos;
    a.fext = fext;
    a.k_rep = k_rep;
    a.seed = seed;
    a.sample = step;
    a.c_det = dt;
    a.c_noise = sqrt(2.0 * kT * dt);
    CK(push_args(c, d.args, &a, sizeof(a), s));
    const bool use_graph = c->params.use_graph >= 0;
    if (use_graph && !c->exec[mode]) {
        st = build_graph<T>(c, mode);
        if (st != PSE_OK) return st;
    }
    if (use_graph) {
        CK(cudaGraphLaunch(c->exec[mode], s));
    } else {
        st = run_plain<T>(c, s, mode);
        if (st != PSE_OK) return st;
    }
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

template <typename T>
pse_status forces_impl(pse_ctx *c, int64_t N, const T *pos, const T *force, uint64_t seed, uint64_t sample,
                       double c_det, double c_noise, T *out, cudaStream_t s) {
    if (!pos || !force || !out || N < 1) return PSE_EINVAL;
    if (!(c_det == c_det) || !(c_noise == c_noise)) return PSE_EINVAL;
    if (c_noise != 0.0 && c->params.wave_noise == 1) return PSE_ENOTSUPPORTED;
    DeviceGuard guard(c->device);
    pse_status st = ensure<T>(c, N);
    if (st != PSE_OK) return st;
    if ((st = ensure_r2c<T>(c)) != PSE_OK) return st;
    if ((st = choose_spread<T>(c)) != PSE_OK) return st;
    const int mode = c_noise != 0.0 ? GM_FORCES_NOISE : GM_FORCES;
    SampleArgs<T> a{};
    a.pos = pos;
    a.out = out;
    a.vin = force;
    a.seed = seed;
    a.sample = sample;
    a.c_det = c_det;
    a.c_noise = c_noise;
    CK(push_args(c, dev<T>(c).args, &a, sizeof(a), s));
    if ((c->params.autotune & 2) && c->params.spread_tile == 0 && !c->spread_tuned) {
        pre<T>(c, N, s);
        if ((st = tune_spread<T>(c, s)) != PSE_OK) return st;
    }
    const bool use_graph = c->params.use_graph >= 0;
    if (use_graph && !c->exec[mode]) {
        st = build_graph<T>(c, mode);
        if (st != PSE_OK) return st;
    }
    if (use_graph) {
        CK(cudaGraphLaunch(c->exec[mode], s));
    } else {
        st = run_plain<T>(c, s, mode);
        if (st != PSE_OK) return st;
    }
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

static int smooth_2357(int n) {
    const int pr[4] = {2, 3, 5, 7};
    for (int i = 0; i < 4; ++i) while (n % pr[i] == 0) n /= pr[i];
    return n == 1;
}

// Device time (ms) of one cuFFT C2R (batch 3) on each grid Ms[i], the mean of
// 3 transforms after one warm-up; 1e30 where no plan or memory was had.
template <typename T> void time_fft_sizes(const int *Ms, int n, float *ms_out) {
    int Mmax = 0;
    for (int i = 0; i < n; ++i) {
        ms_out[i] = 1e30f;
        if (Ms[i] > Mmax) Mmax = Ms[i];
    }
    const size_t cbytes = sizeof(T) * 2 * 3 * (size_t)Mmax * Mmax * (Mmax / 2 + 1);
    const size_t rbytes = sizeof(T) * 3 * (size_t)Mmax * Mmax * Mmax;
    void *spec = nullptr, *grid = nullptr;
    if (cudaMalloc(&spec, cbytes) != cudaSuccess || cudaMalloc(&grid, rbytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(spec);
        return;
    }
    cudaMemset(spec, 0, cbytes);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < n; ++i) {
        const int M = Ms[i];
        cufftHandle h;
        int dims[3] = {M, M, M};
        if (cufftPlanMany(&h, 3, dims, nullptr, 1, M * M * (M / 2 + 1), nullptr, 1, M * M * M,
                          sizeof(T) == 4 ? CUFFT_C2R : CUFFT_Z2D, 3) != CUFFT_SUCCESS)
            continue;
        float ms = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) cudaEventRecord(e0, 0);
            if constexpr (sizeof(T) == 4) cufftExecC2R(h, (cufftComplex *)spec, (cufftReal *)grid);
            else cufftExecZ2D(h, (cufftDoubleComplex *)spec, (cufftDoubleReal *)grid);
        }
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        cufftDestroy(h);
        ms_out[i] = ms / 3.f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(spec);
    cudaFree(grid);
    cudaGetLastError();
}

// Fastest cuFFT C2R (batch 3) grid among the 2,3,5,7-smooth sizes in
// [M, 1.12 M] (a finer grid only lowers the quadrature error).
template <typename T> pse_status tune_fft_size(int M0, int *best_M) {
    *best_M = M0;
    int Ms[64], n = 0;
    for (int M = M0; M <= (int)(M0 * 1.12) + 1 && n < 64; ++M)
        if (smooth_2357(M)) Ms[n++] = M;
    float ms[64];
    time_fft_sizes<T>(Ms, n, ms);
    float best = 1e30f;
    for (int i = 0; i < n; ++i)
        if (ms[i] < best) {
            best = ms[i];
            *best_M = Ms[i];
        }
    return PSE_OK;
}

// Largest xi whose Sec. II C plan fits a grid of M points per side
// (k_cut L / pi <= M, eta <= 1, r_cut < L/2), by bisection: the three
// conditions bound xi from above, above and below.  0 if none fits.
double xi_max_for_grid(double L, double a, const pse_params &p0, int M) {
    pse_params p = p0;
    p.grid_M = M;
    auto fits = [&](double xi) {
        p.xi = xi;
        pse_plan_info pl;
        if (pse_plan(L, a, &p, &pl) != PSE_OK) return false;
        return ceil(pl.k_cut * L / 3.141592653589793 - 1e-9) <= M;
    };
    double lo = sqrt(log(1.0 / p0.tol)) / (0.5 * L) * (1.0 + 1e-9);
    if (!fits(lo)) return 0.0;
    double hi = 2.0 * lo;
    while (fits(hi)) {
        lo = hi;
        hi *= 2.0;
        if (hi > 1e6 / a) return lo;
    }
    for (int it = 0; it < 50; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (fits(mid)) lo = mid;
        else hi = mid;
    }
    return lo;
}

pse_status create_impl(pse_ctx **out, double L, double a, const pse_params *p, int nspec = 0,
                       const double *radii = nullptr) {
    if (!out) return PSE_EINVAL;
    *out = nullptr;
    if (!p) return PSE_EINVAL;
    pse_ctx *c = new (std::nothrow) pse_ctx();
    if (!c) return PSE_ENOMEM;
    c->params = *p;
    c->nspec = nspec;
    for (int sp = 0; sp < nspec; ++sp) c->radii[sp] = radii[sp];
    pse_status st = pse_plan(L, a, p, &c->plan);
    if (st != PSE_OK) { delete c; return st; }
    if ((p->autotune & 1) && p->grid_M <= 0) {
        int Mbest = c->plan.M;
        st = (p->precision == PSE_FP64) ? tune_fft_size<double>(c->plan.M, &Mbest) : tune_fft_size<float>(c->plan.M, &Mbest);
        if (st == PSE_OK && Mbest != c->plan.M) {
            c->params.grid_M = Mbest;
            st = pse_plan(L, a, &c->params, &c->plan);
            if (st != PSE_OK) { delete c; return st; }
        }
    }
    if (p->autotune & 8) {  // the largest xi the final grid admits: same wave cost, shorter r_cut
        const double xi = xi_max_for_grid(L, a, c->params, c->plan.M);
        if (xi > c->plan.xi) {
            c->params.xi = xi;
            c->params.grid_M = c->plan.M;
            st = pse_plan(L, a, &c->params, &c->plan);
            if (st != PSE_OK) { delete c; return st; }
        }
    }
    if (p->max_iter < 0 || p->max_iter > PSE_MAXIT || p->fixed_iter < 0 || p->fixed_iter > PSE_MAXIT ||
        p->system < 0 || p->system > 0x3fffffff) {
        delete c;
        return PSE_EINVAL;
    }
    c->max_iter = p->max_iter > 0 ? p->max_iter : PSE_MAXIT;
    if (c->params.fixed_iter > c->max_iter) c->max_iter = c->params.fixed_iter;
    if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); delete c; return PSE_ECUDA; }
    if (p->wave_noise < 0 || p->wave_noise > 1 ||
        !(p->spread_tile == 0 || p->spread_tile == 1 || p->spread_tile == 2 || p->spread_tile == 4) ||
        p->matvec_shape < 0 || p->matvec_shape > PSE_MV_NOLIST + 1 || p->interp_form < 0 || p->interp_form > 1 ||
        p->wave_fft < 0 || p->wave_fft > 1) {
        delete c;
        return PSE_EINVAL;
    }
    if (nspec > 1 && (c->plan.P < 3 || c->plan.P > 10)) {  // species grids need the node-major interpolation
        delete c;
        return PSE_ENOTSUPPORTED;
    }
    st = (p->precision == PSE_FP64) ? init_ctx<double>(c) : init_ctx<float>(c);
    if (st != PSE_OK) { pse_destroy(c); return st; }
    *out = c;
    return PSE_OK;
}

// Polydisperse contexts hold species tables and grids; the monodisperse
// entry points (and the forces, Brownian, full-mobility and preconditioner
// paths) are not available for them.
inline bool poly_ctx(const pse_ctx *c) { return c && c->nspec > 1; }

}  // namespace

extern "C" {

pse_status pse_create_ex(pse_ctx **out, double L, double a, const pse_params *p) {
    return create_impl(out, L, a, p);
}

pse_status pse_create_poly(pse_ctx **out, double L, int n_species, const double *radii, const pse_params *p) {
    if (!out) return PSE_EINVAL;
    *out = nullptr;
    if (!p || !radii || n_species < 1 || n_species > PSE_MAX_SPECIES) return PSE_EINVAL;
    double amin = radii[0];
    for (int sp = 0; sp < n_species; ++sp) {
        if (!(radii[sp] > 0) || !isfinite(radii[sp])) return PSE_EINVAL;
        amin = radii[sp] < amin ? radii[sp] : amin;
    }
    if (n_species > 1 && (p->precision != PSE_FP32 || p->wave_noise != 0 || p->wave_fft != 0 ||
                          p->interp_form != 0 || p->use_precond != 0))
        return PSE_ENOTSUPPORTED;
    // one species is the monodisperse sampler at that radius
    return create_impl(out, L, amin, p, n_species, radii);
}

pse_status pse_get_species(const pse_ctx *c, int *n_species, double *radii) {
    if (!c || !n_species) return PSE_EINVAL;
    *n_species = c->nspec;
    for (int sp = 0; sp < c->nspec && radii; ++sp) radii[sp] = c->radii[sp];
    return PSE_OK;
}

pse_status pse_sample_poly(pse_ctx *c, int64_t N, const float *d_pos, const int *d_species, uint64_t seed,
                           uint64_t sample_index, float *d_out, float *d_real, float *d_wave, void *stream) {
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    if (c->nspec < 1) return PSE_ENOTSUPPORTED;  // a monodisperse context: use pse_sample
    if (!d_species) return PSE_EINVAL;
    return sample_impl<float>(c, N, d_pos, seed, sample_index, d_out, d_real, d_wave, (cudaStream_t)stream,
                              d_species);
}

pse_status pse_real_matvec_poly(pse_ctx *c, int64_t N, const float *d_pos, const int *d_species, const float *d_v,
                                float *d_out, void *stream) {
    if (!c) return PSE_EINVAL;
    if (c->plan.precision != PSE_FP32 || c->nspec < 1) return PSE_ENOTSUPPORTED;
    if (!d_pos || !d_species || !d_v || !d_out || N < 1) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    SampleArgs<float> a{};
    a.pos = d_pos;
    a.out = d_out;
    a.vin = d_v;
    a.species = d_species;
    CK(push_args(c, c->df.args, &a, sizeof(a), s));
    pre<float>(c, N, s);
    launch_nbr<float>(N, c->gf, c->df, s);
    launch_matvec_caller<float>(N, c->df.args, c->gf, c->df, s);
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

pse_status pse_create(pse_ctx **out, double L, double a, double xi, double tol) {
    pse_params p;
    memset(&p, 0, sizeof(p));
    p.tol = tol;
    p.xi = xi;
    p.precision = PSE_FP32;
    return create_impl(out, L, a, &p);
}

void pse_destroy(pse_ctx *c) {
    if (!c) return;
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    drop_graph(c);
    if (c->fft_made) cufftDestroy(c->fft);
    if (c->r2c_made) cufftDestroy(c->fft_r2c);
    if (c->sp_scratch) cudaFree(c->sp_scratch);
    free_list(c->per_n);
    free_list(c->per_ctx);
    cudaStream_t ss[6] = {c->s_main, c->s_wave, c->s_body, c->s_copy, c->s_back, c->s_init};
    for (cudaStream_t s : ss) if (s) cudaStreamDestroy(s);
    for (int b = 0; b < 2; ++b) {
        if (c->ev_in[b]) cudaEventDestroy(c->ev_in[b]);
        if (c->ev_done[b]) cudaEventDestroy(c->ev_done[b]);
        if (c->ev_back[b]) cudaEventDestroy(c->ev_back[b]);
    }
    for (int k = 0; k < PSE_ARGS_SLOTS; ++k)
        if (c->ev_args[k]) cudaEventDestroy(c->ev_args[k]);
    if (c->args_ring) cudaFreeHost(c->args_ring);
    for (cudaEvent_t e : c->ev) if (e) cudaEventDestroy(e);
    if (c->ev_init) cudaEventDestroy(c->ev_init);
    delete c;
}

pse_status pse_get_plan(const pse_ctx *c, pse_plan_info *out) {
    if (!c || !out) return PSE_EINVAL;
    *out = c->plan;
    return PSE_OK;
}

pse_status pse_sample(pse_ctx *c, int64_t N, const float *d_pos, uint64_t seed, uint64_t sample_index, float *d_out,
                      void *stream) {
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    if (!d_out) return PSE_EINVAL;
    return sample_impl<float>(c, N, d_pos, seed, sample_index, d_out, nullptr, nullptr, (cudaStream_t)stream);
}

pse_status pse_sample_parts(pse_ctx *c, int64_t N, const float *d_pos, uint64_t seed, uint64_t sample_index,
                            float *d_out, float *d_real, float *d_wave, void *stream) {
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return sample_impl<float>(c, N, d_pos, seed, sample_index, d_out, d_real, d_wave, (cudaStream_t)stream);
}

pse_status pse_sample_f64(pse_ctx *c, int64_t N, const double *d_pos, uint64_t seed, uint64_t sample_index,
                          double *d_out, double *d_real, double *d_wave, void *stream) {
    if (!c || c->plan.precision != PSE_FP64) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return sample_impl<double>(c, N, d_pos, seed, sample_index, d_out, d_real, d_wave, (cudaStream_t)stream);
}

pse_status pse_sample_with_forces(pse_ctx *c, int64_t N, const float *d_pos, const float *d_force, uint64_t seed,
                                  uint64_t sample_index, double c_det, double c_noise, float *d_out, void *stream) {
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return forces_impl<float>(c, N, d_pos, d_force, seed, sample_index, c_det, c_noise, d_out, (cudaStream_t)stream);
}

pse_status pse_sample_with_forces_f64(pse_ctx *c, int64_t N, const double *d_pos, const double *d_force,
                                      uint64_t seed, uint64_t sample_index, double c_det, double c_noise,
                                      double *d_out, void *stream) {
    if (!c || c->plan.precision != PSE_FP64) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return forces_impl<double>(c, N, d_pos, d_force, seed, sample_index, c_det, c_noise, d_out,
                               (cudaStream_t)stream);
}

pse_status pse_bd_step(pse_ctx *c, int64_t N, float *d_pos, const float *d_fext, double dt, double kT,
                       double k_rep, uint64_t seed, uint64_t step, void *stream) {
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return bd_impl<float>(c, N, d_pos, d_fext, dt, kT, k_rep, seed, step, (cudaStream_t)stream);
}

pse_status pse_bd_step_f64(pse_ctx *c, int64_t N, double *d_pos, const double *d_fext, double dt, double kT,
                           double k_rep, uint64_t seed, uint64_t step, void *stream) {
    if (!c || c->plan.precision != PSE_FP64) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return bd_impl<double>(c, N, d_pos, d_fext, dt, kT, k_rep, seed, step, (cudaStream_t)stream);
}

pse_status pse_sample_full_lanczos(pse_ctx *c, int64_t N, const float *d_pos, uint64_t seed, uint64_t sample_index,
                                   float *d_out, void *stream) {
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return full_impl<float>(c, N, d_pos, seed, sample_index, d_out, (cudaStream_t)stream);
}

pse_status pse_sample_full_lanczos_f64(pse_ctx *c, int64_t N, const double *d_pos, uint64_t seed,
                                       uint64_t sample_index, double *d_out, void *stream) {
    if (!c || c->plan.precision != PSE_FP64) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    return full_impl<double>(c, N, d_pos, seed, sample_index, d_out, (cudaStream_t)stream);
}

pse_status pse_mobility_apply(pse_ctx *c, int64_t N, const float *d_pos, const float *d_force, float *d_out,
                              void *stream) {
    return pse_sample_with_forces(c, N, d_pos, d_force, 0, 0, 1.0, 0.0, d_out, stream);
}

pse_status pse_sample_host(pse_ctx *c, int64_t N, const float *h_pos, uint64_t seed, uint64_t sample_index,
                           float *h_out, void *stream) {
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!h_pos || !h_out || N < 1) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    CK(cudaMemcpyAsync(c->stage_pos, h_pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s));
    st = sample_impl<float>(c, N, (const float *)c->stage_pos, seed, sample_index, (float *)c->stage_out, nullptr,
                            nullptr, s);
    if (st != PSE_OK) return st;
    CK(cudaMemcpyAsync(h_out, c->stage_out, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return PSE_OK;
}

pse_status pse_real_matvec(pse_ctx *c, int64_t N, const float *d_pos, const float *d_v, float *d_out,
                           void *stream) {
    if (!c) return PSE_EINVAL;
    if (c->plan.precision != PSE_FP32 || poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!d_pos || !d_v || !d_out || N < 1) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    SampleArgs<float> a{};
    a.pos = d_pos;
    a.out = d_out;
    a.vin = d_v;
    CK(push_args(c, c->df.args, &a, sizeof(a), s));
    pre<float>(c, N, s);
    launch_nbr<float>(N, c->gf, c->df, s);
    launch_matvec_caller<float>(N, c->df.args, c->gf, c->df, s);
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

pse_status pse_profile_stages(pse_ctx *c, int64_t N, const float *d_pos, uint64_t seed, uint64_t sample_index,
                              float *d_out, double *ms, int *launches, void *stream) {
    if (!c) return PSE_EINVAL;
    if (c->plan.precision != PSE_FP32 || poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!d_pos || !d_out || !ms || !launches || N < 1) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    Dev<float> &d = c->df;
    SampleArgs<float> a{};
    a.pos = d_pos;
    a.out = d_out;
    a.seed = seed;
    a.sample = sample_index;
    a.c_noise = 1.0;
    CK(push_args(c, d.args, &a, sizeof(a), s));
    if (c->params.wave_noise == 1 && (st = ensure_r2c<float>(c)) != PSE_OK) return st;
    const double ltol = c->params.lanczos_tol > 0 ? c->params.lanczos_tol : c->plan.tol;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int i = 0; i < PSE_NSTAGES; ++i) { ms[i] = 0.0; launches[i] = 0; }
    auto timed = [&](int stage, int nl, auto &&fn) -> pse_status {
        if (cudaEventRecord(e0, s) != cudaSuccess) return PSE_ECUDA;
        pse_status r = fn();
        if (r != PSE_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess) return PSE_ECUDA;
        if (cudaEventSynchronize(e1) != cudaSuccess) return PSE_ECUDA;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[stage] += t;
        launches[stage] += nl;
        return PSE_OK;
    };
    const int nscan = 3;
    pse_status r = PSE_OK;
    if (r == PSE_OK) r = timed(PSE_STAGE_CELLS, 1 + nscan, [&] { launch_bin<float>(N, d.args, c->gf, d, s); return PSE_OK; });
    if (r == PSE_OK) r = timed(PSE_STAGE_SORT, 2, [&] {
        launch_scatter<float>(N, d.args, c->gf, d, s);
        launch_place<float>(N, d.args, c->gf, d, s);
        cudaMemsetAsync(&d.lz->overflow, 0, sizeof(int), s);
        cudaMemsetAsync(&d.lz->n_pairs, 0, sizeof(unsigned long long), s);
        return PSE_OK; });
    const bool fused = c->fused_fft;
    if (r == PSE_OK) r = timed(PSE_STAGE_WAVE_NOISE, c->params.wave_noise ? 2 : 1, [&] {
        if (fused) {  // noise generated inside the first FFT pass (x)
            launch_fused_fft(c->wf, d.args, c->params.system, d, 1, s);
            return PSE_OK;
        }
        if (c->params.wave_noise == 0) {
            launch_wave_noise<float>(c->wf, d.args, c->params.system, d.spec, s);
            return PSE_OK;
        }
        launch_grid_noise<float>(c->wf, d.args, c->params.system, d.grid, s);
        CKF(cufftSetStream(c->fft_r2c, s));
        CKF(cufftExecR2C(c->fft_r2c, (cufftReal *)d.grid, (cufftComplex *)d.spec));
        launch_wave_apply<float>(c->wf, d.args, c->params.system, d.spec, WAVE_MODE_GRIDNOISE, 0, s);
        return PSE_OK; });
    if (r == PSE_OK) r = timed(PSE_STAGE_FFT, fused ? 2 : 0, [&] {
        if (fused) {  // y and z passes, the last one writing the node-major grid
            launch_fused_fft(c->wf, d.args, c->params.system, d, 6, s);
            return PSE_OK;
        }
        CKF(cufftSetStream(c->fft, s));
        CKF(cufftExecC2R(c->fft, (cufftComplex *)d.spec, (cufftReal *)d.grid));
        return PSE_OK; });
    if (r == PSE_OK)
        r = timed(PSE_STAGE_GRID_COPY, (c->wf.interp_lanes == 0 && !fused) ? 1 : 0, [&] {
            if (!fused) launch_grid_copy<float>(c->wf, c->df, s);
            return PSE_OK; });
    if (r == PSE_OK)
        r = timed(PSE_STAGE_INTERP, 1, [&] { launch_interp<float>(N, c->wf, c->gf, c->df, s); return PSE_OK; });
    if (r == PSE_OK) r = timed(PSE_STAGE_NEIGHBOURS, 1, [&] {
        launch_nbr<float>(N, c->gf, d, s);
        return PSE_OK; });
    if (r == PSE_OK) r = timed(PSE_STAGE_REAL_NOISE, c->pc_enabled ? 2 : 1, [&] {
        real_setup<float>(c, N, s);
        return PSE_OK; });
    for (int it = 0; r == PSE_OK && it < c->max_iter + 2; ++it) {
        r = timed(PSE_STAGE_MATVEC, 1, [&] { launch_lz_matvec<float>(N, c->gf, d, s); return PSE_OK; });
        if (r == PSE_OK) r = timed(PSE_STAGE_LANCZOS_UPDATE, 1, [&] { launch_lz_update<float>(N, c->max_iter, d, s); return PSE_OK; });
        if (r == PSE_OK) r = timed(PSE_STAGE_EIGEN, 1, [&] {
            launch_lz_eig(d.lz, c->max_iter, c->params.fixed_iter, ltol, 0, s);
            return PSE_OK; });
        int cont = 0;
        if (r == PSE_OK && cudaMemcpy(&cont, &d.lz->cont, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) r = PSE_ECUDA;
        if (!cont) break;
    }
    if (r == PSE_OK) r = timed(PSE_STAGE_FINAL, 1, [&] { launch_lz_final<float>(N, d.args, d, true, s); return PSE_OK; });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->last_stream = s;
    if (r != PSE_OK) return r;
    CK(cudaGetLastError());
    return PSE_OK;
}

// ---------------------------------------------------------------- choice of xi
// Mean device time of `reps` samples of a fresh context with parameters p
// (two untimed samples first: graph capture and launch-shape tuning), its
// Lanczos count and grid; with `stage`, also the times of one staged sample's
// neighbour list + matvecs, k-space noise and FFT.
static pse_status xi_trial(double L, double a, const pse_params &p, int64_t N, const float *d_pos, float *d_out,
                           int reps, cudaStream_t s, double *ms, int *iters, int *M, double *stage) {
    pse_ctx *c = nullptr;
    pse_status st = create_impl(&c, L, a, &p);
    if (st != PSE_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pse_stats stats;
    for (int i = 0; st == PSE_OK && i < 2; ++i) st = pse_sample(c, N, d_pos, 1, 900000 + i, d_out, s);
    if (st == PSE_OK) st = pse_get_stats(c, &stats);
    if (st == PSE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = PSE_ECUDA;
    if (st == PSE_OK && cudaEventRecord(e0, s) != cudaSuccess) st = PSE_ECUDA;
    for (int i = 0; st == PSE_OK && i < reps; ++i) st = pse_sample(c, N, d_pos, 1, 900002 + i, d_out, s);
    if (st == PSE_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = PSE_ECUDA;
    if (st == PSE_OK) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        st = pse_get_stats(c, &stats);
        *iters = stats.lanczos_iters;
        *M = c->plan.M;
    }
    if (st == PSE_OK && stage) {
        double sm[PSE_NSTAGES];
        int nl[PSE_NSTAGES];
        st = pse_profile_stages(c, N, d_pos, 1, 900001, d_out, sm, nl, s);
        stage[0] = sm[PSE_STAGE_NEIGHBOURS] + sm[PSE_STAGE_MATVEC];
        stage[1] = sm[PSE_STAGE_WAVE_NOISE];
        stage[2] = sm[PSE_STAGE_FFT];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pse_destroy(c);
    return st;
}

static int planned_grid(double L, double a, const pse_params &p0, double xi) {
    pse_params p = p0;
    p.xi = xi;
    p.grid_M = 0;
    pse_plan_info pl;
    return pse_plan(L, a, &p, &pl) == PSE_OK ? pl.M : 0;
}

pse_status pse_tune_xi(double L, double a, const pse_params *p, int64_t N, const float *d_pos, double d_f, int reps,
                       pse_xi_tuning *out, void *stream) {
    if (!p || !out || !d_pos || N < 1) return PSE_EINVAL;
    memset(out, 0, sizeof(*out));
    if (p->precision != PSE_FP32 || p->use_precond) return PSE_ENOTSUPPORTED;
    if (d_f == 0.0) d_f = 3.0;
    if (!(d_f >= 1.0 && d_f <= 3.0) || !(a > 0) || reps < 0 || reps > 1000) return PSE_EINVAL;
    if (reps == 0) reps = 5;
    cudaStream_t s = (cudaStream_t)stream;
    float *d_out = nullptr;
    CK(cudaMalloc(&d_out, sizeof(float) * 3 * N));
    const double xi0 = p->xi > 0 ? p->xi : 0.5 / a;
    pse_params p0 = *p;
    p0.xi = xi0;
    p0.autotune &= ~8;  // every trial keeps the xi it is given
    out->xi_start = xi0;
    double stage[3];
    pse_status st = xi_trial(L, a, p0, N, d_pos, d_out, reps, s, &out->ms_tried[0], &out->iters_tried[0],
                             &out->M_tried[0], stage);
    if (st == PSE_OK) {
        out->t_real = stage[0];
        out->t_wave = stage[1] + stage[2];
        st = pse_xi_model(xi0, out->t_real, out->t_wave, d_f, &out->xi_model);
    }
    if (st != PSE_OK) {
        cudaFree(d_out);
        return st;
    }
    out->xi_tried[0] = xi0;
    out->ms_pred[0] = out->ms_tried[0];
    out->ms_start = out->ms_tried[0];
    const int M0 = out->M_tried[0];
    // Candidate grids: the smooth sizes the plan gives between 0.75 and 1.35
    // times xi*.  On a fixed grid the wave part costs the same for every xi
    // that fits it while the real part shrinks as xi grows, so each grid is
    // taken at the largest xi it admits.
    pse_params pg = p0;
    pg.autotune &= ~1;  // the grid is fixed per candidate
    int Mlo = 0;
    for (double f = 0.75; f < 1.4 && !Mlo; f += 0.05) Mlo = planned_grid(L, a, pg, out->xi_model * f);
    int Mhi = planned_grid(L, a, pg, out->xi_model * 1.35);
    if (!Mlo) Mlo = M0;
    if (!Mhi || Mhi < Mlo) Mhi = Mlo;
    int Ms[PSE_XI_GRIDS];
    double xis[PSE_XI_GRIDS];
    int ng = 0;
    for (int M = Mlo; M <= Mhi && ng < PSE_XI_GRIDS; ++M) {
        if (!smooth_2357(M)) continue;
        const double xi = xi_max_for_grid(L, a, pg, M);
        if (xi <= 0.0) continue;
        Ms[ng] = M;
        xis[ng++] = xi;
    }
    out->n_grids = ng;
    float fft_ms[PSE_XI_GRIDS];
    time_fft_sizes<float>(Ms, ng, fft_ms);
    // predicted sample time per grid: eq. work's xi-dependent terms from the
    // start context, the FFT as timed, the rest unchanged
    double pred[PSE_XI_GRIDS];
    for (int i = 0; i < ng; ++i)
        pred[i] = out->ms_start - out->t_real - out->t_wave + out->t_real * pow(xi0 / xis[i], d_f) +
                  stage[1] * pow((double)Ms[i] / M0, 3) + fft_ms[i];
    int k = 1;
    for (; k < PSE_XI_TRIALS; ++k) {  // time the best predictions in order
        int b = -1;
        for (int i = 0; i < ng; ++i)
            if (pred[i] < 1e29 && (b < 0 || pred[i] < pred[b])) b = i;
        if (b < 0) break;
        pse_params pt = pg;
        pt.xi = xis[b];
        pt.grid_M = Ms[b];
        out->xi_tried[k] = xis[b];
        out->ms_pred[k] = pred[b];
        pred[b] = 1e30;
        const pse_status r = xi_trial(L, a, pt, N, d_pos, d_out, reps, s, &out->ms_tried[k], &out->iters_tried[k],
                                      &out->M_tried[k], nullptr);
        if (r == PSE_ECUDA || r == PSE_ECUFFT) {
            cudaFree(d_out);
            return r;
        }
        if (r != PSE_OK) {  // not usable: list overflow, no convergence within max_iter
            out->ms_tried[k] = -1.0;
            out->M_tried[k] = Ms[b];
        }
    }
    out->n_tried = k;
    out->xi_best = xi0;
    out->M_best = M0;
    out->ms_best = out->ms_start;
    for (int i = 1; i < k; ++i)
        if (out->ms_tried[i] > 0 && out->ms_tried[i] < out->ms_best) {
            out->ms_best = out->ms_tried[i];
            out->xi_best = out->xi_tried[i];
            out->M_best = out->M_tried[i];
        }
    cudaFree(d_out);
    CK(cudaGetLastError());
    return PSE_OK;
}

// ---------------------------------------------------------------- learned preconditioner
static pse_status pc_prepare(pse_ctx *c, int64_t N, const float *d_pos, cudaStream_t s) {
    if (!c) return PSE_EINVAL;
    if (c->plan.precision != PSE_FP32) return PSE_ENOTSUPPORTED;
    if (!d_pos || N < 1) return PSE_EINVAL;
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    SampleArgs<float> a{};
    a.pos = d_pos;
    CK(push_args(c, c->df.args, &a, sizeof(a), s));
    pre<float>(c, N, s);
    launch_nbr<float>(N, c->gf, c->df, s);
    return PSE_OK;
}

pse_status pse_precond_features(pse_ctx *c, int64_t N, const float *d_pos, float *d_feat, float *d_tens,
                                void *stream) {
    if (!d_feat || !d_tens) return PSE_EINVAL;
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    DeviceGuard guard(c ? c->device : 0);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = pc_prepare(c, N, d_pos, s);
    if (st != PSE_OK) return st;
    launch_pc_features(N, c->gf, c->df, d_feat, d_tens, s);
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

pse_status pse_precond_targets(pse_ctx *c, int64_t N, const float *d_pos, float *d_target, void *stream) {
    if (!d_target) return PSE_EINVAL;
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    DeviceGuard guard(c ? c->device : 0);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = pc_prepare(c, N, d_pos, s);
    if (st != PSE_OK) return st;
    launch_pc_targets(N, c->gf, c->df, d_target, s);
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

pse_status pse_precond_set_weights(pse_ctx *c, const float *h_theta, int nparam) {
    if (!c) return PSE_EINVAL;
    if (c->plan.precision != PSE_FP32 || poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (h_theta && nparam != PSE_PRECOND_NPARAM) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    CK(cudaDeviceSynchronize());
    if (h_theta) CK(cudaMemcpy(c->df.pc_theta, h_theta, sizeof(float) * PSE_PRECOND_NPARAM, cudaMemcpyHostToDevice));
    c->pc_enabled = h_theta != nullptr;
    c->df.pc_on = (c->pc_enabled && c->N > 0) ? c->df.pc : nullptr;
    drop_graph(c);  // kernel arguments changed
    return PSE_OK;
}

pse_status pse_precond_blocks(pse_ctx *c, int64_t N, const float *d_pos, float *d_S, void *stream) {
    if (!d_S) return PSE_EINVAL;
    if (c && !c->pc_enabled) return PSE_ENOTREADY;
    DeviceGuard guard(c ? c->device : 0);
    cudaStream_t s = (cudaStream_t)stream;
    pse_status st = pc_prepare(c, N, d_pos, s);
    if (st != PSE_OK) return st;
    launch_pc_infer(N, c->gf, c->df, c->df.pc_theta, c->pc_s0, c->df.pc, s);
    launch_pc_blocks_caller(N, c->df, d_S, s);
    c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

pse_status pse_sample_host_async(pse_ctx *c, int64_t N, const float *h_pos, uint64_t seed, uint64_t sample_index,
                                 float *h_out, void *stream) {
    if (!c || c->plan.precision != PSE_FP32) return c ? PSE_ENOTSUPPORTED : PSE_EINVAL;
    if (poly_ctx(c)) return PSE_ENOTSUPPORTED;
    if (!h_pos || !h_out || N < 1) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (N != c->N) CK(cudaDeviceSynchronize());  // staging buffers are re-allocated for a new N
    pse_status st = ensure<float>(c, N);
    if (st != PSE_OK) return st;
    const int b = c->host_flip;
    c->host_flip ^= 1;
    float *dp = (float *)(b ? c->stage_pos2 : c->stage_pos), *dout = (float *)(b ? c->stage_out2 : c->stage_out);
    const size_t bytes = sizeof(float) * 3 * N;
    // pair b was last used two calls ago: its sample must be done before its
    // input is overwritten, and its result copied out before its output is
    // (the result copies run on their own stream, in call order, so an input
    // copy never queues behind the result copy of the sample still running)
    if (c->host_used[b]) {
        CK(cudaStreamWaitEvent(c->s_copy, c->ev_done[b], 0));
        CK(cudaStreamWaitEvent(s, c->ev_back[b], 0));
    }
    CK(cudaMemcpyAsync(dp, h_pos, bytes, cudaMemcpyHostToDevice, c->s_copy));
    CK(cudaEventRecord(c->ev_in[b], c->s_copy));
    CK(cudaStreamWaitEvent(s, c->ev_in[b], 0));
    st = sample_impl<float>(c, N, dp, seed, sample_index, dout, nullptr, nullptr, s);
    if (st != PSE_OK) return st;
    CK(cudaEventRecord(c->ev_done[b], s));
    c->host_used[b] = true;
    CK(cudaStreamWaitEvent(c->s_back, c->ev_done[b], 0));
    CK(cudaMemcpyAsync(h_out, dout, bytes, cudaMemcpyDeviceToHost, c->s_back));
    CK(cudaEventRecord(c->ev_back[b], c->s_back));
    return PSE_OK;
}

pse_status pse_host_sync(pse_ctx *c) {
    if (!c) return PSE_EINVAL;
    DeviceGuard guard(c->device);
    CK(cudaStreamSynchronize(c->s_copy));
    CK(cudaStreamSynchronize(c->s_back));
    return PSE_OK;
}

pse_status pse_get_stats(pse_ctx *c, pse_stats *out) {
    if (!c || !out) return PSE_EINVAL;
    memset(out, 0, sizeof(*out));
    if (c->N == 0) return PSE_OK;
    DeviceGuard guard(c->device);
    if (c->last_stream) CK(cudaStreamSynchronize(c->last_stream));
    CK(cudaDeviceSynchronize());
    LzState lz;
    const LzState *src = c->plan.precision == PSE_FP64 ? c->dd.lz : c->df.lz;
    CK(cudaMemcpy(&lz, src, sizeof(lz), cudaMemcpyDeviceToHost));
    const int64_t np = (int64_t)lz.n_pairs;
    out->lanczos_iters = lz.J;
    out->converged = lz.converged;
    out->lanczos_rel_change = lz.rel;
    out->n_pairs = np;
    out->overflow = lz.overflow;
    out->matvec_shape = (c->plan.precision == PSE_FP64 ? c->gd.mv : c->gf.mv) + 1;
    if (lz.overflow) return PSE_ENOMEM;
    if (!lz.converged && lz.J > 0) return PSE_ENOTCONVERGED;
    return PSE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batched systems
struct pse_batch {
    std::vector<pse_ctx *> sys;
    int device = 0;
    cudaStream_t root = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> built_N;
    SampleArgs<float> *d_args = nullptr;  // one per system, read by that system's kernels
    std::vector<SampleArgs<float>> h_args;
    // pinned ring of argument tables (nsys entries per slot): the per-call
    // copy then does not wait for the previous batched sample
    SampleArgs<float> *args_ring = nullptr;
    cudaEvent_t ev_args[PSE_ARGS_SLOTS] = {};
    bool args_used[PSE_ARGS_SLOTS] = {};
    int args_slot = 0;
    LzState **d_lzs = nullptr;            // each system's Lanczos state, for the loop condition
    cudaStream_t body = nullptr;          // captures the shared loop body
    LzSys *d_sys = nullptr;               // per-system descriptors of the fused loop kernels
    int *d_blk_mv = nullptr, *d_blk_up = nullptr;  // block -> system of the fused matvec / update
    int nblk_mv = 0, nblk_up = 0;
    BSys *d_bsys = nullptr;               // per-system descriptors of the fused prologue / epilogue
    int *d_btab[PSE_BK] = {};             // block -> system, per fused kernel kind
    int bnblk[PSE_BK] = {};
    cudaStream_t wave = nullptr;          // wave branch of the batch
    int *d_any = nullptr;                 // any system still iterating (host-loop mode)
    // systems whose grids share a size share one pooled spectrum / grid and one
    // batched cuFFT plan (3 transforms per system)
    struct FftGroup {
        int M = 0;
        std::vector<int> members;
        void *spec = nullptr, *grid = nullptr;
        void *grid4 = nullptr;  // node-major copies of the members' grids
        cufftHandle plan = 0;
        bool plan_made = false;
    };
    std::vector<FftGroup> groups;
    int p4 = 0;  // common support P of the node-major interpolation, 0: planar
    cudaEvent_t ev_sorted = nullptr, ev_wave = nullptr, ev_noise = nullptr;
    std::vector<cudaEvent_t> ev_pre;
    cudaGraphConditionalHandle cond = 0;
};

static void batch_drop_graph(pse_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

extern "C" void pse_batch_destroy(pse_batch *b) {
    if (!b) return;
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    batch_drop_graph(b);
    for (pse_ctx *c : b->sys) pse_destroy(c);
    if (b->d_args) cudaFree(b->d_args);
    for (int k = 0; k < PSE_ARGS_SLOTS; ++k)
        if (b->ev_args[k]) cudaEventDestroy(b->ev_args[k]);
    if (b->args_ring) cudaFreeHost(b->args_ring);
    if (b->d_lzs) cudaFree(b->d_lzs);
    if (b->root) cudaStreamDestroy(b->root);
    if (b->body) cudaStreamDestroy(b->body);
    if (b->d_sys) cudaFree(b->d_sys);
    if (b->d_blk_mv) cudaFree(b->d_blk_mv);
    if (b->d_blk_up) cudaFree(b->d_blk_up);
    if (b->d_bsys) cudaFree(b->d_bsys);
    for (int k = 0; k < PSE_BK; ++k) if (b->d_btab[k]) cudaFree(b->d_btab[k]);
    for (auto &g : b->groups) {
        if (g.plan_made) cufftDestroy(g.plan);
        if (g.spec) cudaFree(g.spec);
        if (g.grid) cudaFree(g.grid);
        if (g.grid4) cudaFree(g.grid4);
    }
    if (b->wave) cudaStreamDestroy(b->wave);
    if (b->d_any) cudaFree(b->d_any);
    if (b->ev_sorted) cudaEventDestroy(b->ev_sorted);
    if (b->ev_wave) cudaEventDestroy(b->ev_wave);
    if (b->ev_noise) cudaEventDestroy(b->ev_noise);
    for (cudaEvent_t e : b->ev_pre) if (e) cudaEventDestroy(e);
    delete b;
}

// Grid size classes of a batch: each system's Sec. II C grid is raised to
// the next class (a finer grid only lowers the NUFFT error), so that systems
// of a class share one batched inverse FFT.
static const int kGridClasses[] = {16, 20, 24, 28, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128, 144, 160, 192,
                                   224, 256, 288, 320, 384, 448, 512, 576, 640, 768, 896, 1024};
static constexpr int kNumGridClasses = (int)(sizeof(kGridClasses) / sizeof(kGridClasses[0]));

extern "C" pse_status pse_batch_grid(double L, double a, const pse_params *p, int step, int *M_out) {
    if (!p || !M_out || step < 0) return PSE_EINVAL;
    pse_params q = *p;
    q.autotune &= ~1;
    pse_plan_info pi;
    const pse_status st = pse_plan(L, a, &q, &pi);
    if (st != PSE_OK) return st;
    int ci = -1;
    for (int i = 0; i < kNumGridClasses; ++i)
        if (kGridClasses[i] >= pi.M) { ci = i; break; }
    if (ci < 0) {  // beyond the last class: its own grid
        *M_out = pi.M;
        return PSE_OK;
    }
    ci += step;
    *M_out = kGridClasses[ci < kNumGridClasses ? ci : kNumGridClasses - 1];
    return PSE_OK;
}

extern "C" pse_status pse_batch_create(pse_batch **out, int nsys, const double *L, const double *a,
                                       const pse_params *p) {
    if (!out) return PSE_EINVAL;
    *out = nullptr;
    if (nsys < 1 || !L || !a || !p) return PSE_EINVAL;
    pse_batch *b = new (std::nothrow) pse_batch();
    if (!b) return PSE_ENOMEM;
    if (cudaGetDevice(&b->device) != cudaSuccess) { cudaGetLastError(); delete b; return PSE_ECUDA; }
    pse_status st = PSE_OK;
    for (int k = 0; k < nsys && st == PSE_OK; ++k) {
        if (p[k].precision != PSE_FP32) { st = PSE_ENOTSUPPORTED; break; }
        pse_params q = p[k];
        q.system = k;
        q.autotune &= ~1;  // the size class replaces the per-system FFT-size timing
        q.interp_form = 1;  // the fused batch interpolation reads the pooled planar grids
        if (q.grid_M <= 0) {
            pse_plan_info pi;
            st = pse_plan(L[k], a[k], &q, &pi);
            if (st != PSE_OK) break;
            for (int cl : kGridClasses)
                if (cl >= pi.M) { q.grid_M = cl; break; }
        }
        pse_ctx *c = nullptr;
        st = pse_create_ex(&c, L[k], a[k], &q);
        if (st == PSE_OK) b->sys.push_back(c);
    }
    // pooled spectra / grids and one plan per grid size
    for (int k = 0; k < (int)b->sys.size() && st == PSE_OK; ++k) {
        const int M = b->sys[k]->plan.M;
        size_t gi = 0;
        while (gi < b->groups.size() && b->groups[gi].M != M) ++gi;
        if (gi == b->groups.size()) {
            b->groups.emplace_back();
            b->groups.back().M = M;
        }
        b->groups[gi].members.push_back(k);
    }
    for (auto &g : b->groups) {
        if (st != PSE_OK) break;
        const int64_t M = g.M, plane = M * M * (M / 2 + 1), n = (int64_t)g.members.size();
        if (cudaMalloc(&g.spec, sizeof(cufftComplex) * 3 * plane * n) != cudaSuccess ||
            cudaMalloc(&g.grid, sizeof(float) * 3 * M * M * M * n) != cudaSuccess) {
            cudaGetLastError();
            st = PSE_ENOMEM;
            break;
        }
        int nn[3] = {(int)M, (int)M, (int)M};
        if (cufftPlanMany(&g.plan, 3, nn, nullptr, 1, (int)plane, nullptr, 1, (int)(M * M * M), CUFFT_C2R,
                          (int)(3 * n)) != CUFFT_SUCCESS) {
            st = PSE_ECUFFT;
            break;
        }
        g.plan_made = true;
        for (int i = 0; i < (int)n; ++i) {  // the system's kernels use its slice of the pool
            pse_ctx *c = b->sys[g.members[i]];
            c->df.spec = (cufftComplex *)g.spec + 3 * plane * i;
            c->df.grid = (float *)g.grid + 3 * M * M * M * i;
        }
    }
    // node-major interpolation when every system has the same support P in
    // 3..10 (one instantiation serves all): pooled float4 grids per size
    if (st == PSE_OK) {
        const int P0 = b->sys[0]->plan.P;
        bool same = P0 >= 3 && P0 <= 10;
        for (pse_ctx *c : b->sys) same = same && c->plan.P == P0;
        if (same) {
            for (auto &g : b->groups) {
                const int64_t M = g.M, n = (int64_t)g.members.size();
                if (cudaMalloc(&g.grid4, sizeof(V4<float>) * M * M * M * n) != cudaSuccess) {
                    cudaGetLastError();
                    same = false;
                    break;
                }
                for (int i = 0; i < (int)n; ++i)
                    b->sys[g.members[i]]->df.grid4 = (V4<float> *)g.grid4 + M * M * M * i;
            }
            b->p4 = same ? P0 : 0;
        }
    }
    if (st == PSE_OK && cudaMalloc(&b->d_args, sizeof(SampleArgs<float>) * nsys) != cudaSuccess) {
        cudaGetLastError();
        st = PSE_ENOMEM;
    }
    if (st == PSE_OK && cudaMalloc((void **)&b->d_lzs, sizeof(LzState *) * nsys) != cudaSuccess) {
        cudaGetLastError();
        st = PSE_ENOMEM;
    }
    // as in a lone context: the near-field chain at the highest priority,
    // the wave branch at the lowest
    int p_lo = 0, p_hi = 0;
    if (st == PSE_OK && cudaDeviceGetStreamPriorityRange(&p_lo, &p_hi) != cudaSuccess) st = PSE_ECUDA;
    if (st == PSE_OK && (cudaStreamCreateWithPriority(&b->root, cudaStreamNonBlocking, p_hi) != cudaSuccess ||
                         cudaStreamCreateWithPriority(&b->body, cudaStreamNonBlocking, p_hi) != cudaSuccess ||
                         cudaStreamCreateWithPriority(&b->wave, cudaStreamNonBlocking, p_lo) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ev_sorted, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ev_wave, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ev_noise, cudaEventDisableTiming) != cudaSuccess))
        st = PSE_ECUDA;
    if (st == PSE_OK) {
        b->ev_pre.assign(nsys, nullptr);
        for (int k = 0; k < nsys && st == PSE_OK; ++k)
            if (cudaEventCreateWithFlags(&b->ev_pre[k], cudaEventDisableTiming) != cudaSuccess) st = PSE_ECUDA;
        std::vector<LzState *> lzs(nsys);
        for (int k = 0; k < nsys; ++k) lzs[k] = b->sys[k]->df.lz;
        if (st == PSE_OK && cudaMemcpy(b->d_lzs, lzs.data(), sizeof(LzState *) * nsys, cudaMemcpyHostToDevice) != cudaSuccess)
            st = PSE_ECUDA;
        // every system's kernels read their per-call arguments from the batch array
        for (int k = 0; k < nsys; ++k) b->sys[k]->df.args = b->d_args + k;
        b->h_args.assign(nsys, SampleArgs<float>{});
        b->built_N.assign(nsys, 0);
    }
    if (st != PSE_OK) {
        pse_batch_destroy(b);
        return st;
    }
    *out = b;
    return PSE_OK;
}

// Descriptors and block tables of the fused loop kernels.  Each system gets
// a fixed number of blocks of each fused kernel (one per PSE_BATCH_MV_THREADS
// / PSE_BATCH_MV_TPP particles of the matvec, per 256 of the update, capped
// at the resident blocks per SM), so its reductions add the same partial
// sums in the same order on every launch; its sample equals a lone
// context's to float rounding.
static pse_status batch_descriptors(pse_batch *b) {
    const int S = (int)b->sys.size();
    const int64_t cap_mv = (int64_t)num_sms() * matvec_blocks_per_sm(),
                  cap_up = (int64_t)num_sms() * update_blocks_per_sm();
    std::vector<LzSys> hs(S);
    std::vector<int> blk_mv, blk_up;
    for (int k = 0; k < S; ++k) {
        pse_ctx *c = b->sys[k];
        const int64_t N = c->N;
        auto blocks = [&](int64_t per_block, int64_t cap) {
            const int64_t need = (N + per_block - 1) / per_block;
            return (int)(need < cap ? (need > 0 ? need : 1) : cap);
        };
        LzSys &d = hs[k];
        d.N = N;
        d.K = nbr_k(N, c->df.nbr_cap);
        d.blk_mv = (int)blk_mv.size();
        d.nblk_mv = blocks(PSE_BATCH_MV_THREADS / PSE_BATCH_MV_TPP, cap_mv);
        d.blk_up = (int)blk_up.size();
        d.nblk_up = blocks(256, cap_up);
        blk_mv.insert(blk_mv.end(), d.nblk_mv, k);
        blk_up.insert(blk_up.end(), d.nblk_up, k);
        d.max_iter = c->max_iter;
        d.fixed_iter = c->params.fixed_iter;
        d.tol = c->params.lanczos_tol > 0 ? c->params.lanczos_tol : c->plan.tol;
        d.g = c->gf;
        d.rec = c->df.rec;
        d.count = c->df.nbr_count;
        d.nbr = c->df.nbr;
        d.table = c->df.table;
        d.table_c = c->df.table_c;
        d.u = c->df.u;
        d.part_mv = c->df.partials;
        d.part_up = c->df.partials + num_sms() * 16 + 32;
        d.lz = c->df.lz;
        d.pc = c->df.pc_on;
        d.basis = c->df.basis;
    }
    if (b->d_sys) cudaFree(b->d_sys);
    if (b->d_blk_mv) cudaFree(b->d_blk_mv);
    if (b->d_blk_up) cudaFree(b->d_blk_up);
    b->d_sys = nullptr;
    b->d_blk_mv = b->d_blk_up = nullptr;
    if (cudaMalloc((void **)&b->d_sys, sizeof(LzSys) * S) != cudaSuccess ||
        cudaMalloc((void **)&b->d_blk_mv, sizeof(int) * blk_mv.size()) != cudaSuccess ||
        cudaMalloc((void **)&b->d_blk_up, sizeof(int) * blk_up.size()) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ENOMEM;
    }
    CK(cudaMemcpy(b->d_sys, hs.data(), sizeof(LzSys) * S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_blk_mv, blk_mv.data(), sizeof(int) * blk_mv.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_blk_up, blk_up.data(), sizeof(int) * blk_up.size(), cudaMemcpyHostToDevice));
    b->nblk_mv = (int)blk_mv.size();
    b->nblk_up = (int)blk_up.size();

    // prologue / epilogue kernels: blocks per system for each kind
    std::vector<BSys> hb(S);
    std::vector<int> tabs[PSE_BK];
    for (int k = 0; k < S; ++k) {
        pse_ctx *c = b->sys[k];
        if (c->plan.P > PSE_BATCH_INTERP_G) return PSE_ENOTSUPPORTED;
        BSys &d = hb[k];
        d.N = c->N;
        d.nc3 = c->ncell3;
        d.system = c->params.system;
        d.K = nbr_k(c->N, c->df.nbr_cap);
        d.pc_s0 = c->pc_s0;
        d.g = c->gf;
        d.w = c->wf;
        d.d = c->df;
        const int64_t modes = (int64_t)c->plan.M * c->plan.M * (c->plan.M / 2 + 1);
        const int64_t n_per[PSE_BK] = {
            (d.nc3 + 255) / 256,                               // zero
            (d.N + 255) / 256,                                 // bin
            (d.N + 255) / 256,                                 // scatter
            (d.N + 255) / 256,                                 // placement in cell order
            (d.N + 255) / 256,                                 // neighbours
            0,                                                 // init (set below)
            (modes + 255) / 256,                               // noise
            b->p4 ? (d.N + 4 * (32 / b->p4) - 1) / (4 * (32 / b->p4))  // interpolation: 4 warps of
                  : (d.N * PSE_BATCH_INTERP_G + 127) / 128,       // 32/P particles, or 16 lanes each
            (d.N + 255) / 256,                                 // final (one block per 256, exact)
            c->pc_enabled ? (d.N + 127) / 128 : 0,             // network blocks (only where installed)
            b->p4 ? ((int64_t)c->plan.M * c->plan.M * c->plan.M + 255) / 256 : 0};  // node-major copy
        for (int kind = 0; kind < PSE_BK; ++kind) {
            int64_t n = n_per[kind];
            if (kind == BK_INIT) {  // the lone context's grid, so beta_0 adds the same partials
                const int64_t need = (d.N + 255) / 256, cap = (int64_t)num_sms() * 8;
                n = need < cap ? need : cap;
            }
            if (n < 1 && kind != BK_PC && kind != BK_COPY) n = 1;
            if (n > (1 << 24)) return PSE_EINVAL;
            d.b0[kind] = (int)tabs[kind].size();
            d.nb[kind] = (int)n;
            tabs[kind].insert(tabs[kind].end(), (size_t)n, k);
        }
    }
    if (b->d_bsys) cudaFree(b->d_bsys);
    b->d_bsys = nullptr;
    for (int kind = 0; kind < PSE_BK; ++kind) {
        if (b->d_btab[kind]) cudaFree(b->d_btab[kind]);
        b->d_btab[kind] = nullptr;
    }
    if (cudaMalloc((void **)&b->d_bsys, sizeof(BSys) * S) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ENOMEM;
    }
    CK(cudaMemcpy(b->d_bsys, hb.data(), sizeof(BSys) * S, cudaMemcpyHostToDevice));
    for (int kind = 0; kind < PSE_BK; ++kind) {
        b->bnblk[kind] = 0;
        if (tabs[kind].empty()) continue;
        if (cudaMalloc((void **)&b->d_btab[kind], sizeof(int) * tabs[kind].size()) != cudaSuccess) {
            cudaGetLastError();
            return PSE_ENOMEM;
        }
        CK(cudaMemcpy(b->d_btab[kind], tabs[kind].data(), sizeof(int) * tabs[kind].size(), cudaMemcpyHostToDevice));
        b->bnblk[kind] = (int)tabs[kind].size();
    }
    return PSE_OK;
}

// Pieces of one batched sample, on stream `s` (capturing or not): the fused
// prologue (cell lists; the wave branch -- noise of all systems, one batched
// C2R per grid size, interpolation of all -- beside the neighbour lists,
// preconditioner blocks and q_1), one Lanczos step of every system, and the
// epilogue (final combination of all systems once the wave branch is done).
static pse_status batch_prologue(pse_batch *b, cudaStream_t s) {
    const int S = (int)b->sys.size();
    pse_status st = PSE_OK;
    launch_batch_prologue_cells(b->d_bsys, S, b->d_btab, b->bnblk, s);
    cudaEventRecord(b->ev_sorted, s);
    cudaStreamWaitEvent(b->wave, b->ev_sorted, 0);
    launch_batch_noise(b->d_bsys, b->d_btab, b->bnblk, b->wave);
    cudaEventRecord(b->ev_noise, b->wave);
    for (size_t gi = 0; gi < b->groups.size() && st == PSE_OK; ++gi) {
        auto &g = b->groups[gi];
        pse_ctx *c = b->sys[g.members[0]];  // the first member's stream carries the branch
        cudaStreamWaitEvent(c->s_wave, b->ev_noise, 0);
        if (cufftSetStream(g.plan, c->s_wave) != CUFFT_SUCCESS ||
            cufftExecC2R(g.plan, (cufftComplex *)g.spec, (cufftReal *)g.grid) != CUFFT_SUCCESS)
            st = PSE_ECUFFT;
        cudaEventRecord(b->ev_pre[gi], c->s_wave);
        cudaStreamWaitEvent(b->wave, b->ev_pre[gi], 0);
    }
    launch_batch_interp(b->d_bsys, b->d_btab, b->bnblk, b->p4, b->wave);
    cudaEventRecord(b->ev_wave, b->wave);
    launch_batch_nbr(b->d_bsys, (int)b->sys.size(), b->d_btab, b->bnblk, s);
    launch_batch_pc_infer(b->d_bsys, b->d_btab, b->bnblk, s);
    launch_batch_init(b->d_bsys, b->d_btab, b->bnblk, s);
    return st;
}

static void batch_step(pse_batch *b, cudaStream_t s, cudaGraphConditionalHandle h, int *any_out) {
    const int S = (int)b->sys.size();
    launch_lz_matvec_batch(b->d_sys, b->d_blk_mv, b->nblk_mv, s);
    launch_lz_update_batch(b->d_sys, b->d_blk_up, b->nblk_up, s);
    launch_lz_eig_batch(b->d_sys, S, s);
    launch_batch_cond(b->d_lzs, S, h, s, any_out);
}

static void batch_epilogue(pse_batch *b, cudaStream_t s) {
    cudaStreamWaitEvent(s, b->ev_wave, 0);
    launch_batch_final(b->d_bsys, b->d_btab, b->bnblk, s);
}

extern "C" pse_status pse_batch_sample(pse_batch *b, const int64_t *offsets, const float *d_pos, uint64_t seed,
                                       uint64_t sample_index, float *d_out, void *stream) {
    if (!b || !offsets || !d_pos || !d_out) return PSE_EINVAL;
    const int S = (int)b->sys.size();
    if (offsets[0] != 0) return PSE_EINVAL;
    for (int k = 0; k < S; ++k)
        if (offsets[k + 1] - offsets[k] < 1) return PSE_EINVAL;
    DeviceGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool plain = b->sys[0]->params.use_graph < 0;
    bool rebuild = plain || b->exec == nullptr;
    for (int k = 0; k < S; ++k) {
        const int64_t N = offsets[k + 1] - offsets[k];
        if (N != b->built_N[k]) rebuild = true;
        pse_status st = ensure<float>(b->sys[k], N);
        if (st != PSE_OK) return st;
        if (b->sys[k]->params.wave_noise == 1 && (st = ensure_r2c<float>(b->sys[k])) != PSE_OK) return st;
        b->sys[k]->df.args = b->d_args + k;  // kept across re-allocation
    }
    if (rebuild) {
        batch_drop_graph(b);
        const pse_status sd = batch_descriptors(b);
        if (sd != PSE_OK) return sd;
    }
    if (rebuild && !plain) {
        // prologues of all systems in parallel, one shared WHILE node whose body
        // holds every system's Lanczos step and the batch condition, epilogues
        CK(cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal));
        pse_status st = batch_prologue(b, b->root);
        cudaGraph_t body = nullptr;
        cudaError_t e = add_while(b->root, &b->cond, &body);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b->body, body, nullptr, nullptr, 0,
                                                              cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            batch_step(b, b->body, b->cond, nullptr);
            cudaGraph_t body_out = nullptr;
            e = cudaStreamEndCapture(b->body, &body_out);
        }
        if (e != cudaSuccess && st == PSE_OK) st = PSE_ECUDA;
        batch_epilogue(b, b->root);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->root, &graph);
        if (st != PSE_OK || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != PSE_OK ? st : PSE_ECUDA;
        }
        b->graph = graph;
        if (cudaGraphInstantiate(&b->exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
            cudaGetLastError();
            batch_drop_graph(b);
            return PSE_ECUDA;
        }
        for (int k = 0; k < S; ++k) b->built_N[k] = offsets[k + 1] - offsets[k];
    }
    for (int k = 0; k < S; ++k) {
        SampleArgs<float> &a = b->h_args[k];
        a.pos = d_pos + 3 * offsets[k];
        a.out = d_out + 3 * offsets[k];
        a.real = nullptr;
        a.wave = nullptr;
        a.vin = nullptr;
        a.seed = seed;
        a.sample = sample_index;
        a.c_det = 0.0;
        a.c_noise = 1.0;
    }
    {
        if (!b->args_ring) {
            CK(cudaMallocHost((void **)&b->args_ring, sizeof(SampleArgs<float>) * S * PSE_ARGS_SLOTS));
            for (int k = 0; k < PSE_ARGS_SLOTS; ++k) CK(cudaEventCreateWithFlags(&b->ev_args[k], cudaEventDisableTiming));
        }
        const int k = b->args_slot;
        b->args_slot = (k + 1) % PSE_ARGS_SLOTS;
        if (b->args_used[k]) CK(cudaEventSynchronize(b->ev_args[k]));
        SampleArgs<float> *slot = b->args_ring + (size_t)k * S;
        memcpy(slot, b->h_args.data(), sizeof(SampleArgs<float>) * S);
        CK(cudaMemcpyAsync(b->d_args, slot, sizeof(SampleArgs<float>) * S, cudaMemcpyHostToDevice, s));
        CK(cudaEventRecord(b->ev_args[k], s));
        b->args_used[k] = true;
    }
    if (plain) {  // the same kernels without a graph, host-side loop (one sync per step)
        if (!b->d_any && cudaMalloc((void **)&b->d_any, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return PSE_ENOMEM;
        }
        pse_status st = batch_prologue(b, s);
        if (st != PSE_OK) return st;
        for (int it = 0; it < PSE_MAXIT + 2; ++it) {
            batch_step(b, s, 0, b->d_any);
            int any = 0;
            CK(cudaMemcpyAsync(&any, b->d_any, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!any) break;
        }
        batch_epilogue(b, s);
        for (int k = 0; k < S; ++k) b->built_N[k] = offsets[k + 1] - offsets[k];
    } else {
        CK(cudaGraphLaunch(b->exec, s));
    }
    for (pse_ctx *c : b->sys) c->last_stream = s;
    CK(cudaGetLastError());
    return PSE_OK;
}

extern "C" pse_status pse_batch_set_precond(pse_batch *b, int k, const float *h_theta, int nparam) {
    if (!b || k < 0 || k >= (int)b->sys.size()) return PSE_EINVAL;
    const pse_status st = pse_precond_set_weights(b->sys[k], h_theta, nparam);
    if (st == PSE_OK) batch_drop_graph(b);
    return st;
}

extern "C" pse_status pse_batch_get_stats(pse_batch *b, int k, pse_stats *out) {
    if (!b || k < 0 || k >= (int)b->sys.size()) return PSE_EINVAL;
    return pse_get_stats(b->sys[k], out);
}

extern "C" pse_status pse_batch_get_plan(const pse_batch *b, int k, pse_plan_info *out) {
    if (!b || k < 0 || k >= (int)b->sys.size()) return PSE_EINVAL;
    return pse_get_plan(b->sys[k], out);
}
