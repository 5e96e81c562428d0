// Wave-space sample M_w^{1/2} dW2 (Sec. II B 2): complex Hermitian noise,
// B^{1/2} scaling with the Gaussian deconvolution, inverse FFT (cuFFT C2R,
// launched by the host), and Gaussian interpolation S^dagger = h^3 S^T at the
// particles.  sm_103a.
//
// Per mode k = 2 pi n / L of the half spectrum (nz >= 0):
//   vhat(k) = V^{-1/2} sinc(ka)/k sqrt(1 + k^2/4xi^2) exp(-(1 - eta) k^2 / 8xi^2)
//             (I - kk) dW2(k)
// which, interpolated with g(r) = (2xi^2/(pi eta))^{3/2} exp(-2 xi^2 r^2 / eta)
// (Fourier transform exp(-eta k^2 / 8 xi^2)), reproduces the eq. Mwave
// factor sinc^2(ka) H(k, xi) / (V k^2) in the covariance.
#include "pse_internal.cuh"

namespace pse {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = cufftComplex; };
template <> struct Cplx<double> { using type = cufftDoubleComplex; };

template <typename T> __device__ __forceinline__ T exp_t(T x) {
    if constexpr (sizeof(T) == 4) return expf(x);
    else return exp(x);
}

// Mode (ix, iy, iz) of the half spectrum, iz in [0, M/2]: signed indices,
// and whether it carries noise (k != 0, no Nyquist index).
struct ModeIdx {
    int ix, iy, iz, nx, ny, nz;
    bool live;
};
// n / d for 32-bit n with the multiplier m and shift l of d >= 2
// (Granlund and Montgomery, PLDI 1994, the round-up method).
__device__ __forceinline__ uint32_t udiv_magic(uint32_t n, uint32_t m, int l) {
    const uint32_t t1 = __umulhi(m, n);
    return (t1 + ((n - t1) >> 1)) >> (l - 1);
}
template <typename T> __device__ __forceinline__ ModeIdx mode_of(int64_t t, const WaveGeom<T> &w) {
    ModeIdx m;
    const int M = w.M, Mh1 = w.Mh1;
    if (!w.big) {
        const uint32_t u = (uint32_t)t;
        const uint32_t r = udiv_magic(u, w.dv_h1_m, w.dv_h1_l);
        const uint32_t x = udiv_magic(r, w.dv_M_m, w.dv_M_l);
        m.iz = (int)(u - r * (uint32_t)Mh1);
        m.iy = (int)(r - x * (uint32_t)M);
        m.ix = (int)x;
    } else {
        m.iz = (int)(t % Mh1);
        m.iy = (int)((t / Mh1) % M);
        m.ix = (int)(t / ((int64_t)Mh1 * M));
    }
    const int half = M / 2;
    m.nx = m.ix <= half ? m.ix : m.ix - M;
    m.ny = m.iy <= half ? m.iy : m.iy - M;
    m.nz = m.iz;
    const bool nyq = (M % 2) == 0 && (m.ix == half || m.iy == half || m.iz == half);
    m.live = !nyq && (m.nx | m.ny | m.nz) != 0;
    return m;
}

// dW2 of a live mode: the noise of a {k, -k} pair is keyed by its
// representative (nz > 0, or nz = 0 and (ny > 0 or (ny = 0 and nx > 0))),
// id q = (ix*M + iy)*Mh1 + iz, Philox blocks 2q and 2q+1; a mode holding the
// partner draws the same numbers and conjugates them, so the kz = 0 plane is
// exactly Hermitian.
template <typename T>
__device__ __forceinline__ void mode_noise(const ModeIdx &m, int M, int Mh1, uint32_t strm, uint64_t seed,
                                           uint64_t sample, T wr[3], T wi[3]) {
    int rx = m.ix, ry = m.iy;
    bool conj = false;
    if (m.nz == 0 && !(m.ny > 0 || (m.ny == 0 && m.nx > 0))) {
        rx = (M - m.ix) % M;
        ry = (M - m.iy) % M;
        conj = true;
    }
    const uint32_t q = (uint32_t)(((int64_t)rx * M + ry) * Mh1 + m.iz);
    const Normals4<T> a = normals4<T>(2u * q, strm, seed, sample);
    const Normals4<T> b = normals4<T>(2u * q + 1u, strm, seed, sample);
    const T s2 = T(0.70710678118654752440);
    wr[0] = a.v[0] * s2; wr[1] = a.v[2] * s2; wr[2] = b.v[0] * s2;
    wi[0] = a.v[1] * s2; wi[1] = a.v[3] * s2; wi[2] = b.v[1] * s2;
    if (conj) { wi[0] = -wi[0]; wi[1] = -wi[1]; wi[2] = -wi[2]; }
}

// Unit wave vector and the noise scale
//   sc(k) = V^{-1/2} sinc(ka)/k sqrt(1 + k^2/4xi^2) exp(-(1 - eta) k^2 / 8xi^2)
// of a live mode.  sc and 1/|n| depend on the integer n^2 = nx^2 + ny^2 + nz^2
// only; both come from a table evaluated in FP64 on the host.
template <typename T>
__device__ __forceinline__ T mode_scale(const ModeIdx &m, const WaveGeom<T> &w, T &hx, T &hy, T &hz) {
    const int n2 = m.nx * m.nx + m.ny * m.ny + m.nz * m.nz;
    T sc, inv;
    if constexpr (sizeof(T) == 4) {
        const float2 e = __ldg(reinterpret_cast<const float2 *>(w.sc_tab) + n2);
        sc = e.x;
        inv = e.y;
    } else {
        const double2 e = __ldg(reinterpret_cast<const double2 *>(w.sc_tab) + n2);
        sc = e.x;
        inv = e.y;
    }
    hx = T(m.nx) * inv;
    hy = T(m.ny) * inv;
    hz = T(m.nz) * inv;
    return sc;
}

// One thread per half-spectrum mode: vhat = sc(k) (I - kk) dW2(k); k = 0 and
// Nyquist modes are zero.
template <typename T>
__device__ __forceinline__ void wave_noise_elem(int64_t t, const WaveGeom<T> &w, const SampleArgs<T> *args,
                                                int system, typename Cplx<T>::type *spec, int64_t plane) {
    using C = typename Cplx<T>::type;
    const ModeIdx m = mode_of(t, w);
    C o0, o1, o2;
    o0.x = o0.y = o1.x = o1.y = o2.x = o2.y = T(0);
    T pr[3] = {T(0), T(0), T(0)}, pi[3] = {T(0), T(0), T(0)};  // (I - kk) dW2
    int n2 = 0;
    T sc = T(0);
    if (m.live) {
        T wr[3], wi[3];
        mode_noise<T>(m, w.M, w.Mh1, 2u * system + 1u, args->seed, args->sample, wr, wi);
        T hx, hy, hz;
        sc = mode_scale<T>(m, w, hx, hy, hz);
        n2 = m.nx * m.nx + m.ny * m.ny + m.nz * m.nz;
        const T dr = hx * wr[0] + hy * wr[1] + hz * wr[2];
        const T di = hx * wi[0] + hy * wi[1] + hz * wi[2];
        pr[0] = wr[0] - hx * dr; pi[0] = wi[0] - hx * di;
        pr[1] = wr[1] - hy * dr; pi[1] = wi[1] - hy * di;
        pr[2] = wr[2] - hz * dr; pi[2] = wi[2] - hz * di;
    }
    o0.x = sc * pr[0]; o0.y = sc * pi[0];
    o1.x = sc * pr[1]; o1.y = sc * pi[1];
    o2.x = sc * pr[2]; o2.y = sc * pi[2];
    spec[t] = o0;
    spec[plane + t] = o1;
    spec[2 * plane + t] = o2;
    // polydisperse: species s scales the same noise with its own shape factor
    for (int sp = 1; sp < w.nspec; ++sp) {
        const T scs = m.live ? w.sc_tab[sp * w.sc_stride + 2 * n2] : T(0);
        C *o = spec + (int64_t)sp * 3 * plane;
        C q;
        q.x = scs * pr[0]; q.y = scs * pi[0]; o[t] = q;
        q.x = scs * pr[1]; q.y = scs * pi[1]; o[plane + t] = q;
        q.x = scs * pr[2]; q.y = scs * pi[2]; o[2 * plane + t] = q;
    }
}

template <typename T>
__global__ void k_wave_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, typename Cplx<T>::type *spec,
                             int64_t plane) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)w.M * w.M * w.Mh1) wave_noise_elem<T>(t, w, args, system, spec, plane);
}

// Mode factor applied in place to a forward (R2C) spectrum, one thread per
// half-spectrum mode, k = 0 and Nyquist set to zero:
//   WAVE_MODE_DET:       vhat = c_det norm sc^2 (I - kk) Fhat  [+ c_noise sc (I - kk) dW2]
//     Fhat = DFT of the unnormalised spread grid sum_i w_x w_y w_z F_i; with the
//     Gaussian's constant norm = (2xi^2/(pi eta))^{3/2} h^3 this is
//     h^3 B(k)/V (I - kk) DFT(S F), the deterministic wave product, and the
//     optional k-space noise term fuses the Brownian wave part into the same
//     inverse FFT (Sec. III);
//   WAVE_MODE_GRIDNOISE: vhat = c_noise sc M^{-3/2} (I - kk) What, What the DFT of white
//     grid noise, which on every live mode pair has the law of dW2.
template <typename T>
__global__ void k_wave_apply(WaveGeom<T> w, const SampleArgs<T> *args, int system, typename Cplx<T>::type *spec,
                             int64_t plane, int mode, int with_noise) {
    using C = typename Cplx<T>::type;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nmodes = (int64_t)w.M * w.M * w.Mh1;
    if (t >= nmodes) return;
    const ModeIdx m = mode_of(t, w);
    C o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c].x = o[c].y = T(0);
    if (m.live) {
        T hx, hy, hz;
        const T sc = mode_scale<T>(m, w, hx, hy, hz);
        const C i0 = spec[t], i1 = spec[plane + t], i2 = spec[2 * plane + t];
        T f;
        if (mode == WAVE_MODE_DET) f = (T)args->c_det * w.norm * sc * sc;
        else f = (T)args->c_noise * sc * w.inv_M15;
        T vr[3] = {i0.x, i1.x, i2.x}, vi[3] = {i0.y, i1.y, i2.y};
        const T dr = hx * vr[0] + hy * vr[1] + hz * vr[2];
        const T di = hx * vi[0] + hy * vi[1] + hz * vi[2];
        const T hh[3] = {hx, hy, hz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o[c].x = f * (vr[c] - hh[c] * dr);
            o[c].y = f * (vi[c] - hh[c] * di);
        }
        if (mode == WAVE_MODE_DET && with_noise) {
            T wr[3], wi[3];
            mode_noise<T>(m, w.M, w.Mh1, 2u * system + 1u, args->seed, args->sample, wr, wi);
            const T g = (T)args->c_noise * sc;
            const T er = hx * wr[0] + hy * wr[1] + hz * wr[2];
            const T ei = hx * wi[0] + hy * wi[1] + hz * wi[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[c].x += g * (wr[c] - hh[c] * er);
                o[c].y += g * (wi[c] - hh[c] * ei);
            }
        }
    }
    spec[t] = o[0];
    spec[plane + t] = o[1];
    spec[2 * plane + t] = o[2];
}

// White noise on the grid: node g = (ix*M + iy)*M + iz keys one Philox block
// on the wave stream; its first three normals are the x, y, z components.
template <typename T>
__global__ void k_grid_noise(int64_t M3, const SampleArgs<T> *args, int system, T *grid) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M3) return;
    const Normals4<T> n = normals4<T>((uint32_t)g, 2u * system + 1u, args->seed, args->sample);
    grid[g] = n.v[0];
    grid[M3 + g] = n.v[1];
    grid[2 * M3 + g] = n.v[2];
}

// Support start and fractional offset of one coordinate: s = x M / L as a
// float-float product, i0 = floor(s - P/2) + 1 decided exactly, and
// u = s - i0 in [P/2 - 1, P/2) (grid units).
__device__ __forceinline__ void support(float x, const WaveGeom<float> &w, int &i0, float &u) {
    const float hi = x * w.gl_hi;
    const float lo = fmaf(x, w.gl_lo, fmaf(x, w.gl_hi, -hi));
    const float th = hi - 0.5f * (float)w.P;  // exact: P/2 lies on the ulp grid of hi
    float fl = floorf(th);
    float rem = (th - fl) + lo;
    // rem = s - P/2 - fl to float rounding; its sign decides the floor.  A
    // tiny negative rem moves the support down one node, and rem + 1 may
    // round to 1: keep it just below 1 so that it does not move back.
    if (rem < 0.f) {
        fl -= 1.f;
        rem = fminf(rem + 1.f, 0.99999994f);
    } else if (rem >= 1.f) {
        fl += 1.f;
        rem -= 1.f;
    }
    i0 = (int)fl + 1;
    u = rem + 0.5f * (float)w.P - 1.f;
}
__device__ __forceinline__ void support(double x, const WaveGeom<double> &w, int &i0, double &u) {
    const double hi = x * w.gl_hi;
    const double lo = fma(x, w.gl_hi, -hi);
    const double th = hi - 0.5 * w.P;
    double fl = floor(th);
    double rem = (th - fl) + lo;
    if (rem < 0.0) {  // as in the float form: a tiny negative rem must not round back to 1
        fl -= 1.0;
        rem = fmin(rem + 1.0, 0.99999999999999989);
    } else if (rem >= 1.0) {
        fl += 1.0;
        rem -= 1.0;
    }
    i0 = (int)fl + 1;
    u = rem + 0.5 * w.P - 1.0;
}

#define PSE_PMAX 16

__device__ __forceinline__ int wrap_grid(int i, int M) {  // valid for i in [-M, 2M)
    i = i < 0 ? i + M : i;
    return i >= M ? i - M : i;
}

// ------------------------------------------------------------------ spreading
// Grid force density (unnormalised): grid_c(x_g) += sum_i w_x w_y w_z F_i,c over
// each particle's P^3 support, w = exp(-ch2 (u - p)^2) per axis as in the
// interpolation (the Gaussian's constant is applied in the mode factor).
//
// One CTA per tile of G^3 cells.  The tile's particles (cell-sorted, so each
// cell is a contiguous run) are spread into a padded E^3 node block in shared
// memory with shared-memory atomics, CP components per pass.  The block
// starts at the node orig[t] of each axis (host-computed: the support start of
// the tile's lower corner less one node) and E bounds the support of every
// particle of the tile with one node of margin on each side.  Two ways out:
//   scratch != null: the block is stored to scratch[tile][component] (plain
//     coalesced stores); k_spread_gather then sums, for every grid node, the
//     blocks that cover it (no global atomics);
//   scratch == null: the block is added to the grid with one coalesced float
//     atomic per nonzero node.
// A particle whose support still falls outside the block (not expected, kept
// for safety) adds straight into the global grid, which is cleared first.
#define PSE_SPREAD_THREADS 1024  // threads per CTA (occupancy while the shared atomics wait)
#define PSE_SPREAD_CHUNK 256     // particles staged per pass

__device__ __forceinline__ int pmod(int i, int M) {
    const int r = i % M;
    return r < 0 ? r + M : r;
}

template <typename T> __device__ __forceinline__ int64_t caller_of(T w) {
    if constexpr (sizeof(T) == 4) return (int64_t)__float_as_int(w);
    else return (int64_t)__double_as_longlong(w);
}

template <typename T>
__global__ void __launch_bounds__(PSE_SPREAD_THREADS)
    k_spread(WaveGeom<T> w, Geom<T> g, SpreadTile st, const int *__restrict__ orig, const V4<T> *__restrict__ pos_sorted,
             const int *__restrict__ cell_start, const SampleArgs<T> *args, T *grid, T *scratch,
             const Rec<T> *__restrict__ src) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int E = st.E, E2 = E * E, E3 = E2 * E, P = w.P, CP = st.CP, G = st.G, M = w.M;
    const int64_t M3 = (int64_t)M * M * M;
    T *tile = (T *)smem_raw;                                // CP * E^3
    T *wts = tile + CP * E3;                                // CHUNK * 3P
    T *fv = wts + PSE_SPREAD_CHUNK * 3 * P;                 // CHUNK * 3
    int *base = (int *)(fv + PSE_SPREAD_CHUNK * 3);         // CHUNK
    int *cst = base + PSE_SPREAD_CHUNK;                     // 64: first sorted index of each cell
    int *coff = cst + 64;                                   // 65: prefix of the cells' counts
    __shared__ int s_ncell;

    const int t = blockIdx.x;
    const int tz = t % st.ntx, ty = (t / st.ntx) % st.ntx, tx = t / (st.ntx * st.ntx);
    const int c0x = tx * G, c0y = ty * G, c0z = tz * G;
    const int ox = orig[tx], oy = orig[ty], oz = orig[tz];
    // cells of the tile and their particle runs
    const int G3 = G * G * G;
    if (threadIdx.x < G3) {
        const int a = threadIdx.x / (G * G), b = (threadIdx.x / G) % G, c = threadIdx.x % G;
        const int cx = c0x + a, cy = c0y + b, cz = c0z + c;
        int s0 = 0, n = 0;
        if (cx < g.nc && cy < g.nc && cz < g.nc) {
            const int id = cell_id(cx, cy, cz, g.nb);
            s0 = cell_start[id];
            n = cell_start[id + 1] - s0;
        }
        cst[threadIdx.x] = s0;
        coff[threadIdx.x + 1] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        coff[0] = 0;
        for (int j = 1; j <= G3; ++j) coff[j] += coff[j - 1];
        s_ncell = G3;
    }
    __syncthreads();
    const int ntile = coff[s_ncell];
    T *out = scratch ? scratch + (int64_t)t * 3 * E3 : nullptr;
    if (ntile == 0) {
        if (out)
            for (int i = threadIdx.x; i < 3 * E3; i += blockDim.x) out[i] = T(0);
        return;
    }
    const int PP = P * P;

    for (int cp0 = 0; cp0 < 3; cp0 += CP) {
        for (int i = threadIdx.x; i < CP * E3; i += blockDim.x) tile[i] = T(0);
        __syncthreads();
        for (int p0 = 0; p0 < ntile; p0 += PSE_SPREAD_CHUNK) {
            const int np = min(PSE_SPREAD_CHUNK, ntile - p0);
            if (threadIdx.x < np) {
                const int k = p0 + threadIdx.x;
                int lo = 0, hi = s_ncell - 1;  // last cell j with coff[j] <= k
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (coff[mid] <= k) lo = mid;
                    else hi = mid - 1;
                }
                const int64_t si = cst[lo] + (k - coff[lo]);
                const V4<T> p = pos_sorted[si];
                int i0x, i0y, i0z;
                T ux, uy, uz;
                support(p.x, w, i0x, ux);
                support(p.y, w, i0y, uy);
                support(p.z, w, i0z, uz);
                T *wv = wts + threadIdx.x * 3 * P;
                for (int q = 0; q < P; ++q) {
                    const T dx = ux - T(q), dy = uy - T(q), dz = uz - T(q);
                    wv[q] = exp_t(-w.ch2 * dx * dx);
                    wv[P + q] = exp_t(-w.ch2 * dy * dy);
                    wv[2 * P + q] = exp_t(-w.ch2 * dz * dz);
                }
                T *f = fv + threadIdx.x * 3;
                if (src) {  // a sorted-order vector (the Lanczos vector of the full-mobility iteration)
                    const V4<T> q = src[si].q;
                    f[0] = q.x; f[1] = q.y; f[2] = q.z;
                } else {
                    const T *F = args->vin + 3 * caller_of(p.w);
                    f[0] = F[0]; f[1] = F[1]; f[2] = F[2];
                }
                const int lx = i0x - ox, ly = i0y - oy, lz = i0z - oz;
                const bool inside = lx >= 0 && ly >= 0 && lz >= 0 && lx + P <= E && ly + P <= E && lz + P <= E;
                base[threadIdx.x] = inside ? (lx * E + ly) * E + lz : -1;
                if (!inside) {
                    for (int a = 0; a < P; ++a)
                        for (int b = 0; b < P; ++b)
                            for (int c = 0; c < P; ++c) {
                                const T wt = wv[a] * wv[P + b] * wv[2 * P + c];
                                const int64_t gi =
                                    ((int64_t)pmod(i0x + a, M) * M + pmod(i0y + b, M)) * M + pmod(i0z + c, M);
                                for (int cc = 0; cc < CP; ++cc) atomicAdd(grid + (cp0 + cc) * M3 + gi, wt * f[cp0 + cc]);
                            }
                }
            }
            __syncthreads();
            // thread t owns the (y, z) node pair q = t mod P^2 of particles
            // t / P^2, t / P^2 + stride, ...: no divisions in the loop
            const int stride = blockDim.x / PP;
            if (threadIdx.x < stride * PP) {
                const int q = threadIdx.x % PP, b = q / P, c = q - b * P;
                for (int pp = threadIdx.x / PP; pp < np; pp += stride) {
                    const int b0 = base[pp];
                    if (b0 < 0) continue;
                    const T *wv = wts + pp * 3 * P;
                    const T *f = fv + pp * 3 + cp0;
                    const T wyz = wv[P + b] * wv[2 * P + c];
                    const int row = b0 + b * E + c;
                    for (int a = 0; a < P; ++a) {
                        const T wt = wv[a] * wyz;
                        for (int cc = 0; cc < CP; ++cc) atomicAdd(tile + cc * E3 + row + a * E2, wt * f[cc]);
                    }
                }
            }
            __syncthreads();
        }
        if (out) {
            for (int i = threadIdx.x; i < CP * E3; i += blockDim.x) out[cp0 * E3 + i] = tile[i];
        } else {
            for (int i = threadIdx.x; i < E3; i += blockDim.x) {
                const int lz = i % E, ly = (i / E) % E, lx = i / E2;
                const int64_t gi = ((int64_t)pmod(ox + lx, M) * M + pmod(oy + ly, M)) * M + pmod(oz + lz, M);
                for (int cc = 0; cc < CP; ++cc) {
                    const T v = tile[cc * E3 + i];
                    if (v != T(0)) atomicAdd(grid + (cp0 + cc) * M3 + gi, v);
                }
            }
        }
        __syncthreads();
    }
}

// Second phase of the two-phase spreading: one thread per grid node (z
// fastest, so the reads of one block row are coalesced) adds the values the
// covering tile blocks hold for it.  cover[x * PSE_COVER + k] = (tile index
// along the axis, node offset in that tile's block) for the cnt[x] blocks
// covering node x along one axis (the same on the three axes of a cube).
template <typename T>
__global__ void __launch_bounds__(256) k_spread_gather(int M, int E, int ntx, const int2 *__restrict__ cover,
                                                       const int *__restrict__ cnt, const T *__restrict__ scratch,
                                                       T *grid) {
    const int64_t M3 = (int64_t)M * M * M;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= M3) return;
    const int z = (int)(g % M), y = (int)((g / M) % M), x = (int)(g / ((int64_t)M * M));
    const int E3 = E * E * E;
    const int nx = cnt[x], ny = cnt[y], nz = cnt[z];
    T a0 = 0, a1 = 0, a2 = 0;
    for (int i = 0; i < nx; ++i) {
        const int2 cx = cover[x * PSE_COVER + i];
        for (int j = 0; j < ny; ++j) {
            const int2 cy = cover[y * PSE_COVER + j];
            for (int k = 0; k < nz; ++k) {
                const int2 cz = cover[z * PSE_COVER + k];
                const int64_t tb = ((int64_t)(cx.x * ntx + cy.x) * ntx + cz.x) * 3 * E3;
                const int off = (cx.y * E + cy.y) * E + cz.y;
                a0 += scratch[tb + off];
                a1 += scratch[tb + E3 + off];
                a2 += scratch[tb + 2 * E3 + off];
            }
        }
    }
    grid[g] += a0;
    grid[M3 + g] += a1;
    grid[2 * M3 + g] += a2;
}

size_t spread_smem_bytes(SpreadTile st, int P, size_t elem) {
    return elem * ((size_t)st.CP * st.E * st.E * st.E + (size_t)PSE_SPREAD_CHUNK * (3 * P + 3)) +
           sizeof(int) * (PSE_SPREAD_CHUNK + 64 + 65);
}

// G lanes per sorted particle (G = 8, 16 or 32 divides the warp):
// u_w = norm * sum_{P^3} g_x g_y g_z v(node), separable weights
// exp(-ch2 (u - p)^2) per axis, periodic node indices.  Lane g of the group
// owns the (y, z) node pairs g, g + G, ...; for each x node the group's loads
// are runs of consecutive floats along z (the grid's contiguous axis).  The
// first P lanes of the group evaluate the 3P one-dimensional weights, shared
// by shuffles inside the group.
template <typename T, int G>
__device__ __forceinline__ void interp_particle(int64_t s, bool active, int lg, int gbase, const WaveGeom<T> &w,
                                                const V4<T> *__restrict__ pos_sorted, const T *__restrict__ grid,
                                                V4<T> *uwave) {
    const V4<T> p = pos_sorted[active ? s : 0];
    const int M = w.M, P = w.P;
    const int64_t M3 = (int64_t)M * M * M;
    int i0x, i0y, i0z;
    T ux, uy, uz;
    support(p.x, w, i0x, ux);
    support(p.y, w, i0y, uy);
    support(p.z, w, i0z, uz);
    T wxl = 0, wyl = 0, wzl = 0;
    if (lg < P) {
        const T dx = ux - T(lg), dy = uy - T(lg), dz = uz - T(lg);
        wxl = exp_t(-w.ch2 * dx * dx);
        wyl = exp_t(-w.ch2 * dy * dy);
        wzl = exp_t(-w.ch2 * dz * dz);
    }
    T ax = 0, ay = 0, az = 0;
    const int PP = P * P;
    for (int q0 = 0; q0 < PP; q0 += G) {
        const int q = q0 + lg;
        const bool on = active && q < PP;
        const int b = q < PP ? q / P : 0;
        const int c = q < PP ? q - b * P : 0;
        const T wy = __shfl_sync(0xffffffffu, wyl, gbase + (b < G ? b : 0));
        const T wz = __shfl_sync(0xffffffffu, wzl, gbase + (c < G ? c : 0));
        const int iy = wrap_grid(i0y + b, M), iz = wrap_grid(i0z + c, M);
        const T wyz = wy * wz;
        const int64_t rowyz = (int64_t)iy * M + iz;
        for (int a = 0; a < P; ++a) {
            const T wx = __shfl_sync(0xffffffffu, wxl, gbase + (a < G ? a : 0));
            if (on) {
                const int64_t idx = (int64_t)wrap_grid(i0x + a, M) * M * M + rowyz;
                const T wt = wx * wyz;
                ax += wt * __ldg(grid + idx);
                ay += wt * __ldg(grid + M3 + idx);
                az += wt * __ldg(grid + 2 * M3 + idx);
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (active && lg == 0) {
        V4<T> o;
        o.x = ax * w.norm; o.y = ay * w.norm; o.z = az * w.norm; o.w = T(0);
        uwave[s] = o;
    }
}

// Fused over the systems of a batch (wave noise of every system's half
// spectrum; interpolation with 16 lanes per particle, P <= 16).
__global__ void k_wave_noise_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    const BSys &S = sys[tab[blockIdx.x]];
    const int lb = (int)blockIdx.x - S.b0[BK_NOISE];
    const int64_t plane = (int64_t)S.w.M * S.w.M * S.w.Mh1;
    const int64_t stride = (int64_t)S.nb[BK_NOISE] * blockDim.x;
    for (int64_t t = lb * (int64_t)blockDim.x + threadIdx.x; t < plane; t += stride)
        wave_noise_elem<float>(t, S.w, S.d.args, S.system, (cufftComplex *)S.d.spec, plane);
}

// One lane group per particle, one launch-wide pass.
template <typename T, int G>
__global__ void __launch_bounds__(128) k_interp(int64_t N, WaveGeom<T> w, const V4<T> *__restrict__ pos_sorted,
                                                const T *__restrict__ grid, V4<T> *uwave) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lg = threadIdx.x % G;
    interp_particle<T, G>(tid / G, tid / G < N, lg, (threadIdx.x & 31) - lg, w, pos_sorted, grid, uwave);
}

__global__ void __launch_bounds__(128) k_interp_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    constexpr int G = PSE_BATCH_INTERP_G;
    const BSys &S = sys[tab[blockIdx.x]];
    const int lb = (int)blockIdx.x - S.b0[BK_INTERP];
    const int lg = threadIdx.x % G;
    const int64_t per_block = blockDim.x / G;
    for (int64_t base = lb * per_block; base < S.N; base += (int64_t)S.nb[BK_INTERP] * per_block) {  // uniform
        const int64_t s = base + threadIdx.x / G;
        interp_particle<float, G>(s, s < S.N, lg, (threadIdx.x & 31) - lg, S.w, S.d.pos_sorted, S.d.grid, S.d.uwave);
    }
}

// Node-major copy of the three planar velocity grids: one 16-byte record
// (x, y, z, 0) per node, so that the interpolation reads a node with one load.
__global__ void k_grid_aos(int64_t M3, const float *__restrict__ g, V4<float> *__restrict__ g4) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M3) return;
    V4<float> v;
    v.x = __ldg(g + i);
    v.y = __ldg(g + M3 + i);
    v.z = __ldg(g + 2 * M3 + i);
    v.w = 0.f;
    g4[i] = v;
}

// Interpolation from the node-major grid: a group of P lanes per particle,
// floor(32 / P) particles per warp (consecutive in cell order, so their
// supports overlap in L1).  Lane c of a group owns the z-node c of the
// support and walks the P x P (x, y) columns, one 16-byte load per node; it
// evaluates the 1-D weights of index c on all three axes, which the group's
// lanes exchange by shuffles.  The group's partial sums meet in its first lane.
template <int P>
__device__ __forceinline__ void interp4_warp(int64_t warp0, int64_t N, const WaveGeom<float> &w,
                                             const V4<float> *__restrict__ pos_sorted,
                                             const V4<float> *__restrict__ grid4, V4<float> *uwave,
                                             const V4<float> *__restrict__ loc = nullptr) {
    constexpr int R = 32 / P;  // particles per warp; lanes R P .. 31 idle
    const int lane = threadIdx.x & 31;
    const int g = lane / P, c = lane - (lane / P) * P;
    const int64_t s = warp0 + g;
    const bool act = g < R && s < N;
    const int base = (g < R ? g : 0) * P;  // first lane of the group
    const V4<float> p = pos_sorted[act ? s : 0];
    const int M = w.M;
    if (loc) {  // polydisperse: the grid of this particle's species
        const int sp = (__float_as_int(loc[act ? s : 0].w) >> PSE_SPECIES_SHIFT) & 3;
        grid4 += (int64_t)sp * M * M * M;
    }
    int i0x, i0y, i0z;
    float ux, uy, uz;
    support(p.x, w, i0x, ux);
    support(p.y, w, i0y, uy);
    support(p.z, w, i0z, uz);
    const float fc = float(c);
    const float ex = ux - fc, ey = uy - fc, ez = uz - fc;
    const float wxc = expf(-w.ch2 * ex * ex);
    const float wyc = expf(-w.ch2 * ey * ey);
    const float wzc = expf(-w.ch2 * ez * ez);
    const int izc = wrap_grid(i0z + c, M);
    float wyz[P];
    int row[P];
#pragma unroll
    for (int b = 0; b < P; ++b) {
        wyz[b] = __shfl_sync(0xffffffffu, wyc, base + b) * wzc;
        row[b] = wrap_grid(i0y + b, M) * M + izc;
    }
    const float4 *g4 = reinterpret_cast<const float4 *>(grid4);
    const int64_t MM = (int64_t)M * M;
    float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll 1
    for (int a = 0; a < P; ++a) {
        const float wxa = __shfl_sync(0xffffffffu, wxc, base + a);
        const float4 *plane = g4 + wrap_grid(i0x + a, M) * MM;
        if (act) {
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const float4 v = __ldg(plane + row[b]);
                const float wt = wxa * wyz[b];
                ax = fmaf(wt, v.x, ax);
                ay = fmaf(wt, v.y, ay);
                az = fmaf(wt, v.z, az);
            }
        }
    }
    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        sx += __shfl_sync(0xffffffffu, ax, base + k);
        sy += __shfl_sync(0xffffffffu, ay, base + k);
        sz += __shfl_sync(0xffffffffu, az, base + k);
    }
    if (act && c == 0) {
        V4<float> o;
        o.x = sx * w.norm; o.y = sy * w.norm; o.z = sz * w.norm; o.w = 0.f;
        uwave[s] = o;
    }
}

template <int P>
__global__ void __launch_bounds__(128) k_interp4(int64_t N, WaveGeom<float> w,
                                                 const V4<float> *__restrict__ pos_sorted,
                                                 const V4<float> *__restrict__ grid4, V4<float> *uwave,
                                                 const V4<float> *__restrict__ loc) {
    const int64_t warp0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (32 / P);
    if (warp0 >= N) return;  // whole warps leave together
    interp4_warp<P>(warp0, N, w, pos_sorted, grid4, uwave, loc);
}

// Fused over the systems of a batch: the node-major copy of every system's
// grid, then the interpolation of every system (all with the same P).
__global__ void k_grid_aos_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    const BSys &S = sys[tab[blockIdx.x]];
    const int lb = (int)blockIdx.x - S.b0[BK_COPY];
    const int64_t M3 = (int64_t)S.w.M * S.w.M * S.w.M;
    const int64_t stride = (int64_t)S.nb[BK_COPY] * blockDim.x;
    for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < M3; i += stride) {
        V4<float> v;
        v.x = __ldg(S.d.grid + i);
        v.y = __ldg(S.d.grid + M3 + i);
        v.z = __ldg(S.d.grid + 2 * M3 + i);
        v.w = 0.f;
        S.d.grid4[i] = v;
    }
}
template <int P> __global__ void __launch_bounds__(128) k_interp4_batch(const BSys *__restrict__ sys,
                                                                         const int *__restrict__ tab) {
    constexpr int R = 32 / P;
    const BSys &S = sys[tab[blockIdx.x]];
    const int lb = (int)blockIdx.x - S.b0[BK_INTERP];
    const int64_t per_block = (blockDim.x / 32) * R;
    const int64_t wofs = (threadIdx.x >> 5) * R;
    for (int64_t base = lb * per_block; base < S.N; base += (int64_t)S.nb[BK_INTERP] * per_block)  // uniform
        if (base + wofs < S.N) interp4_warp<P>(base + wofs, S.N, S.w, S.d.pos_sorted, S.d.grid4, S.d.uwave);
}

static inline unsigned nbw(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int P>
static void interp4(int64_t N, const WaveGeom<float> &w, const Dev<float> &d, cudaStream_t s) {
    const int64_t warps = (N + 32 / P - 1) / (32 / P);
    k_interp4<P><<<nbw(warps * 32, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid4, d.uwave,
                                                      w.nspec > 1 ? d.loc_sorted : nullptr);
}

void launch_batch_noise(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s) {
    k_wave_noise_batch<<<nblk[BK_NOISE], 256, 0, s>>>(sys, tab[BK_NOISE]);
}
void launch_batch_interp(const BSys *sys, int *const *tab, const int *nblk, int P4, cudaStream_t s) {
    if (P4 == 0) {
        k_interp_batch<<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]);
        return;
    }
    k_grid_aos_batch<<<nblk[BK_COPY], 256, 0, s>>>(sys, tab[BK_COPY]);
    switch (P4) {
        case 3: k_interp4_batch<3><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 4: k_interp4_batch<4><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 5: k_interp4_batch<5><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 6: k_interp4_batch<6><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 7: k_interp4_batch<7><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 8: k_interp4_batch<8><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        case 9: k_interp4_batch<9><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
        default: k_interp4_batch<10><<<nblk[BK_INTERP], 128, 0, s>>>(sys, tab[BK_INTERP]); break;
    }
}

template <typename T>
void launch_wave_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, void *spec, cudaStream_t s) {
    const int64_t plane = (int64_t)w.M * w.M * w.Mh1;
    k_wave_noise<T><<<nbw(plane, 256), 256, 0, s>>>(w, args, system, (typename Cplx<T>::type *)spec, plane);
}
template <typename T> void launch_grid_copy(WaveGeom<T> w, const Dev<T> &d, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (w.interp_lanes == 0 && w.P >= 3 && w.P <= 10) {
            const int64_t M3 = (int64_t)w.M * w.M * w.M;
            for (int sp = 0; sp < (w.nspec > 1 ? w.nspec : 1); ++sp)  // one grid per species
                k_grid_aos<<<nbw(M3, 256), 256, 0, s>>>(M3, d.grid + (int64_t)sp * 3 * M3, d.grid4 + sp * M3);
        }
    }
}
template <typename T> void launch_interp(int64_t N, WaveGeom<T> w, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (w.interp_lanes == 0 && w.P >= 3 && w.P <= 10) {
            switch (w.P) {
                case 3: interp4<3>(N, w, d, s); break;
                case 4: interp4<4>(N, w, d, s); break;
                case 5: interp4<5>(N, w, d, s); break;
                case 6: interp4<6>(N, w, d, s); break;
                case 7: interp4<7>(N, w, d, s); break;
                case 8: interp4<8>(N, w, d, s); break;
                case 9: interp4<9>(N, w, d, s); break;
                default: interp4<10>(N, w, d, s); break;
            }
            return;
        }
    }
    // the group must hold the P lanes that evaluate the 1-D weights
    const int G = w.interp_lanes >= w.P ? w.interp_lanes : (w.P <= 8 ? 8 : (w.P <= 16 ? 16 : 32));
    if (G <= 8) k_interp<T, 8><<<nbw(N * 8, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
    else if (G <= 16) k_interp<T, 16><<<nbw(N * 16, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
    else k_interp<T, 32><<<nbw(N * 32, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
}

template <typename T>
void launch_wave_apply(WaveGeom<T> w, const SampleArgs<T> *args, int system, void *spec, int mode, int with_noise,
                       cudaStream_t s) {
    const int64_t plane = (int64_t)w.M * w.M * w.Mh1;
    k_wave_apply<T><<<nbw(plane, 256), 256, 0, s>>>(w, args, system, (typename Cplx<T>::type *)spec, plane, mode,
                                                    with_noise);
}
template <typename T> void launch_grid_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, T *grid,
                                             cudaStream_t s) {
    const int64_t M3 = (int64_t)w.M * w.M * w.M;
    k_grid_noise<T><<<nbw(M3, 256), 256, 0, s>>>(M3, args, system, grid);
}
// Opt the spreading kernel in to all the dynamic shared memory a block may
// have on this device (the opt-in limit less the kernel's static shared
// memory); returns that size.  Called once, outside any stream capture.
template <typename T> cudaError_t spread_prepare(size_t *max_dynamic) {
    *max_dynamic = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_spread<T>);
    if (e != cudaSuccess) return e;
    const size_t avail = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    e = cudaFuncSetAttribute(k_spread<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail);
    if (e == cudaSuccess) *max_dynamic = avail;
    return e;
}
// Spread into d.grid (cleared by the caller).  With a cover table the tile
// blocks go through scratch and the gather kernel; otherwise they are added
// with atomics.
template <typename T>
cudaError_t launch_spread(WaveGeom<T> w, Geom<T> g, SpreadTile st, const int *orig, const int2 *cover,
                          const int *cover_cnt, T *scratch, const Dev<T> &d, cudaStream_t s,
                          const Rec<T> *src) {
    const size_t smem = spread_smem_bytes(st, w.P, sizeof(T));
    const unsigned tiles = (unsigned)st.ntx * st.ntx * st.ntx;
    const bool two_phase = scratch && cover && cover_cnt;
    k_spread<T><<<tiles, PSE_SPREAD_THREADS, smem, s>>>(w, g, st, orig, d.pos_sorted, d.cell_start, d.args, d.grid,
                                                         two_phase ? scratch : nullptr, src);
    if (two_phase) {
        const int64_t M3 = (int64_t)w.M * w.M * w.M;
        k_spread_gather<T><<<nbw(M3, 256), 256, 0, s>>>(w.M, st.E, st.ntx, cover, cover_cnt, scratch, d.grid);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fused k-space noise and inverse FFT
// For grids M = R^2 (R = 8, 16: M = 64, 256; FP32, k-space noise): the
// unnormalised C2R of the noise spectrum in three passes of our own, the
// noise generated inside the first pass and the last pass writing the
// node-major records the interpolation reads (no spectrum written by a noise
// kernel, no planar grid, no copy).
//   pass x: per (ky, tile of kz < M/2): noise of the modes, DFT over kx;
//   pass y: per (ix, tile of kz): DFT over ky, in place in the spectrum buffer;
//   pass z: per (ix, tile of iy): the real inverse DFT over kz, two real rows
//           per complex transform (z = IDFT(Ya + i Yb): x_a = Re z, x_b = Im z,
//           Y extended by Y_{M-k} = conj(Y_k), the Nyquist term Y_{M/2} = 0).
// Each line of M = R^2 points is transformed by R threads in two register
// passes (the four-step split n = t + R m, k = k1 + R k2):
//   A_t[k1] = w_M^{t k1} sum_m x[t + R m] w_R^{m k1},
//   X[k1 + R k2] = sum_t A_t[k1] w_R^{t k2},  w_L = e^{2 pi i / L},
// with one padded shared-memory transpose between them.
constexpr int PSE_FFT_TZ = 8;   // kz values per block in the x and y passes
constexpr int PSE_FFT_TY = 8;   // iy rows per block in the z pass

template <int R> __device__ __forceinline__ constexpr int bitrev_c(int v) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (v & 1);
        v >>= 1;
    }
    return r;
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-register radix-2 DIT of R points: v in bit-reversed order, output in
// natural order, w[k] = w_R^k for k < R/2.
template <int R> __device__ __forceinline__ void fft_reg(float2 (&v)[R], const float2 (&w)[R / 2]) {
#pragma unroll
    for (int half = 1; half < R; half <<= 1) {
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const int pos = j & (half - 1);
            const int i0 = ((j - pos) << 1) + pos, i1 = i0 + half;
            const float2 t = cmulf(w[pos * (R / (2 * half))], v[i1]);
            const float2 a = v[i0];
            v[i0] = make_float2(a.x + t.x, a.y + t.y);
            v[i1] = make_float2(a.x - t.x, a.y - t.y);
        }
    }
}

// w_M^j for any j >= 0 from the half-circle table tw[k] = w_M^k, k < M/2.
template <int M> __device__ __forceinline__ float2 tw_full(const float2 *tw, int j) {
    j &= M - 1;
    const float2 e = tw[j & (M / 2 - 1)];
    return j < M / 2 ? e : make_float2(-e.x, -e.y);
}

// One line of M = R^2 points, natural order in `line` (stride 1, R (R + 1)
// entries of room), transformed by the R threads t = 0..R-1 of a group;
// returns X[t + R k2] in out[k2].  The group's threads must lie in one warp.
template <int R>
__device__ __forceinline__ void fft_line_sq(float2 *line, int t, const float2 *tw, const float2 (&wR)[R / 2],
                                            float2 (&out)[R]) {
    constexpr int M = R * R;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = line[t + R * bitrev_c<R>(m)];
    fft_reg<R>(v, wR);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmulf(v[k1], tw_full<M>(tw, t * k1));
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) line[k1 * (R + 1) + t] = v[k1];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R; ++m) out[m] = line[t * (R + 1) + bitrev_c<R>(m)];
    fft_reg<R>(out, wR);
    __syncwarp();
}

// Shared-memory line stride: room for the R (R + 1) transpose, padded to
// 4 mod 16 float2 so that the TZ lines touched by one row of a tile load or
// store start on different banks.
template <int R> constexpr int fft_lsz() { return R * (R + 1) + ((4 - R * (R + 1)) % 16 + 16) % 16; }

template <int R> __device__ __forceinline__ void load_wR(const float2 *tw, float2 (&wR)[R / 2]) {
#pragma unroll
    for (int k = 0; k < R / 2; ++k) wR[k] = tw[k * R];  // w_R^k = w_M^{k R}
}

// pass x: block = (tile of TZ kz values, ky); threads: 3 TZ lines x R.
template <int R>
__global__ void __launch_bounds__(3 * PSE_FFT_TZ * R, 3) k_fftx_noise(WaveGeom<float> w, const SampleArgs<float> *args,
                                                                   int system, const float2 *__restrict__ tw_g,
                                                                   float2 *spec) {
    constexpr int M = R * R, TZ = PSE_FFT_TZ, LSZ = fft_lsz<R>(), Mh1 = M / 2 + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm;           // M/2
    float2 *buf = sm + M / 2;  // [3 TZ lines][LSZ], line = c * TZ + kzl
    for (int k = threadIdx.x; k < M / 2; k += blockDim.x) tw[k] = tw_g[k];
    const int kz0 = blockIdx.x * TZ, ky = blockIdx.y;
    const uint32_t strm = 2u * system + 1u;
    const uint64_t seed = args->seed, sample = args->sample;
    for (int i = threadIdx.x; i < M * TZ; i += blockDim.x) {
        const int kzl = i % TZ, kx = i / TZ;
        ModeIdx m;
        m.ix = kx; m.iy = ky; m.iz = kz0 + kzl;
        m.nx = kx <= M / 2 ? kx : kx - M;
        m.ny = ky <= M / 2 ? ky : ky - M;
        m.nz = m.iz;
        m.live = kx != M / 2 && ky != M / 2 && (m.nx | m.ny | m.nz) != 0;
        float2 o0 = make_float2(0.f, 0.f), o1 = o0, o2 = o0;
        if (m.live) {
            float wr[3], wi[3];
            mode_noise<float>(m, M, Mh1, strm, seed, sample, wr, wi);
            float hx, hy, hz;
            const float sc = mode_scale<float>(m, w, hx, hy, hz);
            const float dr = hx * wr[0] + hy * wr[1] + hz * wr[2];
            const float di = hx * wi[0] + hy * wi[1] + hz * wi[2];
            o0 = make_float2(sc * (wr[0] - hx * dr), sc * (wi[0] - hx * di));
            o1 = make_float2(sc * (wr[1] - hy * dr), sc * (wi[1] - hy * di));
            o2 = make_float2(sc * (wr[2] - hz * dr), sc * (wi[2] - hz * di));
        }
        buf[(0 * TZ + kzl) * LSZ + kx] = o0;
        buf[(1 * TZ + kzl) * LSZ + kx] = o1;
        buf[(2 * TZ + kzl) * LSZ + kx] = o2;
    }
    __syncthreads();
    float2 wR[R / 2];
    load_wR<R>(tw, wR);
    const int line = threadIdx.x / R, t = threadIdx.x % R;
    float2 out[R];
    fft_line_sq<R>(buf + line * LSZ, t, tw, wR, out);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) buf[line * LSZ + t + R * k2] = out[k2];
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * M * TZ; i += blockDim.x) {
        const int kzl = i % TZ, rest = i / TZ, ix = rest % M, c = rest / M;
        spec[(((int64_t)c * M + ix) * M + ky) * Mh1 + kz0 + kzl] = buf[(c * TZ + kzl) * LSZ + ix];
    }
}

// pass y: block = (tile of TZ kz values, ix); in place.
template <int R>
__global__ void __launch_bounds__(3 * PSE_FFT_TZ * R, 3) k_ffty(const float2 *__restrict__ tw_g, float2 *spec) {
    constexpr int M = R * R, TZ = PSE_FFT_TZ, LSZ = fft_lsz<R>(), Mh1 = M / 2 + 1;
    extern __shared__ float2 sm[];
    float2 *tw = sm;
    float2 *buf = sm + M / 2;
    for (int k = threadIdx.x; k < M / 2; k += blockDim.x) tw[k] = tw_g[k];
    const int kz0 = blockIdx.x * TZ, ix = blockIdx.y;
    for (int i = threadIdx.x; i < 3 * M * TZ; i += blockDim.x) {
        const int kzl = i % TZ, rest = i / TZ, ky = rest % M, c = rest / M;
        buf[(c * TZ + kzl) * LSZ + ky] = spec[(((int64_t)c * M + ix) * M + ky) * Mh1 + kz0 + kzl];
    }
    __syncthreads();
    float2 wR[R / 2];
    load_wR<R>(tw, wR);
    const int line = threadIdx.x / R, t = threadIdx.x % R;
    float2 out[R];
    fft_line_sq<R>(buf + line * LSZ, t, tw, wR, out);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) buf[line * LSZ + t + R * k2] = out[k2];
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * M * TZ; i += blockDim.x) {
        const int kzl = i % TZ, rest = i / TZ, ky = rest % M, c = rest / M;
        spec[(((int64_t)c * M + ix) * M + ky) * Mh1 + kz0 + kzl] = buf[(c * TZ + kzl) * LSZ + ky];
    }
}

// pass z: block = (tile of TY iy rows, ix); the 3 TY real rows (c, iyl) are
// transformed in pairs (c, iyl) + i (c, iyl + TY/2).
template <int R>
__global__ void __launch_bounds__(3 * PSE_FFT_TY / 2 * R) k_fftz_c2r(const float2 *__restrict__ tw_g,
                                                                   const float2 *__restrict__ spec, V4<float> *grid4) {
    constexpr int M = R * R, H = M / 2, TY = PSE_FFT_TY, LSZ = fft_lsz<R>(), Mh1 = M / 2 + 1, NP = 3 * TY / 2;
    extern __shared__ float2 sm[];
    float2 *tw = sm;                      // M/2
    float2 *raw = tw + M / 2;             // [3][TY][H]
    float2 *buf = raw + 3 * TY * H;       // [NP][LSZ]
    float *xo = reinterpret_cast<float *>(raw);  // [3][TY][M], over raw once Z is built
    for (int k = threadIdx.x; k < M / 2; k += blockDim.x) tw[k] = tw_g[k];
    const int iy0 = blockIdx.x * TY, ix = blockIdx.y;
    for (int i = threadIdx.x; i < 3 * TY * H; i += blockDim.x) {
        const int k = i % H, rest = i / H, iyl = rest % TY, c = rest / TY;
        raw[i] = spec[(((int64_t)c * M + ix) * M + iy0 + iyl) * Mh1 + k];
    }
    __syncthreads();
    // pair p = c * (TY/2) + j holds rows (c, j) and (c, j + TY/2)
    for (int i = threadIdx.x; i < NP * M; i += blockDim.x) {
        const int k = i % M, p = i / M, c = p / (TY / 2), j = p % (TY / 2);
        const float2 *ra = raw + (c * TY + j) * H, *rb = raw + (c * TY + j + TY / 2) * H;
        float2 ya, yb;
        if (k < H) {
            ya = ra[k];
            yb = rb[k];
        } else if (k == H) {
            ya = yb = make_float2(0.f, 0.f);
        } else {
            const float2 a = ra[M - k], b = rb[M - k];
            ya = make_float2(a.x, -a.y);
            yb = make_float2(b.x, -b.y);
        }
        buf[p * LSZ + k] = make_float2(ya.x - yb.y, ya.y + yb.x);  // Ya + i Yb
    }
    __syncthreads();
    float2 wR[R / 2];
    load_wR<R>(tw, wR);
    const int p = threadIdx.x / R, t = threadIdx.x % R;
    float2 out[R];
    fft_line_sq<R>(buf + p * LSZ, t, tw, wR, out);
    {
        const int c = p / (TY / 2), j = p % (TY / 2);
        float *xa = xo + (c * TY + j) * M, *xb = xo + (c * TY + j + TY / 2) * M;
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) {
            xa[t + R * k2] = out[k2].x;
            xb[t + R * k2] = out[k2].y;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TY * M; i += blockDim.x) {
        const int iz = i % M, iyl = i / M;
        V4<float> v;
        v.x = xo[(0 * TY + iyl) * M + iz];
        v.y = xo[(1 * TY + iyl) * M + iz];
        v.z = xo[(2 * TY + iyl) * M + iz];
        v.w = 0.f;
        grid4[((int64_t)ix * M + iy0 + iyl) * M + iz] = v;
    }
}

template <int R> static size_t fft_smem_xy() {
    return sizeof(float2) * (R * R / 2 + 3 * PSE_FFT_TZ * fft_lsz<R>());
}
template <int R> static size_t fft_smem_z() {
    constexpr int M = R * R;  // raw (3 TY rows of M/2 float2) is reused for the 3 TY rows of M real outputs
    return sizeof(float2) * (M / 2 + 3 * PSE_FFT_TY * (M / 2) + 3 * PSE_FFT_TY / 2 * fft_lsz<R>());
}

template <int R> static void fused_fft_launch(const WaveGeom<float> &w, const SampleArgs<float> *args, int system,
                                              const Dev<float> &d, int parts, cudaStream_t s) {
    constexpr int M = R * R;
    const float2 *tw = reinterpret_cast<const float2 *>(w.fft_tw);
    float2 *spec = reinterpret_cast<float2 *>(d.spec);
    const dim3 gxy(M / 2 / PSE_FFT_TZ, M), gz(M / PSE_FFT_TY, M);
    if (parts & 1) k_fftx_noise<R><<<gxy, 3 * PSE_FFT_TZ * R, fft_smem_xy<R>(), s>>>(w, args, system, tw, spec);
    if (parts & 2) k_ffty<R><<<gxy, 3 * PSE_FFT_TZ * R, fft_smem_xy<R>(), s>>>(tw, spec);
    if (parts & 4) k_fftz_c2r<R><<<gz, 3 * PSE_FFT_TY / 2 * R, fft_smem_z<R>(), s>>>(tw, spec, d.grid4);
}

bool fused_fft_supported(int M) { return M == 64 || M == 256; }

template <int R> static cudaError_t fused_fft_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_fftx_noise<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fft_smem_xy<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ffty<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem_xy<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fftz_c2r<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem_z<R>());
    return e;
}

cudaError_t fused_fft_prepare(int M) {
    if (M == 64) return fused_fft_attrs<8>();
    if (M == 256) return fused_fft_attrs<16>();
    return cudaErrorInvalidValue;
}

void launch_fused_fft(const WaveGeom<float> &w, const SampleArgs<float> *args, int system, const Dev<float> &d,
                      int parts, cudaStream_t s) {
    if (w.M == 64) fused_fft_launch<8>(w, args, system, d, parts, s);
    else fused_fft_launch<16>(w, args, system, d, parts, s);
}

#define PSE_INST(T)                                                                                      \
    template void launch_wave_noise<T>(WaveGeom<T>, const SampleArgs<T> *, int, void *, cudaStream_t); \
    template void launch_interp<T>(int64_t, WaveGeom<T>, Geom<T>, const Dev<T> &, cudaStream_t);       \
    template void launch_grid_copy<T>(WaveGeom<T>, const Dev<T> &, cudaStream_t);                        \
    template void launch_wave_apply<T>(WaveGeom<T>, const SampleArgs<T> *, int, void *, int, int, cudaStream_t); \
    template void launch_grid_noise<T>(WaveGeom<T>, const SampleArgs<T> *, int, T *, cudaStream_t);   \
    template cudaError_t launch_spread<T>(WaveGeom<T>, Geom<T>, SpreadTile, const int *, const int2 *, const int *, \
                                          T *, const Dev<T> &, cudaStream_t, const Rec<T> *);                                      \
    template cudaError_t spread_prepare<T>(size_t *);
PSE_INST(float)
PSE_INST(double)
#undef PSE_INST

}  // namespace pse
