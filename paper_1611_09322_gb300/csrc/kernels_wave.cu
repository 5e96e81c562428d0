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

template <typename T> __device__ __forceinline__ T sinc_over_k(T k, T a) {
    const T ka = k * a;
    if constexpr (sizeof(T) == 4) return sinf(ka) / (ka * k);
    else return sin(ka) / (ka * k);
}
template <typename T> __device__ __forceinline__ T exp_t(T x) {
    if constexpr (sizeof(T) == 4) return expf(x);
    else return exp(x);
}
template <typename T> __device__ __forceinline__ T sqrt_t(T x) {
    if constexpr (sizeof(T) == 4) return sqrtf(x);
    else return sqrt(x);
}

// One thread per half-spectrum mode (ix, iy, iz), iz in [0, M/2].  The noise
// of a {k, -k} pair is keyed by its representative (nz > 0, or nz = 0 and
// (ny > 0 or (ny = 0 and nx > 0))), id q = (ix*M + iy)*Mh1 + iz, Philox
// blocks 2q and 2q+1; a thread holding the partner draws the same numbers
// and conjugates them, so the kz = 0 plane is exactly Hermitian.  k = 0 and
// Nyquist modes are zero.
template <typename T>
__global__ void k_wave_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, typename Cplx<T>::type *spec,
                             int64_t plane) {
    using C = typename Cplx<T>::type;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nmodes = (int64_t)w.M * w.M * w.Mh1;
    if (t >= nmodes) return;
    const int iz = (int)(t % w.Mh1);
    const int iy = (int)((t / w.Mh1) % w.M);
    const int ix = (int)(t / ((int64_t)w.Mh1 * w.M));
    const int M = w.M, half = M / 2;
    const int nx = ix <= half ? ix : ix - M;
    const int ny = iy <= half ? iy : iy - M;
    const int nz = iz;
    const bool even = (M % 2) == 0;
    const bool nyq = even && (ix == half || iy == half || iz == half);
    C o0, o1, o2;
    o0.x = o0.y = o1.x = o1.y = o2.x = o2.y = T(0);
    if (!nyq && (nx | ny | nz) != 0) {
        int rx = ix, ry = iy;
        bool conj = false;
        if (nz == 0 && !(ny > 0 || (ny == 0 && nx > 0))) {
            rx = (M - ix) % M;
            ry = (M - iy) % M;
            conj = true;
        }
        const uint32_t q = (uint32_t)(((int64_t)rx * M + ry) * w.Mh1 + iz);
        const uint32_t strm = 2u * system + 1u;
        const Normals4<T> a = normals4<T>(2u * q, strm, args->seed, args->sample);
        const Normals4<T> b = normals4<T>(2u * q + 1u, strm, args->seed, args->sample);
        const T s2 = T(0.70710678118654752440);
        T wr[3] = {a.v[0] * s2, a.v[2] * s2, b.v[0] * s2};
        T wi[3] = {a.v[1] * s2, a.v[3] * s2, b.v[1] * s2};
        if (conj) { wi[0] = -wi[0]; wi[1] = -wi[1]; wi[2] = -wi[2]; }
        const T kx = w.kscale * nx, ky = w.kscale * ny, kz = w.kscale * nz;
        const T k2 = kx * kx + ky * ky + kz * kz;
        const T k = sqrt_t(k2);
        const T hx = kx / k, hy = ky / k, hz = kz / k;
        const T dr = hx * wr[0] + hy * wr[1] + hz * wr[2];
        const T di = hx * wi[0] + hy * wi[1] + hz * wi[2];
        const T sc = w.inv_sqrtV * sinc_over_k(k, w.a) * sqrt_t(T(1) + k2 * w.inv4xi2) * exp_t(-w.decay * k2);
        o0.x = sc * (wr[0] - hx * dr); o0.y = sc * (wi[0] - hx * di);
        o1.x = sc * (wr[1] - hy * dr); o1.y = sc * (wi[1] - hy * di);
        o2.x = sc * (wr[2] - hz * dr); o2.y = sc * (wi[2] - hz * di);
    }
    spec[t] = o0;
    spec[plane + t] = o1;
    spec[2 * plane + t] = o2;
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
    if (rem < 0.f) { fl -= 1.f; rem += 1.f; }
    if (rem >= 1.f) { fl += 1.f; rem -= 1.f; }
    i0 = (int)fl + 1;
    u = rem + 0.5f * (float)w.P - 1.f;
}
__device__ __forceinline__ void support(double x, const WaveGeom<double> &w, int &i0, double &u) {
    const double hi = x * w.gl_hi;
    const double lo = fma(x, w.gl_hi, -hi);
    const double th = hi - 0.5 * w.P;
    double fl = floor(th);
    double rem = (th - fl) + lo;
    if (rem < 0.0) { fl -= 1.0; rem += 1.0; }
    if (rem >= 1.0) { fl += 1.0; rem -= 1.0; }
    i0 = (int)fl + 1;
    u = rem + 0.5 * w.P - 1.0;
}

#define PSE_PMAX 16

__device__ __forceinline__ int wrap_grid(int i, int M) {  // valid for i in [-M, 2M)
    i = i < 0 ? i + M : i;
    return i >= M ? i - M : i;
}

// G lanes per sorted particle (G = 8, 16 or 32 divides the warp):
// u_w = norm * sum_{P^3} g_x g_y g_z v(node), separable weights
// exp(-ch2 (u - p)^2) per axis, periodic node indices.  Lane g of the group
// owns the (y, z) node pairs g, g + G, ...; for each x node the group's loads
// are runs of consecutive floats along z (the grid's contiguous axis).  The
// first P lanes of the group evaluate the 3P one-dimensional weights, shared
// by shuffles inside the group.
template <typename T, int G>
__global__ void __launch_bounds__(128) k_interp(int64_t N, WaveGeom<T> w, const V4<T> *__restrict__ pos_sorted,
                                                const T *__restrict__ grid, V4<T> *uwave) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = tid / G;
    const int lg = threadIdx.x % G;
    const int gbase = (threadIdx.x & 31) - lg;  // first lane of this group in the warp
    const bool active = s < N;
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

static inline unsigned nbw(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
void launch_wave_noise(WaveGeom<T> w, const SampleArgs<T> *args, int system, void *spec, cudaStream_t s) {
    const int64_t plane = (int64_t)w.M * w.M * w.Mh1;
    k_wave_noise<T><<<nbw(plane, 256), 256, 0, s>>>(w, args, system, (typename Cplx<T>::type *)spec, plane);
}
template <typename T> void launch_interp(int64_t N, WaveGeom<T> w, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    // the group must hold the P lanes that evaluate the 1-D weights
    const int G = w.interp_lanes >= w.P ? w.interp_lanes : (w.P <= 8 ? 8 : (w.P <= 16 ? 16 : 32));
    if (G <= 8) k_interp<T, 8><<<nbw(N * 8, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
    else if (G <= 16) k_interp<T, 16><<<nbw(N * 16, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
    else k_interp<T, 32><<<nbw(N * 32, 128), 128, 0, s>>>(N, w, d.pos_sorted, d.grid, d.uwave);
}

#define PSE_INST(T)                                                                                      \
    template void launch_wave_noise<T>(WaveGeom<T>, const SampleArgs<T> *, int, void *, cudaStream_t); \
    template void launch_interp<T>(int64_t, WaveGeom<T>, Geom<T>, const Dev<T> &, cudaStream_t);
PSE_INST(float)
PSE_INST(double)
#undef PSE_INST

}  // namespace pse
