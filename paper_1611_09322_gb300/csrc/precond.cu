// Learned block-diagonal preconditioner for the real-space Lanczos, sm_103a.
//
// The Lanczos iteration of Sec. II B 1 may run on S M_r S for any invertible
// block-diagonal S: the sample S^{-1} (S M_r S)^{1/2} z1 has covariance M_r
// exactly, only the iteration count changes.  Each 3x3 block is
//     S_i = s0 exp(a_i) (I + tanh(b_i) T_i / (1 + tr T_i)),
//     T_i = sum_j w(r_ij) rr_ij,  w(r) = exp(-((r - 2a)/a)^2)  (j within r_cut),
// rotation-equivariant and SPD by construction; a = b = 0 is the analytic
// self-mobility block s0 I (s0 = self mobility^{-1/2}).  (a_i, b_i) come from
// an 8 -> 16 -> 16 -> 2 tanh MLP on rotation-invariant features of i's
// neighbourhood.  The network is trained here on the GPU (forward, backward
// and Adam kernels) against local inverse-square-root blocks
// [(M_loc)^{-1/2}]_ii, which a Newton-Schulz kernel computes from M_r
// restricted to i and its contact shell.
#include <math.h>
#include <string.h>

#include "pse_internal.cuh"

namespace pse {

constexpr int kPcIn = 8, kPcH = 16;
constexpr int kPcNParam = kPcH * kPcIn + kPcH + kPcH * kPcH + kPcH + 2 * kPcH + 2;  // 450
static_assert(kPcNParam == PSE_PRECOND_NPARAM, "parameter count");
__constant__ float c_feat_scale[kPcIn] = {4.f, 8.f, 16.f, 4.f, 8.f, 16.f, 32.f, 1.f};

namespace {

template <typename T> __device__ __forceinline__ long long wb(T w) {
    if constexpr (sizeof(T) == 4) return (long long)__float_as_int(w);
    else return __double_as_longlong(w);
}
__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// Features (scaled) and structure tensor (xx, yy, zz, xy, xz, yz) of sorted
// particle s from its ELL neighbour list.
__device__ void pc_features(int64_t N, int64_t s, const Geom<float> &g, const Rec<float> *__restrict__ rec,
                            const int *__restrict__ count, const int *__restrict__ nbr, float f[kPcIn],
                            float Tm[6]) {
    const float a = g.a;
    const V4<float> li = rec[s].l;
    float t6[6] = {0, 0, 0, 0, 0, 0};
    float n25 = 0, n35 = 0, n45 = 0, nrc = 0, inv = 0;
    const float rc = sqrtf(g.rc2);
    const int slots = count[s];
    int cnt = 0;  // neighbours, without the slots removed by the float64 decision at r_cut
    for (int k = 0; k < slots; ++k) {
        const int e = __ldg(nbr + (int64_t)k * N + s);
        if (e < 0) continue;
        ++cnt;
        const int t = e >> 6;
        const int ox = ((e >> 4) & 3) - 1, oy = ((e >> 2) & 3) - 1, oz = (e & 3) - 1;
        const V4<float> lt = rec[t].l;
        const float dx = (li.x - lt.x) - (ox * g.cs + ox * g.cs_lo);
        const float dy = (li.y - lt.y) - (oy * g.cs + oy * g.cs_lo);
        const float dz = (li.z - lt.z) - (oz * g.cs + oz * g.cs_lo);
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float ri = r > 0.f ? 1.f / r : 0.f;
        const float hx = dx * ri, hy = dy * ri, hz = dz * ri;
        const float q = (r - 2.f * a) / a;
        const float w = expf(-q * q);
        t6[0] += w * hx * hx; t6[1] += w * hy * hy; t6[2] += w * hz * hz;
        t6[3] += w * hx * hy; t6[4] += w * hx * hz; t6[5] += w * hy * hz;
        n25 += sigm(4.f * (2.5f * a - r) / a);
        n35 += sigm(4.f * (3.5f * a - r) / a);
        n45 += sigm(4.f * (4.5f * a - r) / a);
        nrc += sigm(4.f * (rc - r) / a);
        inv += 2.f * a * ri;
    }
    const float tr = t6[0] + t6[1] + t6[2];
    const float tr2 = t6[0] * t6[0] + t6[1] * t6[1] + t6[2] * t6[2] + 2.f * (t6[3] * t6[3] + t6[4] * t6[4] + t6[5] * t6[5]);
    const float det = t6[0] * (t6[1] * t6[2] - t6[5] * t6[5]) - t6[3] * (t6[3] * t6[2] - t6[5] * t6[4]) +
                      t6[4] * (t6[3] * t6[5] - t6[1] * t6[4]);
    const float raw[kPcIn] = {tr, tr2, det, n25, n35, n45, nrc, cnt > 0 ? inv / cnt : 0.f};
#pragma unroll
    for (int i = 0; i < kPcIn; ++i) f[i] = raw[i] / c_feat_scale[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) Tm[i] = t6[i];
}

// MLP forward: outputs (a, b) and the hidden activations.
__device__ __forceinline__ void pc_mlp(const float *__restrict__ th, const float f[kPcIn], float h1[kPcH],
                                       float h2[kPcH], float o[2]) {
    const float *W1 = th, *b1 = W1 + kPcH * kPcIn, *W2 = b1 + kPcH, *b2 = W2 + kPcH * kPcH, *W3 = b2 + kPcH,
                *b3 = W3 + 2 * kPcH;
#pragma unroll
    for (int i = 0; i < kPcH; ++i) {
        float z = b1[i];
#pragma unroll
        for (int k = 0; k < kPcIn; ++k) z += W1[i * kPcIn + k] * f[k];
        h1[i] = tanhf(z);
    }
#pragma unroll
    for (int i = 0; i < kPcH; ++i) {
        float z = b2[i];
#pragma unroll
        for (int k = 0; k < kPcH; ++k) z += W2[i * kPcH + k] * h1[k];
        h2[i] = tanhf(z);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float z = b3[i];
#pragma unroll
        for (int k = 0; k < kPcH; ++k) z += W3[i * kPcH + k] * h2[k];
        o[i] = z;
    }
}

// S = s0 E (I + c T), c = tanh(b) / (1 + tr T): (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ void pc_block(float s0, float av, float bv, const float Tm[6], float S[6]) {
    const float E = s0 * expf(av);
    const float c = tanhf(bv) / (1.f + Tm[0] + Tm[1] + Tm[2]);
    S[0] = E * (1.f + c * Tm[0]);
    S[1] = E * (1.f + c * Tm[1]);
    S[2] = E * (1.f + c * Tm[2]);
    S[3] = E * c * Tm[3];
    S[4] = E * c * Tm[4];
    S[5] = E * c * Tm[5];
}

__device__ __forceinline__ void sym3_inv(const float S[6], float R[6]) {
    const float a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5];
    const float A = b * c - f * f, B = a * c - e * e, C = a * b - d * d;
    const float D = e * f - c * d, Ee = d * f - b * e, F = d * e - a * f;
    const float det = a * A + d * D + e * Ee;
    const float id = 1.f / det;
    R[0] = A * id; R[1] = B * id; R[2] = C * id; R[3] = D * id; R[4] = Ee * id; R[5] = F * id;
}

}  // namespace

// ------------------------------------------------------------------ inference (sampler)
// S_i and S_i^{-1} of every sorted particle: pc[s*16 + 0..5] = S, [8..13] = S^{-1}.
__global__ void __launch_bounds__(128) k_pc_infer(int64_t N, Geom<float> g, const Rec<float> *__restrict__ rec,
                                                  const int *__restrict__ count, const int *__restrict__ nbr,
                                                  const float *__restrict__ theta, float s0, float *pc) {
    __shared__ float th[kPcNParam];
    for (int i = threadIdx.x; i < kPcNParam; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    float f[kPcIn], Tm[6], h1[kPcH], h2[kPcH], o[2], S[6], R[6];
    pc_features(N, s, g, rec, count, nbr, f, Tm);
    pc_mlp(th, f, h1, h2, o);
    pc_block(s0, o[0], o[1], Tm, S);
    sym3_inv(S, R);
    float *dst = pc + s * 16;
#pragma unroll
    for (int i = 0; i < 6; ++i) { dst[i] = S[i]; dst[8 + i] = R[i]; }
    dst[6] = dst[7] = dst[14] = dst[15] = 0.f;
}

// features and structure tensors in caller order (training data)
__global__ void k_pc_features(int64_t N, Geom<float> g, const Rec<float> *__restrict__ rec,
                              const int *__restrict__ count, const int *__restrict__ nbr,
                              const V4<float> *__restrict__ pos_sorted, float *feat, float *tens) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    float f[kPcIn], Tm[6];
    pc_features(N, s, g, rec, count, nbr, f, Tm);
    const int64_t o = wb(pos_sorted[s].w);
    for (int i = 0; i < kPcIn; ++i) feat[o * kPcIn + i] = f[i];
    for (int i = 0; i < 6; ++i) tens[o * 6 + i] = Tm[i];
}

// ------------------------------------------------------------------ local inverse-sqrt targets
constexpr int kLocK = 16, kLocMax = 3 * (kLocK + 1);  // 51

// One CTA per sorted particle i: contact-shell neighbours (r < 3a, the 16
// nearest, ties by caller index), dense M_loc from the table, coupled
// Newton-Schulz iteration Y -> (A/c)^{1/2}, Z -> (A/c)^{-1/2} with c the
// Gershgorin bound, 40 steps; writes the 3x3 block of Z / sqrt(c).
__global__ void __launch_bounds__(128) k_pc_targets(int64_t N, Geom<float> g, const Rec<float> *__restrict__ rec,
                                                    const int *__restrict__ count, const int *__restrict__ nbr,
                                                    const V4<float> *__restrict__ pos_sorted,
                                                    const V4<float> *__restrict__ table, float *target) {
    __shared__ float A[kLocMax][kLocMax + 1], Y[kLocMax][kLocMax + 1], Z[kLocMax][kLocMax + 1],
        Tt[kLocMax][kLocMax + 1];
    __shared__ float cand_r[64], cand_d[64][3];
    __shared__ long long cand_id[64];
    __shared__ int ncand, m;
    __shared__ float cgersh;
    const int64_t s = blockIdx.x;
    const float a = g.a;
    if (threadIdx.x == 0) {
        // candidates within 3a, insertion-sorted by (r, caller index)
        int nc = 0;
        const V4<float> li = rec[s].l;
        const int cnt = count[s];
        for (int k = 0; k < cnt; ++k) {
            const int e = nbr[(int64_t)k * N + s];
            if (e < 0) continue;  // a pair removed by the float64 decision at r_cut
            const int t = e >> 6;
            const int ox = ((e >> 4) & 3) - 1, oy = ((e >> 2) & 3) - 1, oz = (e & 3) - 1;
            const V4<float> lt = rec[t].l;
            const float dx = (lt.x - li.x) + (ox * g.cs + ox * g.cs_lo);
            const float dy = (lt.y - li.y) + (oy * g.cs + oy * g.cs_lo);
            const float dz = (lt.z - li.z) + (oz * g.cs + oz * g.cs_lo);
            const float r = sqrtf(dx * dx + dy * dy + dz * dz);
            if (r >= 3.f * a || nc >= 64) continue;
            const long long id = wb(pos_sorted[t].w);
            int j = nc++;
            while (j > 0 && (cand_r[j - 1] > r || (cand_r[j - 1] == r && cand_id[j - 1] > id))) {
                cand_r[j] = cand_r[j - 1];
                cand_id[j] = cand_id[j - 1];
                cand_d[j][0] = cand_d[j - 1][0]; cand_d[j][1] = cand_d[j - 1][1]; cand_d[j][2] = cand_d[j - 1][2];
                --j;
            }
            cand_r[j] = r;
            cand_id[j] = id;
            cand_d[j][0] = dx; cand_d[j][1] = dy; cand_d[j][2] = dz;
        }
        ncand = nc < kLocK ? nc : kLocK;
        m = 3 * (ncand + 1);
    }
    __syncthreads();
    const int n = m, np = ncand + 1;
    // A = M_loc: particle 0 at the origin, particle p at cand_d[p-1]
    for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
        const int pa = idx / np, pb = idx % np;
        float blk[6] = {0, 0, 0, 0, 0, 0};
        if (pa == pb) {
            blk[0] = blk[1] = blk[2] = g.self_m;
        } else {
            const float xa = pa ? cand_d[pa - 1][0] : 0.f, ya = pa ? cand_d[pa - 1][1] : 0.f, za = pa ? cand_d[pa - 1][2] : 0.f;
            const float xb = pb ? cand_d[pb - 1][0] : 0.f, yb = pb ? cand_d[pb - 1][1] : 0.f, zb = pb ? cand_d[pb - 1][2] : 0.f;
            const float dx = xa - xb, dy = ya - yb, dz = za - zb;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < g.rc2 && r2 > 0.f) {
                const float ri = rsqrtf(r2), r = r2 * ri;
                const float uu = r * g.tab_inv_dr;
                int it = (int)uu;
                it = it > PSE_TABLE_N - 2 ? PSE_TABLE_N - 2 : it;
                const float fr = uu - it;
                const V4<float> tb = table[it];
                const float F = tb.x + fr * tb.z, GmF = tb.y + fr * tb.w;
                const float hx = dx * ri, hy = dy * ri, hz = dz * ri;
                blk[0] = F + GmF * hx * hx; blk[1] = F + GmF * hy * hy; blk[2] = F + GmF * hz * hz;
                blk[3] = GmF * hx * hy; blk[4] = GmF * hx * hz; blk[5] = GmF * hy * hz;
            }
        }
        const int ra = 3 * pa, cb = 3 * pb;
        A[ra][cb] = blk[0]; A[ra + 1][cb + 1] = blk[1]; A[ra + 2][cb + 2] = blk[2];
        A[ra][cb + 1] = A[ra + 1][cb] = blk[3];
        A[ra][cb + 2] = A[ra + 2][cb] = blk[4];
        A[ra + 1][cb + 2] = A[ra + 2][cb + 1] = blk[5];
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // Gershgorin bound of lambda_max
        float mx = 0.f;
        for (int r = threadIdx.x; r < n; r += 32) {
            float sum = 0.f;
            for (int c = 0; c < n; ++c) sum += fabsf(A[r][c]);
            mx = fmaxf(mx, sum);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) cgersh = mx;
    }
    __syncthreads();
    const float ic = 1.f / cgersh;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        Y[r][c] = A[r][c] * ic;
        Z[r][c] = (r == c) ? 1.f : 0.f;
    }
    __syncthreads();
    for (int step = 0; step < 40; ++step) {
        // Tt = (3 I - Z Y) / 2
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int r = idx / n, c = idx % n;
            float acc = 0.f;
            for (int k = 0; k < n; ++k) acc += Z[r][k] * Y[k][c];
            Tt[r][c] = ((r == c) ? 1.5f : 0.f) - 0.5f * acc;
        }
        __syncthreads();
        // A <- Y Tt (new Y, A reused as scratch)
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int r = idx / n, c = idx % n;
            float acc = 0.f;
            for (int k = 0; k < n; ++k) acc += Y[r][k] * Tt[k][c];
            A[r][c] = acc;
        }
        __syncthreads();
        // Y <- Tt Z (new Z, Y is free now)
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int r = idx / n, c = idx % n;
            float acc = 0.f;
            for (int k = 0; k < n; ++k) acc += Tt[r][k] * Z[k][c];
            Y[r][c] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int r = idx / n, c = idx % n;
            Z[r][c] = Y[r][c];
            Y[r][c] = A[r][c];
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) {
        const float sc = rsqrtf(cgersh);
        const int rr[6] = {0, 1, 2, 0, 0, 1}, cc[6] = {0, 1, 2, 1, 2, 2};
        const int64_t o = wb(pos_sorted[s].w);
        target[o * 6 + threadIdx.x] = Z[rr[threadIdx.x]][cc[threadIdx.x]] * sc;
    }
}

// ------------------------------------------------------------------ training
// Loss mean_i ||S_i - target_i||_F^2 / s0^2 and its gradient: one thread per
// sample runs the forward and backward pass in registers; per-parameter
// gradients are summed over the warp by shuffles, over the block in shared
// memory, and across blocks by atomics.
__global__ void __launch_bounds__(256) k_pc_lossgrad(int64_t n, const float *__restrict__ feat,
                                                     const float *__restrict__ tens, const float *__restrict__ target,
                                                     const float *__restrict__ theta, float s0, float *grad,
                                                     double *loss) {
    __shared__ float th[kPcNParam];
    __shared__ float gsum[kPcNParam];
    __shared__ double lsum;
    for (int i = threadIdx.x; i < kPcNParam; i += blockDim.x) {
        th[i] = theta[i];
        gsum[i] = 0.f;
    }
    if (threadIdx.x == 0) lsum = 0.0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = i < n;
    float f[kPcIn], Tm[6], h1[kPcH], h2[kPcH], o[2], S[6];
    float l = 0.f, da = 0.f, db = 0.f;
    if (active) {
#pragma unroll
        for (int k = 0; k < kPcIn; ++k) f[k] = feat[i * kPcIn + k];
#pragma unroll
        for (int k = 0; k < 6; ++k) Tm[k] = tens[i * 6 + k];
        pc_mlp(th, f, h1, h2, o);
        pc_block(s0, o[0], o[1], Tm, S);
        float d6[6];
        const float inv_n = 1.f / (float)n, is2 = 1.f / (s0 * s0);
#pragma unroll
        for (int k = 0; k < 6; ++k) d6[k] = S[k] - target[i * 6 + k];
        l = (d6[0] * d6[0] + d6[1] * d6[1] + d6[2] * d6[2] + 2.f * (d6[3] * d6[3] + d6[4] * d6[4] + d6[5] * d6[5])) * is2;
        // dL/dS (off-diagonals counted twice), then through S = s0 E (I + c T)
        const float w = 2.f * inv_n * is2;
        const float tr = 1.f + Tm[0] + Tm[1] + Tm[2];
        const float tb = tanhf(o[1]);
        const float E = s0 * expf(o[0]);
        float dSS = 0.f, dST = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float m = k < 3 ? 1.f : 2.f;
            dSS += m * d6[k] * S[k];
            dST += m * d6[k] * Tm[k];
        }
        da = w * dSS;
        db = w * E * (1.f - tb * tb) / tr * dST;
    }
    // backward through the MLP (zero for inactive threads)
    const float *W2 = th + kPcH * kPcIn + kPcH, *W3 = W2 + kPcH * kPcH + kPcH;
    float dz2[kPcH], dz1[kPcH];
#pragma unroll
    for (int k = 0; k < kPcH; ++k) {
        const float dh2 = W3[k] * da + W3[kPcH + k] * db;
        dz2[k] = active ? dh2 * (1.f - h2[k] * h2[k]) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kPcH; ++k) {
        float dh1 = 0.f;
#pragma unroll
        for (int r = 0; r < kPcH; ++r) dh1 += W2[r * kPcH + k] * dz2[r];
        dz1[k] = active ? dh1 * (1.f - h1[k] * h1[k]) : 0.f;
    }
    // per-parameter gradient, summed over the warp then the block
    const int lane = threadIdx.x & 31;
    auto acc = [&](int p, float v) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(&gsum[p], v);
    };
    int p = 0;
    for (int r = 0; r < kPcH; ++r)
        for (int k = 0; k < kPcIn; ++k) acc(p++, active ? dz1[r] * f[k] : 0.f);
    for (int r = 0; r < kPcH; ++r) acc(p++, dz1[r]);
    for (int r = 0; r < kPcH; ++r)
        for (int k = 0; k < kPcH; ++k) acc(p++, active ? dz2[r] * h1[k] : 0.f);
    for (int r = 0; r < kPcH; ++r) acc(p++, dz2[r]);
    for (int k = 0; k < kPcH; ++k) acc(p++, active ? da * h2[k] : 0.f);
    for (int k = 0; k < kPcH; ++k) acc(p++, active ? db * h2[k] : 0.f);
    acc(p++, da);
    acc(p++, db);
    float lw = l;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, off);
    if (lane == 0) atomicAdd(&lsum, (double)lw);
    __syncthreads();
    for (int q = threadIdx.x; q < kPcNParam; q += blockDim.x) atomicAdd(grad + q, gsum[q]);
    if (threadIdx.x == 0) atomicAdd(loss, lsum / (double)n);
}

// Adam step (Kingma & Ba): m, v moments, bias-corrected.
__global__ void k_pc_adam(float *theta, float *m, float *v, const float *grad, float lr, int step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPcNParam) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i];
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v[i] = b2 * v[i] + (1.f - b2) * g * g;
    const float mh = m[i] / (1.f - powf(b1, (float)step));
    const float vh = v[i] / (1.f - powf(b2, (float)step));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_pc_blocks_caller(int64_t N, const float *__restrict__ pc, const V4<float> *__restrict__ pos_sorted,
                                   float *S) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t o = wb(pos_sorted[s].w);
    for (int i = 0; i < 6; ++i) S[o * 6 + i] = pc[s * 16 + i];
}

void launch_pc_blocks_caller(int64_t N, const Dev<float> &d, float *S, cudaStream_t s) {
    k_pc_blocks_caller<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, d.pc, d.pos_sorted, S);
}

// Fused over the systems of a batch that have the network installed (only
// those get blocks in the table).
__global__ void __launch_bounds__(128) k_pc_infer_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    __shared__ float th[kPcNParam];
    const BSys &S = sys[tab[blockIdx.x]];
    for (int i = threadIdx.x; i < kPcNParam; i += blockDim.x) th[i] = S.d.pc_theta[i];
    __syncthreads();
    const int64_t s = ((int64_t)blockIdx.x - S.b0[BK_PC]) * blockDim.x + threadIdx.x;
    if (s >= S.N) return;
    float f[kPcIn], Tm[6], h1[kPcH], h2[kPcH], o[2], Sb[6], R[6];
    pc_features(S.N, s, S.g, S.d.rec, S.d.nbr_count, S.d.nbr, f, Tm);
    pc_mlp(th, f, h1, h2, o);
    pc_block(S.pc_s0, o[0], o[1], Tm, Sb);
    sym3_inv(Sb, R);
    float *dst = S.d.pc + s * 16;
#pragma unroll
    for (int i = 0; i < 6; ++i) { dst[i] = Sb[i]; dst[8 + i] = R[i]; }
    dst[6] = dst[7] = dst[14] = dst[15] = 0.f;
}
void launch_batch_pc_infer(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s) {
    if (nblk[BK_PC] > 0) k_pc_infer_batch<<<nblk[BK_PC], 128, 0, s>>>(sys, tab[BK_PC]);
}

void launch_pc_infer(int64_t N, Geom<float> g, const Dev<float> &d, const float *theta, float s0, float *pc,
                     cudaStream_t s) {
    k_pc_infer<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, g, d.rec, d.nbr_count, d.nbr, theta, s0, pc);
}
void launch_pc_features(int64_t N, Geom<float> g, const Dev<float> &d, float *feat, float *tens, cudaStream_t s) {
    k_pc_features<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, g, d.rec, d.nbr_count, d.nbr, d.pos_sorted, feat,
                                                               tens);
}
void launch_pc_targets(int64_t N, Geom<float> g, const Dev<float> &d, float *target, cudaStream_t s) {
    k_pc_targets<<<(unsigned)N, 128, 0, s>>>(N, g, d.rec, d.nbr_count, d.nbr, d.pos_sorted, d.table, target);
}

}  // namespace pse

using namespace pse;

extern "C" pse_status pse_precond_loss_grad(int64_t n, const float *d_feat, const float *d_tens,
                                            const float *d_target, const float *d_theta, float s0, float *d_grad,
                                            double *d_loss, void *stream) {
    if (n < 1 || !d_feat || !d_tens || !d_target || !d_theta || !d_grad || !d_loss || !(s0 > 0)) return PSE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_grad, 0, sizeof(float) * kPcNParam, s) != cudaSuccess ||
        cudaMemsetAsync(d_loss, 0, sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ECUDA;
    }
    k_pc_lossgrad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, d_feat, d_tens, d_target, d_theta, s0, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? PSE_OK : PSE_ECUDA;
}

extern "C" pse_status pse_precond_train(int64_t n, const float *d_feat, const float *d_tens, const float *d_target,
                                        float *d_theta, float s0, int steps, float lr, float *d_work,
                                        double *d_loss_hist, void *stream) {
    if (n < 1 || steps < 1 || !d_feat || !d_tens || !d_target || !d_theta || !d_work || !(s0 > 0) || !(lr > 0))
        return PSE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float *grad = d_work, *m = d_work + kPcNParam, *v = d_work + 2 * kPcNParam;
    if (cudaMemsetAsync(m, 0, sizeof(float) * 2 * kPcNParam, s) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ECUDA;
    }
    double *loss = reinterpret_cast<double *>(d_work + 3 * kPcNParam + 2);  // 8-byte aligned slot after the moments
    for (int it = 1; it <= steps; ++it) {
        pse_status st = pse_precond_loss_grad(n, d_feat, d_tens, d_target, d_theta, s0, grad,
                                              d_loss_hist ? d_loss_hist + (it - 1) : loss, stream);
        if (st != PSE_OK) return st;
        k_pc_adam<<<(kPcNParam + 127) / 128, 128, 0, s>>>(d_theta, m, v, grad, lr, it);
    }
    return cudaGetLastError() == cudaSuccess ? PSE_OK : PSE_ECUDA;
}
