// Real-space sample M_r^{1/2} z1 by Lanczos (Sec. II B 1; Chow & Saad),
// sm_103a.
//
// Vectors live in cell-sorted order as 16-byte (x, y, z, pad) records.  The
// basis is kept unnormalised: q_1 = z1 and q_{j+1} = w_j, with
// beta_j = ||q_{j+1}||, v_j = q_j / beta_{j-1}.  Per iteration j:
//   matvec  u = M_r q_j                       (+ deterministic q_j . u)
//   update  alpha_j = q_j.u / beta_{j-1}^2,
//           q_{j+1} = u/beta_{j-1} - alpha_j q_j/beta_{j-1} - beta_{j-1} q_{j-1}/beta_{j-2}
//                                               (+ deterministic ||q_{j+1}||^2)
//   eigen   y_j = T_j^{1/2} e_1 in FP64 (one warp), stop test
//           ||y_j - [y_{j-1}; 0]|| / ||y_j|| < tol  (= ||x_j - x_{j-1}|| / ||x_j||
//           for an orthonormal basis)
// and finally x = beta_0 sum_i y_i q_i / beta_{i-1}.  Scalars are FP64; the
// reducing kernels run persistent grids (a fixed multiple of the SM count)
// and their per-block partial sums are added in block order by the last
// block to arrive, so results do not depend on scheduling.
#include "pse_internal.cuh"

namespace pse {

template <typename T> __device__ __forceinline__ T sqrt_hd(T x) {
    if constexpr (sizeof(T) == 4) return sqrtf(x);
    else return sqrt(x);
}
template <typename T> __device__ __forceinline__ T floor_hd(T x) {
    if constexpr (sizeof(T) == 4) return floorf(x);
    else return floor(x);
}

template <typename T> __device__ __forceinline__ long long w_bits_r(T w) {
    if constexpr (sizeof(T) == 4) return (long long)__float_as_int(w);
    else return __double_as_longlong(w);
}

// per-thread partial: float for the float path (summed per warp in float,
// then in double), double for the FP64 path
template <typename T> struct Part { using type = float; };
template <> struct Part<double> { using type = double; };

template <typename T> __device__ __forceinline__ double block_total(typename Part<T>::type v, double *sh) {
    if constexpr (sizeof(T) == 4) return block_sum_fw(v, sh);
    else return block_sum(v, sh);
}

// ------------------------------------------------------------------ init: q_1 = z1, beta_0
template <typename T>
__device__ __forceinline__ void lz_init_body(int64_t N, const SampleArgs<T> *args, int system,
                                             const V4<T> *pos_sorted, V4<T> *q1, Rec<T> *rec, double *partials,
                                             LzState *lz, const float *__restrict__ pc, int bidx, int nblk,
                                             double *sh) {
    typename Part<T>::type part = 0;
    for (int64_t s = bidx * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)nblk * blockDim.x) {
        const uint32_t orig = (uint32_t)w_bits_r(pos_sorted[s].w);
        const Normals4<T> z = normals4<T>(orig, 2u * system, args->seed, args->sample);
        V4<T> v;
        v.x = z.v[0]; v.y = z.v[1]; v.z = z.v[2]; v.w = T(0);
        q1[s] = v;
        if constexpr (sizeof(T) == 4) {
            if (pc) {  // matvec input is S q
                V4<T> p;
                sym3_apply(pc + s * 16, v.x, v.y, v.z, p.x, p.y, p.z);
                p.w = T(0);
                rec[s].q = p;
            } else {
                rec[s].q = v;
            }
        } else {
            rec[s].q = v;
        }
        part += v.x * v.x + v.y * v.y + v.z * v.z;
    }
    const double bsum = block_total<T>(part, sh);
    double total;
    if (grid_sum_last(bsum, partials, &lz->counter_init, sh, &total, bidx, nblk) && threadIdx.x == 0) {
        lz->beta[0] = sqrt(total);
        lz->iter = 1;
        lz->jeig = 0;
        lz->J = 0;
        lz->converged = 0;
        lz->cont = 1;
        lz->active = 1;
        lz->rel = 0.0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lz_init(int64_t N, const SampleArgs<T> *args, int system,
                                                 const V4<T> *pos_sorted, V4<T> *q1, Rec<T> *rec, double *partials,
                                                 LzState *lz, const float *__restrict__ pc) {
    __shared__ double sh[32];
    lz_init_body<T>(N, args, system, pos_sorted, q1, rec, partials, lz, pc, blockIdx.x, gridDim.x, sh);
}

__global__ void __launch_bounds__(256) k_lz_init_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    __shared__ double sh[32];
    const BSys &S = sys[tab[blockIdx.x]];
    lz_init_body<float>(S.N, S.d.args, S.system, S.d.pos_sorted, S.d.basis, S.d.rec, S.d.partials, S.d.lz, S.d.pc_on,
                        (int)blockIdx.x - S.b0[BK_INIT], S.nb[BK_INIT], sh);
}

// ------------------------------------------------------------------ near-field matvec
// u_s = self q_s + sum_t [F (I - rr) + G rr] q_t over the ELL list of s, F and
// G linearly interpolated from the FP64-built table (stored / 6 pi a).  A
// group of TPP consecutive threads shares one particle: thread g of the
// group takes entries g, g + TPP, ... and the group sums by shuffles.  Each
// neighbour costs one 4-byte list entry and one 32-byte record; a thread
// issues ILP list loads, then ILP record loads, before any arithmetic, so
// that many independent gathers are in flight.  The first round's list
// loads do not wait for the particle's count: entries up to the ELL
// capacity K are always in the array, and those past the count are dropped.

template <typename T>
__device__ __forceinline__ void pair_fg(T r, const Geom<T> &g, const V4<T> *__restrict__ table, T &F, T &GmF) {
    if (sizeof(T) == 8 && r >= T(0.2) * g.a) {
        // FP64 context: Appendix A evaluated exactly instead of interpolated
        double Fd, Gd;
        fg_closed_hd((double)r, (double)g.xi, (double)g.a, &Fd, &Gd);
        const double sc = 1.0 / (6.0 * 3.14159265358979323846 * (double)g.a);
        F = (T)(Fd * sc);
        GmF = (T)((Gd - Fd) * sc);
    } else {
        const T uu = r * g.tab_inv_dr;
        int it = (int)uu;
        it = it > PSE_TABLE_N - 2 ? PSE_TABLE_N - 2 : it;
        const T f = uu - T(it);
        const V4<T> tb = table[it];
        F = tb.x + f * tb.z;
        GmF = tb.y + f * tb.w;
    }
}

// One matvec record, read-only for the kernel's lifetime: a single 256-bit
// load for float records (one L1 request per neighbour instead of two).
template <typename T> __device__ __forceinline__ Rec<T> load_rec(const Rec<T> *__restrict__ p) {
    if constexpr (sizeof(T) == 4) {
        Rec<T> r;
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(r.l.x), "=f"(r.l.y), "=f"(r.l.z), "=f"(r.l.w), "=f"(r.q.x), "=f"(r.q.y), "=f"(r.q.z), "=f"(r.q.w)
            : "l"(p));
        return r;
    } else {
        return *p;
    }
}

// Compact-table lookup (two uniform segments, knot at min(2a, r_cut)); `tab`
// is normally the block's shared-memory copy.
template <typename T>
__device__ __forceinline__ void pair_fg_c(T r, const Geom<T> &g, const V4<T> *tab, T &F, T &GmF) {
    const T u = r < g.tc_split ? r * g.tc_invA : T(PSE_TABLEC_A) + (r - g.tc_split) * g.tc_invB;
    int it = (int)u;
    it = it > PSE_TABLEC_N - 2 ? PSE_TABLEC_N - 2 : it;
    const T f = u - T(it);
    const V4<T> tb = tab[it];
    F = tb.x + f * tb.z;
    GmF = tb.y + f * tb.w;
}

// Species index of a cell record (polydisperse contexts).
template <typename T> __device__ __forceinline__ int spec_of(const V4<T> &l) {
    return (int)((w_bits_r(l.w) >> PSE_SPECIES_SHIFT) & 3);
}
// Self mobility of species sp (selects, so that the parameter array is not
// copied to local memory for a dynamic index).
template <typename T> __device__ __forceinline__ T self_of(const Geom<T> &g, int sp) {
    return sp == 0 ? g.self_s[0] : (sp == 1 ? g.self_s[1] : (sp == 2 ? g.self_s[2] : g.self_s[3]));
}

// Row s of M_r q without the self term, summed over the TPP-thread group.
// CT: `table` is the compact table (pair_fg_c), else the uniform one.
// POLY: the uniform table holds one block per species pair (polydisperse).
template <typename T, int TPP, int ILP, bool CT = false, bool POLY = false>
__device__ __forceinline__ void mr_row_part(int64_t N, int64_t s, int lane_g, bool active, int K, const Geom<T> &g,
                                            const Rec<T> *__restrict__ rec, const int *__restrict__ count,
                                            const int *__restrict__ nbr, const V4<T> *__restrict__ table,
                                            V4<T> &li, V4<T> &qi, T &ax, T &ay, T &az) {
    ax = ay = az = T(0);
    if (active) {
        const int cnt = count[s];
        int ent[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const int k = lane_g + u * TPP;
            ent[u] = k < K ? __ldg(nbr + (int64_t)k * N + s) : -1;
        }
        const Rec<T> ri = load_rec(rec + s);
        li = ri.l;
        qi = ri.q;
        for (int k0 = lane_g; k0 < cnt; k0 += ILP * TPP) {
            if (k0 != lane_g) {
#pragma unroll
                for (int u = 0; u < ILP; ++u) {
                    const int k = k0 + u * TPP;
                    ent[u] = k < K ? __ldg(nbr + (int64_t)k * N + s) : -1;
                }
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (k0 + u * TPP >= cnt) ent[u] = -1;
            Rec<T> rt[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) rt[u] = load_rec(rec + (ent[u] >= 0 ? (ent[u] >> 6) : s));
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                if (ent[u] < 0) continue;
                const int e = ent[u];
                const int ox = ((e >> 4) & 3) - 1, oy = ((e >> 2) & 3) - 1, oz = (e & 3) - 1;
                const T dx = (li.x - rt[u].l.x) - (T(ox) * g.cs + T(ox) * g.cs_lo);
                const T dy = (li.y - rt[u].l.y) - (T(oy) * g.cs + T(oy) * g.cs_lo);
                const T dz = (li.z - rt[u].l.z) - (T(oz) * g.cs + T(oz) * g.cs_lo);
                const T r2 = dx * dx + dy * dy + dz * dz;
                T rinv;
                if constexpr (sizeof(T) == 4) rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                else rinv = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
                T F, GmF;
                if constexpr (CT) {
                    pair_fg_c(r2 * rinv, g, table, F, GmF);
                } else if constexpr (POLY) {
                    const V4<T> *tb = table + (int64_t)pair_index(spec_of(li), spec_of(rt[u].l), g.nspec) * PSE_TABLE_N;
                    pair_fg(r2 * rinv, g, tb, F, GmF);
                } else {
                    pair_fg(r2 * rinv, g, table, F, GmF);
                }
                const T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
                const T dot = GmF * (hx * rt[u].q.x + hy * rt[u].q.y + hz * rt[u].q.z);
                ax += F * rt[u].q.x + dot * hx;
                ay += F * rt[u].q.y + dot * hy;
                az += F * rt[u].q.z + dot * hz;
            }
        }
    }
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
}

// Row s of M_r q without the self term and without a neighbour list (FP32):
// one thread walks the 27 stencil cells of its particle over the cell-sorted
// records, which carry q beside the cell-local offsets.  A candidate is kept
// by the neighbour search's own float32 test (below the top of the r_cut
// band), and one inside the band by the float64 decision from the wrapped
// positions, so the row sums exactly the pairs the neighbour list holds
// (summation in stencil order).
__device__ __forceinline__ void mr_row_nolist(int64_t s, bool active, const Geom<float> &g,
                                              const Rec<float> *__restrict__ rec,
                                              const int *__restrict__ cell_start,
                                              const V4<float> *__restrict__ pos, const V4<float> *tab,
                                              V4<float> &li, V4<float> &qi, float &ax, float &ay, float &az) {
    ax = ay = az = 0.f;
    if (!active) return;
    const Rec<float> ri = load_rec(rec + s);
    li = ri.l;
    qi = ri.q;
    const int c = (int)(w_bits_r(li.w) & PSE_CELL_MASK);
    const int nc = g.nc;
    int cx, cy, cz;
    cell_xyz(c, g.nb, cx, cy, cz);
    for (int ox = -1; ox <= 1; ++ox) {
        int axc = cx + ox;
        axc += axc < 0 ? nc : 0;
        axc -= axc >= nc ? nc : 0;
        const float sx = float(ox) * g.cs + float(ox) * g.cs_lo;
        for (int oy = -1; oy <= 1; ++oy) {
            int ayc = cy + oy;
            ayc += ayc < 0 ? nc : 0;
            ayc -= ayc >= nc ? nc : 0;
            const float sy = float(oy) * g.cs + float(oy) * g.cs_lo;
            for (int oz = -1; oz <= 1; ++oz) {
                int azc = cz + oz;
                azc += azc < 0 ? nc : 0;
                azc -= azc >= nc ? nc : 0;
                const float sz = float(oz) * g.cs + float(oz) * g.cs_lo;
                const int c2 = cell_id(axc, ayc, azc, g.nb);
                const int b = cell_start[c2], e = cell_start[c2 + 1];
                const int self = (ox | oy | oz) == 0 ? (int)s : -1;
                for (int t = b; t < e; ++t) {
                    if (t == self) continue;
                    const Rec<float> rt = load_rec(rec + t);
                    const float dx = (li.x - rt.l.x) - sx;
                    const float dy = (li.y - rt.l.y) - sy;
                    const float dz = (li.z - rt.l.z) - sz;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= g.rc2_hi) continue;
                    if (r2 >= g.rc2_lo && !pair_inside_f64(pos[s], pos[t], g)) continue;
                    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                    float F, GmF;
                    pair_fg_c(r2 * rinv, g, tab, F, GmF);
                    const float hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
                    const float dot = GmF * (hx * rt.q.x + hy * rt.q.y + hz * rt.q.z);
                    ax += F * rt.q.x + dot * hx;
                    ay += F * rt.q.y + dot * hy;
                    az += F * rt.q.z + dot * hz;
                }
            }
        }
    }
}

// Body of one Lanczos matvec over the nblk blocks of one system (bidx = this
// block's index among them).  NOLIST: rows by mr_row_nolist (FP32, TPP 1),
// which reads cell_start and the sorted positions instead of the list.
template <typename T, int TPP, int ILP, bool CT, bool POLY = false, bool NOLIST = false>
__device__ __forceinline__ void lz_matvec_body(int64_t N, int K, const Geom<T> &g, const Rec<T> *__restrict__ rec,
                                               const int *__restrict__ count, const int *__restrict__ nbr,
                                               const V4<T> *__restrict__ table, V4<T> *u, double *partials,
                                               LzState *lz, const float *__restrict__ pc,
                                               const V4<T> *__restrict__ basis, const V4<T> *__restrict__ add,
                                               int bidx, int nblk, double *sh,
                                               const int *__restrict__ cell_start = nullptr,
                                               const V4<T> *__restrict__ pos_sorted = nullptr) {
    const int j = lz->iter;
    if (j > PSE_MAXIT || !lz->active) return;  // uniform across the system's blocks
    typename Part<T>::type part = 0;
    const int lane_g = threadIdx.x % TPP;
    const int64_t per_block = blockDim.x / TPP;
    // contiguous chunk of particles per block (spatial locality across
    // iterations); whole groups stride together so group shuffles converge
    const int64_t chunk = ((N + nblk - 1) / nblk + per_block - 1) / per_block * per_block;
    const int64_t end = (bidx + 1) * chunk < N ? (bidx + 1) * chunk : N;
    for (int64_t base = bidx * chunk; base < end; base += per_block) {
        const int64_t s = base + threadIdx.x / TPP;
        const bool active = s < end;
        V4<T> li, qi;
        T ax, ay, az;
        if constexpr (NOLIST) {
            mr_row_nolist(s, active, g, rec, cell_start, pos_sorted, table, li, qi, ax, ay, az);
        } else {
            mr_row_part<T, TPP, ILP, CT, POLY>(N, s, lane_g, active, K, g, rec, count, nbr, table, li, qi, ax, ay,
                                               az);
        }
        if (active && lane_g == 0) {
            V4<T> o;
            const T self = POLY ? self_of(g, spec_of(li)) : g.self_m;
            o.x = ax + self * qi.x;
            o.y = ay + self * qi.y;
            o.z = az + self * qi.z;
            o.w = T(0);
            if (add) {  // full-mobility Lanczos: the wave product M_w q_j of the same vector
                const V4<T> aw = add[s];
                o.x += aw.x;
                o.y += aw.y;
                o.z += aw.z;
            }
            if constexpr (sizeof(T) == 4) {
                if (pc) {  // A = S M_r S: the record holds S q, apply S to the row, dot with q
                    T x, y, z;
                    sym3_apply(pc + s * 16, o.x, o.y, o.z, x, y, z);
                    o.x = x; o.y = y; o.z = z;
                    qi = basis[(int64_t)(j - 1) * N + s];
                }
            }
            u[s] = o;
            part += qi.x * o.x + qi.y * o.y + qi.z * o.z;
        }
    }
    const double bsum = block_total<T>(part, sh);
    double total;
    if (grid_sum_last(bsum, partials, &lz->counter_mv, sh, &total, bidx, nblk) && threadIdx.x == 0) {
        const double b1 = lz->beta[j - 1];
        const bool ok = b1 > 0.0;  // beta_{j-1} = 0: invariant subspace, the eigen kernel stops the loop
        const double alpha = ok ? total / (b1 * b1) : 0.0;
        lz->alpha[j] = alpha;
        lz->c_u = ok ? (float)(1.0 / b1) : 0.f;
        lz->c_q = ok ? (float)(alpha / b1) : 0.f;
        lz->c_p = (ok && j >= 2) ? (float)(b1 / lz->beta[j - 2]) : 0.f;
    }
}

// Float contexts stage the compact F, G table (16 KB) in shared memory:
// table lookups then cost shared-memory wavefronts instead of scattered L1
// lines.  The FP64 path uses the uniform table (r < 0.2a) and the closed form.
// BS threads per block: with large blocks fewer copies of the table share an
// SM, leaving more of its on-chip memory to the L1 that caches the records.
template <typename T, int TPP, int ILP, int BS = 128>
__global__ void __launch_bounds__(BS) k_lz_matvec(int64_t N, int K, Geom<T> g, const Rec<T> *__restrict__ rec,
                                                   const int *__restrict__ count, const int *__restrict__ nbr,
                                                   const V4<T> *__restrict__ table, const V4<T> *__restrict__ table_c,
                                                   V4<T> *u, double *partials, LzState *lz,
                                                   const float *__restrict__ pc, const V4<T> *__restrict__ basis,
                                                   const V4<T> *__restrict__ add) {
    __shared__ double sh[32];
    if constexpr (sizeof(T) == 4) {
        __shared__ V4<float> tab_s[PSE_TABLEC_N];
        for (int i = threadIdx.x; i < PSE_TABLEC_N; i += blockDim.x) tab_s[i] = table_c[i];
        __syncthreads();
        lz_matvec_body<T, TPP, ILP, true>(N, K, g, rec, count, nbr, tab_s, u, partials, lz, pc, basis, add,
                                          blockIdx.x, gridDim.x, sh);
    } else {
        lz_matvec_body<T, TPP, ILP, false>(N, K, g, rec, count, nbr, table, u, partials, lz, pc, basis, add,
                                           blockIdx.x, gridDim.x, sh);
    }
}

// ------------------------------------------------------------------ brick-tiled matvec
// FP32 monodisperse form that serves the neighbour records from shared
// memory.  A block takes one 4x4x4-cell brick at a time (a fixed, strided
// set of bricks: the per-block partial sums, and so alpha, do not depend on
// scheduling).  It stages the records of the brick's 6x6x6-cell
// neighbourhood -- runs of consecutive sorted particles, one per cell, read
// from L2 -- and a per-cell offset, so that the ELL entry (t, stencil code)
// of a particle in brick-local cell (lx, ly, lz) is found at
// t + hoff[((lx + 1 + ox) * 6 + (ly + 1 + oy)) * 6 + (lz + 1 + oz)].  The
// scattered 32-byte gathers then cost shared-memory wavefronts instead of
// L1/L2 lines.  A brick whose neighbourhood holds more than `cap` particles
// gathers from global memory instead.  The pair arithmetic is that of
// mr_row_part with the compact table.
#define PSE_TILE_THREADS 256
#define PSE_TILE_TPP 4
#define PSE_TILE_ILP 4
__global__ void __launch_bounds__(PSE_TILE_THREADS, 4) k_lz_matvec_tiled(
    int64_t N, int K, Geom<float> g, const Rec<float> *__restrict__ rec, const int *__restrict__ cell_start,
    const int *__restrict__ count, const int *__restrict__ nbr, const V4<float> *__restrict__ table_c,
    V4<float> *u, double *partials, LzState *lz, const V4<float> *__restrict__ add, int nbricks, int cap) {
    constexpr int TPP = PSE_TILE_TPP, ILP = PSE_TILE_ILP;
    __shared__ double sh[32];
    __shared__ V4<float> tab_s[PSE_TABLEC_N];
    __shared__ int hpre[217], hoff[216], hcell[216];
    extern __shared__ __align__(32) unsigned char tile_raw[];
    Rec<float> *halo = reinterpret_cast<Rec<float> *>(tile_raw);
    for (int i = threadIdx.x; i < PSE_TABLEC_N; i += blockDim.x) tab_s[i] = table_c[i];
    const int j = lz->iter;
    if (j > PSE_MAXIT || !lz->active) return;  // uniform across the launch
    float part = 0.f;
    const int nb = g.nb, nc = g.nc;
    const int lane_g = threadIdx.x % TPP;
    const int per_pass = blockDim.x / TPP;
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x) {
        const int s0 = cell_start[b * 64], s1 = cell_start[b * 64 + 64];
        if (s0 == s1) continue;  // uniform: an empty brick (or cell slots past ncell)
        const int bz = b % nb, by = (b / nb) % nb, bx = b / (nb * nb);
        __syncthreads();  // the previous brick's readers are done with the tile
        for (int h = threadIdx.x; h < 216; h += blockDim.x) {
            const int hx = h / 36, hy = (h / 6) % 6, hz = h % 6;
            const int cx = ((bx * 4 - 1 + hx) % nc + nc) % nc;
            const int cy = ((by * 4 - 1 + hy) % nc + nc) % nc;
            const int cz = ((bz * 4 - 1 + hz) % nc + nc) % nc;
            const int c = cell_id(cx, cy, cz, nb);
            hcell[h] = c;
            hpre[h + 1] = cell_start[c + 1] - cell_start[c];
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // exclusive prefix of the 216 counts, one warp
            int carry = 0;
            for (int base = 0; base < 216; base += 32) {
                const int h = base + threadIdx.x;
                int v = h < 216 ? hpre[h + 1] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int n = __shfl_up_sync(0xffffffffu, v, o);
                    if (threadIdx.x >= o) v += n;
                }
                if (h < 216) hpre[h + 1] = carry + v;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            if (threadIdx.x == 0) hpre[0] = 0;
        }
        __syncthreads();
        const int total = hpre[216];
        const bool staged = total <= cap;
        if (staged) {
            for (int h = threadIdx.x; h < 216; h += blockDim.x) hoff[h] = hpre[h] - cell_start[hcell[h]];
            for (int i = threadIdx.x; i < total; i += blockDim.x) {
                int lo = 0, hi = 215;  // last halo cell with hpre <= i
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (hpre[mid] <= i) lo = mid;
                    else hi = mid - 1;
                }
                halo[i] = load_rec(rec + cell_start[hcell[lo]] + (i - hpre[lo]));
            }
        }
        __syncthreads();
        for (int base = s0; base < s1; base += per_pass) {
            const int s = base + threadIdx.x / TPP;
            const bool active = s < s1;
            float ax = 0.f, ay = 0.f, az = 0.f;
            Rec<float> ri;
            if (active) {
                ri = load_rec(rec + s);
                const int own = __float_as_int(ri.l.w) & 63;  // brick-local cell (lx, ly, lz)
                const int l0 = ((((own >> 4) & 3) + 1) * 6 + ((own >> 2) & 3) + 1) * 6 + (own & 3) + 1;
                const int cnt = count[s];
                for (int k0 = lane_g; k0 < cnt; k0 += ILP * TPP) {
                    int ent[ILP];
#pragma unroll
                    for (int q = 0; q < ILP; ++q) {
                        const int k = k0 + q * TPP;
                        ent[q] = k < cnt ? __ldg(nbr + (int64_t)k * N + s) : -1;
                    }
                    Rec<float> rt[ILP];
#pragma unroll
                    for (int q = 0; q < ILP; ++q) {
                        const int e = ent[q];
                        if (e < 0) continue;
                        const int t = e >> 6;
                        // stencil code (ox+1)<<4 | (oy+1)<<2 | (oz+1) shifts the halo index
                        const int hc = l0 - 43 + ((e >> 4) & 3) * 36 + ((e >> 2) & 3) * 6 + (e & 3);
                        rt[q] = staged ? halo[t + hoff[hc]] : load_rec(rec + t);
                    }
#pragma unroll
                    for (int q = 0; q < ILP; ++q) {
                        const int e = ent[q];
                        if (e < 0) continue;
                        const int ox = ((e >> 4) & 3) - 1, oy = ((e >> 2) & 3) - 1, oz = (e & 3) - 1;
                        const float dx = (ri.l.x - rt[q].l.x) - (float(ox) * g.cs + float(ox) * g.cs_lo);
                        const float dy = (ri.l.y - rt[q].l.y) - (float(oy) * g.cs + float(oy) * g.cs_lo);
                        const float dz = (ri.l.z - rt[q].l.z) - (float(oz) * g.cs + float(oz) * g.cs_lo);
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                        float F, GmF;
                        pair_fg_c(r2 * rinv, g, tab_s, F, GmF);
                        const float hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
                        const float dot = GmF * (hx * rt[q].q.x + hy * rt[q].q.y + hz * rt[q].q.z);
                        ax += F * rt[q].q.x + dot * hx;
                        ay += F * rt[q].q.y + dot * hy;
                        az += F * rt[q].q.z + dot * hz;
                    }
                }
            }
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                az += __shfl_xor_sync(0xffffffffu, az, o);
            }
            if (active && lane_g == 0) {
                V4<float> o;
                o.x = ax + g.self_m * ri.q.x;
                o.y = ay + g.self_m * ri.q.y;
                o.z = az + g.self_m * ri.q.z;
                o.w = 0.f;
                if (add) {
                    const V4<float> aw = add[s];
                    o.x += aw.x;
                    o.y += aw.y;
                    o.z += aw.z;
                }
                u[s] = o;
                part += ri.q.x * o.x + ri.q.y * o.y + ri.q.z * o.z;
            }
        }
    }
    const double bsum = block_sum_fw(part, sh);
    double total;
    if (grid_sum_last(bsum, partials, &lz->counter_mv, sh, &total) && threadIdx.x == 0) {
        const double b1 = lz->beta[j - 1];
        const bool ok = b1 > 0.0;
        const double alpha = ok ? total / (b1 * b1) : 0.0;
        lz->alpha[j] = alpha;
        lz->c_u = ok ? (float)(1.0 / b1) : 0.f;
        lz->c_q = ok ? (float)(alpha / b1) : 0.f;
        lz->c_p = (ok && j >= 2) ? (float)(b1 / lz->beta[j - 2]) : 0.f;
    }
}

// Polydisperse contexts (FP32): 4 threads x 4 gathers per particle in blocks
// of 1024, F and G from the uniform table block of each species pair.
__global__ void __launch_bounds__(1024) k_lz_matvec_poly(int64_t N, int K, Geom<float> g,
                                                         const Rec<float> *__restrict__ rec,
                                                         const int *__restrict__ count, const int *__restrict__ nbr,
                                                         const V4<float> *__restrict__ table, V4<float> *u,
                                                         double *partials, LzState *lz,
                                                         const V4<float> *__restrict__ basis) {
    __shared__ double sh[32];
    lz_matvec_body<float, 4, 4, false, true>(N, K, g, rec, count, nbr, table, u, partials, lz, nullptr, basis,
                                             nullptr, blockIdx.x, gridDim.x, sh);
}

// List-free Lanczos matvec (FP32 monodisperse, no preconditioner): one
// thread per particle in blocks of PSE_NOLIST_THREADS, compact table in
// shared memory.  The sample then builds no neighbour list.
__global__ void __launch_bounds__(PSE_NOLIST_THREADS) k_lz_matvec_nolist(
    int64_t N, Geom<float> g, const Rec<float> *__restrict__ rec, const int *__restrict__ cell_start,
    const V4<float> *__restrict__ pos_sorted, const V4<float> *__restrict__ table_c, V4<float> *u,
    double *partials, LzState *lz, const V4<float> *__restrict__ add) {
    __shared__ double sh[32];
    __shared__ V4<float> tab_s[PSE_TABLEC_N];
    for (int i = threadIdx.x; i < PSE_TABLEC_N; i += blockDim.x) tab_s[i] = table_c[i];
    __syncthreads();
    lz_matvec_body<float, 1, 1, true, false, true>(N, 0, g, rec, nullptr, nullptr, tab_s, u, partials, lz, nullptr,
                                                   nullptr, add, blockIdx.x, gridDim.x, sh, cell_start, pos_sorted);
}

// Fused over the systems of a batch: block b works for system blk2sys[b].
__global__ void __launch_bounds__(PSE_BATCH_MV_THREADS) k_lz_matvec_batch(const LzSys *__restrict__ sys,
                                                                          const int *__restrict__ blk2sys) {
    __shared__ double sh[32];
    __shared__ V4<float> tab_s[PSE_TABLEC_N];
    const LzSys &S = sys[blk2sys[blockIdx.x]];
    for (int i = threadIdx.x; i < PSE_TABLEC_N; i += blockDim.x) tab_s[i] = S.table_c[i];
    __syncthreads();
    lz_matvec_body<float, PSE_BATCH_MV_TPP, PSE_BATCH_MV_ILP, true>(S.N, S.K, S.g, S.rec, S.count, S.nbr, tab_s, S.u, S.part_mv,
                                                     S.lz, S.pc, S.basis, nullptr, blockIdx.x - S.blk_mv, S.nblk_mv,
                                                     sh);
}

template <typename T>
__device__ __forceinline__ void lz_update_body(int64_t N, V4<T> *basis, Rec<T> *rec, const V4<T> *u, double *partials,
                                               LzState *lz, const float *__restrict__ pc, int bidx, int nblk,
                                               double *sh) {
    const int j = lz->iter;
    if (j > PSE_MAXIT || !lz->active) return;
    // coefficients in the working precision; the FP64 path recomputes them exactly
    T cu, cq, cp;
    if constexpr (sizeof(T) == 4) {
        cu = lz->c_u; cq = lz->c_q; cp = lz->c_p;
    } else {
        const double b1 = lz->beta[j - 1];
        const bool ok = b1 > 0.0;
        cu = ok ? 1.0 / b1 : 0.0;
        cq = ok ? lz->alpha[j] / b1 : 0.0;
        cp = (ok && j >= 2) ? b1 / lz->beta[j - 2] : 0.0;
    }
    const V4<T> *qj = basis + (int64_t)(j - 1) * N;
    const V4<T> *qp = basis + (int64_t)(j - 2) * N;
    V4<T> *qn = basis + (int64_t)j * N;
    typename Part<T>::type part = 0;
    for (int64_t s = bidx * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)nblk * blockDim.x) {
        const V4<T> us = u[s];
        const V4<T> a = qj[s];
        V4<T> w;
        w.x = cu * us.x - cq * a.x;
        w.y = cu * us.y - cq * a.y;
        w.z = cu * us.z - cq * a.z;
        w.w = T(0);
        if (j >= 2) {
            const V4<T> b = qp[s];
            w.x -= cp * b.x;
            w.y -= cp * b.y;
            w.z -= cp * b.z;
        }
        qn[s] = w;
        if constexpr (sizeof(T) == 4) {
            if (pc) {
                V4<T> p;
                sym3_apply(pc + s * 16, w.x, w.y, w.z, p.x, p.y, p.z);
                p.w = T(0);
                rec[s].q = p;
            } else {
                rec[s].q = w;
            }
        } else {
            rec[s].q = w;
        }
        part += w.x * w.x + w.y * w.y + w.z * w.z;
    }
    const double bsum = block_total<T>(part, sh);
    double total;
    if (grid_sum_last(bsum, partials, &lz->counter_up, sh, &total, bidx, nblk) && threadIdx.x == 0) {
        lz->beta[j] = sqrt(total);
        lz->iter = j + 1;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lz_update(int64_t N, V4<T> *basis, Rec<T> *rec, const V4<T> *u,
                                                   double *partials, LzState *lz, const float *__restrict__ pc) {
    __shared__ double sh[32];
    lz_update_body<T>(N, basis, rec, u, partials, lz, pc, blockIdx.x, gridDim.x, sh);
}

__global__ void __launch_bounds__(256) k_lz_update_batch(const LzSys *__restrict__ sys, const int *__restrict__ blk2sys) {
    __shared__ double sh[32];
    const LzSys &S = sys[blk2sys[blockIdx.x]];
    lz_update_body<float>(S.N, S.basis, S.rec, S.u, S.part_up, S.lz, S.pc, blockIdx.x - S.blk_up, S.nblk_up, sh);
}

// ------------------------------------------------------------------ FP64 tridiagonal eigen-solve
// One warp.  T_k (diag alpha_1..alpha_k, off-diag beta_1..beta_{k-1}) is
// diagonalised by implicit QL sweeps with Wilkinson-type shifts (Golub & Van
// Loan, Sec. 8.3); every lane runs the scalar recurrences redundantly and
// applies each plane rotation to its own rows of the eigenvector matrix.
// Then y = Q diag(sqrt(lambda)) Q^T e_1.
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// T_k^{1/2} e_1 for a small SPD tridiagonal T_k (k <= KP, KP * KP <= 64) by
// the coupled Newton-Schulz iteration for the matrix square root: with
// A = T_k / c, where c = the Gershgorin bound >= lambda_max, Y_0 = A,
// Z_0 = I and W_n = (3 I - Z_n Y_n) / 2, the iterates Y_{n+1} = Y_n W_n and
// Z_{n+1} = W_n Z_n converge to A^{1/2} and A^{-1/2}; the residual
// R_n = I - Z_n Y_n obeys R_{n+1} = (3 R_n^2 + R_n^3) / 4 and starts below
// 1 - lambda_min / c < 1.  Only multiply-adds (no FP64 divisions or square
// roots per step), the KP^2 entries spread over the warp's lanes; rows and
// columns k..KP-1 are padded with the identity, which stays its own root.
// Once max|R_n| < 1e-8 one more product gives Y to rounding (the next
// residual is ~1e-16).  Writes y = c^{1/2} Y e_1 and returns true, or false
// (y untouched) if the residual has not fallen below 1e-8 in 60 steps.
template <int KP>
__device__ bool tri_sqrt_e1_ns(int k, const double *alpha, const double *beta, double *y, double *sm) {
    constexpr int NE = KP * KP, PER = (NE + 31) / 32;
    double *Y = sm, *Z = sm + NE, *W = sm + 2 * NE;
    const int lane = threadIdx.x;
    double c = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double r = alpha[i + 1] + (i > 0 ? fabs(beta[i]) : 0.0) + (i + 1 < k ? fabs(beta[i + 1]) : 0.0);
        c = fmax(c, r);
    }
    c = warp_max_d(c);
    if (!(c > 0.0)) return false;
    const double ic = 1.0 / c;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int q = lane + 32 * u;
        if (q < NE) {
            const int i = q / KP, j = q % KP;
            double a = i == j ? 1.0 : 0.0;
            if (i < k && j < k) {
                if (i == j) a = alpha[i + 1] * ic;
                else if (i - j == 1 || j - i == 1) a = beta[i > j ? i : j] * ic;
                else a = 0.0;
            }
            Y[q] = a;
            Z[q] = i == j ? 1.0 : 0.0;
        }
    }
    __syncwarp();
    for (int it = 0; it < 60; ++it) {
        double res = 0.0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int q = lane + 32 * u;
            if (q < NE) {
                const int i = q / KP, j = q % KP;
                double zy = 0.0;
#pragma unroll
                for (int l = 0; l < KP; ++l) zy = fma(Z[i * KP + l], Y[l * KP + j], zy);
                const double r = (i == j ? 1.0 : 0.0) - zy;
                res = fmax(res, fabs(r));
                W[q] = 0.5 * ((i == j ? 3.0 : 0.0) - zy);
            }
        }
        res = warp_max_d(res);
        if (!(res < 1.0)) return false;  // diverging (not SPD) or NaN
        __syncwarp();
        const bool last = res < 1e-8;
        double yn[PER], zn[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int q = lane + 32 * u;
            yn[u] = zn[u] = 0.0;
            if (q < NE) {
                const int i = q / KP, j = q % KP;
#pragma unroll
                for (int l = 0; l < KP; ++l) {
                    yn[u] = fma(Y[i * KP + l], W[l * KP + j], yn[u]);
                    zn[u] = fma(W[i * KP + l], Z[l * KP + j], zn[u]);
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int q = lane + 32 * u;
            if (q < NE) {
                Y[q] = yn[u];
                Z[q] = zn[u];
            }
        }
        __syncwarp();
        if (last) {
            const double sc = sqrt(c);
            for (int i = lane; i < k; i += 32) y[i] = sc * Y[i * KP];
            __syncwarp();
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ void lz_eig_body(LzState *lz, int max_iter, int fixed_iter, double tol,
                                            cudaGraphConditionalHandle handle) {
    __shared__ double Q[PSE_MAXIT][PSE_MAXIT + 1];
    __shared__ double d[PSE_MAXIT + 1], e[PSE_MAXIT + 1], y[PSE_MAXIT + 1];
    __shared__ double nsm[3 * 64];
    const int lane = threadIdx.x;
    if (!lz->active) return;  // this system has stopped (batched loop)
    const int k = lz->iter - 1;  // T_k is complete: alpha_k from the matvec, beta_k from the update
    // Every FP64 warp instruction costs many cycles of this GPU's FP64 pipe,
    // active lanes or not, so T_1 and T_2 take closed forms: T_1^{1/2} e_1 =
    // sqrt(alpha_1); for the SPD 2x2 T = [[a, b], [b, c]], T^{1/2} =
    // (T + s I) / t with s = sqrt(det T), t = sqrt(tr T + 2 s) (Cayley-Hamilton),
    // the same matrix the eigendecomposition gives, to rounding.
    if (k <= 2) {
        if (lane == 0) {
            const double a = lz->alpha[1];
            if (k == 1) {
                y[0] = sqrt(fmax(a, 0.0));
            } else {
                const double c = lz->alpha[2], b = lz->beta[1];
                const double sd = sqrt(fmax(fma(a, c, -b * b), 0.0)), t = sqrt(a + c + 2.0 * sd);
                y[0] = (a + sd) / t;
                y[1] = b / t;
            }
        }
        __syncwarp();
    } else if ((k <= 4 && tri_sqrt_e1_ns<4>(k, lz->alpha, lz->beta, y, nsm)) ||
               (k > 4 && k <= 8 && tri_sqrt_e1_ns<8>(k, lz->alpha, lz->beta, y, nsm))) {
        // T_3 .. T_8: multiply-add iteration (k_lz_eig's FP64 QL sweeps took
        // ~20 and ~38 us for k = 3 and 4: divisions and square roots per rotation)
    } else {
        for (int i = lane; i < k; i += 32) {
            d[i] = lz->alpha[i + 1];
            e[i] = (i + 1 < k) ? lz->beta[i + 1] : 0.0;
            for (int c = 0; c < k; ++c) Q[i][c] = (i == c) ? 1.0 : 0.0;
        }
        __syncwarp();
        const double eps = 2.220446049250313e-16;
        for (int l = 0; l < k; ++l) {
            for (int sweep = 0; sweep < 60; ++sweep) {
                int m = l;
                for (; m < k - 1; ++m) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= eps * dd) break;
                }
                if (m == l) break;
                // shift from the leading 2x2 block (entries are O(mobility), far
                // from overflow, so plain square roots replace hypot)
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = sqrt(fma(g, g, 1.0));
                g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
                double s = 1.0, c = 1.0, p = 0.0;
                int i = m - 1;
                bool deflated = false;
                for (; i >= l; --i) {
                    const double f = s * e[i], b = c * e[i];
                    r = sqrt(fma(f, f, g * g));
                    __syncwarp();
                    if (lane == 0) e[i + 1] = r;
                    __syncwarp();
                    if (r == 0.0) {
                        if (lane == 0) { d[i + 1] -= p; e[m] = 0.0; }
                        __syncwarp();
                        deflated = true;
                        break;
                    }
                    const double rinv = 1.0 / r;  // one division per rotation
                    s = f * rinv;
                    c = g * rinv;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    p = s * r;
                    __syncwarp();
                    if (lane == 0) d[i + 1] = g + p;
                    __syncwarp();
                    g = c * r - b;
                    for (int row = lane; row < k; row += 32) {
                        const double qa = Q[row][i], qb = Q[row][i + 1];
                        Q[row][i + 1] = s * qa + c * qb;
                        Q[row][i] = c * qa - s * qb;
                    }
                    __syncwarp();
                }
                if (deflated && i >= l) continue;
                __syncwarp();
                if (lane == 0) { d[l] -= p; e[l] = g; e[m] = 0.0; }
                __syncwarp();
            }
        }
        __syncwarp();
        // y = Q diag(sqrt(max(lambda, 0))) Q^T e_1, each square root taken once
        for (int c = lane; c < k; c += 32) e[c] = sqrt(fmax(d[c], 0.0)) * Q[0][c];
        __syncwarp();
        for (int row = lane; row < k; row += 32) {
            double acc = 0.0;
            for (int c = 0; c < k; ++c) acc += Q[row][c] * e[c];
            y[row] = acc;
        }
        __syncwarp();
    }
    double num = 0.0, den = 0.0;
    for (int row = lane; row < k; row += 32) {
        const double prev = (row < k - 1) ? lz->y[row] : 0.0;
        num += (y[row] - prev) * (y[row] - prev);
        den += y[row] * y[row];
    }
    num = warp_sum(num);
    den = warp_sum(den);
    const double rel = (k >= 2 && den > 0) ? sqrt(num / den) : 1.0;
    bool stop;
    int conv = 0;
    if (fixed_iter > 0) {
        stop = (k >= fixed_iter);
        conv = stop;
    } else {
        // beta_k = 0: the Krylov space is invariant and T_k^{1/2} e_1 is exact
        const bool breakdown = !(lz->beta[k] > 0.0);
        conv = breakdown || (k >= 2 && rel < tol);
        stop = conv || (k >= max_iter);
    }
    const double b0 = lz->beta[0];
    __syncwarp();
    for (int row = lane; row < k; row += 32) {
        lz->y[row] = y[row];
        lz->coef[row] = (float)(b0 * y[row] / lz->beta[row]);
    }
    if (lane == 0) {
        lz->rel = rel;
        if (stop) {
            lz->J = k;
            lz->converged = conv;
        }
        lz->cont = stop ? 0 : 1;
        if (handle) cudaGraphSetConditional(handle, stop ? 0u : 1u);
    }
}

__global__ void __launch_bounds__(32) k_lz_eig(LzState *lz, int max_iter, int fixed_iter, double tol,
                                               cudaGraphConditionalHandle handle) {
    lz_eig_body(lz, max_iter, fixed_iter, tol, handle);
}

// One warp per system of a batch.
__global__ void __launch_bounds__(32) k_lz_eig_batch(const LzSys *__restrict__ sys) {
    const LzSys &S = sys[blockIdx.x];
    lz_eig_body(S.lz, S.max_iter, S.fixed_iter, S.tol, 0);
}

// One thread per system: the systems whose stop test passed in this loop
// body become inactive for the next one; the shared WHILE node continues
// while any system is still active.
__global__ void k_batch_cond(LzState *const *lzs, int nsys, cudaGraphConditionalHandle h, int *any_out) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < nsys; k += blockDim.x) {
        LzState *lz = lzs[k];
        const int c = lz->active && lz->cont;
        lz->active = c;
        if (c) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (h) cudaGraphSetConditional(h, any ? 1u : 0u);
        if (any_out) *any_out = any;
    }
}

// ------------------------------------------------------------------ final combination
// x_s = sum_{i=1..J} coef_i q_i[s]  (+ wave part), written in caller order.
// On the forces path (udet != null) out = c_noise x + c_det M_r F + wave, the
// wave part already carrying both weights.
// Three consecutive floats of a caller-order (N, 3) array in two stores:
// of two consecutive 4-byte aligned addresses one is 8-byte aligned, and the
// pair starting there goes out as one float2 (the scattered output writes
// are a third fewer).
__device__ __forceinline__ void store3(float *p, float x, float y, float z) {
    if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        *reinterpret_cast<float2 *>(p) = make_float2(x, y);
        p[2] = z;
    } else {
        p[0] = x;
        *reinterpret_cast<float2 *>(p + 1) = make_float2(y, z);
    }
}

template <typename T>
__device__ __forceinline__ void lz_final_body(int64_t N, const SampleArgs<T> *args, const V4<T> *pos_sorted,
                                              const V4<T> *basis, const V4<T> *uwave, const LzState *lz,
                                              bool with_wave, const float *__restrict__ pc, const V4<T> *udet,
                                              int64_t s) {
    __shared__ T cf[PSE_MAXIT + 2];
    __shared__ double cfd[PSE_MAXIT + 2];
    const int J = lz->J;
    for (int i = threadIdx.x; i < J; i += blockDim.x) {
        if constexpr (sizeof(T) == 4) cf[i] = lz->coef[i];
        else cfd[i] = lz->beta[0] * lz->y[i] / lz->beta[i];
    }
    __syncthreads();
    if (s >= N) return;
    T x = 0, y = 0, z = 0;
    for (int i = 0; i < J; ++i) {
        T c;
        if constexpr (sizeof(T) == 4) c = cf[i];
        else c = cfd[i];
        const V4<T> q = basis[(int64_t)i * N + s];
        x += c * q.x;
        y += c * q.y;
        z += c * q.z;
    }
    if constexpr (sizeof(T) == 4) {
        if (pc) {  // real part = S^{-1} (S M_r S)^{1/2} z1
            T a, b, c;
            sym3_apply(pc + s * 16 + 8, x, y, z, a, b, c);
            x = a; y = b; z = c;
        }
    }
    const int64_t o = 3 * w_bits_r(pos_sorted[s].w);
    T wx = 0, wy = 0, wz = 0;
    if (with_wave) {
        const V4<T> w = uwave[s];
        wx = w.x; wy = w.y; wz = w.z;
    }
    if (args->real) { args->real[o] = x; args->real[o + 1] = y; args->real[o + 2] = z; }
    if (args->wave && with_wave) { args->wave[o] = wx; args->wave[o + 1] = wy; args->wave[o + 2] = wz; }
    if (udet) {
        const T cn = (T)args->c_noise, cd = (T)args->c_det;
        const V4<T> m = udet[s];
        x = cn * x + cd * m.x;
        y = cn * y + cd * m.y;
        z = cn * z + cd * m.z;
    }
    if (args->out) {
        if constexpr (sizeof(T) == 4) {
            store3(args->out + o, x + wx, y + wy, z + wz);
        } else {
            args->out[o] = x + wx; args->out[o + 1] = y + wy; args->out[o + 2] = z + wz;
        }
    }
}

template <typename T>
__global__ void k_lz_final(int64_t N, const SampleArgs<T> *args, const V4<T> *pos_sorted, const V4<T> *basis,
                           const V4<T> *uwave, const LzState *lz, bool with_wave, const float *__restrict__ pc,
                           const V4<T> *udet) {
    lz_final_body<T>(N, args, pos_sorted, basis, uwave, lz, with_wave, pc, udet,
                     blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// One block of 256 particles per launch block: each block's particles belong
// to one system (blocks never straddle systems).
__global__ void k_lz_final_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    const BSys &S = sys[tab[blockIdx.x]];
    const int lb = (int)blockIdx.x - S.b0[BK_FINAL];
    lz_final_body<float>(S.N, S.d.args, S.d.pos_sorted, S.d.basis, S.d.uwave, S.d.lz, true, S.d.pc_on, nullptr,
                         lb * (int64_t)blockDim.x + threadIdx.x);
}

// Forces path without noise: out = c_det M_r F + wave part (c_det M_w F), caller order.
template <typename T>
__global__ void k_det_final(int64_t N, const SampleArgs<T> *args, const V4<T> *pos_sorted, const V4<T> *udet,
                            const V4<T> *uwave) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t o = 3 * w_bits_r(pos_sorted[s].w);
    const T cd = (T)args->c_det;
    const V4<T> m = udet[s], w = uwave[s];
    args->out[o] = cd * m.x + w.x;
    args->out[o + 1] = cd * m.y + w.y;
    args->out[o + 2] = cd * m.z + w.z;
}

// ------------------------------------------------------------------ Brownian dynamics step
// Overlap repulsion F_s = k_rep sum_t (2a - r) rhat over the list entries of
// s closer than 2a (pair vectors from cell-local offsets, as in the matvec),
// plus the external force, written in caller order.
template <typename T>
__global__ void k_repulsion(int64_t N, Geom<T> g, const SampleArgs<T> *args, const Rec<T> *__restrict__ rec,
                            const int *__restrict__ count, const int *__restrict__ nbr,
                            const V4<T> *__restrict__ pos_sorted, T *F) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const V4<T> li = rec[s].l;
    const T two_a = T(2) * g.a, k = (T)args->k_rep;
    T fx = 0, fy = 0, fz = 0;
    const int cnt = count[s];
    for (int q = 0; q < cnt; ++q) {
        const int e = nbr[(int64_t)q * N + s];
        if (e < 0) continue;  // a pair removed by the float64 decision at r_cut
        const V4<T> lt = rec[e >> 6].l;
        const int ox = ((e >> 4) & 3) - 1, oy = ((e >> 2) & 3) - 1, oz = (e & 3) - 1;
        const T dx = (li.x - lt.x) - (T(ox) * g.cs + T(ox) * g.cs_lo);
        const T dy = (li.y - lt.y) - (T(oy) * g.cs + T(oy) * g.cs_lo);
        const T dz = (li.z - lt.z) - (T(oz) * g.cs + T(oz) * g.cs_lo);
        const T r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < two_a * two_a && r2 > T(0)) {
            const T r = sqrt_hd(r2);
            const T f = k * (two_a - r) / r;
            fx += f * dx;
            fy += f * dy;
            fz += f * dz;
        }
    }
    const int64_t o = 3 * w_bits_r(pos_sorted[s].w);
    if (args->fext) {
        fx += args->fext[o];
        fy += args->fext[o + 1];
        fz += args->fext[o + 2];
    }
    F[o] = fx;
    F[o + 1] = fy;
    F[o + 2] = fz;
}

// x <- x + dx, wrapped into [0, L) (caller order).
template <typename T> __global__ void k_advance(int64_t N, Geom<T> g, const SampleArgs<T> *args) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * N || !args->advance) return;
    T x = args->advance[i] + args->out[i];
    x -= g.L * floor_hd(x / g.L);
    if (x >= g.L || x < T(0)) x = T(0);
    args->advance[i] = x;
}

// ------------------------------------------------------------------ caller-vector matvec
template <typename T>
__global__ void k_gather_vec(int64_t N, const SampleArgs<T> *args, const V4<T> *pos_sorted, Rec<T> *rec) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t o = 3 * w_bits_r(pos_sorted[s].w);
    V4<T> v;
    v.x = args->vin[o]; v.y = args->vin[o + 1]; v.z = args->vin[o + 2]; v.w = T(0);
    rec[s].q = v;
}

template <typename T, int TPP, bool POLY = false>
__global__ void __launch_bounds__(128) k_matvec_scatter(int64_t N, int K, const SampleArgs<T> *args, Geom<T> g,
                                                        const Rec<T> *rec, const int *count, const int *nbr,
                                                        const V4<T> *table, const V4<T> *pos_sorted) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = tid / TPP;
    const int lane_g = (int)(tid % TPP);
    const bool active = s < N;
    V4<T> li, qi;
    T ax, ay, az;
    mr_row_part<T, TPP, 4, false, POLY>(N, s, lane_g, active, K, g, rec, count, nbr, table, li, qi, ax, ay, az);
    if (!active || lane_g != 0) return;
    const int64_t i = 3 * w_bits_r(pos_sorted[s].w);
    const T self = POLY ? self_of(g, spec_of(li)) : g.self_m;
    args->out[i] = ax + self * qi.x;
    args->out[i + 1] = ay + self * qi.y;
    args->out[i + 2] = az + self * qi.z;
}

// M_r v for v already gathered into the records; output in sorted order.
template <typename T, int TPP>
__global__ void __launch_bounds__(128) k_matvec_sorted(int64_t N, int K, Geom<T> g, const Rec<T> *rec,
                                                       const int *count, const int *nbr, const V4<T> *table,
                                                       V4<T> *out) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = tid / TPP;
    const int lane_g = (int)(tid % TPP);
    const bool active = s < N;
    V4<T> li, qi;
    T ax, ay, az;
    mr_row_part<T, TPP, 4>(N, s, lane_g, active, K, g, rec, count, nbr, table, li, qi, ax, ay, az);
    if (!active || lane_g != 0) return;
    V4<T> o;
    o.x = ax + g.self_m * qi.x;
    o.y = ay + g.self_m * qi.y;
    o.z = az + g.self_m * qi.z;
    o.w = T(0);
    out[s] = o;
}

// ------------------------------------------------------------------ launchers
static inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
// persistent grid: at most `per_sm` resident blocks per SM
static inline unsigned pgrid(int64_t work_items, int items_per_block, int per_sm) {
    const int64_t need = (work_items + items_per_block - 1) / items_per_block;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}

static constexpr int kMvTpp = 4;

template <typename T>
void launch_lz_init(int64_t N, const SampleArgs<T> *args, int system, const Dev<T> &d, cudaStream_t s) {
    k_lz_init<T><<<pgrid(N, 256, 8), 256, 0, s>>>(N, args, system, d.pos_sorted, d.basis, d.rec, d.partials, d.lz,
                                                  sizeof(T) == 4 ? d.pc_on : nullptr);
}
// Matvec launch shapes (threads per particle, independent gathers per thread),
// selected by Geom::mv; the sampler may time them all and keep the fastest.
// Persistent grid: one wave of resident blocks (at most 16 per SM), so that
// no second, partly filled wave of equal-work blocks trails the first.
template <typename T, int TPP, int ILP, int BS = 128> int mv_blocks_per_sm() {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lz_matvec<T, TPP, ILP, BS>, BS, 0) != cudaSuccess ||
            nb < 1) {
            cudaGetLastError();
            nb = BS >= 1024 ? 1 : 2048 / BS;
        }
        per_sm = nb < 16 ? nb : 16;
    }
    return per_sm;
}
// resident blocks per SM of the fused batch matvec (at most 16)
int matvec_blocks_per_sm() {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lz_matvec_batch, PSE_BATCH_MV_THREADS, 0) !=
                cudaSuccess ||
            nb < 1) {
            cudaGetLastError();
            nb = 1;
        }
        per_sm = nb < 16 ? nb : 16;
    }
    return per_sm;
}
// the same for the Lanczos update (FP32 and FP64), at most 8 per SM
template <typename T> int up_blocks_per_sm() {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lz_update<T>, 256, 0) != cudaSuccess || nb < 1) {
            cudaGetLastError();
            nb = 8;
        }
        per_sm = nb < 8 ? nb : 8;
    }
    return per_sm;
}
int update_blocks_per_sm() { return up_blocks_per_sm<float>(); }
// occupancy of every matvec shape, queried once outside any stream capture
static int mv_poly_blocks_per_sm() {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lz_matvec_poly, 1024, 0) != cudaSuccess || nb < 1) {
            cudaGetLastError();
            nb = 1;
        }
        per_sm = nb;
    }
    return per_sm;
}
static int mv_nolist_blocks_per_sm() {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lz_matvec_nolist, PSE_NOLIST_THREADS, 0) !=
                cudaSuccess ||
            nb < 1) {
            cudaGetLastError();
            nb = 1;
        }
        per_sm = nb;
    }
    return per_sm;
}
// Launch geometry of the brick-tiled matvec: the staging capacity follows the
// mean neighbourhood occupancy 216 N / ncell^3 with six standard deviations
// of Poisson slack; blocks per SM from the shared memory that leaves.
static size_t g_tile_static_smem = 0, g_sm_smem = 0;
static int g_tile_regs = 0;
static int tile_cap(int64_t N, int nc) {
    const double mean = 216.0 * (double)N / ((double)nc * nc * nc);
    int cap = (int)(mean + 6.0 * sqrt(mean) + 32.0);
    cap = (cap + 31) & ~31;
    return cap < 256 ? 256 : (cap > 4096 ? 4096 : cap);
}
static void tile_prepare() {
    if (g_sm_smem) return;
    int dev = 0, v = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, k_lz_matvec_tiled) == cudaSuccess &&
        cudaFuncSetAttribute(k_lz_matvec_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             4096 * (int)sizeof(Rec<float>)) == cudaSuccess) {
        g_tile_static_smem = fa.sharedSizeBytes;
        g_tile_regs = fa.numRegs;
        g_sm_smem = (size_t)v;
    } else {
        cudaGetLastError();
    }
}
static int tile_blocks_per_sm(size_t dyn) {
    if (!g_sm_smem) return 1;
    const size_t per_block = g_tile_static_smem + dyn + 1024;  // 1 KB per block reserved by the runtime
    int nb = (int)(g_sm_smem / per_block);
    const int by_regs = 65536 / ((g_tile_regs > 0 ? g_tile_regs : 64) * PSE_TILE_THREADS);
    nb = nb < by_regs ? nb : by_regs;
    nb = nb < 2048 / PSE_TILE_THREADS ? nb : 2048 / PSE_TILE_THREADS;
    return nb > 0 ? nb : 1;
}

template <typename T> void mv_prepare_all() {
    mv_blocks_per_sm<T, 4, 4>(); mv_blocks_per_sm<T, 8, 2>();
    mv_blocks_per_sm<T, 16, 1>(); mv_blocks_per_sm<T, 4, 2>();
    mv_blocks_per_sm<T, 4, 4, 1024>(); mv_blocks_per_sm<T, 4, 4, 512>();
    mv_blocks_per_sm<T, 8, 2, 1024>(); mv_blocks_per_sm<T, 4, 2, 1024>();
    mv_blocks_per_sm<T, 1, 4, 1024>(); mv_blocks_per_sm<T, 2, 4, 1024>();
    if constexpr (sizeof(T) == 4) {
        mv_poly_blocks_per_sm();
        mv_nolist_blocks_per_sm();
    }
}
void matvec_prepare() {
    tile_prepare();
    mv_prepare_all<float>();
    mv_prepare_all<double>();
    up_blocks_per_sm<float>(); up_blocks_per_sm<double>();
    matvec_blocks_per_sm();
}

template <typename T, int TPP, int ILP, int BS = 128>
void mv_launch(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_lz_matvec<T, TPP, ILP, BS><<<pgrid(N, BS / TPP, mv_blocks_per_sm<T, TPP, ILP, BS>()), BS, 0, s>>>(
        N, nbr_k(N, d.nbr_cap), g, d.rec, d.nbr_count, d.nbr, d.table, d.table_c, d.u, d.partials, d.lz,
        sizeof(T) == 4 ? d.pc_on : nullptr, d.basis, d.mv_add);
}
template <typename T> void launch_lz_matvec(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (g.mv == PSE_MV_TILED && g.nspec <= 1 && !d.pc_on && g_sm_smem) {
            const int cap = tile_cap(N, g.nc);
            const size_t dyn = (size_t)cap * sizeof(Rec<float>);
            const int nbricks = g.nb * g.nb * g.nb;
            k_lz_matvec_tiled<<<pgrid(nbricks, 1, tile_blocks_per_sm(dyn)), PSE_TILE_THREADS, dyn, s>>>(
                N, nbr_k(N, d.nbr_cap), g, d.rec, d.cell_start, d.nbr_count, d.nbr, d.table_c, d.u, d.partials, d.lz,
                d.mv_add, nbricks, cap);
            return;
        }
        if (g.mv == PSE_MV_NOLIST && g.nspec <= 1 && !d.pc_on) {
            k_lz_matvec_nolist<<<pgrid(N, PSE_NOLIST_THREADS, mv_nolist_blocks_per_sm()), PSE_NOLIST_THREADS, 0, s>>>(
                N, g, d.rec, d.cell_start, d.pos_sorted, d.table_c, d.u, d.partials, d.lz, d.mv_add);
            return;
        }
        if (g.nspec > 1) {
            k_lz_matvec_poly<<<pgrid(N, 1024 / 4, mv_poly_blocks_per_sm()), 1024, 0, s>>>(
                N, nbr_k(N, d.nbr_cap), g, d.rec, d.nbr_count, d.nbr, d.table, d.u, d.partials, d.lz, d.basis);
            return;
        }
    }
    switch (g.mv) {
        case 1: mv_launch<T, 8, 2>(N, g, d, s); break;
        case 2: mv_launch<T, 16, 1>(N, g, d, s); break;
        case 3: mv_launch<T, 4, 2>(N, g, d, s); break;
        case 4:
        case PSE_MV_TILED: mv_launch<T, 4, 4, 1024>(N, g, d, s); break;
        case 5: mv_launch<T, 4, 4, 512>(N, g, d, s); break;
        case 6: mv_launch<T, 8, 2, 1024>(N, g, d, s); break;
        case 7: mv_launch<T, 4, 2, 1024>(N, g, d, s); break;
        case 8: mv_launch<T, 1, 4, 1024>(N, g, d, s); break;
        case 9: mv_launch<T, 2, 4, 1024>(N, g, d, s); break;
        default: mv_launch<T, 4, 4>(N, g, d, s); break;
    }
}
template <typename T> void launch_lz_update(int64_t N, int, const Dev<T> &d, cudaStream_t s) {
    k_lz_update<T><<<pgrid(N, 256, up_blocks_per_sm<T>()), 256, 0, s>>>(N, d.basis, d.rec, d.u, d.partials + num_sms() * 16 + 32, d.lz,
                                                    sizeof(T) == 4 ? d.pc_on : nullptr);
}
void launch_lz_eig(LzState *lz, int max_iter, int fixed_iter, double tol, cudaGraphConditionalHandle h,
                   cudaStream_t s) {
    k_lz_eig<<<1, 32, 0, s>>>(lz, max_iter, fixed_iter, tol, h);
}
void launch_batch_cond(LzState *const *lzs, int nsys, cudaGraphConditionalHandle h, cudaStream_t s, int *any_out) {
    k_batch_cond<<<1, 256, 0, s>>>(lzs, nsys, h, any_out);
}
void launch_lz_matvec_batch(const LzSys *sys, const int *blk2sys, int nblocks, cudaStream_t s) {
    k_lz_matvec_batch<<<nblocks, PSE_BATCH_MV_THREADS, 0, s>>>(sys, blk2sys);
}
void launch_lz_update_batch(const LzSys *sys, const int *blk2sys, int nblocks, cudaStream_t s) {
    k_lz_update_batch<<<nblocks, 256, 0, s>>>(sys, blk2sys);
}
void launch_lz_eig_batch(const LzSys *sys, int nsys, cudaStream_t s) { k_lz_eig_batch<<<nsys, 32, 0, s>>>(sys); }
void launch_batch_init(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s) {
    k_lz_init_batch<<<nblk[BK_INIT], 256, 0, s>>>(sys, tab[BK_INIT]);
}
void launch_batch_final(const BSys *sys, int *const *tab, const int *nblk, cudaStream_t s) {
    k_lz_final_batch<<<nblk[BK_FINAL], 256, 0, s>>>(sys, tab[BK_FINAL]);
}
template <typename T>
void launch_lz_final(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, bool with_wave, cudaStream_t s) {
    k_lz_final<T><<<nb(N, 256), 256, 0, s>>>(N, args, d.pos_sorted, d.basis, d.uwave, d.lz, with_wave,
                                             sizeof(T) == 4 ? d.pc_on : nullptr, nullptr);
}
template <typename T>
void launch_lz_final_forces(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s) {
    k_lz_final<T><<<nb(N, 256), 256, 0, s>>>(N, args, d.pos_sorted, d.basis, d.uwave, d.lz, true,
                                             sizeof(T) == 4 ? d.pc_on : nullptr, d.udet);
}
template <typename T> void launch_repulsion(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_repulsion<T><<<nb(N, 128), 128, 0, s>>>(N, g, d.args, d.rec, d.nbr_count, d.nbr, d.pos_sorted, d.bd_force);
}
template <typename T> void launch_advance(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_advance<T><<<nb(3 * N, 256), 256, 0, s>>>(N, g, d.args);
}
template <typename T> void launch_det_final(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s) {
    k_det_final<T><<<nb(N, 256), 256, 0, s>>>(N, args, d.pos_sorted, d.udet, d.uwave);
}
template <typename T> void launch_gather_vec(int64_t N, const SampleArgs<T> *args, const Dev<T> &d, cudaStream_t s) {
    k_gather_vec<T><<<nb(N, 256), 256, 0, s>>>(N, args, d.pos_sorted, d.rec);
}
template <typename T> void launch_matvec_sorted(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_matvec_sorted<T, kMvTpp><<<nb(N * kMvTpp, 128), 128, 0, s>>>(N, nbr_k(N, d.nbr_cap), g, d.rec, d.nbr_count,
                                                                    d.nbr, d.table, d.udet);
}
template <typename T>
void launch_matvec_caller(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_gather_vec<T><<<nb(N, 256), 256, 0, s>>>(N, args, d.pos_sorted, d.rec);
    if (g.nspec > 1)
        k_matvec_scatter<T, kMvTpp, true><<<nb(N * kMvTpp, 128), 128, 0, s>>>(N, nbr_k(N, d.nbr_cap), args, g, d.rec,
                                                                              d.nbr_count, d.nbr, d.table,
                                                                              d.pos_sorted);
    else
        k_matvec_scatter<T, kMvTpp><<<nb(N * kMvTpp, 128), 128, 0, s>>>(N, nbr_k(N, d.nbr_cap), args, g, d.rec,
                                                                         d.nbr_count, d.nbr, d.table,
                                                                         d.pos_sorted);
}

#define PSE_INST(T)                                                                                          \
    template void launch_lz_init<T>(int64_t, const SampleArgs<T> *, int, const Dev<T> &, cudaStream_t);        \
    template void launch_lz_matvec<T>(int64_t, Geom<T>, const Dev<T> &, cudaStream_t);                       \
    template void launch_lz_update<T>(int64_t, int, const Dev<T> &, cudaStream_t);                           \
    template void launch_lz_final<T>(int64_t, const SampleArgs<T> *, const Dev<T> &, bool, cudaStream_t);    \
    template void launch_lz_final_forces<T>(int64_t, const SampleArgs<T> *, const Dev<T> &, cudaStream_t);   \
    template void launch_det_final<T>(int64_t, const SampleArgs<T> *, const Dev<T> &, cudaStream_t);         \
    template void launch_repulsion<T>(int64_t, Geom<T>, const Dev<T> &, cudaStream_t);                       \
    template void launch_advance<T>(int64_t, Geom<T>, const Dev<T> &, cudaStream_t);                         \
    template void launch_gather_vec<T>(int64_t, const SampleArgs<T> *, const Dev<T> &, cudaStream_t);        \
    template void launch_matvec_sorted<T>(int64_t, Geom<T>, const Dev<T> &, cudaStream_t);                   \
    template void launch_matvec_caller<T>(int64_t, const SampleArgs<T> *, Geom<T>, const Dev<T> &, cudaStream_t);
PSE_INST(float)
PSE_INST(double)
#undef PSE_INST

}  // namespace pse
