// Cell list, device scan and near-field neighbour list (the linked-cell
// search the paper's real-space sum uses, Sec. III), sm_103a.
//
// Particles are binned into ncell^3 cells of side >= r_cut (ids in 4x4x4
// brick-major order), counting-sorted into cell order (deterministic: ties in a cell are ordered by caller
// index), and every sorted particle gets an ELL list of the particles within
// r_cut.  Each entry packs the neighbour's sorted index with the 3x3x3
// stencil offset of its cell, so pair vectors are formed from cell-local
// offsets: d = (l_i - l_t) - dc * cs, accurate to a few float ulps of the
// cell side whatever the box size, with no wrap logic in the matvec.
#include "pse_internal.cuh"

namespace pse {

template <typename T> __device__ __forceinline__ T wrap_box(T x, T L) {
    if (x < T(0) || x >= L) {
        x -= L * floor(x / L);
        if (x >= L || x < T(0)) x = T(0);
    }
    return x;
}

template <typename T> __device__ __forceinline__ int cell_coord(T x, T inv_cs, int nc) {
    int c = (int)(x * inv_cs);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// offset of x from its cell corner c*cs, compensated: fma gives x - c*cs_hi
// with one rounding, then the low part of cs is removed.
__device__ __forceinline__ float cell_offset(float x, int c, float cs, float cs_lo) {
    return fmaf(-(float)c, cs, x) - (float)c * cs_lo;
}
__device__ __forceinline__ double cell_offset(double x, int c, double cs, double) { return x - c * cs; }

template <typename T>
__device__ __forceinline__ void bin_elem(int64_t i, const SampleArgs<T> *args, const Geom<T> &g, int *cell_of,
                                         int *slot, int *count) {
    const T *p = args->pos + 3 * i;
    const T x = wrap_box(p[0], g.L), y = wrap_box(p[1], g.L), z = wrap_box(p[2], g.L);
    const int cx = cell_coord(x, g.inv_cs, g.nc), cy = cell_coord(y, g.inv_cs, g.nc),
              cz = cell_coord(z, g.inv_cs, g.nc);
    const int c = cell_id(cx, cy, cz, g.nb);
    cell_of[i] = c;
    slot[i] = atomicAdd(count + c, 1);
}

template <typename T>
__global__ void k_bin(int64_t N, const SampleArgs<T> *args, Geom<T> g, int *cell_of, int *slot, int *count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) bin_elem<T>(i, args, g, cell_of, slot, count);
}

// Counting-sort scatter: slot start[c] + slot[i] gets the caller index i
// (inside a cell the slots follow k_bin's atomics; the placement below makes
// the order deterministic).
__global__ void k_scatter(int64_t N, const int *__restrict__ cell_of, const int *__restrict__ slot,
                          const int *__restrict__ start, int *perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) perm[start[cell_of[i]] + slot[i]] = (int)i;
}

template <typename T> __device__ __forceinline__ long long w_bits(T w) {
    if constexpr (sizeof(T) == 4) return (long long)__float_as_int(w);
    else return __double_as_longlong(w);
}

// Placement of counting-sort slot k: its particle i goes to position
// b + rank in its cell [b, e), rank = the number of the cell's members with
// a smaller caller index, so each cell is ordered by caller index whatever
// the atomics did (one thread per particle, no serial per-cell sort).  The
// position there gets the wrapped position (w = caller index bits), the
// offsets from the cell corner (w = cell id, species in the high bits) and
// the offsets half of the matvec record.
template <typename T>
__device__ __forceinline__ void place_elem(int64_t k, const SampleArgs<T> *args, const Geom<T> &g,
                                           const int *__restrict__ cell_of, const int *__restrict__ start,
                                           const int *__restrict__ perm, V4<T> *pos_sorted, V4<T> *loc_sorted,
                                           Rec<T> *rec) {
    const int i = perm[k];
    const int c = cell_of[i];
    const int b = start[c], e = start[c + 1];
    int rank = 0;
    for (int t = b; t < e; ++t) rank += perm[t] < i;
    const int64_t dst = b + rank;
    const T *p = args->pos + 3 * (int64_t)i;
    const T x = wrap_box(p[0], g.L), y = wrap_box(p[1], g.L), z = wrap_box(p[2], g.L);
    int cx, cy, cz;
    cell_xyz(c, g.nb, cx, cy, cz);
    V4<T> a;
    a.x = x; a.y = y; a.z = z;
    if constexpr (sizeof(T) == 4) a.w = __int_as_float(i);
    else a.w = __longlong_as_double((long long)i);
    pos_sorted[dst] = a;
    V4<T> l;
    l.x = cell_offset(x, cx, g.cs, g.cs_lo);
    l.y = cell_offset(y, cy, g.cs, g.cs_lo);
    l.z = cell_offset(z, cz, g.cs, g.cs_lo);
    // polydisperse: the species (clamped to the context's species) rides in
    // the high bits of the cell id
    int cw = c;
    if (args->species) {
        int sp = args->species[i];
        sp = sp < 0 ? 0 : (sp >= g.nspec ? g.nspec - 1 : sp);
        cw |= sp << PSE_SPECIES_SHIFT;
    }
    if constexpr (sizeof(T) == 4) l.w = __int_as_float(cw);
    else l.w = __longlong_as_double((long long)cw);
    loc_sorted[dst] = l;
    rec[dst].l = l;
}

template <typename T>
__global__ void k_place(int64_t N, const SampleArgs<T> *args, Geom<T> g, const int *__restrict__ cell_of,
                        const int *__restrict__ start, const int *__restrict__ perm, V4<T> *pos_sorted,
                        V4<T> *loc_sorted, Rec<T> *rec) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N) place_elem<T>(k, args, g, cell_of, start, perm, pos_sorted, loc_sorted, rec);
}

// One thread per sorted particle, one pass: every neighbour within r_cut over
// the 27 stencil cells goes to ELL column cnt (nbr[cnt * N + s], coalesced
// across a warp when counts agree) as (t << 6) | stencil code.  With
// ncell = 2 the same cell appears under two offsets; r_cut < L/2 leaves at
// most one image of each pair inside r_cut, so the distance test keeps the
// right one.  Lists longer than K are cut and flag an overflow.
// A float32 pair distance within rounding of r_cut (|r^2 - r_cut^2| below
// 4e-6 r_cut^2, about three times the error of the cell-offset arithmetic)
// does not decide the pair.  The search keeps every pair below the top of
// that band and only notes that a particle met one in it; such particles (a
// few per 10^5) walk their cells a second time, off the main loop, and
// record each band pair (s, t, code, list slot) in a small edge buffer;
// k_nbr_edges then decides it again in float64 from the wrapped positions
// with the nearest periodic image and removes the entries beyond r_cut (set
// to -1, which every list reader skips).  The lists then hold exactly the
// pairs with r < r_cut in float64, as the oracle's do.
//
// One walk over the 27 stencil cells.  RECORD = false: fill the ELL row and
// flag a pair in the band; RECORD = true: write nothing but the band's pairs
// to the edge buffer, with the list slot the first walk gave them.
// The stencil shift is folded into the particle's own offset once per cell
// row (d = (l_i - shift) - l_t; its rounding stays far inside the band), and
// the self test runs only on candidates inside r_cut.
template <typename T, bool RECORD>
__device__ __forceinline__ int nbr_walk(int64_t s, int64_t N, const Geom<T> &g, const V4<T> *__restrict__ loc,
                                        const int *__restrict__ cell_start, int *nbr, int K, bool &band,
                                        int4 *edge, int *edge_n, int edge_cap) {
    int cnt = 0;
    const V4<T> li = loc[s];
    const int c = (int)(w_bits(li.w) & PSE_CELL_MASK);
    const int nc = g.nc;
    int cx, cy, cz;
    cell_xyz(c, g.nb, cx, cy, cz);
    int *dst = nbr + s;  // ELL column cnt of row s
    for (int ox = -1; ox <= 1; ++ox) {
        int ax = cx + ox;
        ax += ax < 0 ? nc : 0;
        ax -= ax >= nc ? nc : 0;
        const T px = li.x - (T(ox) * g.cs + T(ox) * g.cs_lo);
        for (int oy = -1; oy <= 1; ++oy) {
            int ay = cy + oy;
            ay += ay < 0 ? nc : 0;
            ay -= ay >= nc ? nc : 0;
            const T py = li.y - (T(oy) * g.cs + T(oy) * g.cs_lo);
            for (int oz = -1; oz <= 1; ++oz) {
                int az = cz + oz;
                az += az < 0 ? nc : 0;
                az -= az >= nc ? nc : 0;
                const T pz = li.z - (T(oz) * g.cs + T(oz) * g.cs_lo);
                const int code = ((ox + 1) << 4) | ((oy + 1) << 2) | (oz + 1);
                const int c2 = cell_id(ax, ay, az, g.nb);
                const int b = cell_start[c2], e = cell_start[c2 + 1];
                const int self = code == 21 ? (int)s : -1;  // the particle itself, in its own cell
#pragma unroll 2
                for (int t = b; t < e; ++t) {
                    const V4<T> lt = loc[t];
                    const T dx = px - lt.x, dy = py - lt.y, dz = pz - lt.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    // the float test keeps every pair up to the top of the band; the
                    // float64 decision later removes those beyond r_cut.  The
                    // particle itself (r2 = 0) passes it and is dropped here.
                    if (r2 < g.rc2_hi && t != self) {
                        if constexpr (RECORD) {
                            if (r2 >= g.rc2_lo) {
                                const int k = atomicAdd(edge_n, 1);
                                if (k < edge_cap) edge[k] = make_int4((int)s, t, code, cnt < K ? cnt : -2);
                            }
                        } else {
                            if constexpr (sizeof(T) == 4) {
                                if (r2 >= g.rc2_lo) band = true;
                            }
                            if (cnt < K) {
                                *dst = (t << 6) | code;
                                dst += N;
                            }
                        }
                        ++cnt;
                    }
                }
            }
        }
    }
    return cnt;
}

// The second walk, out of line: the main loop's registers and schedule do
// not pay for it.
template <typename T>
__device__ __noinline__ void nbr_record_band(int64_t s, int64_t N, Geom<T> g, const V4<T> *__restrict__ loc,
                                             const int *__restrict__ cell_start, int *nbr, int K, int4 *edge,
                                             int *edge_n, int edge_cap) {
    bool unused = false;
    nbr_walk<T, true>(s, N, g, loc, cell_start, nbr, K, unused, edge, edge_n, edge_cap);
}

template <typename T>
__device__ __forceinline__ int nbr_elem(int64_t s, int64_t N, const Geom<T> &g, const V4<T> *__restrict__ loc,
                                        const int *__restrict__ cell_start, int *count, int *nbr, int K,
                                        int *overflow, int4 *edge, int *edge_n, int edge_cap) {
    bool band = false;
    int cnt = nbr_walk<T, false>(s, N, g, loc, cell_start, nbr, K, band, edge, edge_n, edge_cap);
    if constexpr (sizeof(T) == 4) {
        if (band) nbr_record_band<T>(s, N, g, loc, cell_start, nbr, K, edge, edge_n, edge_cap);
    }
    if (cnt > K) {
        atomicExch(overflow, 1);
        cnt = K;
    }
    count[s] = cnt;
    return cnt;
}

// Blocks of 256 threads with no minimum block count, the candidate loop
// unrolled twice: at N = 1e6 (phi = 0.1) 185 us, against 188 in blocks of
// 128, 192 in blocks of 64, 190-202 us with a minimum of 10, 12 or 16 blocks
// of 128 per SM, and 218-227 us unrolled 1, 3 or 4 times (ptxas' register
// allocation and load scheduling decide it; all give the same lists).
template <typename T>
__global__ void __launch_bounds__(256) k_nbr(int64_t N, Geom<T> g, const V4<T> *__restrict__ loc,
                                             const int *__restrict__ cell_start, int *count, int *nbr, int K,
                                             int *overflow, unsigned long long *n_pairs, int4 *edge, int *edge_n,
                                             int edge_cap) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int cnt = s < N ? nbr_elem<T>(s, N, g, loc, cell_start, count, nbr, K, overflow, edge, edge_n, edge_cap)
                          : 0;
    // pair total for the statistics: one atomic per warp
    int tot = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(n_pairs, (unsigned long long)tot);
}

// The float64 decision for the pairs k_nbr recorded within rounding of
// r_cut (one block; a few per 10^5 particles).  Entry (s, t, code, slot):
// slot >= 0 the float search stored the pair there, -2 it accepted it with a
// full list, -1 it rejected it.  Clears the edge count for the next search.
__device__ __forceinline__ void nbr_edges_body(int64_t N, const Geom<float> &g, const V4<float> *__restrict__ pos,
                                               int *count, int *nbr, int K, int *overflow,
                                               unsigned long long *n_pairs, const int4 *edge, int *edge_n,
                                               int edge_cap) {
    const int n = min(*edge_n, edge_cap);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int4 e = edge[i];
        const int64_t s = e.x;
        const bool in32 = e.w != -1, in64 = pair_inside_f64(pos[s], pos[e.y], g);
        if (in32 && !in64) {
            if (e.w >= 0) {
                nbr[(int64_t)e.w * N + s] = -1;
                atomicAdd(n_pairs, ~0ull);  // - 1
            }
        } else if (!in32 && in64) {
            const int k = atomicAdd(count + s, 1);
            if (k < K) {
                nbr[(int64_t)k * N + s] = (e.y << 6) | e.z;
                atomicAdd(n_pairs, 1ull);
            } else {
                atomicSub(count + s, 1);
                atomicExch(overflow, 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *edge_n = 0;
}

__global__ void __launch_bounds__(256) k_nbr_edges(int64_t N, Geom<float> g, const V4<float> *__restrict__ pos,
                                                   int *count, int *nbr, int K, int *overflow,
                                                   unsigned long long *n_pairs, const int4 *edge, int *edge_n,
                                                   int edge_cap) {
    nbr_edges_body(N, g, pos, count, nbr, K, overflow, n_pairs, edge, edge_n, edge_cap);
}

// ------------------------------------------------------------------ fused multi-system kernels
// Block b of a fused launch works for system tab[b]; lb is its index among
// that system's nb blocks.  Element-wise kernels stride over the system's
// elements with its blocks.
#define PSE_BATCH_SYS(kind)                                  \
    const BSys &S = sys[tab[blockIdx.x]];                    \
    const int lb = (int)blockIdx.x - S.b0[kind];             \
    const int64_t stride = (int64_t)S.nb[kind] * blockDim.x

__global__ void k_zero_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    PSE_BATCH_SYS(BK_ZERO);
    for (int64_t c = lb * (int64_t)blockDim.x + threadIdx.x; c < S.nc3; c += stride) S.d.cell_count[c] = 0;
    if (lb == 0 && threadIdx.x == 0) {
        S.d.lz->overflow = 0;
        S.d.lz->n_pairs = 0ull;
    }
}
__global__ void k_bin_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    PSE_BATCH_SYS(BK_BIN);
    for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < S.N; i += stride)
        bin_elem<float>(i, S.d.args, S.g, S.d.cell_of, S.d.slot, S.d.cell_count);
}
// One block of 1024 threads per system: exclusive scan of the cell counts
// into cell_start (nc3 + 1 entries), 4096 counts per pass with a carry.
__global__ void __launch_bounds__(1024) k_scan_batch(const BSys *__restrict__ sys) {
    const BSys &S = sys[blockIdx.x];
    __shared__ int sh[1024];
    int carry = 0;
    const int n = S.nc3;
    for (int base0 = 0; base0 < n; base0 += PSE_SCAN_ITEMS) {
        const int base = base0 + threadIdx.x * 4;
        int v[4], tot = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = base + k < n ? S.d.cell_count[base + k] : 0;
            tot += v[k];
        }
        sh[threadIdx.x] = tot;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        int run = carry + sh[threadIdx.x] - tot;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < n) S.d.cell_start[base + k] = run;
            run += v[k];
        }
        carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) S.d.cell_start[n] = carry;
}
__global__ void k_scatter_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    PSE_BATCH_SYS(BK_SCATTER);
    for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < S.N; i += stride)
        S.d.perm[S.d.cell_start[S.d.cell_of[i]] + S.d.slot[i]] = (int)i;
}
__global__ void k_place_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    PSE_BATCH_SYS(BK_SORT);
    for (int64_t k = lb * (int64_t)blockDim.x + threadIdx.x; k < S.N; k += stride)
        place_elem<float>(k, S.d.args, S.g, S.d.cell_of, S.d.cell_start, S.d.perm, S.d.pos_sorted, S.d.loc_sorted,
                          S.d.rec);
}
__global__ void __launch_bounds__(256) k_nbr_batch(const BSys *__restrict__ sys, const int *__restrict__ tab) {
    PSE_BATCH_SYS(BK_NBR);
    for (int64_t s0 = lb * (int64_t)blockDim.x; s0 < S.N; s0 += stride) {  // uniform per block
        const int64_t s = s0 + threadIdx.x;
        const int cnt = s < S.N ? nbr_elem<float>(s, S.N, S.g, S.d.loc_sorted, S.d.cell_start, S.d.nbr_count,
                                                   S.d.nbr, S.K, &S.d.lz->overflow, S.d.edge, S.d.edge_n,
                                                   S.d.edge_cap)
                                : 0;
        int tot = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&S.d.lz->n_pairs, (unsigned long long)tot);
    }
}

static unsigned tab_blocks(const int *nblk, int kind) { return (unsigned)nblk[kind]; }

void launch_batch_prologue_cells(const BSys *sys, int nsys, int *const *tab, const int *nblk, cudaStream_t s) {
    k_zero_batch<<<tab_blocks(nblk, BK_ZERO), 256, 0, s>>>(sys, tab[BK_ZERO]);
    k_bin_batch<<<tab_blocks(nblk, BK_BIN), 256, 0, s>>>(sys, tab[BK_BIN]);
    k_scan_batch<<<nsys, 1024, 0, s>>>(sys);
    k_scatter_batch<<<tab_blocks(nblk, BK_SCATTER), 256, 0, s>>>(sys, tab[BK_SCATTER]);
    k_place_batch<<<tab_blocks(nblk, BK_SORT), 256, 0, s>>>(sys, tab[BK_SORT]);
}
// one block per system for the float64 decisions at r_cut
__global__ void __launch_bounds__(256) k_nbr_edges_batch(const BSys *__restrict__ sys) {
    const BSys &S = sys[blockIdx.x];
    nbr_edges_body(S.N, S.g, S.d.pos_sorted, S.d.nbr_count, S.d.nbr, S.K, &S.d.lz->overflow, &S.d.lz->n_pairs,
                   S.d.edge, S.d.edge_n, S.d.edge_cap);
}

void launch_batch_nbr(const BSys *sys, int nsys, int *const *tab, const int *nblk, cudaStream_t s) {
    k_nbr_batch<<<tab_blocks(nblk, BK_NBR), 256, 0, s>>>(sys, tab[BK_NBR]);
    k_nbr_edges_batch<<<nsys, 256, 0, s>>>(sys);
}

// ------------------------------------------------------------------ exclusive scan
// Three passes: per-block scan of PSE_SCAN_ITEMS ints (1024 threads x 4),
// a one-block scan of the block totals, then the carry-in add.
__global__ void k_scan_block(const int *in, int *out, int64_t n, int *sums) {
    __shared__ int sh[1024];
    const int64_t base = (int64_t)blockIdx.x * PSE_SCAN_ITEMS + threadIdx.x * 4;
    int v[4];
    int tot = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tot += v[k];
    }
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan
        const int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = sh[threadIdx.x] - tot;  // exclusive prefix of this thread
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) sums[blockIdx.x] = sh[1023];
}

__global__ void k_scan_sums(int *sums, int nb, int *total_out) {
    __shared__ int sh[1024];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
        const int chunk = sh[1023];
        __syncthreads();
        carry += chunk;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int *out, int64_t n, const int *sums) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / PSE_SCAN_ITEMS];
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 132;
    }
    return n;
}

void launch_scan(const int *in, int *out, int64_t n, int *sums, cudaStream_t s) {
    const int nb = (int)((n + PSE_SCAN_ITEMS - 1) / PSE_SCAN_ITEMS);
    if (nb > 0) k_scan_block<<<nb, 1024, 0, s>>>(in, out, n, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, out + n);
    if (n > 0) k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
}

// ------------------------------------------------------------------ launchers
static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
void launch_bin(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    const int64_t nc3 = cell_slots(g.nc);
    cudaMemsetAsync(d.cell_count, 0, sizeof(int) * nc3, s);
    k_bin<T><<<nblk(N, 256), 256, 0, s>>>(N, args, g, d.cell_of, d.slot, d.cell_count);
    launch_scan(d.cell_count, d.cell_start, nc3, d.scan_sums, s);
}

template <typename T>
void launch_scatter(int64_t N, const SampleArgs<T> *, Geom<T>, const Dev<T> &d, cudaStream_t s) {
    k_scatter<<<nblk(N, 256), 256, 0, s>>>(N, d.cell_of, d.slot, d.cell_start, d.perm);
}

template <typename T>
void launch_place(int64_t N, const SampleArgs<T> *args, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_place<T><<<nblk(N, 256), 256, 0, s>>>(N, args, g, d.cell_of, d.cell_start, d.perm, d.pos_sorted,
                                            d.loc_sorted, d.rec);
}

template <typename T> void launch_nbr(int64_t N, Geom<T> g, const Dev<T> &d, cudaStream_t s) {
    k_nbr<T><<<nblk(N, 256), 256, 0, s>>>(N, g, d.loc_sorted, d.cell_start, d.nbr_count, d.nbr,
                                          nbr_k(N, d.nbr_cap), &d.lz->overflow, &d.lz->n_pairs, d.edge, d.edge_n,
                                          d.edge_cap);
    if constexpr (sizeof(T) == 4)
        k_nbr_edges<<<1, 256, 0, s>>>(N, g, d.pos_sorted, d.nbr_count, d.nbr, nbr_k(N, d.nbr_cap), &d.lz->overflow,
                                      &d.lz->n_pairs, d.edge, d.edge_n, d.edge_cap);
}

#define PSE_INST(T)                                                                                       \
    template void launch_bin<T>(int64_t, const SampleArgs<T> *, Geom<T>, const Dev<T> &, cudaStream_t);     \
    template void launch_scatter<T>(int64_t, const SampleArgs<T> *, Geom<T>, const Dev<T> &, cudaStream_t); \
    template void launch_place<T>(int64_t, const SampleArgs<T> *, Geom<T>, const Dev<T> &, cudaStream_t);   \
    template void launch_nbr<T>(int64_t, Geom<T>, const Dev<T> &, cudaStream_t);
PSE_INST(float)
PSE_INST(double)
#undef PSE_INST

}  // namespace pse
