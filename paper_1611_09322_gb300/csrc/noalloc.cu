// Near-field product M_r v without any device allocation.
//
// Some callers cannot call cudaMalloc: code running where the allocator is
// off limits (inside an application that owns all device memory through its
// own pool, a plugin that may not grow the process footprint, or a caller
// that needs a fixed, known-in-advance memory budget).  For them this file
// keeps every scratch buffer of the matvec in one file-scope static device
// array of fixed size.  With CUDA's lazy module loading the array is
// reserved on a device when this module is first used there (the first
// call's cudaGetSymbolAddress), and it stays reserved until the process
// exits; a caller with a fixed memory budget makes that first call during
// its own set-up.
#include <string.h>

#include "pse_internal.cuh"

namespace pse {
namespace {

constexpr int64_t kNoAllocMaxN = 16384;              // particles
constexpr int64_t kNoAllocMaxCells = 32768;          // cell slots (ncell <= 32)
constexpr int64_t kNoAllocMaxPairs = kNoAllocMaxN * 160;  // directed neighbour entries
constexpr int kNoAllocEdges = 4096;                        // pairs decided again in float64 at r_cut

struct NoAllocScratch {
    V4<float> pos_sorted[kNoAllocMaxN];
    V4<float> loc_sorted[kNoAllocMaxN];
    Rec<float> rec[kNoAllocMaxN];
    V4<float> table[PSE_TABLE_N];
    int cell_of[kNoAllocMaxN];
    int slot[kNoAllocMaxN];
    int perm[kNoAllocMaxN];
    int nbr_count[kNoAllocMaxN];
    int cell_count[kNoAllocMaxCells];
    int cell_start[kNoAllocMaxCells + 1];
    int scan_sums[PSE_SCAN_ITEMS];
    int nbr[kNoAllocMaxPairs];
    int4 edge[kNoAllocEdges];
    int edge_n;  // zero at load; the float64 decision kernel clears it after each use
    SampleArgs<float> args;
    LzState lz;
};

}  // namespace
}  // namespace pse

// The scratch itself (about 12 MB).  In host code this name is only a
// stand-in for the device symbol; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(pse::NoAllocScratch)];

namespace {

constexpr int kMaxDevices = 64;
pse::NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};
// table cache per device: the parameters the device table was last built for
double g_tab_key[kMaxDevices][3] = {};
bool g_tab_valid[kMaxDevices] = {};
pse::V4<float> g_host_table[PSE_TABLE_N];

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
pse_status scratch_for_current_device(pse::NoAllocScratch **out, int *dev) {
    if (cudaGetDevice(dev) != cudaSuccess) { cudaGetLastError(); return PSE_ECUDA; }
    if (*dev < 0 || *dev >= kMaxDevices) return PSE_ENOTSUPPORTED;
    if (!g_scratch_ptr[*dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PSE_ECUDA;
        }
        g_scratch_ptr[*dev] = (pse::NoAllocScratch *)p;
    }
    *out = g_scratch_ptr[*dev];
    return PSE_OK;
}

}  // namespace

using namespace pse;

extern "C" pse_status pse_real_matvec_noalloc(double L, double a, double xi, double tol, int64_t N,
                                              const float *d_pos, const float *d_v, float *d_out, void *stream) {
    if (!d_pos || !d_v || !d_out || N < 1) return PSE_EINVAL;
    if (N > kNoAllocMaxN) return PSE_EINVAL;  // beyond the static scratch
    pse_params prm;
    memset(&prm, 0, sizeof(prm));
    prm.tol = tol;
    prm.xi = xi;
    prm.precision = PSE_FP32;
    pse_plan_info plan;
    pse_status st = pse_plan(L, a, &prm, &plan);
    if (st != PSE_OK) return st;
    const int64_t nc3 = cell_slots(plan.ncell);
    if (nc3 > kNoAllocMaxCells) return PSE_EINVAL;  // box too large for the static cell arrays

    NoAllocScratch *sc = nullptr;
    int dev = 0;
    if ((st = scratch_for_current_device(&sc, &dev)) != PSE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // F, G table: rebuilt only when (xi, a, r_cut) change on this device
    const double key[3] = {plan.xi, plan.a, plan.r_cut};
    if (!g_tab_valid[dev] || memcmp(key, g_tab_key[dev], sizeof(key)) != 0) {
        static double F[PSE_TABLE_N], G[PSE_TABLE_N];
        build_fg_table(plan.r_cut, plan.xi, plan.a, PSE_TABLE_N, F, G);
        const double sc6 = 1.0 / (6 * M_PI * plan.a);
        for (int i = 0; i < PSE_TABLE_N; ++i) {
            const double f0 = F[i] * sc6, g0 = (G[i] - F[i]) * sc6;
            const double f1 = (i + 1 < PSE_TABLE_N) ? F[i + 1] * sc6 : f0;
            const double g1 = (i + 1 < PSE_TABLE_N) ? (G[i + 1] - F[i + 1]) * sc6 : g0;
            g_host_table[i].x = (float)f0;
            g_host_table[i].y = (float)g0;
            g_host_table[i].z = (float)(f1 - f0);
            g_host_table[i].w = (float)(g1 - g0);
        }
        // pageable source: the call returns once the data is staged
        if (cudaMemcpyAsync(sc->table, g_host_table, sizeof(g_host_table), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return PSE_ECUDA;
        }
        memcpy(g_tab_key[dev], key, sizeof(key));
        g_tab_valid[dev] = true;
    }

    Geom<float> g{};
    const double cs = plan.L / plan.ncell;
    g.L = (float)plan.L;
    g.cs = (float)cs;
    g.cs_lo = (float)(cs - (double)(float)cs);
    g.inv_cs = (float)(plan.ncell / plan.L);
    g.rc2 = (float)(plan.r_cut * plan.r_cut);
    g.tab_inv_dr = (float)((PSE_TABLE_N - 1) / plan.r_cut);
    g.self_m = (float)plan.self_mobility;
    g.a = (float)plan.a;
    g.xi = (float)plan.xi;
    g.nc = plan.ncell;
    g.nb = bricks_per_side(plan.ncell);
    g.rc2_d = plan.r_cut * plan.r_cut;
    g.L_d = plan.L;
    g.invL_d = 1.0 / plan.L;
    g.rc2_lo = (float)(g.rc2_d * (1.0 - 4e-6));
    g.rc2_hi = (float)(g.rc2_d * (1.0 + 4e-6));

    Dev<float> d{};
    d.pos_sorted = sc->pos_sorted;
    d.loc_sorted = sc->loc_sorted;
    d.cell_of = sc->cell_of;
    d.slot = sc->slot;
    d.perm = sc->perm;
    d.cell_count = sc->cell_count;
    d.cell_start = sc->cell_start;
    d.nbr_count = sc->nbr_count;
    d.nbr = sc->nbr;
    d.nbr_cap = kNoAllocMaxPairs;
    d.edge = sc->edge;
    d.edge_n = &sc->edge_n;
    d.edge_cap = kNoAllocEdges;
    d.scan_sums = sc->scan_sums;
    d.rec = sc->rec;
    d.table = sc->table;
    d.lz = &sc->lz;
    d.args = &sc->args;

    SampleArgs<float> args{};
    args.pos = d_pos;
    args.out = d_out;
    args.vin = d_v;
    if (cudaMemcpyAsync(&sc->args, &args, sizeof(args), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(&sc->lz.overflow, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ECUDA;
    }
    launch_bin<float>(N, d.args, g, d, s);  // clears the cell counts first
    launch_scatter<float>(N, d.args, g, d, s);
    launch_place<float>(N, d.args, g, d, s);
    launch_nbr<float>(N, g, d, s);
    launch_matvec_caller<float>(N, d.args, g, d, s);
    // a launch that failed to start (configuration, resources) is reported
    // here, not by the synchronisation below
    if (cudaGetLastError() != cudaSuccess) return PSE_ECUDA;
    int overflow = 0;
    if (cudaMemcpyAsync(&overflow, &sc->lz.overflow, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PSE_ECUDA;
    }
    if (overflow) return PSE_ENOMEM;  // more neighbour pairs than the static list holds
    return PSE_OK;
}
