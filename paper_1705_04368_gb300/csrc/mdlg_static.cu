// mdlg_static.cu -- mdlg_forces_static: forces and observables of one
// configuration computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need a
// force evaluation: code running inside a CUDA graph that is being captured
// (a cudaMalloc there breaks the capture), memory-pool-managed frameworks that
// own every allocation, or real-time loops that must not block in the
// allocator.  This entry point serves them: everything the computation needs
// beyond the caller's inputs and outputs lives in one statically sized device
// array of this file.  The array exists on every GPU that loads the library
// and is held until the process exits.  All calls on a device share it and it
// keeps the last call's contents, so calls whose work overlaps on the GPU
// (different streams, or host threads racing) corrupt each other's results:
// serialize them.
//
// The computation is the one the context path uses at statistics time: the
// configuration is packed into integer cell origins plus binary32 offsets,
// counting-sorted into neighbour cells, and the step kernel runs in its
// statistics mode with a zero time step (forces and reductions only; the
// cell-stencil force path, since no Verlet list is kept).
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mdlg.h"
#include "mdlg_kernels.h"

using namespace mdlg;

namespace {

constexpr int64_t kMaxN = MDLG_STATIC_MAX_N;
constexpr int64_t kMaxCells = MDLG_STATIC_MAX_CELLS;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the sub-arrays inside the scratch array.
struct Layout {
    size_t cell[2], cl[2], vel[2], pid[2], key, slot, entry, count, cell_start, block_sums,
        ctl, vsync, fsync, total;
};

constexpr Layout make_layout() {
    Layout L{};
    size_t o = 0;
    for (int b = 0; b < 2; ++b) {
        L.cell[b] = o; o += align256(sizeof(uint32_t) * kMaxN);
        L.cl[b] = o;   o += align256(sizeof(float2) * kMaxN);
        L.vel[b] = o;  o += align256(sizeof(float2) * kMaxN);
        L.pid[b] = o;  o += align256(sizeof(int32_t) * kMaxN);
    }
    L.key = o;        o += align256(sizeof(uint32_t) * kMaxN);
    L.slot = o;       o += align256(sizeof(int32_t) * kMaxN);
    L.entry = o;      o += align256(sizeof(unsigned long long) * kMaxN);
    L.count = o;      o += align256(sizeof(int32_t) * kMaxCells);
    L.cell_start = o; o += align256(sizeof(int32_t) * (kMaxCells + 1));
    L.block_sums = o; o += align256(sizeof(int32_t) * 64);
    L.ctl = o;        o += align256(sizeof(Control));
    L.vsync = o;      o += align256(sizeof(float2) * kMaxN);
    L.fsync = o;      o += align256(sizeof(float2) * kMaxN);
    L.total = o;
    return L;
}

constexpr Layout kLayout = make_layout();

// The scratch itself (about 6 MB).  Host code must not use this name as a
// device address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kLayout.total];

std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
int scratch_base(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MDLG_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MDLG_ECUDA;
        }
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_base[dev];
    return MDLG_OK;
}

bool pow2(double g) {
    if (!(g > 0.0) || !std::isfinite(g)) return false;
    int e = 0;
    return std::frexp(g, &e) == 0.5;
}

int64_t ratio_of(double value, double unit) {
    if (!(unit > 0.0) || !(value > 0.0)) return -1;
    const double r = value / unit, k = std::nearbyint(r);
    if (k < 1.0 || k > 2147483647.0 || std::fabs(r - k) > 1e-9 * k) return -1;
    return (int64_t)k;
}

}  // namespace

extern "C" int mdlg_forces_static(const mdlg_params *p, const double *x, const double *v,
                                  double *f, double *obs, int32_t *status, void *stream) {
    if (!p || !x || !v || !f || !obs) return MDLG_EINVAL;
    if (p->dim != 2 || p->n < 1 ||
        (p->potential != MDLG_POT_LJ_TS && p->potential != MDLG_POT_LJ_SF))
        return MDLG_EINVAL;
    if (!(p->rcut > 0.0) || !(p->sigma > 0.0) || !std::isfinite(p->eps) || !(p->mass > 0.0) ||
        !(p->skin >= 0.0) || !pow2(p->grid))
        return MDLG_EINVAL;
    if (p->n > kMaxN) return MDLG_EOVERFLOW;

    // geometry: the same rule as a context's (cells of k base cells, k g >= rc + skin)
    Geom geo{};
    geo.g = (float)p->grid;
    geo.inv_g = (float)(1.0 / p->grid);
    geo.k = (int32_t)std::ceil((p->rcut + p->skin) / p->grid - 1e-12);
    if (geo.k < 1) geo.k = 1;
    geo.ratio = 1;
    geo.vmax = 1;
    for (int a = 0; a < 2; ++a) {
        const int64_t lg = ratio_of(p->box[a], p->grid);
        if (lg < 1 || lg > 65535 || !(p->rcut < 0.5 * p->box[a])) return MDLG_EINVAL;
        geo.lg[a] = (int32_t)lg;
        geo.nc[a] = geo.lg[a] / geo.k;
        geo.lat[a] = 1;
        if (geo.nc[a] < 3) return MDLG_EINVAL;
    }
    const int64_t ncells = (int64_t)geo.nc[0] * geo.nc[1];
    if (ncells > kMaxCells) return MDLG_EOVERFLOW;

    unsigned char *base = nullptr;
    int rc = scratch_base(&base);
    if (rc != MDLG_OK) return rc;
    auto at = [&](size_t off) { return static_cast<void *>(base + off); };
    const Layout &L = kLayout;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Control *ctl = static_cast<Control *>(at(L.ctl));
    const int64_t n = p->n;

    // the control block (status word, displacement bound, launch counter) must
    // start at zero; every other scratch value is written before it is read
    if (cudaMemsetAsync(ctl, 0, sizeof(Control), s) != cudaSuccess) return MDLG_ECUDA;
    uint32_t *cell[2];
    float2 *cl[2], *vel[2];
    int32_t *pid[2];
    for (int b = 0; b < 2; ++b) {
        cell[b] = static_cast<uint32_t *>(at(L.cell[b]));
        cl[b] = static_cast<float2 *>(at(L.cl[b]));
        vel[b] = static_cast<float2 *>(at(L.vel[b]));
        pid[b] = static_cast<int32_t *>(at(L.pid[b]));
    }
    if (launch_pack(geo, n, x, v, cell[1], cl[1], vel[1], pid[1], ctl, s) != cudaSuccess)
        return MDLG_ECUDA;

    SortArgs so{};
    so.geo = geo;
    so.n = n;
    so.nlags = 0;
    so.ncells = ncells;
    so.cell_in = cell[1];
    so.cl_in = cl[1];
    so.v_in = vel[1];
    so.pid_in = pid[1];
    so.cell_out = cell[0];
    so.cl_out = cl[0];
    so.v_out = vel[0];
    so.pid_out = pid[0];
    so.cell_start = static_cast<int32_t *>(at(L.cell_start));
    so.key = static_cast<uint32_t *>(at(L.key));
    so.slot = static_cast<int32_t *>(at(L.slot));
    so.count = static_cast<int32_t *>(at(L.count));
    so.entry = static_cast<unsigned long long *>(at(L.entry));
    so.block_sums = static_cast<int32_t *>(at(L.block_sums));
    so.ctl = ctl;
    so.nbr = nullptr;   // no Verlet list: forces through the cell stencil
    if (launch_sort(so, s) != cudaSuccess) return MDLG_ECUDA;

    StepArgs a{};
    a.geo = geo;
    a.n = n;
    a.cell = cell[0];
    a.cell_start = so.cell_start;
    a.cl_in = cl[0];
    a.v_in = vel[0];
    a.v_sync = static_cast<float2 *>(at(L.vsync));
    a.f_sync = static_cast<float2 *>(at(L.fsync));
    const double rcut = p->rcut, sg = p->sigma, ep = p->eps;
    a.rc2 = (float)(rcut * rcut);
    a.sig2 = (float)(sg * sg);
    a.eps24 = (float)(24.0 * ep);
    a.eps4 = (float)(4.0 * ep);
    const double sr6 = std::pow(sg / rcut, 6.0);
    a.vshift = (float)(4.0 * ep * (sr6 * sr6 - sr6));
    a.dt = 0.f;          // zero time step: v_sync = v, forces and reductions only
    a.dt_m = 0.f;
    a.half_dt_m = 0.f;
    a.mass = (float)p->mass;
    a.cell_w = (float)(geo.k * p->grid);
    a.rc = (float)rcut;
    a.potential = p->potential == MDLG_POT_LJ_SF ? 2 : 1;
    a.fc = (float)(24.0 * ep * (2.0 * sr6 * sr6 - sr6) / rcut);
    a.stats = 1;
    a.ctl = ctl;
    a.nbr = nullptr;
    if (launch_step(a, kModeSync, s) != cudaSuccess) return MDLG_ECUDA;
    if (launch_unpack(geo, n, cell[0], cl[0], a.v_sync, a.f_sync, pid[0], nullptr, nullptr, f, s) !=
        cudaSuccess)
        return MDLG_ECUDA;
    // obs[0..4] = kinetic, potential, virial, momentum x, y (FP64 from the exact sums)
    if (cudaMemcpyAsync(obs, ctl->stats, 5 * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return MDLG_ECUDA;
    if (status && cudaMemcpyAsync(status, &ctl->status, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  s) != cudaSuccess)
        return MDLG_ECUDA;
    return MDLG_OK;
}
