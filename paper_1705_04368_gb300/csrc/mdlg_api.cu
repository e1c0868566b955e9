// mdlg_api.cu -- the C ABI of include/mdlg.h: context lifecycle, step
// scheduling and host <-> device marshalling.  All arithmetic of the method
// runs in the kernels of mdlg_md.cu and mdlg_bin.cu.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/mdlg.h"
#include "mdlg_kernels.h"

using namespace mdlg;

// Adaptive re-sort schedule: the host decides whether step t re-sorts from the
// device values of step t - kPaceLag, so that many steps stay queued.
constexpr int64_t kPaceLag = 3;
static_assert(kPaceLag < kPaceRing, "the slot waited for must not be overwritten");

struct mdlg_ctx {
    mdlg_params p{};
    Geom geo{};
    cudaStream_t stream = nullptr;
    mdlg_allocator alloc{};
    bool use_cuda_malloc = true;
    std::vector<void *> owned;
    int64_t ncells = 0;            // all cells (a batch: every system's cells + its ghost cell)
    int64_t slots = 0;             // particle array length (a batch: padded per system)
    int32_t nsys = 0;              // 0: one system (geo); >0: a batch of nsys systems
    std::vector<SysInfo> sys_host;
    SysInfo *sys_dev = nullptr;
    uint16_t *chunk_sys = nullptr;
    long long *bstats = nullptr;   // nsys x 5 fixed-point sums (batch statistics)
    int32_t ratio_shift = -1;
    int32_t q1 = 0;
    // double-buffered state: position/velocity swap every step, the rest at sorts
    uint32_t *cell[2]{};
    float2 *cl[2]{};
    float2 *vel[2]{};
    int32_t *pid[2]{};
    uint32_t *lprev[2][kMaxLags]{};
    float2 *mprev[2][kMaxLags]{};  // mean-square displacement origins (params.msd)
    double *msd_acc = nullptr;     // nlags x 2
    float2 *vprev[2][kMaxLags]{};  // velocity-correlation origins (params.vacf)
    double *vacf_acc = nullptr;    // nlags x 2
    int pos_cur = 0, meta_cur = 0;
    int32_t *cell_start = nullptr;
    // scratch
    uint32_t *key = nullptr;
    int32_t *slot = nullptr, *count = nullptr, *block_sums = nullptr;
    unsigned long long *entry = nullptr;
    uint8_t *col = nullptr;        // base column inside the new cell (lists on)
    Control *ctl = nullptr;
    unsigned long long *counts = nullptr;   // nlags x q1
    uint32_t *site_n = nullptr, *site_counts = nullptr;
    // collision operator (MDLG_SITES_XI): the field before the latest one and Xi
    uint32_t *site_counts_alt = nullptr;
    int32_t *xi = nullptr, *dmass = nullptr, *dmom = nullptr;
    // moving lattice: per-step shift in units of g 2^-24 per axis
    int64_t shift_m[2]{};
    bool moving = false;
    float2 *vsync = nullptr, *fsync = nullptr;
    double *xbuf = nullptr, *vbuf = nullptr, *fbuf = nullptr;
    uint32_t *nbr = nullptr;      // Verlet list (cap x n)
    int32_t *ncount = nullptr;
    int32_t cap = 0;
    float list_radius = 0.f;
    // host-side schedule
    int64_t step = 0, last_sort = 0, stats_step = -1;
    int64_t intervals[kMaxLags]{};
    int32_t sort_every = 1;
    // adaptive re-sort schedule (params.sort_every = 0, no graphs): every step
    // launch writes its displacement bound and largest speed into a host-mapped
    // ring; before queuing step t the host waits for the slot of step
    // t - kPaceLag and re-sorts if the bound of step t's input, predicted from
    // it, would reach half the skin (pace_decide).  sort_every is then the
    // length of the last interval.
    bool adaptive = false;
    double vmax0 = 0.0;            // fastest uploaded speed
    double skin_eff = 0.0;         // MD cell width minus rc
    PaceSlot *pace = nullptr;      // host-mapped ring (kPaceRing slots), host view
    PaceSlot *pace_dev = nullptr;  // the same ring, device view
    float rc = 0.f, round_margin = 0.f;
    // CUDA graph of two schedule periods (use_graphs)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_start = -1, graph_len = 0;
    bool graph_failed = false;
    int64_t graph_launches[MDLG_PROF_KINDS]{};
    // profiling: event pairs around launch groups
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;
    int64_t launches[MDLG_PROF_KINDS]{};
};

namespace {

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return MDLG_OK;
    fprintf(stderr, "mdlg: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
    return MDLG_ECUDA;
}

#define MDLG_TRY(expr)                 \
    do {                               \
        int rc__ = (expr);             \
        if (rc__ != MDLG_OK) return rc__; \
    } while (0)

#define MDLG_TRY_OR(expr, handler)            \
    do {                                      \
        int rc__ = (expr);                    \
        if (rc__ != MDLG_OK) return handler(rc__); \
    } while (0)

void *dev_alloc(mdlg_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (c->use_cuda_malloc) {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    } else {
        p = c->alloc.alloc(bytes, c->alloc.user);
    }
    if (p) c->owned.push_back(p);
    return p;
}

template <typename T>
int alloc_n(mdlg_ctx *c, T **out, size_t count) {
    *out = static_cast<T *>(dev_alloc(c, sizeof(T) * (count ? count : 1)));
    return *out ? MDLG_OK : MDLG_ENOMEM;
}

void free_all(mdlg_ctx *c) {
    for (void *p : c->owned) {
        if (c->use_cuda_malloc) cudaFree(p);
        else c->alloc.free(p, c->alloc.user);
    }
    c->owned.clear();
    if (c->pace) cudaFreeHost(c->pace);
    c->pace = nullptr;
    c->pace_dev = nullptr;
}

// Launch-group bracketing for mdlg_profile.
struct ProfScope {
    mdlg_ctx *c;
    int kind;
    bool on;
    ProfScope(mdlg_ctx *ctx, int k, int nlaunch) : c(ctx), kind(k), on(ctx->prof) {
        c->launches[k] += nlaunch;
        if (on) record();
    }
    ~ProfScope() {
        if (on) record();
    }
    void record() {
        if (c->ev_used == c->ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
            c->ev_pool.push_back(e);
        }
        cudaEventRecord(c->ev_pool[c->ev_used++], c->stream);
        c->ev_kind.push_back(kind);
    }
};

bool is_pow2(double g) {
    if (!(g > 0.0) || !std::isfinite(g)) return false;
    int e = 0;
    return std::frexp(g, &e) == 0.5;
}

// value / unit as an exact positive integer, or -1
int64_t exact_ratio(double value, double unit) {
    if (!(unit > 0.0) || !(value > 0.0)) return -1;
    double r = value / unit;
    double k = std::nearbyint(r);
    if (k < 1.0 || k > 2147483647.0 || std::fabs(r - k) > 1e-9 * k) return -1;
    return (int64_t)k;
}

int log2_exact(int32_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int s = 0;
    while ((1 << s) < v) ++s;
    return s;
}

int validate(const mdlg_params *p) {
    if (!p) return MDLG_EINVAL;
    if (p->dim != 2 || p->n < 1 || p->n > 2000000000LL) return MDLG_EINVAL;
    if (p->potential != MDLG_POT_LJ_TS && p->potential != MDLG_POT_LJ_SF &&
        p->potential != MDLG_POT_NONE)
        return MDLG_EINVAL;
    const bool lj = p->potential != MDLG_POT_NONE;
    if (!(p->dt > 0.0) || !(p->mass > 0.0) || !is_pow2(p->grid)) return MDLG_EINVAL;
    if (lj &&
        (!(p->rcut > 0.0) || !(p->sigma > 0.0) || !std::isfinite(p->eps)))
        return MDLG_EINVAL;
    if (!(p->skin >= 0.0)) return MDLG_EINVAL;
    if (p->vmax < 1 || p->vmax > MDLG_MAX_VMAX) return MDLG_EINVAL;
    if (p->nlags < 1 || p->nlags > MDLG_MAX_LAGS) return MDLG_EINVAL;
    for (int l = 0; l < p->nlags; ++l)
        if (p->lag_steps[l] < 1) return MDLG_EINVAL;
    if (p->site_mode & ~(MDLG_SITES_FIELD | MDLG_SITES_ACCUM | MDLG_SITES_XI)) return MDLG_EINVAL;
    if ((p->site_mode & MDLG_SITES_FIELD) && (p->site_mode & MDLG_SITES_ACCUM)) return MDLG_EINVAL;
    if ((p->site_mode & MDLG_SITES_XI) && !(p->site_mode & MDLG_SITES_FIELD)) return MDLG_EINVAL;
    if (p->msd != 0 && p->msd != 1) return MDLG_EINVAL;
    if (p->vacf != 0 && p->vacf != 1) return MDLG_EINVAL;
    for (int a = 0; a < 2; ++a)   // per-step shift below 2^16 base cells
        if (!std::isfinite(p->lattice_u[a]) || std::fabs(p->lattice_u[a] * p->dt) >= 65536.0 * p->grid)
            return MDLG_EINVAL;
    if (p->sort_every < 0 || p->stats_every < 0) return MDLG_EINVAL;
    int64_t ratio = exact_ratio(p->dx, p->grid);
    if (ratio < 1) return MDLG_EINVAL;
    for (int a = 0; a < 2; ++a) {
        int64_t lat = exact_ratio(p->box[a], p->dx);
        if (lat < 1 || lat > 65535) return MDLG_EINVAL;
        int64_t lg = exact_ratio(p->box[a], p->grid);
        if (lg < 1 || lg > 65535) return MDLG_EINVAL;
        if (lj && !(p->rcut < 0.5 * p->box[a])) return MDLG_EINVAL;
    }
    // Verlet-list entries carry the particle index in 28 bits
    if (lj && p->n >= (1LL << 28)) return MDLG_EINVAL;
    return MDLG_OK;
}

Batch batch_of(mdlg_ctx *c) {
    Batch b{};
    if (c->nsys > 0) {
        b.sys = c->sys_dev;
        b.chunk_sys = c->chunk_sys;
        b.stats = c->bstats;
        b.nsys = c->nsys;
    }
    return b;
}

// Magnitude of the Lennard-Jones pair force at the cutoff, F(rc) =
// 24 eps (2 (s/rc)^12 - (s/rc)^6) / rc, and its derivative in sigma (the
// shifted-force potential subtracts F(rc) so the force vanishes at rc).
double lj_fc(const mdlg_params &p) {
    const double sr6 = std::pow(p.sigma / p.rcut, 6.0);
    return 24.0 * p.eps * (2.0 * sr6 * sr6 - sr6) / p.rcut;
}

double lj_dfc_dsigma(const mdlg_params &p) {
    const double sr6 = std::pow(p.sigma / p.rcut, 6.0);
    return 24.0 * p.eps * (24.0 * sr6 * sr6 - 6.0 * sr6) / (p.sigma * p.rcut);
}

StepArgs step_args(mdlg_ctx *c) {
    StepArgs a{};
    a.geo = c->geo;
    a.n = c->slots;
    a.batch = batch_of(c);
    a.cell = c->cell[c->meta_cur];
    a.cell_start = c->cell_start;
    a.cl_in = c->cl[c->pos_cur];
    a.v_in = c->vel[c->pos_cur];
    a.cl_out = c->cl[c->pos_cur ^ 1];
    a.v_out = c->vel[c->pos_cur ^ 1];
    a.v_sync = c->vsync;
    a.f_sync = c->fsync;
    const double rc = c->p.rcut, s = c->p.sigma, e = c->p.eps;
    a.rc2 = (float)(rc * rc);
    a.sig2 = (float)(s * s);
    a.eps24 = (float)(24.0 * e);
    a.eps4 = (float)(4.0 * e);
    const double sr6 = std::pow(s / rc, 6.0);
    a.vshift = (float)(4.0 * e * (sr6 * sr6 - sr6));
    a.dt = (float)c->p.dt;
    a.dt_m = (float)(c->p.dt / c->p.mass);
    a.half_dt_m = (float)(0.5 * c->p.dt / c->p.mass);
    a.mass = (float)c->p.mass;
    a.cell_w = (float)(c->geo.k * c->p.grid);
    a.rc = c->p.potential ? (float)rc : 0.f;
    a.round_margin = c->round_margin;
    a.potential = c->p.potential == MDLG_POT_LJ_TS ? 1 : (c->p.potential == MDLG_POT_LJ_SF ? 2 : 0);
    a.fc = (float)lj_fc(c->p);
    a.ctl = c->ctl;
    a.nbr = c->nbr;
    a.ncount = c->ncount;
    a.cap = c->cap;
    a.list_skin = c->list_radius - (float)rc;
    a.pace = c->pace_dev;
    a.step = c->step;
    return a;
}

StateBinArgs bin_args(mdlg_ctx *c, uint32_t mask) {
    StateBinArgs b{};
    b.geo = c->geo;
    b.n = c->slots;
    b.batch = batch_of(c);
    b.ratio_shift = c->ratio_shift;
    b.nlags = c->p.nlags;
    b.mask = mask;
    b.cell = c->cell[c->meta_cur];
    b.cl = c->cl[c->pos_cur];
    for (int l = 0; l < c->p.nlags; ++l) {
        b.lprev[l] = c->lprev[c->meta_cur][l];
        b.counts[l] = c->counts + (size_t)l * c->q1;
    }
    b.site_n = c->site_n;
    b.site_counts = c->site_counts;
    if (c->moving) {
        // S(step) = step * m modulo the box (lg 2^24 units per axis), split into
        // whole base cells K and the fraction b = frac 2^-24
        b.shift.on = 1;
        for (int a = 0; a < 2; ++a) {
            const __int128 M = (__int128)c->geo.lg[a] << 24;
            __int128 r = ((__int128)c->step * c->shift_m[a]) % M;
            if (r < 0) r += M;
            const int64_t rr = (int64_t)r;
            b.shift.K[a] = (int32_t)(rr >> 24);
            b.shift.omb[a] = (float)(16777216 - (rr & 0xffffff)) * (1.0f / 16777216.0f);
        }
    }
    if (c->p.msd) {
        for (int l = 0; l < c->p.nlags; ++l) b.mprev[l] = c->mprev[c->meta_cur][l];
        b.msd_acc = c->msd_acc;
    }
    b.vel = c->vel[c->pos_cur];
    if (c->p.vacf) {
        for (int l = 0; l < c->p.nlags; ++l) b.vprev[l] = c->vprev[c->meta_cur][l];
        b.vacf_acc = c->vacf_acc;
    }
    return b;
}

// MD steps between re-sorts for a speed bound v: half the skin covered.
int32_t interval_for(const mdlg_ctx *c, double v) {
    const double k = std::floor(0.5 * c->skin_eff / (std::fmax(v, 1e-12) * c->p.dt));
    return (int32_t)std::fmax(1.0, std::fmin(k, 1000.0));
}

// Adaptive schedule: whether step t re-sorts.  The slot of step t - kPaceLag
// holds the displacement bound of step t - kPaceLag + 1's input positions and
// that step's largest speed v.  The bound of step t's input is predicted from
// it: the slot's bound plus the remaining kPaceLag - 1 steps at 1.1 v (plus the
// per-step rounding margin), or, when the last re-sort came after that slot's
// step (the bound restarted from zero there), the steps since the re-sort at
// 1.1 v.  Step t re-sorts if twice the prediction exceeds the skin.  The host
// waits only for step t - kPaceLag, so kPaceLag steps stay queued, and the
// decision depends only on device values of fixed steps: a run and its
// repetition (or a resumed checkpoint) re-sort at the same steps.  Before the
// first kPaceLag steps of a context, or when no step of this context wrote the
// slot, the last interval's length decides.
int pace_decide(mdlg_ctx *c, bool *sort) {
    const int64_t t = c->step, since = t - c->last_sort;
    *sort = since >= c->sort_every;
    const int64_t s = t - kPaceLag;
    if (s < 0) return MDLG_OK;
    volatile PaceSlot *ps = c->pace + (s & (kPaceRing - 1));
    // Busy-wait: only kPaceLag steps (a few hundred microseconds) are queued, so
    // giving the core away (a yield can cost a scheduler quantum on a loaded
    // host) would leave the device idle.  Only after ~2^20 polls, a wait far
    // longer than a step, does the loop also yield.
    for (int64_t k = 1; ps->step != s; ++k) {
        if (k % 1024 == 0) {
            const cudaError_t q = cudaStreamQuery(c->stream);
            if (q != cudaSuccess && q != cudaErrorNotReady) return cuda_err(q);
            // the stream is idle and the slot was never written (no step launch
            // for step s in this context): keep the interval rule
            if (q == cudaSuccess && ps->step != s) return MDLG_OK;
            if (k >= (int64_t)1 << 20) std::this_thread::yield();
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const float D = ps->dbound;
    const uint32_t bits = ps->vmax2_bits;
    float v2;
    memcpy(&v2, &bits, sizeof(v2));
    const double per_step = 1.1 * std::sqrt((double)v2) * c->p.dt + c->round_margin;
    const double pred = since >= kPaceLag ? (double)D + (kPaceLag - 1) * per_step
                                          : (double)since * per_step;
    *sort = 2.0 * pred > c->skin_eff;
    return MDLG_OK;
}

int do_sort(mdlg_ctx *c, bool launch = true) {
    if (!launch) {   // bookkeeping of a sort that a replayed graph performs
        c->pos_cur ^= 1;
        c->meta_cur ^= 1;
        c->last_sort = c->step;
        return MDLG_OK;
    }
    if (c->adaptive && c->step > c->last_sort) c->sort_every = (int32_t)(c->step - c->last_sort);
    SortArgs s{};
    s.geo = c->geo;
    s.n = c->slots;
    s.batch = batch_of(c);
    s.nlags = c->p.nlags;
    s.ncells = c->ncells;
    const int pi = c->pos_cur, mi = c->meta_cur;
    s.cell_in = c->cell[mi];
    s.cl_in = c->cl[pi];
    s.v_in = c->vel[pi];
    s.pid_in = c->pid[mi];
    s.cell_out = c->cell[mi ^ 1];
    s.cl_out = c->cl[pi ^ 1];
    s.v_out = c->vel[pi ^ 1];
    s.pid_out = c->pid[mi ^ 1];
    for (int l = 0; l < c->p.nlags; ++l) {
        s.lprev_in[l] = c->lprev[mi][l];
        s.lprev_out[l] = c->lprev[mi ^ 1][l];
        if (c->p.msd) {
            s.mprev_in[l] = c->mprev[mi][l];
            s.mprev_out[l] = c->mprev[mi ^ 1][l];
        }
        if (c->p.vacf) {
            s.vprev_in[l] = c->vprev[mi][l];
            s.vprev_out[l] = c->vprev[mi ^ 1][l];
        }
    }
    s.cell_start = c->cell_start;
    s.key = c->key;
    s.slot = c->slot;
    s.count = c->count;
    s.entry = c->entry;
    s.col = c->col;
    s.block_sums = c->block_sums;
    s.ctl = c->ctl;
    s.nbr = c->nbr;
    s.ncount = c->ncount;
    s.cap = c->cap;
    s.rl2 = c->list_radius * c->list_radius;
    {
        ProfScope ps(c, MDLG_PROF_SORT, c->nbr ? 7 : 6);
        MDLG_TRY(cuda_err(launch_sort(s, c->stream)));
    }
    c->pos_cur ^= 1;
    c->meta_cur ^= 1;
    c->last_sort = c->step;
    return MDLG_OK;
}

// A batch's per-system statistics are accumulated with atomics: zero them
// before every statistics launch.
int zero_bstats(mdlg_ctx *c) {
    if (c->nsys == 0) return MDLG_OK;
    return cuda_err(cudaMemsetAsync(c->bstats, 0, sizeof(long long) * 5 * c->nsys, c->stream));
}

int sync_stats(mdlg_ctx *c, bool with_force) {
    MDLG_TRY(zero_bstats(c));
    StepArgs a = step_args(c);
    a.stats = 1;
    if (!with_force) a.f_sync = c->fsync;   // buffer always present; harmless
    ProfScope ps(c, MDLG_PROF_SYNC, 1);
    MDLG_TRY(cuda_err(launch_step(a, kModeSync, c->stream)));
    c->stats_step = c->step;
    return MDLG_OK;
}

int read_status(mdlg_ctx *c, int32_t *status, double *stats, double *vmax0 = nullptr) {
    Control h{};
    MDLG_TRY(cuda_err(cudaMemcpyAsync(&h, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost,
                                      c->stream)));
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    if (status) *status = h.status;
    if (stats) memcpy(stats, h.stats, sizeof(h.stats));
    if (vmax0) {
        double s2;
        memcpy(&s2, &h.vmax0_bits, sizeof(s2));
        *vmax0 = std::sqrt(s2);
    }
    return MDLG_OK;
}

}  // namespace

extern "C" {

const char *mdlg_strerror(int code) {
    switch (code) {
        case MDLG_OK: return "ok";
        case MDLG_EINVAL: return "invalid argument";
        case MDLG_ENOMEM: return "device allocation failed";
        case MDLG_ECUDA: return "CUDA runtime error";
        case MDLG_EOVERFLOW: return "counter or index range exceeded";
        case MDLG_ENONFINITE: return "non-finite or out-of-box particle state";
        case MDLG_ETIMEOUT: return "bounded device wait timed out";
        case MDLG_ENOTIMPL: return "not implemented";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// Geometry of one system (box per axis) under the shared parameters.
int system_geom(const mdlg_params &p, const double box[2], Geom &g) {
    g.g = (float)p.grid;
    g.inv_g = (float)(1.0 / p.grid);
    g.ratio = (int32_t)exact_ratio(p.dx, p.grid);
    const double reach = p.potential != MDLG_POT_NONE ? p.rcut + p.skin : 4.0;
    g.k = (int32_t)std::ceil(reach / p.grid - 1e-12);
    if (g.k < 1) g.k = 1;
    for (int a = 0; a < 2; ++a) {
        g.lg[a] = (int32_t)exact_ratio(box[a], p.grid);
        g.lat[a] = (int32_t)exact_ratio(box[a], p.dx);
        g.nc[a] = g.lg[a] / g.k;
        if (g.lg[a] % g.ratio) return MDLG_EINVAL;
    }
    g.vmax = p.vmax;
    if (p.potential != MDLG_POT_NONE && (g.nc[0] < 3 || g.nc[1] < 3)) return MDLG_EINVAL;
    if (g.nc[0] < 1) g.nc[0] = 1;
    if (g.nc[1] < 1) g.nc[1] = 1;
    return MDLG_OK;
}

// One system (nsys = 0: params->n, params->box) or a batch of nsys systems
// (ns[s] particles in box boxes[2s], boxes[2s+1]; x0/v0 concatenated).
int create_impl(const mdlg_params *params, int32_t nsys, const int64_t *ns, const double *boxes,
                const double *x0, const double *v0, const mdlg_allocator *allocator, void *stream,
                mdlg_ctx **out) {
    if (!out) return MDLG_EINVAL;
    *out = nullptr;
    if (!params || !x0 || !v0) return MDLG_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free)) return MDLG_EINVAL;
    int64_t ntot = params->n;
    if (nsys > 0) {
        if (!ns || !boxes || nsys > 65535) return MDLG_EINVAL;
        // per-site outputs, the moving lattice and the displacement sums: single systems only
        if (params->site_mode || params->msd || params->vacf || params->lattice_u[0] != 0.0 ||
            params->lattice_u[1] != 0.0)
            return MDLG_EINVAL;
        ntot = 0;
        int64_t slots = 0;
        for (int32_t k = 0; k < nsys; ++k) {
            mdlg_params q = *params;
            q.n = ns[k];
            q.box[0] = boxes[2 * k];
            q.box[1] = boxes[2 * k + 1];
            MDLG_TRY(validate(&q));
            ntot += ns[k];
            slots += (ns[k] + kChunk - 1) / kChunk * kChunk;
        }
        // Verlet-list entries carry the slot index (padding included) in 28 bits
        if (ntot >= (1LL << 28) || slots >= (1LL << 28)) return MDLG_EINVAL;
    } else if (nsys < 0) {
        return MDLG_EINVAL;
    } else {
        MDLG_TRY(validate(params));
    }

    mdlg_ctx *c = new (std::nothrow) mdlg_ctx();
    if (!c) return MDLG_ENOMEM;
    c->p = *params;
    c->p.n = ntot;
    c->nsys = nsys;
    c->stream = static_cast<cudaStream_t>(stream);
    if (allocator) {
        c->alloc = *allocator;
        c->use_cuda_malloc = false;
    }
    const mdlg_params &p = c->p;
    const int64_t n = ntot;
    auto early = [&](int code) {
        delete c;
        return code;
    };

    // geometry (a batch: per system, slots padded to whole chunks, cells numbered
    // system after system with one ghost cell each)
    Geom &g = c->geo;
    double rho_max = 0.0;
    if (nsys == 0) {
        MDLG_TRY_OR(system_geom(p, p.box, g), early);
        c->ncells = (int64_t)g.nc[0] * g.nc[1];
        c->slots = n;
        rho_max = (double)n / (p.box[0] * p.box[1]);
    } else {
        c->sys_host.resize(nsys);
        int64_t slot = 0, q = 0, cell = 0;
        for (int32_t k = 0; k < nsys; ++k) {
            SysInfo &si = c->sys_host[k];
            memset(&si, 0, sizeof(si));
            const double box[2] = {boxes[2 * k], boxes[2 * k + 1]};
            MDLG_TRY_OR(system_geom(p, box, si.geo), early);
            si.p0 = slot;
            si.q0 = q;
            si.n = ns[k];
            si.cell0 = cell;
            si.ncells = si.geo.nc[0] * si.geo.nc[1];
            slot += (ns[k] + kChunk - 1) / kChunk * kChunk;
            q += ns[k];
            cell += (int64_t)si.ncells + 1;
            rho_max = std::fmax(rho_max, (double)ns[k] / (box[0] * box[1]));
        }
        g = c->sys_host[0].geo;   // k, g, ratio, vmax shared by every system
        c->slots = slot;
        c->ncells = cell;
    }
    if (c->ncells > (int64_t)4096 * 4096) return early(MDLG_EINVAL);
    c->ratio_shift = log2_exact(g.ratio);
    c->q1 = (2 * p.vmax + 1) * (2 * p.vmax + 1) + 1;
    for (int a = 0; a < 2; ++a) c->shift_m[a] = std::llround(p.lattice_u[a] * p.dt / p.grid * 16777216.0);
    c->moving = c->shift_m[0] != 0 || c->shift_m[1] != 0;
    if (c->moving) c->graph_failed = true;   // the shift of each binning is a launch argument
    c->rc = (float)p.rcut;
    // rounding slack of one drift update: a few ulps of the largest offset
    c->round_margin = (float)(4.0 * std::ldexp(1.0, -23) * (2.0 * g.k * p.grid));

    int rc = MDLG_OK;
    auto fail = [&](int code) {
        free_all(c);
        delete c;
        return code;
    };
    const size_t N = (size_t)c->slots;
    const size_t NQ = (size_t)(n > c->slots ? n : c->slots);
    const int32_t nsb = nsys > 0 ? nsys : 1;
    for (int b = 0; b < 2; ++b) {
        if ((rc = alloc_n(c, &c->cell[b], N)) || (rc = alloc_n(c, &c->cl[b], N)) ||
            (rc = alloc_n(c, &c->vel[b], N)) || (rc = alloc_n(c, &c->pid[b], N)))
            return fail(rc);
        for (int l = 0; l < p.nlags; ++l) {
            if ((rc = alloc_n(c, &c->lprev[b][l], N))) return fail(rc);
            if (p.msd && (rc = alloc_n(c, &c->mprev[b][l], N))) return fail(rc);
            if (p.vacf && (rc = alloc_n(c, &c->vprev[b][l], N))) return fail(rc);
        }
    }
    if (p.msd && (rc = alloc_n(c, &c->msd_acc, (size_t)2 * p.nlags))) return fail(rc);
    if (p.vacf && (rc = alloc_n(c, &c->vacf_acc, (size_t)2 * p.nlags))) return fail(rc);
    const int64_t nb = sort_scratch_blocks(c->ncells);
    if ((rc = alloc_n(c, &c->cell_start, (size_t)c->ncells + 1)) ||
        (rc = alloc_n(c, &c->key, N)) || (rc = alloc_n(c, &c->slot, N)) ||
        (rc = alloc_n(c, &c->count, (size_t)c->ncells)) ||
        (rc = alloc_n(c, &c->block_sums, (size_t)nb)) || (rc = alloc_n(c, &c->entry, N)) ||
        (rc = alloc_n(c, &c->ctl, 1)) ||
        (rc = alloc_n(c, &c->counts, (size_t)nsb * p.nlags * c->q1)) ||
        (rc = alloc_n(c, &c->vsync, N)) || (rc = alloc_n(c, &c->fsync, N)) ||
        (rc = alloc_n(c, &c->xbuf, 2 * NQ)) || (rc = alloc_n(c, &c->vbuf, 2 * NQ)) ||
        (rc = alloc_n(c, &c->fbuf, 2 * NQ)))
        return fail(rc);
    if (nsys > 0) {
        if ((rc = alloc_n(c, &c->sys_dev, (size_t)nsys)) ||
            (rc = alloc_n(c, &c->chunk_sys, N / kChunk)) ||
            (rc = alloc_n(c, &c->bstats, (size_t)nsys * 5)))
            return fail(rc);
    }
    if (p.site_mode) {
        const size_t sites = (size_t)g.lat[0] * g.lat[1];
        if ((rc = alloc_n(c, &c->site_n, sites)) || (rc = alloc_n(c, &c->site_counts, sites * c->q1)))
            return fail(rc);
        if ((p.site_mode & MDLG_SITES_XI) &&
            ((rc = alloc_n(c, &c->site_counts_alt, sites * c->q1)) ||
             (rc = alloc_n(c, &c->xi, sites * (c->q1 - 1))) || (rc = alloc_n(c, &c->dmass, sites)) ||
             (rc = alloc_n(c, &c->dmom, 2 * sites))))
            return fail(rc);
    }
    if (p.potential != MDLG_POT_NONE) {
        // Verlet list of radius = the MD cell width (rc + the whole skin);
        // capacity three times the mean count at the highest density, plus 16,
        // a multiple of 4 (the step kernel's list batch: lists are padded to it)
        c->list_radius = (float)(g.k * p.grid);
        const double mean = rho_max * 3.14159265358979 * (double)c->list_radius * c->list_radius;
        c->cap = (int32_t)std::ceil((3.0 * mean + 16.0) / 4.0) * 4;
        if (c->cap > 512) c->cap = 512;   // list-build staging: 64 threads x (cap + 1) words of shared memory
        if ((rc = alloc_n(c, &c->nbr, (size_t)c->cap * N)) || (rc = alloc_n(c, &c->ncount, N)) ||
            (rc = alloc_n(c, &c->col, N)))
            return fail(rc);
    }

    cudaStream_t s = c->stream;
    auto chk = [&](cudaError_t e) { return cuda_err(e); };
    if ((rc = chk(cudaMemsetAsync(c->ctl, 0, sizeof(Control), s))) ||
        (rc = chk(cudaMemsetAsync(c->counts, 0, sizeof(unsigned long long) * nsb * p.nlags * c->q1, s))))
        return fail(rc);
    for (int b = 0; b < 2; ++b)
        for (int l = 0; l < p.nlags; ++l)
            if ((rc = chk(cudaMemsetAsync(c->lprev[b][l], 0, sizeof(uint32_t) * N, s))))
                return fail(rc);
    if (p.site_mode) {
        const size_t sites = (size_t)g.lat[0] * g.lat[1];
        if ((rc = chk(cudaMemsetAsync(c->site_n, 0, sizeof(uint32_t) * sites, s))) ||
            (rc = chk(cudaMemsetAsync(c->site_counts, 0, sizeof(uint32_t) * sites * c->q1, s))))
            return fail(rc);
        if (c->site_counts_alt &&
            ((rc = chk(cudaMemsetAsync(c->site_counts_alt, 0, sizeof(uint32_t) * sites * c->q1, s))) ||
             (rc = chk(cudaMemsetAsync(c->xi, 0, sizeof(int32_t) * sites * (c->q1 - 1), s))) ||
             (rc = chk(cudaMemsetAsync(c->dmass, 0, sizeof(int32_t) * sites, s))) ||
             (rc = chk(cudaMemsetAsync(c->dmom, 0, sizeof(int32_t) * 2 * sites, s)))))
            return fail(rc);
    }
    if (p.msd && (rc = chk(cudaMemsetAsync(c->msd_acc, 0, sizeof(double) * 2 * p.nlags, s))))
        return fail(rc);
    if (p.vacf && (rc = chk(cudaMemsetAsync(c->vacf_acc, 0, sizeof(double) * 2 * p.nlags, s))))
        return fail(rc);
    if (nsys > 0) {
        std::vector<uint16_t> cs(N / kChunk);
        for (int32_t k = 0; k < nsys; ++k) {
            const SysInfo &si = c->sys_host[k];
            const int64_t np = (si.n + kChunk - 1) / kChunk * kChunk;
            for (int64_t ch = si.p0 / kChunk; ch < (si.p0 + np) / kChunk; ++ch) cs[ch] = (uint16_t)k;
        }
        // pageable sources: the copies complete before the call returns
        if ((rc = chk(cudaMemcpyAsync(c->sys_dev, c->sys_host.data(), sizeof(SysInfo) * nsys,
                                      cudaMemcpyHostToDevice, s))) ||
            (rc = chk(cudaMemcpyAsync(c->chunk_sys, cs.data(), sizeof(uint16_t) * cs.size(),
                                      cudaMemcpyHostToDevice, s))))
            return fail(rc);
    }
    // upload (pageable host memory: the copy completes before the call returns)
    if ((rc = chk(cudaMemcpyAsync(c->xbuf, x0, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s))) ||
        (rc = chk(cudaMemcpyAsync(c->vbuf, v0, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s))))
        return fail(rc);
    // pack into buffer 1 (original order), sort into buffer 0
    c->pos_cur = 1;
    c->meta_cur = 1;
    if (nsys > 0) {
        const Batch bt = batch_of(c);
        if ((rc = chk(launch_pack_batch(bt, c->slots, c->xbuf, c->vbuf, c->cell[1], c->cl[1],
                                        c->vel[1], c->pid[1], c->ctl, s))))
            return fail(rc);
    } else if ((rc = chk(launch_pack(g, n, c->xbuf, c->vbuf, c->cell[1], c->cl[1], c->vel[1],
                                     c->pid[1], c->ctl, s)))) {
        return fail(rc);
    }
    if ((rc = do_sort(c))) return fail(rc);
    // v_{-1/2} = v_0 - F(x_0) dt / (2m), in place; FP64 observables of step 0
    if ((rc = zero_bstats(c))) return fail(rc);
    StepArgs a = step_args(c);
    a.v_out = c->vel[c->pos_cur];
    a.stats = 1;
    if ((rc = chk(launch_step(a, kModeInit, s)))) return fail(rc);
    c->stats_step = 0;
    // every lag starts from the lattice cells at t = 0
    StateBinArgs b = bin_args(c, (1u << p.nlags) - 1u);
    if ((rc = chk(launch_bin_seed(b, s)))) return fail(rc);
    if ((rc = chk(cudaStreamSynchronize(s)))) return fail(rc);
    int32_t status = 0;
    double vmax0 = 0.0;   // fastest uploaded speed (reduced by the upload kernel)
    if ((rc = read_status(c, &status, nullptr, &vmax0))) return fail(rc);
    if (status) return fail(status);
    // re-sort interval: half the skin covered at 1.15x the fastest initial speed
    // (nothing above depends on it).  If the bound tracked on the device grows
    // past it earlier, the step kernel uses the cell stencil for the remaining
    // steps, so a late sort costs time, not accuracy.
    c->vmax0 = vmax0;
    c->skin_eff = g.k * p.grid - (p.potential ? p.rcut : 0.0);
    if (p.sort_every > 0) {
        c->sort_every = p.sort_every;
    } else {
        c->sort_every = interval_for(c, 1.15 * vmax0);
        // with graphs the captured schedule needs a fixed interval
        if (!p.use_graphs) {
            void *ring = nullptr;
            if (cudaHostAlloc(&ring, kPaceRing * sizeof(PaceSlot), cudaHostAllocMapped) != cudaSuccess) {
                cudaGetLastError();
                return fail(MDLG_ENOMEM);
            }
            c->pace = static_cast<PaceSlot *>(ring);
            for (int k = 0; k < kPaceRing; ++k) c->pace[k] = PaceSlot{-1, 0.0f, 0u};
            void *dev = nullptr;
            if ((rc = chk(cudaHostGetDevicePointer(&dev, ring, 0)))) return fail(rc);
            c->pace_dev = static_cast<PaceSlot *>(dev);
            c->adaptive = true;
        }
    }
    *out = c;
    return MDLG_OK;
}

// FP64 observables [ke, pe, virial, px, py] of system k (k < 0: all systems).
int read_observables(mdlg_ctx *c, int32_t k, double *st, int32_t *status) {
    double one[8];
    MDLG_TRY(read_status(c, status, one));
    if (c->nsys == 0) {
        memcpy(st, one, 5 * sizeof(double));
        return MDLG_OK;
    }
    std::vector<long long> h((size_t)c->nsys * 5);
    MDLG_TRY(cuda_err(cudaMemcpyAsync(h.data(), c->bstats, sizeof(long long) * h.size(),
                                      cudaMemcpyDeviceToHost, c->stream)));
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    for (int q = 0; q < 5; ++q) {
        long long t = 0;
        for (int32_t s = (k < 0 ? 0 : k); s < (k < 0 ? c->nsys : k + 1); ++s) t += h[(size_t)s * 5 + q];
        st[q] = (double)t * (1.0 / 16777216.0);
    }
    return MDLG_OK;
}

}  // namespace

extern "C" {

int mdlg_create(const mdlg_params *params, const double *x0, const double *v0,
                const mdlg_allocator *allocator, void *stream, mdlg_ctx **out) {
    return create_impl(params, 0, nullptr, nullptr, x0, v0, allocator, stream, out);
}

int mdlg_create_batch(const mdlg_params *params, int32_t nsys, const int64_t *n,
                      const double *box, const double *x0, const double *v0,
                      const mdlg_allocator *allocator, void *stream, mdlg_ctx **out) {
    if (nsys < 1) return MDLG_EINVAL;
    return create_impl(params, nsys, n, box, x0, v0, allocator, stream, out);
}

}  // extern "C"

namespace {

// nsteps MD steps as the host schedules them: re-sorts every sort_every
// steps, statistics on multiples of stats_every, binning on multiples of each
// lag.  launch = false only advances the bookkeeping (a replayed graph runs the
// kernels).
int step_loop(mdlg_ctx *c, int64_t nsteps, bool launch) {
    const mdlg_params &p = c->p;
    for (int64_t it = 0; it < nsteps; ++it) {
        bool sort = c->step - c->last_sort >= c->sort_every;
        if (c->pace && launch) MDLG_TRY(pace_decide(c, &sort));
        if (sort) MDLG_TRY(do_sort(c, launch));
        const bool stats = p.stats_every > 0 && c->step % p.stats_every == 0;
        if (launch) {
            StepArgs a = step_args(c);
            a.stats = stats ? 1 : 0;
            if (a.stats) MDLG_TRY(zero_bstats(c));
            ProfScope ps(c, MDLG_PROF_STEP, 1);
            MDLG_TRY(cuda_err(launch_step(a, kModeStep, c->stream)));
        }
        if (stats) c->stats_step = c->step;
        c->pos_cur ^= 1;
        c->step += 1;
        uint32_t mask = 0;
        for (int l = 0; l < p.nlags; ++l)
            if (c->step % p.lag_steps[l] == 0) mask |= 1u << l;
        if (mask) {
            // the collision operator keeps the previous interval's field: the
            // older buffer becomes the one this interval writes
            const bool xi = (mask & 1u) && (p.site_mode & MDLG_SITES_XI);
            if (xi) std::swap(c->site_counts, c->site_counts_alt);
            if (launch) {
                if ((mask & 1u) && (p.site_mode & MDLG_SITES_FIELD)) {
                    const size_t sites = (size_t)c->geo.lat[0] * c->geo.lat[1];
                    MDLG_TRY(cuda_err(cudaMemsetAsync(c->site_n, 0, sizeof(uint32_t) * sites, c->stream)));
                    MDLG_TRY(cuda_err(cudaMemsetAsync(c->site_counts, 0,
                                                      sizeof(uint32_t) * sites * c->q1, c->stream)));
                }
                StateBinArgs b = bin_args(c, mask);
                if (!(mask & 1u)) { b.site_n = nullptr; b.site_counts = nullptr; }
                ProfScope ps(c, MDLG_PROF_BIN, xi ? 2 : 1);
                MDLG_TRY(cuda_err(launch_bin_state(b, c->stream)));
                if (xi) {
                    CollArgs ca{};
                    ca.lat[0] = c->geo.lat[0];
                    ca.lat[1] = c->geo.lat[1];
                    ca.vmax = p.vmax;
                    ca.prev = c->site_counts_alt;
                    ca.cur = c->site_counts;
                    ca.xi = c->xi;
                    ca.dmass = c->dmass;
                    ca.dmom = c->dmom;
                    MDLG_TRY(cuda_err(launch_collision(ca, c->stream)));
                }
            }
            for (int l = 0; l < p.nlags; ++l)
                if ((mask >> l) & 1u) c->intervals[l] += 1;
        }
    }
    return MDLG_OK;
}

int64_t gcd64(int64_t a, int64_t b) {
    while (b) { const int64_t t = a % b; a = b; b = t; }
    return a;
}

// Two periods of the launch schedule: after them the ping-pong buffers are
// back in place, so one captured graph can be replayed every graph_len steps.
int64_t schedule_len(const mdlg_ctx *c) {
    int64_t L = c->sort_every;
    for (int l = 0; l < c->p.nlags; ++l) L = L / gcd64(L, c->p.lag_steps[l]) * c->p.lag_steps[l];
    if (c->p.stats_every > 0) L = L / gcd64(L, c->p.stats_every) * c->p.stats_every;
    return 2 * L;
}

void drop_graph(mdlg_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_start = -1;
}

// Capture the next graph_len steps into a graph and launch it.
int capture_and_launch(mdlg_ctx *c) {
    const int64_t s0 = c->step;
    const int pc = c->pos_cur, mc = c->meta_cur;
    const uint32_t *sc = c->site_counts;
    int64_t before[MDLG_PROF_KINDS];
    for (int k = 0; k < MDLG_PROF_KINDS; ++k) before[k] = c->launches[k];
    const bool prof = c->prof;
    c->prof = false;   // no event records inside the graph
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        c->prof = prof;
        cudaGetLastError();
        c->graph_failed = true;
        return MDLG_OK;   // fall back to direct launches
    }
    const int rc = step_loop(c, c->graph_len, true);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
    c->prof = prof;
    MDLG_TRY(rc);
    MDLG_TRY(cuda_err(ec));
    c->graph = g;
    if (c->pos_cur != pc || c->meta_cur != mc || c->site_counts != sc) {   // cannot be replayed in place
        c->graph_failed = true;
        cudaGraphExec_t once = nullptr;
        MDLG_TRY(cuda_err(cudaGraphInstantiate(&once, g, 0)));
        const cudaError_t el = cudaGraphLaunch(once, c->stream);
        cudaGraphExecDestroy(once);
        drop_graph(c);
        return cuda_err(el);
    }
    MDLG_TRY(cuda_err(cudaGraphInstantiate(&c->graph_exec, g, 0)));
    for (int k = 0; k < MDLG_PROF_KINDS; ++k) c->graph_launches[k] = c->launches[k] - before[k];
    c->graph_start = s0;
    ProfScope ps(c, MDLG_PROF_STEP, 0);
    return cuda_err(cudaGraphLaunch(c->graph_exec, c->stream));
}

}  // namespace

extern "C" {

int mdlg_step(mdlg_ctx *c, int64_t nsteps) {
    if (!c || nsteps < 0) return MDLG_EINVAL;
    if (c->p.use_graphs && !c->graph_failed && c->graph_len == 0) {
        c->graph_len = schedule_len(c);
        if (c->graph_len > 8192) c->graph_failed = true;   // too long to be worth a graph
    }
    while (nsteps > 0) {
        if (c->p.use_graphs && !c->graph_failed && nsteps >= c->graph_len) {
            if (c->graph_exec && (c->step - c->graph_start) % c->graph_len == 0) {
                {
                    ProfScope ps(c, MDLG_PROF_STEP, 0);
                    MDLG_TRY(cuda_err(cudaGraphLaunch(c->graph_exec, c->stream)));
                }
                for (int k = 0; k < MDLG_PROF_KINDS; ++k) c->launches[k] += c->graph_launches[k];
                MDLG_TRY(step_loop(c, c->graph_len, false));
                nsteps -= c->graph_len;
                continue;
            }
            if (!c->graph_exec) {
                const int64_t s0 = c->step;
                MDLG_TRY(capture_and_launch(c));
                nsteps -= c->step - s0;
                continue;
            }
        }
        MDLG_TRY(step_loop(c, 1, true));
        nsteps -= 1;
    }
    return MDLG_OK;
}

}  // extern "C"

namespace {

// Observables and MDLG totals of system k of a batch, or (k < 0) of the whole
// context: one system, or every system of a batch added together.
int stats_impl(mdlg_ctx *c, int32_t k, mdlg_stats_out *out, uint64_t *counts, double *fi) {
    if (!c || !out) return MDLG_EINVAL;
    if (k >= 0 && (c->nsys == 0 || k >= c->nsys)) return MDLG_EINVAL;
    if (c->stats_step != c->step) MDLG_TRY(sync_stats(c, false));
    double st[5];
    int32_t status = 0;
    MDLG_TRY(read_observables(c, k, st, &status));
    const mdlg_params &p = c->p;
    int64_t n = p.n;
    double area = p.box[0] * p.box[1];
    int32_t nsub = 1;
    if (c->nsys > 0) {
        n = 0;
        area = 0.0;
        nsub = 0;
        for (int32_t s = (k < 0 ? 0 : k); s < (k < 0 ? c->nsys : k + 1); ++s) {
            const SysInfo &si = c->sys_host[s];
            n += si.n;
            area += (double)si.geo.lg[0] * si.geo.lg[1] * p.grid * p.grid;
            ++nsub;
        }
    }
    memset(out, 0, sizeof(*out));
    out->step = c->step;
    out->stats_step = c->stats_step;
    out->kinetic = st[0];
    out->potential = st[1];
    out->virial = st[2];
    out->momentum[0] = st[3];
    out->momentum[1] = st[4];
    out->temperature = n > nsub ? st[0] / (double)(n - nsub) : 0.0;
    out->pressure = (st[0] + 0.5 * st[2]) / area;
    for (int l = 0; l < p.nlags; ++l) out->intervals[l] = c->intervals[l];
    out->status = status;
    for (int a = 0; a < 2; ++a)
        out->lattice_u[a] = (double)c->shift_m[a] * p.grid * (1.0 / 16777216.0) / p.dt;
    {
        Control h{};
        MDLG_TRY(cuda_err(cudaMemcpyAsync(&h, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost,
                                          c->stream)));
        MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
        out->stale_steps = h.stale_steps;
        out->sort_every = c->sort_every;
    }
    if (p.msd) {
        double h[2 * kMaxLags];
        MDLG_TRY(cuda_err(cudaMemcpyAsync(h, c->msd_acc, sizeof(double) * 2 * p.nlags,
                                          cudaMemcpyDeviceToHost, c->stream)));
        MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
        for (int l = 0; l < p.nlags; ++l)
            for (int a = 0; a < 2; ++a) {
                const double denom = (double)n * (double)c->intervals[l];
                out->msd[l][a] = denom > 0 ? h[2 * l + a] / denom : 0.0;
            }
    }
    if (p.vacf) {
        double h[2 * kMaxLags];
        MDLG_TRY(cuda_err(cudaMemcpyAsync(h, c->vacf_acc, sizeof(double) * 2 * p.nlags,
                                          cudaMemcpyDeviceToHost, c->stream)));
        MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
        for (int l = 0; l < p.nlags; ++l)
            for (int a = 0; a < 2; ++a) {
                const double denom = (double)n * (double)c->intervals[l];
                out->vacf[l][a] = denom > 0 ? h[2 * l + a] / denom : 0.0;
            }
    }
    if (counts || fi) {
        const int32_t nsb = c->nsys > 0 ? c->nsys : 1;
        std::vector<unsigned long long> h((size_t)nsb * p.nlags * c->q1);
        MDLG_TRY(cuda_err(cudaMemcpyAsync(h.data(), c->counts, sizeof(unsigned long long) * h.size(),
                                          cudaMemcpyDeviceToHost, c->stream)));
        MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
        for (int l = 0; l < p.nlags; ++l)
            for (int i = 0; i < c->q1; ++i) {
                unsigned long long t = 0;
                for (int32_t s = (k < 0 ? 0 : k); s < (k < 0 ? nsb : k + 1); ++s)
                    t += h[((size_t)s * p.nlags + l) * c->q1 + i];
                const size_t o = (size_t)l * c->q1 + i;
                if (counts) counts[o] = t;
                if (fi) {
                    const double denom = (double)n * (double)c->intervals[l];
                    fi[o] = denom > 0 ? (double)t / denom : 0.0;
                }
            }
    }
    return status ? status : MDLG_OK;
}

}  // namespace

extern "C" {

int mdlg_stats(mdlg_ctx *c, mdlg_stats_out *out, uint64_t *counts, double *fi) {
    return stats_impl(c, -1, out, counts, fi);
}

int mdlg_stats_system(mdlg_ctx *c, int32_t system, mdlg_stats_out *out, uint64_t *counts,
                      double *fi) {
    if (system < 0) return MDLG_EINVAL;
    return stats_impl(c, system, out, counts, fi);
}

int mdlg_get_state(mdlg_ctx *c, double *x, double *v, double *f) {
    if (!c) return MDLG_EINVAL;
    const size_t N = (size_t)c->p.n;
    if (v || f) {
        MDLG_TRY(zero_bstats(c));
        StepArgs a = step_args(c);
        a.stats = 1;
        MDLG_TRY(cuda_err(launch_step(a, kModeSync, c->stream)));
        c->stats_step = c->step;
    }
    const Batch bt = batch_of(c);
    MDLG_TRY(cuda_err(launch_unpack(c->geo, c->slots, c->cell[c->meta_cur], c->cl[c->pos_cur],
                                    c->vsync, c->fsync, c->pid[c->meta_cur], x ? c->xbuf : nullptr,
                                    v ? c->vbuf : nullptr, f ? c->fbuf : nullptr, c->stream, &bt)));
    if (x) MDLG_TRY(cuda_err(cudaMemcpyAsync(x, c->xbuf, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->stream)));
    if (v) MDLG_TRY(cuda_err(cudaMemcpyAsync(v, c->vbuf, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->stream)));
    if (f) MDLG_TRY(cuda_err(cudaMemcpyAsync(f, c->fbuf, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->stream)));
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    return MDLG_OK;
}

int mdlg_get_sites(mdlg_ctx *c, uint32_t *site_counts, uint32_t *ncell) {
    if (!c) return MDLG_EINVAL;
    if (!c->p.site_mode) return MDLG_EINVAL;
    const size_t sites = (size_t)c->geo.lat[0] * c->geo.lat[1];
    if (site_counts)
        MDLG_TRY(cuda_err(cudaMemcpyAsync(site_counts, c->site_counts, sizeof(uint32_t) * sites * c->q1,
                                          cudaMemcpyDeviceToHost, c->stream)));
    if (ncell)
        MDLG_TRY(cuda_err(cudaMemcpyAsync(ncell, c->site_n, sizeof(uint32_t) * sites,
                                          cudaMemcpyDeviceToHost, c->stream)));
    return cuda_err(cudaStreamSynchronize(c->stream));
}

int mdlg_get_collision(mdlg_ctx *c, int32_t *xi, int32_t *dmass, int32_t *dmom) {
    if (!c || !(c->p.site_mode & MDLG_SITES_XI) || c->intervals[0] < 2) return MDLG_EINVAL;
    const size_t sites = (size_t)c->geo.lat[0] * c->geo.lat[1];
    if (xi)
        MDLG_TRY(cuda_err(cudaMemcpyAsync(xi, c->xi, sizeof(int32_t) * sites * (c->q1 - 1),
                                          cudaMemcpyDeviceToHost, c->stream)));
    if (dmass)
        MDLG_TRY(cuda_err(cudaMemcpyAsync(dmass, c->dmass, sizeof(int32_t) * sites,
                                          cudaMemcpyDeviceToHost, c->stream)));
    if (dmom)
        MDLG_TRY(cuda_err(cudaMemcpyAsync(dmom, c->dmom, sizeof(int32_t) * 2 * sites,
                                          cudaMemcpyDeviceToHost, c->stream)));
    return cuda_err(cudaStreamSynchronize(c->stream));
}

int mdlg_reset_counts(mdlg_ctx *c) {
    if (!c) return MDLG_EINVAL;
    const size_t nsb = c->nsys > 0 ? (size_t)c->nsys : 1;
    MDLG_TRY(cuda_err(cudaMemsetAsync(c->counts, 0, sizeof(unsigned long long) * nsb * c->p.nlags * c->q1,
                                      c->stream)));
    if (c->p.site_mode) {
        const size_t sites = (size_t)c->geo.lat[0] * c->geo.lat[1];
        MDLG_TRY(cuda_err(cudaMemsetAsync(c->site_n, 0, sizeof(uint32_t) * sites, c->stream)));
        MDLG_TRY(cuda_err(cudaMemsetAsync(c->site_counts, 0, sizeof(uint32_t) * sites * c->q1, c->stream)));
        if (c->site_counts_alt)
            MDLG_TRY(cuda_err(cudaMemsetAsync(c->site_counts_alt, 0, sizeof(uint32_t) * sites * c->q1,
                                              c->stream)));
    }
    if (c->msd_acc)
        MDLG_TRY(cuda_err(cudaMemsetAsync(c->msd_acc, 0, sizeof(double) * 2 * c->p.nlags, c->stream)));
    if (c->vacf_acc)
        MDLG_TRY(cuda_err(cudaMemsetAsync(c->vacf_acc, 0, sizeof(double) * 2 * c->p.nlags, c->stream)));
    for (int l = 0; l < kMaxLags; ++l) c->intervals[l] = 0;
    return MDLG_OK;
}

}  // extern "C"

namespace {

// Device allocations that live for one call (through the context's allocator).
struct TempAlloc {
    mdlg_ctx *c;
    std::vector<void *> ptrs;
    explicit TempAlloc(mdlg_ctx *ctx) : c(ctx) {}
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        const size_t bytes = sizeof(T) * (count ? count : 1);
        if (c->use_cuda_malloc) {
            if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
        } else {
            p = c->alloc.alloc(bytes, c->alloc.user);
        }
        if (p) ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~TempAlloc() {
        cudaStreamSynchronize(c->stream);
        for (void *p : ptrs) {
            if (c->use_cuda_malloc) cudaFree(p);
            else c->alloc.free(p, c->alloc.user);
        }
    }
};

struct Checkpoint {
    float2 *cl, *v;
    uint32_t *cell, *nbr;
    int32_t *pid, *cell_start, *ncount;
};

}  // namespace

extern "C" {

int mdlg_adjoint(mdlg_ctx *c, int64_t nsteps, int32_t ckpt_every, double width,
                 const double *dloss, double *ftilde, double *loss, double *grad_eps,
                 double *grad_sigma, double *grad_x0, double *grad_v0) {
    if (!c || c->nsys != 0 || nsteps < 1 || ckpt_every < 1 || nsteps % ckpt_every) return MDLG_EINVAL;
    if (c->sort_every != ckpt_every || c->step != c->last_sort) return MDLG_EINVAL;
    const mdlg_params &p = c->p;
    if (!(width > 0.0) || width > 0.875 * p.dx || p.vmax > 7) return MDLG_EINVAL;
    const int64_t N = c->slots;
    const int Q = (2 * p.vmax + 1) * (2 * p.vmax + 1);
    const int64_t nseg = nsteps / ckpt_every;
    const size_t nc1 = (size_t)c->ncells + 1;
    cudaStream_t s = c->stream;
    TempAlloc tmp(c);
    auto chk = [](cudaError_t e) { return cuda_err(e); };
#define ADJ_ALLOC(ptr, T, count)                 \
    do {                                         \
        ptr = tmp.get<T>(count);                 \
        if (!ptr) return MDLG_ENOMEM;            \
    } while (0)
    double *x_start, *gx0, *theta, *fsum, *lossd, *wts = nullptr;
    float2 *traj = nullptr, *vbuf = nullptr, *xb[2] = {nullptr, nullptr}, *w[2] = {nullptr, nullptr};
    float2 *xb_orig = nullptr, *w_orig = nullptr;
    float *dck, *dfinal;
    ADJ_ALLOC(x_start, double, 2 * N);
    ADJ_ALLOC(gx0, double, 2 * N);
    ADJ_ALLOC(theta, double, 2);
    ADJ_ALLOC(fsum, double, Q);
    ADJ_ALLOC(lossd, double, 1);
    ADJ_ALLOC(dck, float, nseg);
    ADJ_ALLOC(dfinal, float, 1);
    std::vector<Checkpoint> ck((size_t)nseg);
    for (auto &k : ck) {
        ADJ_ALLOC(k.cl, float2, N);
        ADJ_ALLOC(k.v, float2, N);
        ADJ_ALLOC(k.cell, uint32_t, N);
        ADJ_ALLOC(k.pid, int32_t, N);
        ADJ_ALLOC(k.cell_start, int32_t, nc1);
        k.nbr = nullptr;
        k.ncount = nullptr;
        if (c->nbr) {
            ADJ_ALLOC(k.nbr, uint32_t, (size_t)c->cap * N);
            ADJ_ALLOC(k.ncount, int32_t, N);
        }
    }
    if (dloss) {
        ADJ_ALLOC(wts, double, Q);
        ADJ_ALLOC(traj, float2, (size_t)(ckpt_every + 1) * N);
        ADJ_ALLOC(vbuf, float2, 2 * N);
        for (int b = 0; b < 2; ++b) {
            ADJ_ALLOC(xb[b], float2, N);
            ADJ_ALLOC(w[b], float2, N);
        }
        ADJ_ALLOC(xb_orig, float2, N);
        ADJ_ALLOC(w_orig, float2, N);
    }
#undef ADJ_ALLOC
    MDLG_TRY(chk(cudaMemsetAsync(theta, 0, 2 * sizeof(double), s)));
    MDLG_TRY(chk(cudaMemsetAsync(fsum, 0, Q * sizeof(double), s)));
    MDLG_TRY(chk(cudaMemsetAsync(lossd, 0, sizeof(double), s)));
    if (dloss)
        MDLG_TRY(chk(cudaMemcpyAsync(wts, dloss, Q * sizeof(double), cudaMemcpyHostToDevice, s)));

    // start positions (original order)
    MDLG_TRY(chk(launch_unpack(c->geo, N, c->cell[c->meta_cur], c->cl[c->pos_cur], c->vsync,
                               c->fsync, c->pid[c->meta_cur], x_start, nullptr, nullptr, s)));
    // forward: a checkpoint after every re-sort (the segment boundaries)
    const int64_t s0 = c->step;
    for (int64_t g = 0; g < nseg; ++g) {
        if (g > 0) MDLG_TRY(do_sort(c));
        Checkpoint &k = ck[(size_t)g];
        MDLG_TRY(chk(cudaMemcpyAsync(k.cl, c->cl[c->pos_cur], N * sizeof(float2), cudaMemcpyDeviceToDevice, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(k.v, c->vel[c->pos_cur], N * sizeof(float2), cudaMemcpyDeviceToDevice, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(k.cell, c->cell[c->meta_cur], N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(k.pid, c->pid[c->meta_cur], N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(k.cell_start, c->cell_start, nc1 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s)));
        if (c->nbr) {
            MDLG_TRY(chk(cudaMemcpyAsync(k.nbr, c->nbr, (size_t)c->cap * N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)));
            MDLG_TRY(chk(cudaMemcpyAsync(k.ncount, c->ncount, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s)));
        }
        MDLG_TRY(chk(cudaMemcpyAsync(dck + g, &c->ctl->dbound, sizeof(float), cudaMemcpyDeviceToDevice, s)));
        MDLG_TRY(step_loop(c, ckpt_every, true));
    }
    MDLG_TRY(chk(cudaMemcpyAsync(dfinal, &c->ctl->dbound, sizeof(float), cudaMemcpyDeviceToDevice, s)));

    // soft loss on the final state (order of the last segment)
    SoftArgs la{};
    la.geo = c->geo;
    la.n = N;
    la.ntot = p.n;
    la.cell = c->cell[c->meta_cur];
    la.cl = c->cl[c->pos_cur];
    la.pid = c->pid[c->meta_cur];
    la.x_start = x_start;
    la.dx = p.dx;
    la.width = width;
    la.vmax = p.vmax;
    la.M = (int32_t)std::ceil(8.0 * width / p.dx) + 1;
    la.weights = wts;
    la.fsum = fsum;
    la.loss = lossd;
    la.xb = dloss ? xb[0] : nullptr;
    la.gx_start = dloss ? gx0 : nullptr;
    if (dloss) MDLG_TRY(chk(cudaMemsetAsync(gx0, 0, 2 * N * sizeof(double), s)));
    MDLG_TRY(chk(launch_soft_loss(la, s)));

    if (dloss) {
        // adjoint state in original order between segments
        MDLG_TRY(chk(launch_permute(N, c->pid[c->meta_cur], xb[0], xb_orig, true, s)));
        MDLG_TRY(chk(cudaMemsetAsync(w_orig, 0, N * sizeof(float2), s)));
        AdjArgs aa{};
        aa.geo = c->geo;
        aa.n = N;
        aa.cap = c->cap;
        aa.list_skin = c->list_radius - (float)p.rcut;
        aa.rc = (float)p.rcut;
        aa.rc2 = (float)(p.rcut * p.rcut);
        aa.cell_w = (float)(c->geo.k * p.grid);
        aa.eps24 = (float)(24.0 * p.eps);
        aa.sig2 = (float)(p.sigma * p.sigma);
        aa.inv_eps = p.eps != 0.0 ? (float)(1.0 / p.eps) : 0.f;
        aa.inv_sigma = (float)(1.0 / p.sigma);
        aa.theta = theta;
        aa.ctl = c->ctl;
        aa.potential = p.potential == MDLG_POT_LJ_TS ? 1 : (p.potential == MDLG_POT_LJ_SF ? 2 : 0);
        aa.fc = (float)lj_fc(p);
        aa.dfc_dsigma = (float)lj_dfc_dsigma(p);
        const float dt = (float)p.dt, dt_m = (float)(p.dt / p.mass);
        for (int64_t g = nseg - 1; g >= 0; --g) {
            const Checkpoint &k = ck[(size_t)g];
            MDLG_TRY(chk(launch_permute(N, k.pid, xb_orig, xb[0], false, s)));
            MDLG_TRY(chk(launch_permute(N, k.pid, w_orig, w[0], false, s)));
            // recompute the segment from its checkpoint, keeping every position
            MDLG_TRY(chk(cudaMemcpyAsync(&c->ctl->dbound, dck + g, sizeof(float), cudaMemcpyDeviceToDevice, s)));
            MDLG_TRY(chk(cudaMemcpyAsync(traj, k.cl, N * sizeof(float2), cudaMemcpyDeviceToDevice, s)));
            MDLG_TRY(chk(cudaMemcpyAsync(vbuf, k.v, N * sizeof(float2), cudaMemcpyDeviceToDevice, s)));
            for (int t = 0; t < ckpt_every; ++t) {
                StepArgs a = step_args(c);
                a.cell = k.cell;
                a.cell_start = k.cell_start;
                a.nbr = k.nbr;
                a.ncount = k.ncount;
                a.cl_in = traj + (size_t)t * N;
                a.cl_out = traj + (size_t)(t + 1) * N;
                a.v_in = vbuf + (size_t)(t & 1) * N;
                a.v_out = vbuf + (size_t)((t + 1) & 1) * N;
                const int64_t step = s0 + g * ckpt_every + t;
                a.stats = (p.stats_every > 0 && step % p.stats_every == 0) ? 1 : 0;
                MDLG_TRY(chk(launch_step(a, kModeStep, s)));
            }
            // reverse the segment's steps
            aa.cell = k.cell;
            aa.cell_start = k.cell_start;
            aa.nbr = k.nbr;
            aa.ncount = k.ncount;
            int cur = 0;
            for (int t = ckpt_every - 1; t >= 0; --t) {
                aa.x = traj + (size_t)t * N;
                aa.a_coef = dt;
                aa.b_coef = dt_m;
                aa.w_prev = w[cur];
                aa.xb = xb[cur];
                aa.w_out = w[cur ^ 1];
                aa.xb_out = xb[cur ^ 1];
                MDLG_TRY(chk(launch_adjoint_step(aa, s)));
                cur ^= 1;
            }
            if (g == 0) {
                // the half kick that turns the integer-step velocity into v_{-1/2}
                MDLG_TRY(chk(cudaMemcpyAsync(&c->ctl->dbound, dck, sizeof(float), cudaMemcpyDeviceToDevice, s)));
                aa.x = traj;
                aa.a_coef = 0.f;
                aa.b_coef = -0.5f * dt_m;
                aa.w_prev = w[cur];
                aa.xb = xb[cur];
                aa.w_out = w[cur ^ 1];
                aa.xb_out = xb[cur ^ 1];
                MDLG_TRY(chk(launch_adjoint_step(aa, s)));
                cur ^= 1;
            }
            MDLG_TRY(chk(launch_permute(N, k.pid, xb[cur], xb_orig, true, s)));
            MDLG_TRY(chk(launch_permute(N, k.pid, w[cur], w_orig, true, s)));
        }
        MDLG_TRY(chk(cudaMemcpyAsync(&c->ctl->dbound, dfinal, sizeof(float), cudaMemcpyDeviceToDevice, s)));
    }
    c->stats_step = -1;   // the recompute overwrote the last statistics

    // results to the host
    std::vector<double> hf(Q), hx((size_t)2 * p.n), hg((size_t)2 * p.n);
    std::vector<float2> hxo, hwo;
    double hl = 0.0, ht[2] = {0.0, 0.0};
    MDLG_TRY(chk(cudaMemcpyAsync(hf.data(), fsum, Q * sizeof(double), cudaMemcpyDeviceToHost, s)));
    MDLG_TRY(chk(cudaMemcpyAsync(&hl, lossd, sizeof(double), cudaMemcpyDeviceToHost, s)));
    if (dloss) {
        hxo.resize((size_t)p.n);
        hwo.resize((size_t)p.n);
        MDLG_TRY(chk(cudaMemcpyAsync(ht, theta, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(hg.data(), gx0, 2 * p.n * sizeof(double), cudaMemcpyDeviceToHost, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(hxo.data(), xb_orig, p.n * sizeof(float2), cudaMemcpyDeviceToHost, s)));
        MDLG_TRY(chk(cudaMemcpyAsync(hwo.data(), w_orig, p.n * sizeof(float2), cudaMemcpyDeviceToHost, s)));
    }
    MDLG_TRY(chk(cudaStreamSynchronize(s)));
    int32_t status = 0;
    MDLG_TRY(read_status(c, &status, nullptr));
    if (ftilde) memcpy(ftilde, hf.data(), Q * sizeof(double));
    if (loss) *loss = hl;
    if (dloss) {
        if (grad_eps) *grad_eps = ht[0];
        if (grad_sigma) *grad_sigma = ht[1];
        for (int64_t i = 0; i < p.n; ++i) {
            if (grad_x0) {
                grad_x0[2 * i] = (double)hxo[i].x + hg[2 * i];
                grad_x0[2 * i + 1] = (double)hxo[i].y + hg[2 * i + 1];
            }
            if (grad_v0) {
                grad_v0[2 * i] = hwo[i].x;
                grad_v0[2 * i + 1] = hwo[i].y;
            }
        }
    }
    return status ? status : MDLG_OK;
}

}  // extern "C"

namespace {

// Checkpoint layout: a header, then the device regions below in this order.
constexpr uint64_t kCkptMagic = 0x54504b43474c444dull;   // "MDLGCKPT"
constexpr uint32_t kCkptVersion = 3;

struct CkptHeader {
    uint64_t magic;
    uint32_t version, nsys;
    uint64_t total;             // bytes including this header
    uint64_t shape_hash;        // parameters and geometry the regions depend on
    int64_t step, last_sort, stats_step;
    int64_t intervals[kMaxLags];
    int32_t pos_cur, meta_cur;
    // the re-sort schedule: current interval, the fastest uploaded speed and
    // (adaptive schedule) the slots of the last kPaceLag steps (step -1: none)
    int32_t sort_every;
    int32_t pad_;
    double vmax0;
    PaceSlot pace[kPaceLag];
};

struct Region {
    void *p;
    size_t bytes;
};

uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t k = 0; k < n; ++k) {
        h ^= b[k];
        h *= 0x100000001b3ull;
    }
    return h;
}

template <typename T>
uint64_t mix(uint64_t h, const T &v) { return fnv1a(h, &v, sizeof(T)); }

// Everything the saved regions and the schedule depend on (use_graphs and
// stats_every excluded: they do not change the state).
uint64_t shape_hash(const mdlg_ctx *c) {
    const mdlg_params &p = c->p;
    uint64_t h = 0xcbf29ce484222325ull;
    h = mix(h, p.n); h = mix(h, p.box[0]); h = mix(h, p.box[1]); h = mix(h, p.potential);
    h = mix(h, p.eps); h = mix(h, p.sigma); h = mix(h, p.mass); h = mix(h, p.rcut);
    h = mix(h, p.dt); h = mix(h, p.grid); h = mix(h, p.skin); h = mix(h, p.dx);
    h = mix(h, p.nlags);
    for (int l = 0; l < p.nlags; ++l) h = mix(h, p.lag_steps[l]);
    h = mix(h, p.vmax); h = mix(h, p.site_mode); h = mix(h, p.msd); h = mix(h, p.vacf);
    h = mix(h, p.lattice_u[0]); h = mix(h, p.lattice_u[1]);
    h = mix(h, p.sort_every); h = mix(h, c->adaptive); h = mix(h, c->slots); h = mix(h, c->ncells);
    h = mix(h, c->cap);
    h = mix(h, c->nsys);
    if (c->nsys > 0) h = fnv1a(h, c->sys_host.data(), sizeof(SysInfo) * c->sys_host.size());
    return h;
}

std::vector<Region> ckpt_regions(mdlg_ctx *c) {
    const size_t N = (size_t)c->slots;
    const int nl = c->p.nlags;
    const int pc = c->pos_cur, mc = c->meta_cur;
    std::vector<Region> r;
    r.push_back({c->cell[mc], N * sizeof(uint32_t)});
    r.push_back({c->pid[mc], N * sizeof(int32_t)});
    r.push_back({c->cl[pc], N * sizeof(float2)});
    r.push_back({c->vel[pc], N * sizeof(float2)});
    for (int l = 0; l < nl; ++l) r.push_back({c->lprev[mc][l], N * sizeof(uint32_t)});
    if (c->p.msd) {
        for (int l = 0; l < nl; ++l) r.push_back({c->mprev[mc][l], N * sizeof(float2)});
        r.push_back({c->msd_acc, 2 * nl * sizeof(double)});
    }
    if (c->p.vacf) {
        for (int l = 0; l < nl; ++l) r.push_back({c->vprev[mc][l], N * sizeof(float2)});
        r.push_back({c->vacf_acc, 2 * nl * sizeof(double)});
    }
    r.push_back({c->cell_start, ((size_t)c->ncells + 1) * sizeof(int32_t)});
    if (c->nbr) {
        r.push_back({c->nbr, (size_t)c->cap * N * sizeof(uint32_t)});
        r.push_back({c->ncount, N * sizeof(int32_t)});
    }
    r.push_back({c->ctl, sizeof(Control)});
    const size_t nsb = c->nsys > 0 ? (size_t)c->nsys : 1;
    r.push_back({c->counts, nsb * nl * c->q1 * sizeof(unsigned long long)});
    if (c->nsys > 0) r.push_back({c->bstats, (size_t)c->nsys * 5 * sizeof(long long)});
    if (c->p.site_mode) {
        const size_t sites = (size_t)c->geo.lat[0] * c->geo.lat[1];
        r.push_back({c->site_n, sites * sizeof(uint32_t)});
        r.push_back({c->site_counts, sites * c->q1 * sizeof(uint32_t)});
        if (c->site_counts_alt) {
            r.push_back({c->site_counts_alt, sites * c->q1 * sizeof(uint32_t)});
            r.push_back({c->xi, sites * (c->q1 - 1) * sizeof(int32_t)});
            r.push_back({c->dmass, sites * sizeof(int32_t)});
            r.push_back({c->dmom, 2 * sites * sizeof(int32_t)});
        }
    }
    return r;
}

uint64_t ckpt_total(mdlg_ctx *c) {
    uint64_t t = sizeof(CkptHeader);
    for (const Region &g : ckpt_regions(c)) t += g.bytes;
    return t;
}

}  // namespace

extern "C" {

int mdlg_checkpoint_size(mdlg_ctx *c, uint64_t *bytes) {
    if (!c || !bytes) return MDLG_EINVAL;
    *bytes = ckpt_total(c);
    return MDLG_OK;
}

int mdlg_save(mdlg_ctx *c, void *buf, uint64_t bytes) {
    if (!c || !buf) return MDLG_EINVAL;
    const uint64_t total = ckpt_total(c);
    if (bytes < total) return MDLG_EINVAL;
    CkptHeader h{};
    h.magic = kCkptMagic;
    h.version = kCkptVersion;
    h.nsys = (uint32_t)c->nsys;
    h.total = total;
    h.shape_hash = shape_hash(c);
    h.step = c->step;
    h.last_sort = c->last_sort;
    h.stats_step = c->stats_step;
    for (int l = 0; l < kMaxLags; ++l) h.intervals[l] = c->intervals[l];
    h.pos_cur = c->pos_cur;
    h.meta_cur = c->meta_cur;
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));   // every slot has been written
    h.sort_every = c->sort_every;
    h.vmax0 = c->vmax0;
    for (int64_t k = 0; k < kPaceLag; ++k) {
        const int64_t st = c->step - kPaceLag + k;
        h.pace[k] = PaceSlot{-1, 0.0f, 0u};
        if (c->pace && st >= 0 && c->pace[st & (kPaceRing - 1)].step == st)
            h.pace[k] = c->pace[st & (kPaceRing - 1)];
    }
    memcpy(buf, &h, sizeof(h));
    unsigned char *o = static_cast<unsigned char *>(buf) + sizeof(h);
    for (const Region &g : ckpt_regions(c)) {
        MDLG_TRY(cuda_err(cudaMemcpyAsync(o, g.p, g.bytes, cudaMemcpyDeviceToHost, c->stream)));
        o += g.bytes;
    }
    return cuda_err(cudaStreamSynchronize(c->stream));
}

int mdlg_load(mdlg_ctx *c, const void *buf, uint64_t bytes) {
    if (!c || !buf || bytes < sizeof(CkptHeader)) return MDLG_EINVAL;
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kCkptMagic || h.version != kCkptVersion || h.nsys != (uint32_t)c->nsys)
        return MDLG_EINVAL;
    if (h.shape_hash != shape_hash(c) || bytes < h.total) return MDLG_EINVAL;
    if ((h.pos_cur & ~1) || (h.meta_cur & ~1)) return MDLG_EINVAL;
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    drop_graph(c);                 // a captured schedule refers to the old step count
    c->pos_cur = h.pos_cur;
    c->meta_cur = h.meta_cur;
    if (ckpt_total(c) != h.total) return MDLG_EINVAL;
    const unsigned char *o = static_cast<const unsigned char *>(buf) + sizeof(h);
    for (const Region &g : ckpt_regions(c)) {
        MDLG_TRY(cuda_err(cudaMemcpyAsync(g.p, o, g.bytes, cudaMemcpyHostToDevice, c->stream)));
        o += g.bytes;
    }
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    c->step = h.step;
    c->last_sort = h.last_sort;
    c->stats_step = h.stats_step;
    if (h.sort_every < 1) return MDLG_EINVAL;
    c->sort_every = h.sort_every;
    c->vmax0 = h.vmax0;
    if (c->pace) {
        for (int k = 0; k < kPaceRing; ++k) c->pace[k] = PaceSlot{-1, 0.0f, 0u};
        for (int64_t k = 0; k < kPaceLag; ++k)
            if (h.pace[k].step >= 0 && h.pace[k].step == c->step - kPaceLag + k)
                c->pace[h.pace[k].step & (kPaceRing - 1)] = h.pace[k];
    }
    for (int l = 0; l < kMaxLags; ++l) c->intervals[l] = h.intervals[l];
    return MDLG_OK;
}

int mdlg_profile(mdlg_ctx *c, int enable, double *ms, int64_t *launches) {
    if (!c) return MDLG_EINVAL;
    if (enable) {
        c->prof = true;
        c->ev_used = 0;
        c->ev_kind.clear();
        for (int k = 0; k < MDLG_PROF_KINDS; ++k) c->launches[k] = 0;
        return MDLG_OK;
    }
    c->prof = false;
    MDLG_TRY(cuda_err(cudaStreamSynchronize(c->stream)));
    double acc[MDLG_PROF_KINDS] = {0, 0, 0, 0};
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float t = 0.f;
        MDLG_TRY(cuda_err(cudaEventElapsedTime(&t, c->ev_pool[i], c->ev_pool[i + 1])));
        acc[c->ev_kind[i]] += t;
    }
    for (int k = 0; k < MDLG_PROF_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = c->launches[k];
    }
    c->ev_used = 0;
    c->ev_kind.clear();
    return MDLG_OK;
}

void mdlg_destroy(mdlg_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    free_all(c);
    delete c;
}

int mdlg_bin(const mdlg_lattice *lat, int64_t n, const int32_t *idx_prev, const int32_t *idx_cur,
             uint64_t *counts, uint32_t *ncell, uint32_t *field, void *stream) {
    if (!lat || n < 0 || !counts) return MDLG_EINVAL;
    if (n > 0 && (!idx_prev || !idx_cur)) return MDLG_EINVAL;
    if (lat->ratio < 1 || lat->vmax < 1 || lat->vmax > MDLG_MAX_VMAX) return MDLG_EINVAL;
    LatticeArgs la{};
    for (int a = 0; a < 2; ++a) {
        if (lat->base[a] < 1 || lat->base[a] % lat->ratio) return MDLG_EINVAL;
        la.base[a] = lat->base[a];
        la.lat[a] = lat->base[a] / lat->ratio;
    }
    la.ratio = lat->ratio;
    la.shift = log2_exact(lat->ratio);
    la.vmax = lat->vmax;
    if (n == 0) return MDLG_OK;
    return cuda_err(launch_bin_snapshots(la, n, idx_prev, idx_cur,
                                         reinterpret_cast<unsigned long long *>(counts), ncell,
                                         field, static_cast<cudaStream_t>(stream)));
}

int mdlg_collision(const mdlg_lattice *lat, const uint32_t *field_prev,
                   const uint32_t *field_cur, int32_t *xi, int32_t *dmass, int32_t *dmom,
                   void *stream) {
    if (!lat || !field_prev || !field_cur) return MDLG_EINVAL;
    if (lat->ratio < 1 || lat->vmax < 1 || lat->vmax > MDLG_MAX_VMAX) return MDLG_EINVAL;
    CollArgs ca{};
    for (int a = 0; a < 2; ++a) {
        if (lat->base[a] < 1 || lat->base[a] % lat->ratio) return MDLG_EINVAL;
        ca.lat[a] = lat->base[a] / lat->ratio;
    }
    ca.vmax = lat->vmax;
    ca.prev = field_prev;
    ca.cur = field_cur;
    ca.xi = xi;
    ca.dmass = dmass;
    ca.dmom = dmom;
    if (!xi && !dmass && !dmom) return MDLG_OK;
    return cuda_err(launch_collision(ca, static_cast<cudaStream_t>(stream)));
}

int mdlg_idealgas_bin(int64_t n, const float *pos, const float *vel, int32_t ncombo,
                      const float *dxs, const float *dts, const float *us, int32_t vmax,
                      uint64_t *counts, void *stream) {
    if (n < 0 || !counts || !dxs || !dts) return MDLG_EINVAL;
    if (ncombo < 1 || ncombo > MDLG_MAX_COMBOS || vmax < 1 || vmax > MDLG_MAX_VMAX) return MDLG_EINVAL;
    if (n > 0 && (!pos || !vel)) return MDLG_EINVAL;
    IdealGasArgs ga{};
    ga.ncombo = ncombo;
    ga.vmax = vmax;
    for (int k = 0; k < ncombo; ++k) {
        if (!(dxs[k] > 0.f) || !std::isfinite(dxs[k]) || !std::isfinite(dts[k])) return MDLG_EINVAL;
        ga.dx[k] = dxs[k];
        ga.dt[k] = dts[k];
        ga.pow2[k] = is_pow2((double)dxs[k]) ? 1 : 0;
        ga.inv_dx[k] = ga.pow2[k] ? (float)(1.0 / (double)dxs[k]) : 0.f;
        if (us) {
            if (!std::isfinite(us[2 * k]) || !std::isfinite(us[2 * k + 1])) return MDLG_EINVAL;
            ga.ux[k] = us[2 * k];
            ga.uy[k] = us[2 * k + 1];
        }
    }
    ga.boost = us ? 1 : 0;
    if (n == 0) return MDLG_OK;
    return cuda_err(launch_idealgas_bin(ga, n, pos, vel, reinterpret_cast<unsigned long long *>(counts),
                                        static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
