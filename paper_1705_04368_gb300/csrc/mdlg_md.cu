// mdlg_md.cu -- Lennard-Jones velocity-Verlet step, neighbour-cell sort, Verlet
// list and the global reductions (Newton equations of Sec. III and potential of
// Sec. IV of arXiv:1705.04368).
//
// Time stepping is the leapfrog form of velocity Verlet: the stored velocity is
// the half-step velocity v_{n-1/2}, and one launch per MD step does
//     F_n = F(x_n),  v_{n+1/2} = v_{n-1/2} + F_n dt/m,  x_{n+1} = x_n + v_{n+1/2} dt,
// which reproduces the kick-drift-kick positions exactly in exact arithmetic;
// the integer-step velocity v_n = v_{n-1/2} + F_n dt/(2m) is formed when it is
// needed (statistics, state download).
//
// Neighbour search: particles are sorted by MD cell (side k g >= rc + skin) and
// a Verlet list of radius k g is built right after every sort.  Between sorts a
// particle moves at most D (tracked on the device from the largest speed of
// every step).  While 2D <= skin the list holds every pair closer than rc; past
// that the step kernel falls back to the cell stencil of radius
// R = ceil((rc + 2D) / (k g)), so forces are correct whatever the sort schedule.
//
// MD cells are stored packed as (c_x | c_y << 16); cell_start is indexed by
// the row-major cell number c_y nc_x + c_x.
#include "mdlg_kernels.h"

namespace mdlg {

namespace {

constexpr int kStepThreads = 256;   // one system; a batch uses one 128-slot chunk per block
constexpr int kListBatch = 4;       // list entries loaded before any is used (lists are
                                    // padded to a multiple of this)
constexpr int kNlistThreads = 128;  // list-build block (entries staged in shared memory;
                                    // 64 when the list capacity is large)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;   // 4096 cells per scan block
constexpr int kStatsN = 5;
constexpr int kErrNonFinite = -5;
constexpr int kErrOverflow = -4;
// Fixed-point scale of the exact reductions: per-particle terms are rounded to
// multiples of 2^-24 and summed as 64-bit integers.
constexpr float kFixScale = 16777216.0f;
constexpr double kFixInv = 1.0 / 16777216.0;

__device__ __forceinline__ void set_status(Control *ctl, int code) {
    atomicCAS(&ctl->status, 0, code);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int32_t cell_x(uint32_t cw) { return (int32_t)(cw & 0xffffu); }
__device__ __forceinline__ int32_t cell_y(uint32_t cw) { return (int32_t)(cw >> 16); }

// Stencil bounds of one axis: [-R, R], or every cell once if that would wrap.
__device__ __forceinline__ void stencil(int R, int nc, int &lo, int &hi) {
    if (2 * R + 1 <= nc) { lo = -R; hi = R; }
    else { lo = -(nc >> 1); hi = lo + nc - 1; }
}

// Per-particle pair sums (FP32; the cross-particle reductions are exact).
struct PairAcc {
    float fx, fy, pe, vir;
};

// One pair term of the Lennard-Jones interaction (SF: the shifted-force variant,
// a compile-time choice so the truncated-shifted step carries none of its code):
// force on i from j is 24 eps (2 s^12 - s^6) / r^2 (x_i - x_j), s = sigma / r;
// pe adds V(r) - V(rc), vir adds r . F (both halved later: each pair is seen twice).
template <bool STATS, bool SF>
__device__ __forceinline__ void pair_term(const StepArgs &a, float dx, float dy, PairAcc &acc) {
    const float r2 = fmaf(dx, dx, dy * dy);
    if (r2 < a.rc2) {
        const float ir2 = __fdividef(1.0f, r2);   // hardware reciprocal, <= 2 ulp
        const float sr2 = a.sig2 * ir2;
        const float sr6 = sr2 * sr2 * sr2;
        float fs = a.eps24 * ir2 * sr6 * (2.0f * sr6 - 1.0f);
        float ir = 0.f;
        if (SF) {          // shifted force: subtract F(rc) along the pair
            ir = rsqrtf(r2);
            fs -= a.fc * ir;
        }
        acc.fx = fmaf(fs, dx, acc.fx);
        acc.fy = fmaf(fs, dy, acc.fy);
        if (STATS) {
            float e = a.eps4 * sr6 * (sr6 - 1.0f) - a.vshift;
            if (SF) e = fmaf(a.fc, r2 * ir - a.rc, e);   // + (r - rc) F(rc)
            acc.pe += e;
            acc.vir = fmaf(fs, r2, acc.vir);
        }
    }
}

// The same term without a branch: evaluated for every list slot and masked, so
// the lanes of a warp never diverge inside a batch.  Far or empty slots give a
// tiny finite r^-2, replaced by zero (a select, not a product with a mask).
template <bool STATS, bool SF>
__device__ __forceinline__ void pair_term_masked(const StepArgs &a, float dx, float dy,
                                                 PairAcc &acc) {
    const float r2 = fmaf(dx, dx, dy * dy);
    const bool on = r2 < a.rc2;
    const float ir2 = __fdividef(1.0f, r2);   // hardware reciprocal, <= 2 ulp
    const float sr2 = a.sig2 * ir2;
    const float sr6 = sr2 * sr2 * sr2;
    float fs = a.eps24 * ir2 * sr6 * (2.0f * sr6 - 1.0f);
    float ir = 0.f;
    if (SF) {              // shifted force: subtract F(rc) along the pair
        ir = rsqrtf(r2);
        fs -= a.fc * ir;
    }
    fs = on ? fs : 0.0f;
    acc.fx = fmaf(fs, dx, acc.fx);
    acc.fy = fmaf(fs, dy, acc.fy);
    if (STATS) {
        float e = a.eps4 * sr6 * (sr6 - 1.0f) - a.vshift;
        if (SF) e = fmaf(a.fc, r2 * ir - a.rc, e);       // + (r - rc) F(rc)
        acc.pe += on ? e : 0.0f;
        acc.vir = fmaf(fs, r2, acc.vir);
    }
}

// Origin shift o_j - o_i of the neighbouring cell at offset `off` along one axis.
__device__ __forceinline__ float cell_shift(int32_t c, int off, int32_t nc, int32_t k, int32_t lg,
                                            float g) {
    return (float)wrap_half((wrap_mod(c + off, nc) - c) * k, lg) * g;
}

// All pairs through the cell stencil (always correct for the current bound D).
template <bool STATS, bool SF>
__device__ __forceinline__ void forces_cells(const StepArgs &a, const Geom &geo, const int32_t *cs,
                                             int64_t i, int32_t cx, int32_t cy, float2 p, int lox,
                                             int hix, int loy, int hiy, PairAcc &acc) {
    for (int oy = loy; oy <= hiy; ++oy) {
        const int32_t ny = wrap_mod(cy + oy, geo.nc[1]);
        const float ody = (float)wrap_half((ny - cy) * geo.k, geo.lg[1]) * geo.g;
        for (int ox = lox; ox <= hix; ++ox) {
            const int32_t nx = wrap_mod(cx + ox, geo.nc[0]);
            const float odx = (float)wrap_half((nx - cx) * geo.k, geo.lg[0]) * geo.g;
            const int32_t cn = ny * geo.nc[0] + nx;
            const int32_t s = __ldg(cs + cn), e = __ldg(cs + cn + 1);
            for (int32_t j = s; j < e; ++j) {
                if (j == i) continue;
                const float2 q = __ldg(a.cl_in + j);
                // x_i - x_j = (cl_i - cl_j) - (origin_j - origin_i)
                pair_term<STATS, SF>(a, (p.x - q.x) - odx, (p.y - q.y) - ody, acc);
            }
        }
    }
}

// Pairs from the Verlet list built at the last sort: entry t of particle i is
// nbr[4 (floor(t/4) n + i) + t mod 4] = j | (ox + 1) << 28 | (oy + 1) << 30 with
// (ox, oy) the offset of j's cell from i's cell, so that each batch of four
// entries of a particle is one 16-byte load and a warp's batches are adjacent.
// Each list is padded to a multiple of kListBatch with entries
// i | 3 << 28 | 3 << 30: the particle itself two cell widths away on both axes,
// always beyond rc (cells are wider than rc), so every load is unconditional
// and a padding slot adds zero.  The position loads of a batch are issued
// together so that they overlap.
// For a particle whose neighbouring cells are all full-width and unwrapped
// (REGULAR) the origin shifts are ((c_x - 1) w, (c_y - 1) w), read from a
// 16-entry shared-memory table indexed by the entry's four code bits; at the
// periodic edges and next to the wider last cell they are selected from the
// four per-particle shifts.
template <bool STATS, bool REGULAR, bool SF>
__device__ __forceinline__ void forces_list(const StepArgs &a, int64_t i, float2 p, int cnt,
                                            const float2 *tab, float sxm, float sxp, float sym,
                                            float syp, PairAcc &acc) {
    const uint4 *e = reinterpret_cast<const uint4 *>(a.nbr) + i;
    const int64_t n = a.n;
    const float w = a.cell_w;
    const int nb = (cnt + kListBatch - 1) / kListBatch;
    for (int b = 0; b < nb; ++b) {
        const uint4 e4 = __ldg(e + (int64_t)b * n);
        const uint32_t ent[kListBatch] = {e4.x, e4.y, e4.z, e4.w};
        float2 q[kListBatch];
#pragma unroll
        for (int u = 0; u < kListBatch; ++u) q[u] = __ldg(a.cl_in + (ent[u] & 0x0fffffffu));
#pragma unroll
        for (int u = 0; u < kListBatch; ++u) {
            float sx, sy;
            if (REGULAR) {
                const float2 o = tab[ent[u] >> 28];
                sx = o.x;
                sy = o.y;
            } else {
                const uint32_t ox = (ent[u] >> 28) & 3u, oy = ent[u] >> 30;
                sx = ox == 0u ? sxm : (ox == 2u ? sxp : (ox == 3u ? 2.0f * w : 0.0f));
                sy = oy == 0u ? sym : (oy == 2u ? syp : (oy == 3u ? 2.0f * w : 0.0f));
            }
            pair_term_masked<STATS, SF>(a, (p.x - q[u].x) - sx, (p.y - q[u].y) - sy, acc);
        }
    }
}

// The velocity-Verlet update of one particle for the launch mode, with its
// integer-step velocity vn (statistics) and squared half-step speed (MODE step).
template <int MODE>
__device__ __forceinline__ void integrate_one(const StepArgs &a, int64_t i, float2 p, float2 v,
                                              float fx, float fy, float2 &vn, float &vmax2) {
    if (MODE == kModeStep) {
        vn = make_float2(fmaf(fx, a.half_dt_m, v.x), fmaf(fy, a.half_dt_m, v.y));
        const float2 vh = make_float2(fmaf(fx, a.dt_m, v.x), fmaf(fy, a.dt_m, v.y));
        const float2 pn = make_float2(fmaf(vh.x, a.dt, p.x), fmaf(vh.y, a.dt, p.y));
        a.v_out[i] = vh;
        a.cl_out[i] = pn;
        vmax2 = fmaf(vh.x, vh.x, vh.y * vh.y);
        if (!(vmax2 < 3.0e38f) || !(fabsf(pn.x) < 3.0e38f) || !(fabsf(pn.y) < 3.0e38f))
            set_status(a.ctl, kErrNonFinite);
    } else if (MODE == kModeInit) {
        vn = v;
        a.v_out[i] = make_float2(fmaf(-fx, a.half_dt_m, v.x), fmaf(-fy, a.half_dt_m, v.y));
    } else {
        vn = make_float2(fmaf(fx, a.half_dt_m, v.x), fmaf(fy, a.half_dt_m, v.y));
        a.v_sync[i] = vn;
        if (a.f_sync) a.f_sync[i] = make_float2(fx, fy);
    }
}

// Integration, statistics and the launch-wide reductions of one step launch
// (everything after the forces), shared by the list and the tiled kernels.
// THREADS is the block size; every thread of every block of the launch calls
// it exactly once.
template <int MODE, bool STATS, bool B, int THREADS>
__device__ __forceinline__ void step_finish(const StepArgs &a, const SysView &sv, int64_t i,
                                            bool act, float2 p, float2 v, const PairAcc &acc,
                                            float D) {
    float2 vn = v;   // velocity at the integer step (statistics)
    float vmax2 = 0.f;
    if (act) integrate_one<MODE>(a, i, p, v, acc.fx, acc.fy, vn, vmax2);

    constexpr int kWarps = THREADS / 32;
    __shared__ long long s_red[kWarps][kStatsN];
    __shared__ float s_max[kWarps];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MODE == kModeStep) {
        const float m = warp_max(vmax2);
        if (lane == 0) s_max[warp] = m;
    }
    if (STATS) {
        // per-particle FP32 terms -> multiples of 2^-24 -> exact 64-bit sums
        float t[kStatsN] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (act) {
            t[0] = 0.5f * a.mass * fmaf(vn.x, vn.x, vn.y * vn.y);
            t[1] = 0.5f * acc.pe;
            t[2] = 0.5f * acc.vir;
            t[3] = a.mass * vn.x;
            t[4] = a.mass * vn.y;
        }
#pragma unroll
        for (int k = 0; k < kStatsN; ++k) {
            const long long r = warp_sum_ll(__float2ll_rn(t[k] * kFixScale));
            if (lane == 0) s_red[warp][k] = r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (MODE == kModeStep) {
            float m = 0.f;
            for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s_max[w]);
            atomicMax(&a.ctl->vmax2_bits, __float_as_uint(m));
        }
        if (STATS) {
            for (int k = 0; k < kStatsN; ++k) {
                long long t = 0;
                for (int w = 0; w < kWarps; ++w) t += s_red[w][k];
                // batched: a block is one chunk of one system.  Integer sums are
                // exact, so the order of these atomics does not matter
                atomicAdd(B ? (unsigned long long *)&a.batch.stats[sv.sys * kStatsN + k]
                            : (unsigned long long *)&a.ctl->stats_acc[k],
                          (unsigned long long)t);
            }
        }
        __threadfence();
        const unsigned ticket = atomicAdd(&a.ctl->done, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // Last block of the launch: every other block has published its results.
    __threadfence();
    if (STATS && !B && threadIdx.x < kStatsN) {
        // the launch's totals, and the accumulators back to zero for the next
        const long long t =
            (long long)atomicExch((unsigned long long *)&a.ctl->stats_acc[threadIdx.x], 0ull);
        a.ctl->stats[threadIdx.x] = (double)t * kFixInv;
    }
    if (threadIdx.x == 0) {
        if (MODE == kModeStep) {
            const uint32_t bits = atomicExch(&a.ctl->vmax2_bits, 0u);
            const float vmax = sqrtf(__uint_as_float(bits));
            a.ctl->dbound = D + vmax * a.dt * 1.000001f + a.round_margin;
        }
        a.ctl->done = 0u;
    }
}

// B: batched systems (geometry per 128-slot chunk, ghosts skipped, statistics
// per system); otherwise one system described by a.geo.
template <int MODE, bool STATS, bool B, bool SF>
__device__ __forceinline__ void step_body(const StepArgs &a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const SysView sv = sys_view<B>(a.geo, a.batch, i < a.n ? i : 0);
    const Geom &geo = sv.geo;
    const uint32_t cw = i < a.n ? a.cell[i] : kGhostCell;
    const bool act = i < a.n && (!B || cw != kGhostCell);
    // origin shifts ((c_x - 1) w, (c_y - 1) w) of the 16 list offset codes of a
    // regular neighbourhood (code 3: the padding entries' 2 w)
    __shared__ float2 s_tab[16];
    if (threadIdx.x < 16)
        s_tab[threadIdx.x] = make_float2(fmaf((float)(threadIdx.x & 3u), a.cell_w, -a.cell_w),
                                         fmaf((float)(threadIdx.x >> 2), a.cell_w, -a.cell_w));
    __syncthreads();

    // Neighbour-cell radius for the displacement bound of the input positions
    // (evaluated only where it is used: the cell-stencil path and the check).
    const float D = a.ctl->dbound;
    const auto stencil_radius = [&]() {
        const float Rf = ceilf((a.rc + 2.0f * D) / a.cell_w);
        // NaN -> 1; anything past the box is capped (stencil() then visits every cell once)
        return (Rf >= 1.0f) ? (Rf < 65536.0f ? (int)Rf : 65536) : 1;
    };
    if (a.potential && threadIdx.x == 0 && blockIdx.x == 0) {
        const int R = stencil_radius();
        if (2 * R + 1 > geo.nc[0] || 2 * R + 1 > geo.nc[1])
            set_status(a.ctl, kErrOverflow);   // cell list far out of date: whole box searched
    }
    // the Verlet list holds every pair that can be closer than rc while 2D <= skin
    const bool list_ok = a.nbr != nullptr && 2.0f * D <= a.list_skin;

    PairAcc acc = {0.f, 0.f, 0.f, 0.f};
    float2 p = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
    if (act) {
        p = a.cl_in[i];
        v = a.v_in[i];
        if (a.potential) {
            const int32_t cx = cell_x(cw), cy = cell_y(cw);
            const int cnt = list_ok ? a.ncount[i] : a.cap + 1;
            if (cnt <= a.cap) {
                // neighbouring cells of full width and no periodic wrap: shifts (code - 1) w
                if (cx >= 1 && cx + 2 <= geo.nc[0] && cy >= 1 && cy + 2 <= geo.nc[1]) {
                    forces_list<STATS, true, SF>(a, i, p, cnt, s_tab, 0.f, 0.f, 0.f, 0.f, acc);
                } else {
                    const float sxm = cell_shift(cx, -1, geo.nc[0], geo.k, geo.lg[0], geo.g);
                    const float sxp = cell_shift(cx, +1, geo.nc[0], geo.k, geo.lg[0], geo.g);
                    const float sym = cell_shift(cy, -1, geo.nc[1], geo.k, geo.lg[1], geo.g);
                    const float syp = cell_shift(cy, +1, geo.nc[1], geo.k, geo.lg[1], geo.g);
                    forces_list<STATS, false, SF>(a, i, p, cnt, s_tab, sxm, sxp, sym, syp, acc);
                }
            } else {
                const int R = stencil_radius();
                int lox, hix, loy, hiy;
                stencil(R, geo.nc[0], lox, hix);
                stencil(R, geo.nc[1], loy, hiy);
                forces_cells<STATS, SF>(a, geo, a.cell_start + sv.cell0, i, cx, cy, p, lox, hix, loy,
                                    hiy, acc);
            }
        }
    }
    step_finish<MODE, STATS, B, (B ? kChunk : kStepThreads)>(a, sv, i, act, p, v, acc, D);
}

// One system: 256-thread blocks, the register count left to the compiler.
template <int MODE, bool STATS, bool SF>
__global__ void __launch_bounds__(kStepThreads) k_step(StepArgs a) {
    step_body<MODE, STATS, false, SF>(a);
}

// A batch: one 128-slot chunk per block, 16 blocks per SM (32 registers: the
// per-chunk geometry would otherwise take the count to 40 and the occupancy
// to 48 warps; 4 % faster for the 256-system batch).
template <int MODE, bool STATS, bool SF>
__global__ void __launch_bounds__(kChunk, 16) k_step_batch(StepArgs a) {
    step_body<MODE, STATS, true, SF>(a);
}

// ---- neighbour-cell sort (counting sort keyed by MD cell, particle-number
//      order inside a cell) ---------------------------------------------------


template <bool B>
__global__ void k_sort_key(SortArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const SysView sv = sys_view<B>(a.geo, a.batch, i);
        const Geom &geo = sv.geo;
        const uint32_t cw = a.cell_in[i];
        uint32_t key = kGhostCell;
        int64_t c = sv.cell0 + sv.ncells;   // a system's ghost cell
        if (!B || cw != kGhostCell) {
            const float2 p = a.cl_in[i];
            const int32_t bx = base_cell(cell_x(cw) * geo.k, p.x, geo.inv_g, geo.lg[0]);
            const int32_t by = base_cell(cell_y(cw) * geo.k, p.y, geo.inv_g, geo.lg[1]);
            int32_t nx = bx / geo.k, ny = by / geo.k;
            nx = nx < geo.nc[0] ? nx : geo.nc[0] - 1;
            ny = ny < geo.nc[1] ? ny : geo.nc[1] - 1;
            key = (uint32_t)nx | ((uint32_t)ny << 16);
            c = sv.cell0 + ny * geo.nc[0] + nx;
        }
        a.key[i] = key;
        a.slot[i] = atomicAdd(&a.count[c], 1);
    }
}

// Exclusive scan of one 4096-entry chunk in place; chunk total to *total.
__device__ __forceinline__ void block_exclusive_scan(int32_t *data, int64_t base, int64_t m,
                                                     int32_t *total) {
    __shared__ int32_t s_warp[kScanThreads / 32];
    int32_t v[kScanItems];
    int32_t sum = 0;
    const int64_t o = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (o + k < m) ? data[o + k] : 0;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = s_warp[lane];
        int32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += t;
        }
        s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    int32_t run = s_warp[warp] + inc - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (o + k < m) data[o + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_local(int32_t *count, int64_t m,
                                                             int32_t *block_sums) {
    __shared__ int32_t total;
    block_exclusive_scan(count, (int64_t)blockIdx.x * kScanChunk, m, &total);
    __syncthreads();
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int32_t *block_sums, int64_t nb) {
    __shared__ int32_t total;
    block_exclusive_scan(block_sums, 0, nb, &total);
}

__device__ __forceinline__ int32_t cell_begin(const SortArgs &a, int64_t c) {
    return a.count[c] + a.block_sums[c / kScanChunk];
}

// Global cell of a sort key (the system's ghost cell for a ghost).
template <bool B>
__device__ __forceinline__ int64_t key_cell(const SysView &sv, uint32_t key) {
    if (B && key == kGhostCell) return sv.cell0 + sv.ncells;
    return sv.cell0 + cell_y(key) * sv.geo.nc[0] + cell_x(key);
}

template <bool B>
__global__ void k_sort_place(SortArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const SysView sv = sys_view<B>(a.geo, a.batch, i);
        const int64_t at = (int64_t)cell_begin(a, key_cell<B>(sv, a.key[i])) + a.slot[i];
        a.entry[at] = ((unsigned long long)(uint32_t)a.pid_in[i] << 32) | (uint32_t)i;
    }
}

// Cell start offsets (one thread per MD cell) and the reset of the
// displacement bound: after the sort every particle is inside its cell.
__global__ void k_cell_start(SortArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.cell_start[a.ncells] = (int32_t)a.n;
        a.ctl->dbound = 0.0f;
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.ncells; c += stride)
        a.cell_start[c] = cell_begin(a, c);
}

// One thread per slot of the new order: the particle that arrived in that slot
// finds its rank by particle number among its cell's arrivals, then is copied
// from the old order to its final place, its position re-expressed against the
// new cell's origin.
template <bool B>
__global__ void k_sort_scatter(SortArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += stride) {
        const SysView sv = sys_view<B>(a.geo, a.batch, t);
        const Geom &geo = sv.geo;
        const unsigned long long et = a.entry[t];
        const int32_t from = (int32_t)(et & 0xffffffffu);
        const uint32_t my_pid = (uint32_t)(et >> 32);
        // every gather from the old order first (independent of the rank), and
        // every load before any store (see k_bin_state)
        const uint32_t cw = a.key[from];
        const uint32_t ow = a.cell_in[from];
        const float2 p = a.cl_in[from];
        const float2 vv = a.v_in[from];
        const int32_t pid = a.pid_in[from];
        uint32_t lp[kMaxLags];
        float2 mp[kMaxLags];
        const bool msd = a.mprev_in[0] != nullptr;
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l) {
            lp[l] = l < a.nlags ? a.lprev_in[l][from] : 0u;
            mp[l] = (msd && l < a.nlags) ? a.mprev_in[l][from] : make_float2(0.f, 0.f);
        }
        const int64_t c = key_cell<B>(sv, cw);
        const int32_t s = a.cell_start[c], e = a.cell_start[c + 1];
        int32_t rank = 0;
        for (int32_t u = s; u < e; ++u) rank += (uint32_t)(a.entry[u] >> 32) < my_pid;
        const int32_t to = s + rank;
        float2 pn = p;
        float sx = 0.f, sy = 0.f;
        if (!B || cw != kGhostCell) {
            sx = (float)wrap_half((cell_x(ow) - cell_x(cw)) * geo.k, geo.lg[0]) * geo.g;
            sy = (float)wrap_half((cell_y(ow) - cell_y(cw)) * geo.k, geo.lg[1]) * geo.g;
            pn = make_float2(p.x + sx, p.y + sy);
        }
        a.cl_out[to] = pn;
        a.v_out[to] = vv;
        a.pid_out[to] = pid;
        a.cell_out[to] = cw;
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            if (l < a.nlags) {
                a.lprev_out[l][to] = lp[l];
                if (msd) a.mprev_out[l][to] = make_float2(mp[l].x + sx, mp[l].y + sy);
            }
    }
}

// Verlet list of the freshly sorted state: every j != i closer than the list
// radius, found in the 3 x 3 cell stencil (cells are at least that wide and
// every particle is inside its cell).  Candidates are fetched four at a time
// (predicated) so their loads overlap.  Every candidate's entry is written to
// the next free staging slot and the count advances only on a hit, so the
// lanes of a warp do not diverge over the test (staging holds cap + 1 slots per
// thread: entries past the capacity all land in the spare one, and such a list
// is not used).  Entry t of particle i is
// written to nbr[4 (floor(t/4) n + i) + t mod 4], padded to a multiple of four
// (see forces_list).  A particle with more than `cap` entries stores cap + 1 as
// its count and is handled through the cell stencil by the step kernel.
template <bool B>
__global__ void __launch_bounds__(kNlistThreads) k_nlist(SortArgs a) {
    // entries are staged in shared memory and written after the search, so
    // that no global store precedes a candidate load (see k_bin_state)
    extern __shared__ uint32_t s_ent[];          // blockDim.x x (cap + 1), column-major
    const int nt = blockDim.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < a.n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        int cnt = 0;
        const uint32_t cw = i < a.n ? a.cell_out[i] : kGhostCell;
        if (i < a.n && B && cw == kGhostCell) a.ncount[i] = 0;
        if (i < a.n && (!B || cw != kGhostCell)) {
            const SysView sv = sys_view<B>(a.geo, a.batch, i);
            const Geom &geo = sv.geo;
            const int32_t *cs = a.cell_start + sv.cell0;
            const int32_t cx = cell_x(cw), cy = cell_y(cw);
            const float2 p = a.cl_out[i];
            const int last = a.cap;   // spare staging slot: every entry past the capacity
            // x offsets of the three columns (wrapped at the periodic edges)
            const float sxm = (float)wrap_half((wrap_mod(cx - 1, geo.nc[0]) - cx) * geo.k, geo.lg[0]) * geo.g;
            const float sxp = (float)wrap_half((wrap_mod(cx + 1, geo.nc[0]) - cx) * geo.k, geo.lg[0]) * geo.g;
            const bool interior = cx >= 1 && cx + 1 < geo.nc[0];
            for (int oy = -1; oy <= 1; ++oy) {
                const int32_t ny = wrap_mod(cy + oy, geo.nc[1]);
                const float ody = (float)wrap_half((ny - cy) * geo.k, geo.lg[1]) * geo.g;
                const uint32_t ycode = (uint32_t)(oy + 1) << 30;
                const int32_t row = ny * geo.nc[0];
                if (interior) {
                    // cells cx-1, cx, cx+1 of this row are one contiguous range
                    const int32_t s = __ldg(cs + row + cx - 1);
                    const int32_t m1 = __ldg(cs + row + cx);
                    const int32_t m2 = __ldg(cs + row + cx + 1);
                    const int32_t e = __ldg(cs + row + cx + 2);
                    for (int32_t b = s; b < e; b += 4) {
                        float2 q[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            q[u] = (b + u < e) ? __ldg(a.cl_out + b + u)
                                               : make_float2(1.0e18f, 1.0e18f);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int32_t j = b + u;
                            const bool g1 = j >= m1, g2 = j >= m2;   // in cell cx, cx + 1
                            const float odx = g2 ? sxp : (g1 ? 0.0f : sxm);
                            const float dx = (p.x - q[u].x) - odx, dy = (p.y - q[u].y) - ody;
                            const bool hit = j < e && j != i && fmaf(dx, dx, dy * dy) < a.rl2;
                            s_ent[min(cnt, last) * nt + threadIdx.x] =
                                ((uint32_t)j | ycode) + (g1 ? (1u << 28) : 0u) + (g2 ? (1u << 28) : 0u);
                            cnt += hit;
                        }
                    }
                    continue;
                }
                for (int ox = -1; ox <= 1; ++ox) {
                    const int32_t nx = wrap_mod(cx + ox, geo.nc[0]);
                    const float odx = ox < 0 ? sxm : (ox > 0 ? sxp : 0.0f);
                    const int32_t cn = row + nx;
                    const int32_t s = __ldg(cs + cn), e = __ldg(cs + cn + 1);
                    const uint32_t code = ((uint32_t)(ox + 1) << 28) | ycode;
                    for (int32_t b = s; b < e; b += 4) {
                        float2 q[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            q[u] = (b + u < e) ? __ldg(a.cl_out + b + u)
                                               : make_float2(1.0e18f, 1.0e18f);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int32_t j = b + u;
                            const float dx = (p.x - q[u].x) - odx, dy = (p.y - q[u].y) - ody;
                            const bool hit = j < e && j != i && fmaf(dx, dx, dy * dy) < a.rl2;
                            s_ent[min(cnt, last) * nt + threadIdx.x] = (uint32_t)j | code;
                            cnt += hit;
                        }
                    }
                }
            }
            // batches of four entries, padded (cap is a multiple of the batch)
            if (cnt <= a.cap) {
                const uint32_t pad = (uint32_t)i | 0xf0000000u;
                uint4 *out = reinterpret_cast<uint4 *>(a.nbr) + i;
                for (int t = 0; t < cnt; t += kListBatch) {
                    uint32_t b[kListBatch];
#pragma unroll
                    for (int u = 0; u < kListBatch; ++u)
                        b[u] = t + u < cnt ? s_ent[(t + u) * nt + threadIdx.x] : pad;
                    out[(int64_t)(t / kListBatch) * a.n] = make_uint4(b[0], b[1], b[2], b[3]);
                }
            }
            a.ncount[i] = cnt <= a.cap ? cnt : a.cap + 1;
        }
    }
}

// ---- tiles: shared-memory windows of the sorted state ------------------------
//
// After each sort the slots of every MD-cell row are cut into tiles of up to
// kTileT slots (TileDesc).  The list build runs one block per tile and writes
// the tile's entries as window indices, grouped by step-kernel lane.  The step
// kernel is persistent: each block walks its share of the tiles, and while it
// computes one tile the next tile's window, own positions and velocities, lane
// table and entries are being copied into the other half of its shared memory
// by the TMA engine, so the pair loop only ever reads shared memory.

constexpr int kTileDescWords = (int)(sizeof(TileDesc) / sizeof(int32_t));
constexpr uint32_t kTileWaitPolls = 1u << 20;   // bounded wait for the staged copies
constexpr int kErrTimeout = -6;
constexpr int kStepTileThreads = kTileLanes;    // lane l takes ranks l and kTileT - 1 - l
constexpr uint8_t kNoSlot = 0xff;

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bulk copy (TMA engine) of `bytes` (a multiple of 16) from global memory
// to shared memory, both 16-byte aligned, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Wait for the barrier's phase `parity` to complete, polling at most `limit`
// times; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t k = 0; k < limit; ++k) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Elements staged for a segment: from its even first slot, rounded up to even.
__device__ __forceinline__ int32_t seg_staged(int32_t src, int32_t len) {
    return len > 0 ? (((src & 1) + len + 1) & ~1) : 0;
}

// Exclusive prefix of the tiles of cell rows before r (the scan of row_tiles).
__device__ __forceinline__ int32_t tile_prefix(const SortArgs &a, int64_t r) {
    return a.tile.row_tiles[r] + a.block_sums[r / kScanChunk];
}

// Tiles of every cell row, and a zero past the last row so that the scan also
// yields the total.
__global__ void k_tile_count(SortArgs a) {
    const int32_t ncx = a.geo.nc[0], ncy = a.geo.nc[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= ncy; r += stride) {
        int32_t t = 0;
        if (r < ncy) {
            const int32_t pop = a.cell_start[(r + 1) * ncx] - a.cell_start[r * ncx];
            t = (pop + kTileT - 1) / kTileT;
        }
        a.tile.row_tiles[r] = t;
    }
}

// One thread per tile: its slots, cell columns and window segments.
__global__ void k_tile_desc(SortArgs a) {
    const int32_t ncx = a.geo.nc[0], ncy = a.geo.nc[1];
    const int32_t *cs = a.cell_start;
    const int32_t total = tile_prefix(a, ncy);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.tile.ntiles = total;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        // the row: the last r whose prefix is <= t
        int32_t lo = 0, hi = ncy - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (tile_prefix(a, mid) <= t) lo = mid;
            else hi = mid - 1;
        }
        const int32_t r = lo, k = (int32_t)t - tile_prefix(a, r);
        const int32_t rs = cs[(int64_t)r * ncx], pop = cs[(int64_t)(r + 1) * ncx] - rs;
        TileDesc d;
        d.t0 = rs + k * kTileT;
        d.cnt = min(kTileT, pop - k * kTileT);
        d.ne = 0;
        d.row = r;
        d.cxa = cell_x(a.cell_out[d.t0]);
        d.cxb = cell_x(a.cell_out[d.t0 + d.cnt - 1]);
        const bool whole = d.cxb - d.cxa + 3 > ncx;
        d.whole = whole ? 1 : 0;
        int32_t off = 0;
        for (int oy = 0; oy < 3; ++oy) {
            const int64_t rb = (int64_t)wrap_mod(r + oy - 1, ncy) * ncx;
            int32_t s3[3], l3[3];
            if (whole) {
                s3[0] = s3[2] = 0;
                l3[0] = l3[2] = 0;
                s3[1] = cs[rb];
                l3[1] = cs[rb + ncx] - s3[1];
            } else {
                const int32_t clo = d.cxa > 0 ? d.cxa - 1 : 0;
                const int32_t chi = d.cxb + 1 < ncx ? d.cxb + 1 : ncx - 1;
                s3[0] = d.cxa == 0 ? cs[rb + ncx - 1] : 0;
                l3[0] = d.cxa == 0 ? cs[rb + ncx] - s3[0] : 0;
                s3[1] = cs[rb + clo];
                l3[1] = cs[rb + chi + 1] - s3[1];
                s3[2] = d.cxb == ncx - 1 ? cs[rb] : 0;
                l3[2] = d.cxb == ncx - 1 ? cs[rb + 1] - s3[2] : 0;
            }
            for (int q = 0; q < 3; ++q) {
                const int sg = 3 * oy + q;
                d.src[sg] = s3[q];
                d.len[sg] = l3[q];
                d.off[sg] = off;
                off += seg_staged(s3[q], l3[q]);
            }
        }
        d.wlen = off;
        for (int q = 0; q < 5; ++q) d.pad_[q] = 0;
        a.tile.desc[t] = d;
    }
}

// Window element of slot j of segment sg.
__device__ __forceinline__ int32_t win_index(const TileDesc &d, int sg, int32_t j) {
    return d.off[sg] + (d.src[sg] & 1) + (j - d.src[sg]);
}

// Slot of window element w (tiles whose window is not staged).
__device__ __forceinline__ int32_t win_slot(const TileDesc &d, int32_t w) {
    int32_t slot = 0;
#pragma unroll
    for (int sg = 0; sg < kTileSegs; ++sg) {
        const int32_t st = seg_staged(d.src[sg], d.len[sg]);
        if (w >= d.off[sg] && w < d.off[sg] + st) slot = (d.src[sg] & ~1) + (w - d.off[sg]);
    }
    return slot;
}

// Segment and cell column of the neighbouring column vc = cx + ox - 1 in
// window row oy.
__device__ __forceinline__ void win_cell(const TileDesc &d, int oy, int32_t vc, int32_t ncx,
                                         int &sg, int32_t &c) {
    if (!d.whole && vc < 0) {
        sg = 3 * oy;
        c = ncx - 1;
    } else if (!d.whole && vc >= ncx) {
        sg = 3 * oy + 2;
        c = 0;
    } else {
        sg = 3 * oy + 1;
        c = wrap_mod(vc, ncx);
    }
}

// Shift code (ShiftCode) of the neighbouring column or row c + o - 1,
// o in {0, 1, 2}, of a particle in column or row c of nc.
__device__ __forceinline__ uint32_t shift_code(int o, int32_t c, int32_t nc) {
    return o == 1 ? (uint32_t)kShiftZero
                  : (o == 0 ? (uint32_t)(c == 0 ? kShiftWrapMinus : kShiftMinus)
                            : (uint32_t)(c == nc - 1 ? kShiftWrapPlus : kShiftPlus));
}

// Verlet list of one tile per block in the tiled format.  Candidates come from
// the staged window; every entry is the neighbour's window index with its
// shift codes, staged per thread in shared memory (cap + 1 slots, the last one
// catching everything past the capacity).  The tile's particles are then
// ranked by entry count (ties by slot), lane l gets ranks l and kTileT-1-l,
// and the entries are written lane after lane, each lane's first particle
// first.  A window beyond kTileWinMax elements cannot be indexed: the tile's
// particles then take the cell stencil (lane counts kTileOverflow).
__global__ void __launch_bounds__(kTileT) k_nlist_tile(SortArgs a) {
    extern __shared__ uint16_t s_ent16[];        // kTileT x (cap + 1), column-major
    __shared__ __align__(16) float2 win[kTileWinMax];
    __shared__ __align__(16) TileDesc d;
    __shared__ int32_t s_cnt[kTileT];            // entries; -1: no particle, -2: overflowed
    __shared__ uint8_t s_rank_slot[kTileT];
    __shared__ int32_t s_dst[kTileT];
    __shared__ int32_t s_wsum[2];
    const int tid = threadIdx.x;
    const Geom &geo = a.geo;
    const int32_t ncx = geo.nc[0], ncy = geo.nc[1];
    const int32_t total = *a.tile.ntiles;
    const int64_t region = (int64_t)kTileT * a.cap;
    for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        if (tid < kTileDescWords)
            reinterpret_cast<int32_t *>(&d)[tid] = reinterpret_cast<const int32_t *>(a.tile.desc + tile)[tid];
        __syncthreads();
        const bool listable = d.wlen <= kTileWinMax;
        if (listable) {
            for (int sg = 0; sg < kTileSegs; ++sg) {
                const int32_t st = seg_staged(d.src[sg], d.len[sg]);
                const float2 *src = a.cl_out + (d.src[sg] & ~1);
                for (int e = tid; e < st; e += kTileT) win[d.off[sg] + e] = src[e];
            }
        }
        __syncthreads();
        int cnt = -1;
        if (tid < d.cnt) {
            const int64_t i = d.t0 + tid;
            const uint32_t cw = a.cell_out[i];
            const int32_t cx = cell_x(cw), cy = cell_y(cw);
            const float2 p = a.cl_out[i];
            const int last = a.cap;
            const float sxm = (float)wrap_half((wrap_mod(cx - 1, ncx) - cx) * geo.k, geo.lg[0]) * geo.g;
            const float sxp = (float)wrap_half((wrap_mod(cx + 1, ncx) - cx) * geo.k, geo.lg[0]) * geo.g;
            // the three neighbouring columns lie in one contiguous run of the
            // window row's main segment unless a wrapped cell is involved
            const bool run = !d.whole && cx >= 1 && cx + 1 < ncx;
            cnt = 0;
            // every row's cell boundaries are loaded before any candidate is
            // tested: the run's four boundaries, or (wrapped or whole rows) the
            // start of each of the three cells
            int32_t bnd[3][4];
#pragma unroll
            for (int oy = 0; oy < 3; ++oy) {
                const int64_t rb = (int64_t)wrap_mod(cy + oy - 1, ncy) * ncx;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    bnd[oy][q] = !listable ? 0
                                 : run ? __ldg(a.cell_start + rb + cx - 1 + q)
                                       : (q < 3 ? __ldg(a.cell_start + rb + wrap_mod(cx + q - 1, ncx)) : 0);
            }
#pragma unroll
            for (int oy = 0; oy < 3; ++oy) {
                if (!listable) break;
                const int32_t ry = wrap_mod(cy + oy - 1, ncy);
                const float ody = (float)wrap_half((ry - cy) * geo.k, geo.lg[1]) * geo.g;
                const uint32_t ycode = shift_code(oy, cy, ncy) << 13;
                if (run) {
                    // cells cx-1, cx, cx+1: window indices [w0, w0 + m), inner
                    // boundaries at the starts of cells cx and cx+1
                    const int32_t j0 = bnd[oy][0], m = bnd[oy][3] - j0;
                    const int32_t g1 = bnd[oy][1] - j0, g2 = bnd[oy][2] - j0;
                    const int32_t w0 = win_index(d, 3 * oy + 1, j0);
                    const int32_t islot = (int32_t)(i - j0);   // the particle itself, if in this run
                    const float2 *src = win + w0;
                    for (int32_t b = 0; b < m; b += 4) {
                        float2 q[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            q[u] = (b + u < m) ? src[b + u] : make_float2(1.0e18f, 1.0e18f);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int32_t k = b + u;
                            const bool in1 = k >= g1, in2 = k >= g2;
                            const float odx = in2 ? sxp : (in1 ? 0.0f : sxm);
                            const float dx = (p.x - q[u].x) - odx, dy = (p.y - q[u].y) - ody;
                            const bool hit = k < m && k != islot && fmaf(dx, dx, dy * dy) < a.rl2;
                            const uint32_t xcode = in2 ? (uint32_t)kShiftPlus
                                                       : (in1 ? (uint32_t)kShiftZero : (uint32_t)kShiftMinus);
                            s_ent16[min(cnt, last) * kTileT + tid] =
                                (uint16_t)((uint32_t)(w0 + k) | (xcode << 10) | ycode);
                            cnt += hit;
                        }
                    }
                    continue;
                }
                const int64_t rb = (int64_t)ry * ncx;
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    int sg;
                    int32_t c;
                    win_cell(d, oy, cx + ox - 1, ncx, sg, c);
                    const int32_t j0 = bnd[oy][ox], j1 = __ldg(a.cell_start + rb + c + 1);
                    const int32_t w0 = win_index(d, sg, j0);
                    const float odx = ox == 0 ? sxm : (ox == 2 ? sxp : 0.0f);
                    const uint32_t code = (shift_code(ox, cx, ncx) << 10) | ycode;
                    for (int32_t k = 0; k < j1 - j0; ++k) {
                        const float2 q = win[w0 + k];
                        const float dx = (p.x - q.x) - odx, dy = (p.y - q.y) - ody;
                        const bool hit = j0 + k != i && fmaf(dx, dx, dy * dy) < a.rl2;
                        s_ent16[min(cnt, last) * kTileT + tid] = (uint16_t)((uint32_t)(w0 + k) | code);
                        cnt += hit;
                    }
                }
            }
            const bool ovf = !listable || cnt > a.cap;
            a.ncount[i] = ovf ? a.cap + 1 : cnt;
            cnt = ovf ? -2 : cnt;
        }
        s_cnt[tid] = cnt;
        __syncthreads();
        // rank by entry count, most first (overflowed particles count as none)
        if (cnt != -1) {
            const int key = cnt < 0 ? 0 : cnt;
            int rank = 0;
            for (int j = 0; j < d.cnt; ++j) {
                const int kj = s_cnt[j] < 0 ? 0 : s_cnt[j];
                rank += (kj > key) || (kj == key && j < tid);
            }
            s_rank_slot[rank] = (uint8_t)tid;
        }
        __syncthreads();
        // lane table: lane l takes ranks l and kTileT-1-l; its entries at the
        // exclusive prefix of the lane sums
        int lsum = 0;
        uint8_t sa = kNoSlot, sb = kNoSlot;
        uint16_t ca = 0, cb = 0;
        if (tid < kTileLanes) {
            const int rb = kTileT - 1 - tid;
            if (tid < d.cnt) {
                sa = s_rank_slot[tid];
                const int c = s_cnt[sa];
                ca = c == -2 ? kTileOverflow : (uint16_t)c;
                lsum += c > 0 ? c : 0;
            }
            if (rb < d.cnt) {
                sb = s_rank_slot[rb];
                const int c = s_cnt[sb];
                cb = c == -2 ? kTileOverflow : (uint16_t)c;
                lsum += c > 0 ? c : 0;
            }
        }
        // exclusive scan over the kTileLanes lanes (two warps)
        const int lane = tid & 31, warp = tid >> 5;
        int inc = lsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31 && warp < 2) s_wsum[warp] = inc;
        __syncthreads();
        if (tid < kTileLanes) {
            const int off = inc - lsum + (warp == 1 ? s_wsum[0] : 0);
            if (sa != kNoSlot) s_dst[sa] = off;
            if (sb != kNoSlot) s_dst[sb] = off + (ca == kTileOverflow ? 0 : ca);
            TileLane ln;
            ln.a = sa;
            ln.b = sb;
            ln.ca = ca;
            ln.cb = cb;
            ln.off = (uint16_t)off;
            a.tile.lanes[tile * kTileLanes + tid] = ln;
            if (tid == kTileLanes - 1) a.tile.desc[tile].ne = off + lsum;
        }
        __syncthreads();
        if (cnt > 0) {
            uint16_t *dst = a.tile.list + tile * region + s_dst[tid];
            for (int k = 0; k < cnt; ++k) dst[k] = s_ent16[k * kTileT + tid];
        }
        __syncthreads();   // the next tile reuses the shared arrays
    }
}

// Per-block reductions of a persistent step launch (every thread once):
// the largest squared speed and the exact statistics sums of the block's
// particles go to the control block; the last block publishes the launch's
// totals and the new displacement bound.
template <int MODE, bool STATS>
__device__ __forceinline__ void tile_finish(const StepArgs &a, float vmax2, const long long *lsum,
                                            float D) {
    constexpr int kWarps = kStepTileThreads / 32;
    __shared__ long long s_red[kWarps][kStatsN];
    __shared__ float s_max[kWarps];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MODE == kModeStep) {
        const float m = warp_max(vmax2);
        if (lane == 0) s_max[warp] = m;
    }
    if (STATS) {
#pragma unroll
        for (int k = 0; k < kStatsN; ++k) {
            const long long r = warp_sum_ll(lsum[k]);
            if (lane == 0) s_red[warp][k] = r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (MODE == kModeStep) {
            float m = 0.f;
            for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s_max[w]);
            atomicMax(&a.ctl->vmax2_bits, __float_as_uint(m));
        }
        if (STATS) {
            for (int k = 0; k < kStatsN; ++k) {
                long long t = 0;
                for (int w = 0; w < kWarps; ++w) t += s_red[w][k];
                atomicAdd((unsigned long long *)&a.ctl->stats_acc[k], (unsigned long long)t);
            }
        }
        __threadfence();
        const unsigned ticket = atomicAdd(&a.ctl->done, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (STATS && threadIdx.x < kStatsN) {
        const long long t =
            (long long)atomicExch((unsigned long long *)&a.ctl->stats_acc[threadIdx.x], 0ull);
        a.ctl->stats[threadIdx.x] = (double)t * kFixInv;
    }
    if (threadIdx.x == 0) {
        if (MODE == kModeStep) {
            const uint32_t bits = atomicExch(&a.ctl->vmax2_bits, 0u);
            const float vmax = sqrtf(__uint_as_float(bits));
            a.ctl->dbound = D + vmax * a.dt * 1.000001f + a.round_margin;
        }
        a.ctl->done = 0u;
    }
}

// Shared-memory layout of one stage of the persistent step kernel.
struct TileStage {
    static constexpr int kWin = 0;                                        // float2[kTileWinCap]
    static constexpr int kCl = kWin + 8 * kTileWinCap;                    // float2[kTileT + 2]
    static constexpr int kV = kCl + 8 * (kTileT + 2);                     // float2[kTileT + 2]
    static constexpr int kLanes = kV + 8 * (kTileT + 2);                  // TileLane[kTileLanes]
    static constexpr int kList = kLanes + (int)sizeof(TileLane) * kTileLanes;   // uint16[list_stage]
    static __host__ __device__ int bytes(int list_stage) {
        return kList + ((2 * list_stage + 15) & ~15);
    }
};

// Issue the copies of tile `tile` into stage buffer `st` (one thread).  The
// window and the entries are staged only when the list is in use; own
// positions, velocities and the lane table always.
__device__ __forceinline__ void tile_issue(const StepArgs &a, const TileDesc &d, int64_t tile,
                                           unsigned char *st, uint64_t *bar, bool use_list) {
    const int32_t a0 = d.t0 & 1;
    const uint32_t own = 8u * (uint32_t)((a0 + d.cnt + 1) & ~1);
    const bool win = use_list && d.wlen <= kTileWinCap;
    const int32_t nst = use_list ? min(d.ne, a.tile.list_stage) : 0;
    const uint32_t lbytes = (uint32_t)((2 * nst + 15) & ~15);
    uint32_t bytes = 2u * own + (uint32_t)sizeof(TileLane) * kTileLanes + lbytes;
    if (win)
        for (int sg = 0; sg < kTileSegs; ++sg) bytes += 8u * (uint32_t)seg_staged(d.src[sg], d.len[sg]);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(st + TileStage::kCl, a.cl_in + (d.t0 - a0), own, bar);
    bulk_g2s(st + TileStage::kV, a.v_in + (d.t0 - a0), own, bar);
    bulk_g2s(st + TileStage::kLanes, a.tile.lanes + tile * kTileLanes,
             (uint32_t)sizeof(TileLane) * kTileLanes, bar);
    if (lbytes) bulk_g2s(st + TileStage::kList, a.tile.list + tile * (int64_t)kTileT * a.cap, lbytes, bar);
    if (win) {
        for (int sg = 0; sg < kTileSegs; ++sg) {
            const int32_t ns = seg_staged(d.src[sg], d.len[sg]);
            if (ns > 0)
                bulk_g2s(st + TileStage::kWin + 8 * d.off[sg], a.cl_in + (d.src[sg] & ~1), 8u * (uint32_t)ns, bar);
        }
    }
}

// Pairs of one particle from its entries [e0, e0 + c) of the tile's list.
template <bool STATS, bool SF, bool WIN>
__device__ __forceinline__ void forces_tile(const StepArgs &a, const TileDesc &d, int64_t tile,
                                            const unsigned char *st, const float2 *tab, float2 p,
                                            int e0, int c, PairAcc &acc) {
    const uint16_t *sl = reinterpret_cast<const uint16_t *>(st + TileStage::kList);
    const float2 *win = reinterpret_cast<const float2 *>(st + TileStage::kWin);
    const uint16_t *gl = a.tile.list + tile * (int64_t)kTileT * a.cap;
    const int nst = min(d.ne, a.tile.list_stage);
    const int e1 = e0 + c;
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
        const uint32_t ent = e < nst ? sl[e] : gl[e];
        const int32_t wi = (int32_t)(ent & 0x3ffu);
        const float2 q = WIN ? win[wi] : __ldg(a.cl_in + win_slot(d, wi));
        const float2 sh = tab[ent >> 10];
        pair_term_masked<STATS, SF>(a, (p.x - q.x) - sh.x, (p.y - q.y) - sh.y, acc);
    }
}

// Step kernel of a tiled context, persistent: block b computes tiles b,
// b + gridDim.x, ...  While it computes one, the copies of its next tile are
// in flight into the other stage buffer; the descriptor after that is loaded
// into registers one tile ahead.  Lane l of the block handles the particles
// of ranks l and kTileT-1-l of the tile.  Statistics and the speed bound are
// accumulated over all of a block's particles and reduced once.
template <int MODE, bool STATS, bool SF>
__global__ void __launch_bounds__(kStepTileThreads) k_step_tile(StepArgs a) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ __align__(16) TileDesc s_desc[2];
    __shared__ float2 s_tab[64];
    const int tid = threadIdx.x;
    const Geom &geo = a.geo;
    const int stage_bytes = TileStage::bytes(a.tile.list_stage);
    const int32_t total = *a.tile.ntiles;
    const int64_t G = gridDim.x;
    {
        // origin shift of every (x code, y code) pair (ShiftCode)
        const float w = a.cell_w;
        const float wlx = (float)(geo.lg[0] - (geo.nc[0] - 1) * geo.k) * geo.g;
        const float wly = (float)(geo.lg[1] - (geo.nc[1] - 1) * geo.k) * geo.g;
        const int xc = tid & 7, yc = tid >> 3;
        const auto shift_of = [&](int code, float wl) {
            return code == kShiftMinus ? -w : code == kShiftPlus ? w
                 : code == kShiftWrapMinus ? -wl : code == kShiftWrapPlus ? wl : 0.f;
        };
        s_tab[tid] = make_float2(shift_of(xc, wlx), shift_of(yc, wly));
    }
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
    }
    const float D = a.ctl->dbound;
    const auto stencil_radius = [&]() {
        const float Rf = ceilf((a.rc + 2.0f * D) / a.cell_w);
        return (Rf >= 1.0f) ? (Rf < 65536.0f ? (int)Rf : 65536) : 1;
    };
    if (a.potential && tid == 0 && blockIdx.x == 0) {
        const int R = stencil_radius();
        if (2 * R + 1 > geo.nc[0] || 2 * R + 1 > geo.nc[1]) set_status(a.ctl, kErrOverflow);
    }
    const bool use_list = a.potential && a.tile.list != nullptr && 2.0f * D <= a.list_skin;
    int lox = 0, hix = 0, loy = 0, hiy = 0;
    if (a.potential && !use_list) {
        const int R = stencil_radius();
        stencil(R, geo.nc[0], lox, hix);
        stencil(R, geo.nc[1], loy, hiy);
    }
    int64_t t = blockIdx.x;
    if (t < total && tid < kTileDescWords)
        reinterpret_cast<int32_t *>(&s_desc[0])[tid] = reinterpret_cast<const int32_t *>(a.tile.desc + t)[tid];
    __syncthreads();   // barriers initialised, first descriptor in place
    if (t < total && tid == 0) tile_issue(a, s_desc[0], t, s_dyn, &s_bar[0], use_list);
    // the descriptor after the next one travels one tile ahead in registers
    int32_t dnext = (t + G < total && tid < kTileDescWords)
                        ? reinterpret_cast<const int32_t *>(a.tile.desc + t + G)[tid] : 0;

    float vmax2 = 0.f;
    long long lsum[kStatsN] = {0, 0, 0, 0, 0};
    bool timed_out = false;
    for (int k = 0; t < total; ++k, t += G) {
        const int s = k & 1;
        unsigned char *st = s_dyn + s * stage_bytes;
        const int64_t tn = t + G;
        if (tn < total) {
            if (tid < kTileDescWords) reinterpret_cast<int32_t *>(&s_desc[s ^ 1])[tid] = dnext;
            __syncthreads();
            if (tid == 0)
                tile_issue(a, s_desc[s ^ 1], tn, s_dyn + (s ^ 1) * stage_bytes, &s_bar[s ^ 1], use_list);
            dnext = (tn + G < total && tid < kTileDescWords)
                        ? reinterpret_cast<const int32_t *>(a.tile.desc + tn + G)[tid] : 0;
        }
        if (!mbar_wait(&s_bar[s], (uint32_t)((k >> 1) & 1), kTileWaitPolls)) timed_out = true;
        const TileDesc &d = s_desc[s];
        const bool win = d.wlen <= kTileWinCap;
        const TileLane ln = reinterpret_cast<const TileLane *>(st + TileStage::kLanes)[tid];
        const float2 *scl = reinterpret_cast<const float2 *>(st + TileStage::kCl) + (d.t0 & 1);
        const float2 *sv = reinterpret_cast<const float2 *>(st + TileStage::kV) + (d.t0 & 1);
        int e0 = ln.off;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const uint8_t slot = h == 0 ? ln.a : ln.b;
            const uint16_t c = h == 0 ? ln.ca : ln.cb;
            if (slot == kNoSlot) continue;
            const int64_t i = (int64_t)d.t0 + slot;
            const float2 p = scl[slot], v = sv[slot];
            PairAcc acc = {0.f, 0.f, 0.f, 0.f};
            if (a.potential) {
                if (use_list && c != kTileOverflow) {
                    if (win) forces_tile<STATS, SF, true>(a, d, t, st, s_tab, p, e0, c, acc);
                    else forces_tile<STATS, SF, false>(a, d, t, st, s_tab, p, e0, c, acc);
                    e0 += c;
                } else {
                    int lx = lox, hx = hix, ly = loy, hy = hiy;
                    if (use_list) {   // this particle's list overflowed: the current bound's stencil
                        const int R = stencil_radius();
                        stencil(R, geo.nc[0], lx, hx);
                        stencil(R, geo.nc[1], ly, hy);
                    }
                    const uint32_t cw = a.cell[i];
                    forces_cells<STATS, SF>(a, geo, a.cell_start, i, cell_x(cw), cell_y(cw), p, lx, hx,
                                            ly, hy, acc);
                }
            }
            float2 vn = v;
            float m2 = 0.f;
            integrate_one<MODE>(a, i, p, v, acc.fx, acc.fy, vn, m2);
            vmax2 = fmaxf(vmax2, m2);
            if (STATS) {
                const float tt[kStatsN] = {0.5f * a.mass * fmaf(vn.x, vn.x, vn.y * vn.y), 0.5f * acc.pe,
                                           0.5f * acc.vir, a.mass * vn.x, a.mass * vn.y};
#pragma unroll
                for (int q = 0; q < kStatsN; ++q) lsum[q] += __float2ll_rn(tt[q] * kFixScale);
            }
        }
        __syncthreads();   // this stage and its descriptor are free for the tile after next
    }
    if (timed_out) set_status(a.ctl, kErrTimeout);
    tile_finish<MODE, STATS>(a, vmax2, lsum, D);
}

// ---- upload / download conversions ----------------------------------------

// Largest |v|^2 of the block's uploaded velocities into ctl->vmax0_bits: the
// bits of non-negative doubles order like the values, so an integer max is
// exact and independent of the order of the blocks.  Every thread calls it.
__device__ void block_max_speed2(double s2, Control *ctl) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 = fmax(s2, __shfl_xor_sync(0xffffffffu, s2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomicMax(&ctl->vmax0_bits, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_pack(Geom geo, int64_t n, const double *x, const double *v, uint32_t *cell,
                       float2 *cl, float2 *vel, int32_t *pid, Control *ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s2 = 0.0;   // largest |v|^2 seen by this thread
    const double g = geo.g, inv_g = geo.inv_g;   // g a power of two: x * (1/g) is exact
    const double L0 = (double)geo.lg[0] * g, L1 = (double)geo.lg[1] * g;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double px = x[2 * i], py = x[2 * i + 1];
        if (!(px > 0.0 && px <= L0 && py > 0.0 && py <= L1) || !isfinite(v[2 * i]) ||
            !isfinite(v[2 * i + 1])) {
            set_status(ctl, kErrNonFinite);
        }
        // base cell b with b g < x <= (b+1) g
        int64_t bx = (int64_t)ceil(px * inv_g) - 1, by = (int64_t)ceil(py * inv_g) - 1;
        bx = bx < 0 ? 0 : (bx >= geo.lg[0] ? geo.lg[0] - 1 : bx);
        by = by < 0 ? 0 : (by >= geo.lg[1] ? geo.lg[1] - 1 : by);
        int32_t cx = (int32_t)(bx / geo.k), cy = (int32_t)(by / geo.k);
        cx = cx < geo.nc[0] ? cx : geo.nc[0] - 1;
        cy = cy < geo.nc[1] ? cy : geo.nc[1] - 1;
        cell[i] = (uint32_t)cx | ((uint32_t)cy << 16);
        cl[i] = make_float2((float)(px - (double)(cx * geo.k) * g),
                            (float)(py - (double)(cy * geo.k) * g));
        vel[i] = make_float2((float)v[2 * i], (float)v[2 * i + 1]);
        pid[i] = (int32_t)i;
        s2 = fmax(s2, __dadd_rn(__dmul_rn(v[2 * i], v[2 * i]), __dmul_rn(v[2 * i + 1], v[2 * i + 1])));
    }
    block_max_speed2(s2, ctl);
}

// Batched upload: slot t of system s holds particle q0 + (t - p0) of the
// caller's concatenated arrays, or a ghost in the padding.
__global__ void k_pack_batch(Batch b, int64_t slots, const double *x, const double *v,
                             uint32_t *cell, float2 *cl, float2 *vel, int32_t *pid, Control *ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s2 = 0.0;   // largest |v|^2 seen by this thread
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < slots; t += stride) {
        const SysInfo &si = b.sys[b.chunk_sys[t / kChunk]];
        const Geom &geo = si.geo;
        const int64_t local = t - si.p0;
        if (local >= si.n) {
            // ghosts need distinct particle numbers: the sort ranks a cell's
            // particles by number, and equal numbers would share a slot
            cell[t] = kGhostCell;
            cl[t] = make_float2(0.f, 0.f);
            vel[t] = make_float2(0.f, 0.f);
            pid[t] = -1 - (int32_t)(local - si.n);
            continue;
        }
        const int64_t q = si.q0 + local;
        const double g = geo.g, inv_g = geo.inv_g;
        const double L0 = (double)geo.lg[0] * g, L1 = (double)geo.lg[1] * g;
        const double px = x[2 * q], py = x[2 * q + 1];
        if (!(px > 0.0 && px <= L0 && py > 0.0 && py <= L1) || !isfinite(v[2 * q]) ||
            !isfinite(v[2 * q + 1]))
            set_status(ctl, kErrNonFinite);
        int64_t bx = (int64_t)ceil(px * inv_g) - 1, by = (int64_t)ceil(py * inv_g) - 1;
        bx = bx < 0 ? 0 : (bx >= geo.lg[0] ? geo.lg[0] - 1 : bx);
        by = by < 0 ? 0 : (by >= geo.lg[1] ? geo.lg[1] - 1 : by);
        int32_t cx = (int32_t)(bx / geo.k), cy = (int32_t)(by / geo.k);
        cx = cx < geo.nc[0] ? cx : geo.nc[0] - 1;
        cy = cy < geo.nc[1] ? cy : geo.nc[1] - 1;
        cell[t] = (uint32_t)cx | ((uint32_t)cy << 16);
        cl[t] = make_float2((float)(px - (double)(cx * geo.k) * g),
                            (float)(py - (double)(cy * geo.k) * g));
        vel[t] = make_float2((float)v[2 * q], (float)v[2 * q + 1]);
        pid[t] = (int32_t)q;
        s2 = fmax(s2, __dadd_rn(__dmul_rn(v[2 * q], v[2 * q]), __dmul_rn(v[2 * q + 1], v[2 * q + 1])));
    }
    block_max_speed2(s2, ctl);
}

template <bool B>
__global__ void k_unpack(Geom single, Batch batch, int64_t n, const uint32_t *cell,
                         const float2 *cl, const float2 *vsync, const float2 *fsync,
                         const int32_t *pid, double *x, double *v, double *f) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t cw = cell[j];
        if (B && cw == kGhostCell) continue;
        const SysView sv = sys_view<B>(single, batch, j);
        const Geom &geo = sv.geo;
        const double g = geo.g;
        const double L0 = (double)geo.lg[0] * g, L1 = (double)geo.lg[1] * g;
        const float2 p = cl[j];
        double px = (double)(cell_x(cw) * geo.k) * g + (double)p.x;
        double py = (double)(cell_y(cw) * geo.k) * g + (double)p.y;
        px = px <= 0.0 ? px + L0 : (px > L0 ? px - L0 : px);
        py = py <= 0.0 ? py + L1 : (py > L1 ? py - L1 : py);
        const int64_t o = pid[j];
        if (x) { x[2 * o] = px; x[2 * o + 1] = py; }
        if (v) { const float2 w = vsync[j]; v[2 * o] = w.x; v[2 * o + 1] = w.y; }
        if (f) { const float2 w = fsync[j]; f[2 * o] = w.x; f[2 * o + 1] = w.y; }
    }
}

int grid_for(int64_t n, int threads, int per_sm = 8) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t need = (n + threads - 1) / threads;
    int64_t g = (int64_t)sms * per_sm;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <int MODE, bool STATS, bool B, bool SF>
void launch_step_k(const StepArgs &a, dim3 grid, dim3 block, cudaStream_t s) {
    if (B) k_step_batch<MODE, STATS, SF><<<grid, block, 0, s>>>(a);
    else k_step<MODE, STATS, SF><<<grid, block, 0, s>>>(a);
}

template <bool B, bool SF>
void launch_step_t(const StepArgs &a, int mode, dim3 grid, dim3 block, cudaStream_t s) {
    if (mode == kModeStep) {
        if (a.stats) launch_step_k<kModeStep, true, B, SF>(a, grid, block, s);
        else launch_step_k<kModeStep, false, B, SF>(a, grid, block, s);
    } else if (mode == kModeInit) {
        launch_step_k<kModeInit, true, B, SF>(a, grid, block, s);
    } else {
        launch_step_k<kModeSync, true, B, SF>(a, grid, block, s);
    }
}

// Persistent launch: as many blocks as fit on the device at once (at most one per tile).
template <int MODE, bool STATS, bool SF>
cudaError_t launch_tile_k(const StepArgs &a, cudaStream_t s) {
    void (*kern)(StepArgs) = k_step_tile<MODE, STATS, SF>;
    const size_t smem = 2 * (size_t)TileStage::bytes(a.tile.list_stage);
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kStepTileThreads, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)sms * (per > 0 ? per : 1);
    if (grid > a.tile.max_tiles) grid = a.tile.max_tiles;
    kern<<<(unsigned)(grid < 1 ? 1 : grid), kStepTileThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool SF>
cudaError_t launch_step_tile_t(const StepArgs &a, int mode, cudaStream_t s) {
    if (mode == kModeStep)
        return a.stats ? launch_tile_k<kModeStep, true, SF>(a, s) : launch_tile_k<kModeStep, false, SF>(a, s);
    if (mode == kModeInit) return launch_tile_k<kModeInit, true, SF>(a, s);
    return launch_tile_k<kModeSync, true, SF>(a, s);
}

cudaError_t launch_step(const StepArgs &a, int mode, cudaStream_t s) {
    if (!a.batch.sys && a.tile.desc)
        return a.potential == 2 ? launch_step_tile_t<true>(a, mode, s) : launch_step_tile_t<false>(a, mode, s);
    const int threads = a.batch.sys ? kChunk : kStepThreads;
    const int64_t blocks = (a.n + threads - 1) / threads;
    if (blocks < 1) return cudaSuccess;
    const dim3 grid((unsigned)blocks), block(threads);
    const bool sf = a.potential == 2;
    if (a.batch.sys) {
        if (sf) launch_step_t<true, true>(a, mode, grid, block, s);
        else launch_step_t<true, false>(a, mode, grid, block, s);
    } else {
        if (sf) launch_step_t<false, true>(a, mode, grid, block, s);
        else launch_step_t<false, false>(a, mode, grid, block, s);
    }
    return cudaGetLastError();
}

int64_t sort_scratch_blocks(int64_t ncells) { return (ncells + kScanChunk - 1) / kScanChunk; }

template <bool B>
cudaError_t launch_sort_t(const SortArgs &a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.count, 0, sizeof(int32_t) * (size_t)a.ncells, s);
    if (e != cudaSuccess) return e;
    const int t = 256;
    k_sort_key<B><<<grid_for(a.n, t), t, 0, s>>>(a);
    const int64_t nb = sort_scratch_blocks(a.ncells);
    k_scan_local<<<(unsigned)nb, kScanThreads, 0, s>>>(a.count, a.ncells, a.block_sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(a.block_sums, nb);
    k_sort_place<B><<<grid_for(a.n, t), t, 0, s>>>(a);
    k_cell_start<<<grid_for(a.ncells, t), t, 0, s>>>(a);
    k_sort_scatter<B><<<grid_for(a.n, t, 16), t, 0, s>>>(a);
    if (!B && a.tile.desc) {
        // tiles of the new order (the cell scan's block sums are free again
        // and hold the row scan's), then the tiled list
        const int32_t rows = a.geo.nc[1];
        k_tile_count<<<grid_for(rows + 1, t), t, 0, s>>>(a);
        const int64_t nbr = sort_scratch_blocks(rows + 1);
        k_scan_local<<<(unsigned)nbr, kScanThreads, 0, s>>>(a.tile.row_tiles, rows + 1, a.block_sums);
        k_scan_top<<<1, kScanThreads, 0, s>>>(a.block_sums, nbr);
        k_tile_desc<<<grid_for(a.tile.max_tiles, t), t, 0, s>>>(a);
        const size_t smem = sizeof(uint16_t) * (size_t)kTileT * (a.cap + 1);
        if (smem > 32 * 1024) {
            e = cudaFuncSetAttribute(k_nlist_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_nlist_tile<<<grid_for(a.tile.max_tiles, kTileT, 16), kTileT, smem, s>>>(a);
        return cudaGetLastError();
    }
    if (a.nbr) {
        const int nt = (size_t)kNlistThreads * (a.cap + 1) * sizeof(uint32_t) <= 96 * 1024 ? kNlistThreads : 64;
        const size_t smem = sizeof(uint32_t) * (size_t)nt * (a.cap + 1);
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_nlist<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_nlist<B><<<grid_for(a.n, nt, 32), nt, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_nlist(const SortArgs &a, cudaStream_t s) {
    const int nt = (size_t)kNlistThreads * (a.cap + 1) * sizeof(uint32_t) <= 96 * 1024 ? kNlistThreads : 64;
    const size_t smem = sizeof(uint32_t) * (size_t)nt * (a.cap + 1);
    void (*kern)(SortArgs) = a.batch.sys ? k_nlist<true> : k_nlist<false>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid_for(a.n, nt, 32), nt, smem, s>>>(a);
    return cudaGetLastError();
}

int64_t max_tiles(int64_t n, int32_t rows) { return n / kTileT + rows + 1; }

// In a batch, a.ncells counts every system's cells plus its ghost cell.
cudaError_t launch_sort(const SortArgs &a, cudaStream_t s) {
    return a.batch.sys ? launch_sort_t<true>(a, s) : launch_sort_t<false>(a, s);
}

cudaError_t launch_pack(const Geom &geo, int64_t n, const double *x, const double *v,
                        uint32_t *cell, float2 *cl, float2 *vel, int32_t *pid, Control *ctl,
                        cudaStream_t s) {
    k_pack<<<grid_for(n, 256), 256, 0, s>>>(geo, n, x, v, cell, cl, vel, pid, ctl);
    return cudaGetLastError();
}

cudaError_t launch_pack_batch(const Batch &b, int64_t slots, const double *x, const double *v,
                              uint32_t *cell, float2 *cl, float2 *vel, int32_t *pid, Control *ctl,
                              cudaStream_t s) {
    k_pack_batch<<<grid_for(slots, 256), 256, 0, s>>>(b, slots, x, v, cell, cl, vel, pid, ctl);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom &geo, int64_t n, const uint32_t *cell, const float2 *cl,
                          const float2 *vsync, const float2 *fsync, const int32_t *pid,
                          double *x, double *v, double *f, cudaStream_t s, const Batch *batch) {
    const Batch b = batch ? *batch : Batch{};
    if (b.sys)
        k_unpack<true><<<grid_for(n, 256), 256, 0, s>>>(geo, b, n, cell, cl, vsync, fsync, pid, x, v, f);
    else
        k_unpack<false><<<grid_for(n, 256), 256, 0, s>>>(geo, b, n, cell, cl, vsync, fsync, pid, x, v, f);
    return cudaGetLastError();
}

}  // namespace mdlg
