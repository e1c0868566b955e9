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
// plain steps: resident blocks per SM of the looping kernels (at 32 registers,
// 8 of 256 threads or 16 of one 128-slot chunk fill an SM)
constexpr int kStepLoopBlocksPerSM = 8;
constexpr int kStepBatchBlocksPerSM = 16;
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

// Two list entries A and B at once, on packed binary32 pairs (the f32x2
// arithmetic of sm_100 and later: one instruction for two lanes' worth of
// work).  Each entry's separation is the float2 (cl_i - cl_j) - shift, formed
// as p + (-1) q (exact product, one rounding: the subtraction) plus the
// negated origin shift; the Lennard-Jones factor chain then runs on the pair
// (entry A, entry B).  Every component is rounded exactly as in
// pair_term_masked, in the same order, so the forces are the same bit for bit.
template <bool STATS, bool SF>
__device__ __forceinline__ void pair_terms2_masked(const StepArgs &a, float2 p, float2 qA, float2 nsA,
                                                   float2 qB, float2 nsB, PairAcc &acc) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 dA = __fadd2_rn(__ffma2_rn(qA, m1, p), nsA);
    const float2 dB = __fadd2_rn(__ffma2_rn(qB, m1, p), nsB);
    const float r2A = fmaf(dA.x, dA.x, dA.y * dA.y), r2B = fmaf(dB.x, dB.x, dB.y * dB.y);
    const bool onA = r2A < a.rc2, onB = r2B < a.rc2;
    const float2 ir2 = make_float2(__fdividef(1.0f, r2A), __fdividef(1.0f, r2B));   // hardware reciprocal
    const float2 sr2 = __fmul2_rn(make_float2(a.sig2, a.sig2), ir2);
    const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
    float2 fs = __fmul2_rn(__fmul2_rn(__fmul2_rn(make_float2(a.eps24, a.eps24), ir2), sr6),
                           __ffma2_rn(make_float2(2.0f, 2.0f), sr6, m1));
    if (SF) {              // shifted force: subtract F(rc) along the pair
        fs.x -= a.fc * rsqrtf(r2A);
        fs.y -= a.fc * rsqrtf(r2B);
    }
    fs.x = onA ? fs.x : 0.0f;
    fs.y = onB ? fs.y : 0.0f;
    float2 f = make_float2(acc.fx, acc.fy);
    f = __ffma2_rn(make_float2(fs.x, fs.x), dA, f);
    f = __ffma2_rn(make_float2(fs.y, fs.y), dB, f);
    acc.fx = f.x;
    acc.fy = f.y;
    if (STATS) {
        float2 e = __fadd2_rn(__fmul2_rn(__fmul2_rn(make_float2(a.eps4, a.eps4), sr6),
                                         __fadd2_rn(sr6, m1)),
                              make_float2(-a.vshift, -a.vshift));
        if (SF) {          // + (r - rc) F(rc)
            e.x = fmaf(a.fc, r2A * rsqrtf(r2A) - a.rc, e.x);
            e.y = fmaf(a.fc, r2B * rsqrtf(r2B) - a.rc, e.y);
        }
        acc.pe += onA ? e.x : 0.0f;
        acc.pe += onB ? e.y : 0.0f;
        acc.vir = fmaf(fs.x, r2A, acc.vir);
        acc.vir = fmaf(fs.y, r2B, acc.vir);
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
// (REGULAR) the origin shifts are ((c_x - 1) w, (c_y - 1) w), read (negated)
// from a 16-entry shared-memory table indexed by the entry's four code bits;
// at the periodic edges and next to the wider last cell they are selected
// from the four per-particle shifts.  Entries are evaluated two at a time on
// packed pairs (pair_terms2_masked).  IDX25: every slot number is below 2^25,
// so bits 25-27 of an entry are zero and entry >> 25 is its code times 8, the
// byte offset of the code's float2 in the table (one shift instead of a shift
// and a scaling).
template <bool STATS, bool REGULAR, bool SF, bool IDX25>
__device__ __forceinline__ void forces_list(const StepArgs &a, int64_t i, float2 p, int cnt,
                                            const float2 *tab, float sxm, float sxp, float sym,
                                            float syp, PairAcc &acc) {
    const uint4 *e = reinterpret_cast<const uint4 *>(a.nbr) + i;
    const int64_t n = a.n;
    const float w = a.cell_w;
    const int nb = (int)((uint32_t)(cnt + kListBatch - 1) / kListBatch);   // cnt >= 0
    for (int b = 0; b < nb; ++b) {
        // one 32 x 32 -> 64-bit product (slot numbers below 2^28, batches below 2^7:
        // the capacity is at most 512 entries)
        const uint4 e4 = __ldcs(e + (uint64_t)(uint32_t)b * (uint32_t)n);
        const uint32_t ent[kListBatch] = {e4.x, e4.y, e4.z, e4.w};
        float2 q[kListBatch];
#pragma unroll
        for (int u = 0; u < kListBatch; ++u) q[u] = __ldg(a.cl_in + (ent[u] & 0x0fffffffu));
        // negated origin shifts of the four entries
        float2 ns[kListBatch];
#pragma unroll
        for (int u = 0; u < kListBatch; ++u) {
            if (REGULAR && IDX25) {
                ns[u] = *reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(tab) +
                                                          (ent[u] >> 25));
            } else if (REGULAR) {
                ns[u] = tab[ent[u] >> 28];
            } else {
                const uint32_t ox = (ent[u] >> 28) & 3u, oy = ent[u] >> 30;
                ns[u].x = -(ox == 0u ? sxm : (ox == 2u ? sxp : (ox == 3u ? 2.0f * w : 0.0f)));
                ns[u].y = -(oy == 0u ? sym : (oy == 2u ? syp : (oy == 3u ? 2.0f * w : 0.0f)));
            }
        }
#pragma unroll
        for (int u = 0; u < kListBatch; u += 2)
            pair_terms2_masked<STATS, SF>(a, p, q[u], ns[u], q[u + 1], ns[u + 1], acc);
    }
}

// Negated origin shifts -((c_x - 1) w, (c_y - 1) w) of the 16 list offset
// codes of a regular neighbourhood (code 3: the padding entries' 2 w), built
// by the first 16 threads of a block.
__device__ __forceinline__ void init_shift_table(const StepArgs &a, float2 *s_tab) {
    if (threadIdx.x < 16)
        s_tab[threadIdx.x] = make_float2(-fmaf((float)(threadIdx.x & 3u), a.cell_w, -a.cell_w),
                                         -fmaf((float)(threadIdx.x >> 2), a.cell_w, -a.cell_w));
}

// Neighbour-cell radius for the displacement bound D of the input positions.
__device__ __forceinline__ int stencil_radius(const StepArgs &a, float D) {
    const float Rf = ceilf((a.rc + 2.0f * D) / a.cell_w);
    // NaN -> 1; anything past the box is capped (stencil() then visits every cell once)
    return (Rf >= 1.0f) ? (Rf < 65536.0f ? (int)Rf : 65536) : 1;
}

// Launch-wide check, once per launch (block 0, thread 0): the cell list far out
// of date for the stencil radius of D.
__device__ __forceinline__ void check_stencil(const StepArgs &a, const Geom &geo, float D) {
    if (a.potential && threadIdx.x == 0 && blockIdx.x == 0) {
        const int R = stencil_radius(a, D);
        if (2 * R + 1 > geo.nc[0] || 2 * R + 1 > geo.nc[1])
            set_status(a.ctl, kErrOverflow);   // cell list far out of date: whole box searched
    }
}

// The Verlet list holds every pair that can be closer than rc while 2D <= skin;
// a launch that finds it stale takes the cell stencil and is counted.
__device__ __forceinline__ bool list_current(const StepArgs &a, float D) {
    const bool ok = a.nbr != nullptr && 2.0f * D <= a.list_skin;
    if (a.potential && a.nbr && !ok && threadIdx.x == 0 && blockIdx.x == 0)
        atomicAdd(&a.ctl->stale_steps, 1u);
    return ok;
}

// One slot's force and update.  Returns |v|^2 of the new half-step velocity
// (kModeStep) and, with STATS, the slot's fixed-point inputs t[] (kinetic
// energy at the integer step, halved pair energy and virial, momentum).
// IDX25: slot numbers below 2^25 (see forces_list); INR: the caller has
// checked i < n.
template <int MODE, bool STATS, bool B, bool SF, bool IDX25 = false, bool INR = false>
__device__ __forceinline__ float step_slot(const StepArgs &a, const Geom &geo, int64_t cell0,
                                           int64_t i, const float2 *s_tab, bool list_ok,
                                           float (&t)[kStatsN]) {
    const bool inr = INR || i < a.n;
    const uint32_t cw = inr ? __ldcs(a.cell + i) : kGhostCell;
    const bool act = inr && (!B || cw != kGhostCell);
    PairAcc acc = {0.f, 0.f, 0.f, 0.f};
    float2 p = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
    if (act) {
        p = a.cl_in[i];
        v = __ldcs(a.v_in + i);
        if (a.potential) {
            const int32_t cx = cell_x(cw), cy = cell_y(cw);
            const int cnt = list_ok ? __ldcs(a.ncount + i) : a.cap + 1;
            if (cnt <= a.cap) {
                // neighbouring cells of full width and no periodic wrap: shifts (code - 1) w
                if (cx >= 1 && cx + 2 <= geo.nc[0] && cy >= 1 && cy + 2 <= geo.nc[1]) {
                    forces_list<STATS, true, SF, IDX25>(a, i, p, cnt, s_tab, 0.f, 0.f, 0.f, 0.f, acc);
                } else {
                    const float sxm = cell_shift(cx, -1, geo.nc[0], geo.k, geo.lg[0], geo.g);
                    const float sxp = cell_shift(cx, +1, geo.nc[0], geo.k, geo.lg[0], geo.g);
                    const float sym = cell_shift(cy, -1, geo.nc[1], geo.k, geo.lg[1], geo.g);
                    const float syp = cell_shift(cy, +1, geo.nc[1], geo.k, geo.lg[1], geo.g);
                    forces_list<STATS, false, SF, IDX25>(a, i, p, cnt, s_tab, sxm, sxp, sym, syp, acc);
                }
            } else {
                // D re-read here (the bound only changes at the end of the launch)
                // so that it is not held in a register across the list path
                const int R = stencil_radius(a, a.ctl->dbound);
                int lox, hix, loy, hiy;
                stencil(R, geo.nc[0], lox, hix);
                stencil(R, geo.nc[1], loy, hiy);
                forces_cells<STATS, SF>(a, geo, a.cell_start + cell0, i, cx, cy, p, lox, hix, loy,
                                        hiy, acc);
            }
        }
    }
    const float fx = acc.fx, fy = acc.fy;

    float2 vn = v;   // velocity at the integer step (statistics)
    float vmax2 = 0.f;
    if (act) {
        if (MODE == kModeStep) {
            vn = make_float2(fmaf(fx, a.half_dt_m, v.x), fmaf(fy, a.half_dt_m, v.y));
            const float2 vh = make_float2(fmaf(fx, a.dt_m, v.x), fmaf(fy, a.dt_m, v.y));
            const float2 pn = make_float2(fmaf(vh.x, a.dt, p.x), fmaf(vh.y, a.dt, p.y));
            __stcs(a.v_out + i, vh);
            a.cl_out[i] = pn;
            vmax2 = fmaf(vh.x, vh.x, vh.y * vh.y);
            // a non-finite velocity or offset (from the forces, or restored from
            // a corrupt checkpoint) makes the sum NaN or infinite; the values of
            // any sane run are many orders of magnitude below the bound
            if (!(vmax2 + fabsf(pn.x) + fabsf(pn.y) < 3.0e38f)) set_status(a.ctl, kErrNonFinite);
        } else if (MODE == kModeInit) {
            vn = v;
            a.v_out[i] = make_float2(fmaf(-fx, a.half_dt_m, v.x), fmaf(-fy, a.half_dt_m, v.y));
        } else {
            vn = make_float2(fmaf(fx, a.half_dt_m, v.x), fmaf(fy, a.half_dt_m, v.y));
            a.v_sync[i] = vn;
            if (a.f_sync) a.f_sync[i] = make_float2(fx, fy);
        }
    }
    if (STATS && act) {
        t[0] = 0.5f * a.mass * fmaf(vn.x, vn.x, vn.y * vn.y);
        t[1] = 0.5f * acc.pe;
        t[2] = 0.5f * acc.vir;
        t[3] = a.mass * vn.x;
        t[4] = a.mass * vn.y;
    }
    return vmax2;
}

// End of a block: the block's largest |v|^2 and statistics are published, and
// the last block of the launch (ticket) turns them into the launch's results.
template <int MODE, bool STATS, bool B>
__device__ __forceinline__ void step_epilogue(const StepArgs &a, int64_t sys, float D, float vmax2,
                                              const float (&t)[kStatsN]) {
    constexpr int kWarps = (B ? kChunk : kStepThreads) / 32;
    __shared__ long long s_red[kWarps][kStatsN];
    __shared__ float s_max[kWarps];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MODE == kModeStep) {
        const float m = warp_max(vmax2);
        if (lane == 0) s_max[warp] = m;
    }
    if (STATS) {
        // per-slot FP32 terms -> multiples of 2^-24 -> exact 64-bit sums
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
                long long s = 0;
                for (int w = 0; w < kWarps; ++w) s += s_red[w][k];
                // batched: a block is one chunk of one system.  Integer sums are
                // exact, so the order of these atomics does not matter
                atomicAdd(B ? (unsigned long long *)&a.batch.stats[sys * kStatsN + k]
                            : (unsigned long long *)&a.ctl->stats_acc[k],
                          (unsigned long long)s);
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
        const long long s =
            (long long)atomicExch((unsigned long long *)&a.ctl->stats_acc[threadIdx.x], 0ull);
        a.ctl->stats[threadIdx.x] = (double)s * kFixInv;
    }
    if (threadIdx.x == 0) {
        if (MODE == kModeStep) {
            const uint32_t bits = atomicExch(&a.ctl->vmax2_bits, 0u);
            const float vmax = sqrtf(__uint_as_float(bits));
            const float dn = D + vmax * a.dt * 1.000001f + a.round_margin;
            a.ctl->dbound = dn;
            if (a.pace) {
                // host-mapped slot: the values first, then (after a system-scope
                // fence) the step number that marks them complete
                volatile PaceSlot *ps = a.pace + (a.step & (kPaceRing - 1));
                ps->dbound = dn;
                ps->vmax2_bits = bits;
                __threadfence_system();
                ps->step = a.step;
            }
        }
        a.ctl->done = 0u;
    }
}

// B: batched systems (geometry per 128-slot chunk, ghosts skipped, statistics
// per system); otherwise one system described by a.geo.  One slot per thread.
template <int MODE, bool STATS, bool B, bool SF>
__device__ __forceinline__ void step_body(const StepArgs &a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const SysView sv = sys_view<B>(a.geo, a.batch, i < a.n ? i : 0);
    __shared__ float2 s_tab[16];
    init_shift_table(a, s_tab);
    __syncthreads();
    const float D = a.ctl->dbound;
    check_stencil(a, sv.geo, D);
    const bool list_ok = list_current(a, D);
    float t[kStatsN] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const float vmax2 = step_slot<MODE, STATS, B, SF>(a, sv.geo, sv.cell0, i, s_tab, list_ok, t);
    step_epilogue<MODE, STATS, B>(a, sv.sys, D, vmax2, t);
}

// One chunk of 256 slots per block: the statistics, initial and sync launches
// of one system (the register count left to the compiler).
template <int MODE, bool STATS, bool SF>
__global__ void __launch_bounds__(kStepThreads) k_step(StepArgs a) {
    step_body<MODE, STATS, false, SF>(a);
}

// The same launches of a batch: one 128-slot chunk per block, 16 blocks per
// SM (32 registers: the per-chunk geometry would otherwise take the count to 40
// and the occupancy to 48 warps; 4 % faster for the 256-system batch).
template <int MODE, bool STATS, bool SF>
__global__ void __launch_bounds__(kChunk, kStepBatchBlocksPerSM) k_step_batch(StepArgs a) {
    step_body<MODE, STATS, true, SF>(a);
}

// Plain steps of one system (no statistics): a grid of resident blocks, each
// block taking the 256-slot chunks blockIdx, blockIdx + gridDim, ...  A warp
// runs through its chunks without waiting for the other warps of its block,
// and the block epilogue (barriers, the launch ticket) runs once per block
// instead of once per chunk.  Same arithmetic per slot as k_step.  IDX25: a
// system of at most 2^25 slots (see forces_list).
template <bool SF, bool IDX25>
__global__ void __launch_bounds__(kStepThreads, kStepLoopBlocksPerSM) k_step_loop(StepArgs a) {
    __shared__ float2 s_tab[16];
    init_shift_table(a, s_tab);
    __syncthreads();
    const float D = a.ctl->dbound;
    check_stencil(a, a.geo, D);
    const bool list_ok = list_current(a, D);
    float t[kStatsN] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float vmax2 = 0.f;
    // slot numbers fit 28 bits wherever lists are used (the entries' j field)
    const int32_t n = (int32_t)a.n, stride = (int32_t)gridDim.x * kStepThreads;
    for (int32_t i = (int32_t)blockIdx.x * kStepThreads + threadIdx.x; i < n; i += stride)
        vmax2 = fmaxf(vmax2, step_slot<kModeStep, false, false, SF, IDX25, true>(a, a.geo, 0, i,
                                                                                s_tab, list_ok, t));
    step_epilogue<kModeStep, false, false>(a, 0, D, vmax2, t);
}

// Plain steps of a batch: the same loop over 128-slot chunks (one chunk per
// block and round, 16 resident blocks per SM), each chunk with its own
// system's geometry.  IDX25: at most 2^25 slots in all.
template <bool SF, bool IDX25>
__global__ void __launch_bounds__(kChunk, kStepBatchBlocksPerSM) k_step_batch_loop(StepArgs a) {
    __shared__ float2 s_tab[16];
    init_shift_table(a, s_tab);
    __syncthreads();
    const float D = a.ctl->dbound;
    check_stencil(a, sys_view<true>(a.geo, a.batch, 0).geo, D);
    const bool list_ok = list_current(a, D);
    float t[kStatsN] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float vmax2 = 0.f;
    // slot numbers fit 28 bits wherever lists are used (the entries' j field)
    const int32_t n = (int32_t)a.n, stride = (int32_t)gridDim.x * kChunk;
    for (int32_t i = (int32_t)blockIdx.x * kChunk + threadIdx.x; i < n; i += stride) {
        const SysView sv = sys_view<true>(a.geo, a.batch, i);
        vmax2 = fmaxf(vmax2, step_slot<kModeStep, false, true, SF, IDX25>(a, sv.geo, sv.cell0, i,
                                                                         s_tab, list_ok, t));
    }
    step_epilogue<kModeStep, false, true>(a, 0, D, vmax2, t);
}

// ---- neighbour-cell sort (counting sort keyed by MD cell; inside a cell by
//      base column, then particle number, when Verlet lists are built, else by
//      particle number) -------------------------------------------------------


template <bool B>
__global__ void k_sort_key(SortArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const SysView sv = sys_view<B>(a.geo, a.batch, i);
        const Geom &geo = sv.geo;
        const uint32_t cw = a.cell_in[i];
        uint32_t key = kGhostCell;
        int64_t c = sv.cell0 + sv.ncells;   // a system's ghost cell
        int32_t col = 0;                    // base column inside the new cell
        if (!B || cw != kGhostCell) {
            const float2 p = a.cl_in[i];
            const int32_t bx = base_cell(cell_x(cw) * geo.k, p.x, geo.inv_g, geo.lg[0]);
            const int32_t by = base_cell(cell_y(cw) * geo.k, p.y, geo.inv_g, geo.lg[1]);
            int32_t nx = bx / geo.k, ny = by / geo.k;
            nx = nx < geo.nc[0] ? nx : geo.nc[0] - 1;
            ny = ny < geo.nc[1] ? ny : geo.nc[1] - 1;
            key = (uint32_t)nx | ((uint32_t)ny << 16);
            c = sv.cell0 + ny * geo.nc[0] + nx;
            col = bx - nx * geo.k;
        }
        a.key[i] = key;
        if (a.col) a.col[i] = (uint8_t)(col < 15 ? col : 15);
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
        // rank key of the scatter: base column (lists on; particle numbers are
        // then below 2^28), then particle number
        const uint32_t rk = (uint32_t)a.pid_in[i] + (a.col ? (uint32_t)a.col[i] << 28 : 0u);
        a.entry[at] = ((unsigned long long)rk << 32) | (uint32_t)i;
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
// finds its rank by its entry's rank key (base column, then particle number)
// among its cell's arrivals, then is copied
// from the old order to its final place, its position re-expressed against the
// new cell's origin.
// Without MSD the kernel fits 32 registers (8 blocks of 256 per SM: full
// occupancy for the gathers from the old order).
template <bool B, bool MSD>
__global__ void __launch_bounds__(256, MSD ? 4 : 8) k_sort_scatter(SortArgs a) {
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
        // MSD (a compile-time choice): the offsets and velocities at each lag's
        // last binning (mean-square displacement, velocity correlation; each
        // when its arrays are set) move too, so without it they take no registers
        const bool mo = MSD && a.mprev_in[0] != nullptr, vo = MSD && a.vprev_in[0] != nullptr;
        uint32_t lp[kMaxLags];
        float2 mp[MSD ? kMaxLags : 1], vp[MSD ? kMaxLags : 1];
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l) {
            lp[l] = l < a.nlags ? a.lprev_in[l][from] : 0u;
            if (MSD) {
                mp[l] = (mo && l < a.nlags) ? a.mprev_in[l][from] : make_float2(0.f, 0.f);
                vp[l] = (vo && l < a.nlags) ? a.vprev_in[l][from] : make_float2(0.f, 0.f);
            }
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
                if (MSD && mo) a.mprev_out[l][to] = make_float2(mp[l].x + sx, mp[l].y + sy);
                if (MSD && vo) a.vprev_out[l][to] = vp[l];
            }
    }
}

// Verlet list of the freshly sorted state: every j != i closer than the list
// radius, found in the 3 x 3 cell stencil (cells are at least that wide and
// every particle is inside its cell).  Candidates are fetched a few at a time
// (two in the interior rows, whose ranges are short after the skip below; four
// elsewhere; predicated: past the end of a range the position is a far sentinel
// whose distance fails the radius test) so their loads overlap.  Every candidate's entry is written to
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
        const int32_t i32 = (int32_t)i;   // slot numbers are below 2^28 wherever lists are built
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
                    // the particle's offset minus each column's origin shift and
                    // the row's, formed once: one subtraction per axis and
                    // candidate; the entry codes of the three columns likewise
                    const float pyr = p.y - ody, pxm = p.x - sxm, pxp = p.x - sxp;
                    const uint32_t codeM = ycode + (1u << 28), codeR = ycode + (2u << 28);
                    // cells cx-1, cx, cx+1 of this row are one contiguous range
                    const int32_t s0 = __ldg(cs + row + cx - 1);
                    const int32_t m1 = __ldg(cs + row + cx);
                    const int32_t m2 = __ldg(cs + row + cx + 1);
                    const int32_t e0 = __ldg(cs + row + cx + 2);
                    // A candidate of cell cx-1 whose offset is below p.x, or of
                    // cell cx+1 above it, lies more than a whole cell width (the
                    // list radius) away along x, so it cannot come within rc
                    // before the displacement bound forces the next sort.  Cells
                    // are ordered by base column, so such candidates lead cell
                    // cx-1 and trail cell cx+1; up to four are dropped at each
                    // end of the range.
                    int32_t s = s0, e = e0;
                    {
                        const float *clx = reinterpret_cast<const float *>(a.cl_out);
                        float lx[4], rx[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            lx[u] = s0 + u < m1 ? __ldg(clx + 2 * (int64_t)(s0 + u)) : 3.0e38f;
                            rx[u] = e0 - 1 - u >= m2 ? __ldg(clx + 2 * (int64_t)(e0 - 1 - u)) : -3.0e38f;
                        }
                        bool gl = true, gr = true;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            gl = gl && lx[u] < p.x;
                            gr = gr && rx[u] > p.x;
                            s += gl;
                            e -= gr;
                        }
                    }
                    for (int32_t b = s; b < e; b += 2) {
                        float2 q[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u)
                            q[u] = (b + u < e) ? __ldg(a.cl_out + b + u)
                                               : make_float2(1.0e18f, 1.0e18f);
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int32_t j = b + u;
                            const bool g1 = j >= m1, g2 = j >= m2;   // in cell cx, cx + 1
                            const float pxs = g2 ? pxp : (g1 ? p.x : pxm);
                            const float dx = pxs - q[u].x, dy = pyr - q[u].y;
                            const bool hit = j != i32 && fmaf(dx, dx, dy * dy) < a.rl2;
                            s_ent[min(cnt, last) * nt + threadIdx.x] =
                                (uint32_t)j + (g2 ? codeR : (g1 ? codeM : ycode));
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
                            const bool hit = j != i32 && fmaf(dx, dx, dy * dy) < a.rl2;
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
        // statistics steps one chunk per block; plain steps the looping kernels
        // (slot numbers below 2^25: the one-shift table index of forces_list)
        const bool small = a.n <= ((int64_t)1 << 25);
        const int gb = grid_for(a.n, kChunk, kStepBatchBlocksPerSM);
        const int gs = grid_for(a.n, kStepThreads, kStepLoopBlocksPerSM);
        if (a.stats) launch_step_k<kModeStep, true, B, SF>(a, grid, block, s);
        else if (B && small) k_step_batch_loop<SF, true><<<gb, block, 0, s>>>(a);
        else if (B) k_step_batch_loop<SF, false><<<gb, block, 0, s>>>(a);
        else if (small) k_step_loop<SF, true><<<gs, block, 0, s>>>(a);
        else k_step_loop<SF, false><<<gs, block, 0, s>>>(a);
    } else if (mode == kModeInit) {
        launch_step_k<kModeInit, true, B, SF>(a, grid, block, s);
    } else {
        launch_step_k<kModeSync, true, B, SF>(a, grid, block, s);
    }
}

cudaError_t launch_step(const StepArgs &a, int mode, cudaStream_t s) {
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
    // scatter and list build: 64 and 128 blocks per SM in the grid (several
    // rounds of resident blocks; uneven cells and lists balance better than
    // with one)
    if (a.mprev_in[0] || a.vprev_in[0]) k_sort_scatter<B, true><<<grid_for(a.n, t, 64), t, 0, s>>>(a);
    else k_sort_scatter<B, false><<<grid_for(a.n, t, 64), t, 0, s>>>(a);
    if (a.nbr) {
        const int nt = (size_t)kNlistThreads * (a.cap + 1) * sizeof(uint32_t) <= 96 * 1024 ? kNlistThreads : 64;
        const size_t smem = sizeof(uint32_t) * (size_t)nt * (a.cap + 1);
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_nlist<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_nlist<B><<<grid_for(a.n, nt, 128), nt, smem, s>>>(a);
    }
    return cudaGetLastError();
}

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
