// mdlg_bin.cu -- MDLG occupation-number kernels (Eq. MDni of arXiv:1705.04368).
//
// n_i(x,t) = sum_j Delta_x(x_j(t)) Delta_{x - v_i}(x_j(t - dt)): each particle
// contributes one count at its lattice cell at t, in the velocity given by its
// lattice displacement since t - dt.  All three kernels are grid-stride loops
// over particles with a block-private shared-memory histogram of the Q+1
// velocity bins, flushed once per block with 64-bit global atomics; optional
// per-site outputs (N(x,t), n_i(x,t)) are 32-bit global atomics.
#include <cmath>

#include "mdlg_kernels.h"

namespace mdlg {

namespace {

__device__ __forceinline__ int32_t lattice_of_base(int32_t b, int32_t ratio, int32_t shift) {
    return shift >= 0 ? (b >> shift) : (b / ratio);
}

__device__ __forceinline__ void flush_hist(const uint32_t *sh, int q1, unsigned long long *counts) {
    for (int b = threadIdx.x; b < q1; b += blockDim.x)
        if (sh[b]) atomicAdd(&counts[b], (unsigned long long)sh[b]);
}

// Context-free binning of two snapshots given as integer base-cell indices.
__global__ void k_bin_snapshots(LatticeArgs la, int64_t n, const int2 *__restrict__ prev,
                                const int2 *__restrict__ cur, unsigned long long *counts,
                                uint32_t *ncell, uint32_t *field) {
    extern __shared__ uint32_t sh[];
    const int w = 2 * la.vmax + 1, q = w * w, q1 = q + 1;
    const int center = la.vmax * w + la.vmax;
    for (int b = threadIdx.x; b < q1; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool act = j < n;
        int32_t bin = 0;
        if (act) {
            int2 a = prev[j], c = cur[j];
            int32_t ax = a.x % la.base[0], ay = a.y % la.base[1];
            int32_t cx = c.x % la.base[0], cy = c.y % la.base[1];
            ax += ax < 0 ? la.base[0] : 0;
            ay += ay < 0 ? la.base[1] : 0;
            cx += cx < 0 ? la.base[0] : 0;
            cy += cy < 0 ? la.base[1] : 0;
            const int32_t l0x = lattice_of_base(ax, la.ratio, la.shift);
            const int32_t l0y = lattice_of_base(ay, la.ratio, la.shift);
            const int32_t l1x = lattice_of_base(cx, la.ratio, la.shift);
            const int32_t l1y = lattice_of_base(cy, la.ratio, la.shift);
            const int32_t vx = lattice_disp(l1x - l0x, la.lat[0]);
            const int32_t vy = lattice_disp(l1y - l0y, la.lat[1]);
            bin = vel_index(vx, vy, la.vmax);
            const int64_t site = (int64_t)l1y * la.lat[0] + l1x;
            if (ncell) atomicAdd(&ncell[site], 1u);
            if (field) atomicAdd(&field[site * q1 + bin], 1u);
        }
        hist_add(sh, bin, center, act);
    }
    __syncthreads();
    flush_hist(sh, q1, counts);
}

// Non-interacting gas: stream each particle for every (dx, dt) pair and bin
// its start and end point.  Cell decisions in binary32 with explicit rounding
// (no contraction into FMA): x' = fl(x + fl(v dt)), cell = ceil(fl(x / dx)) - 1,
// with v boosted first, v = fl(v + U), when the pair has a lattice drift U.
// The pair count is a template parameter, so the loop is unrolled and every
// pair's parameters are compile-time offsets into the argument block; when
// every dx is a power of two (ALLPOW2) the division path is not compiled in.
// Multiplying by 1/dx equals dividing by dx when dx is a power of two.  The
// rest velocity, where most decisions of a short coarse step land, is counted
// per pair in registers and added to the block histogram once per thread; the
// other bins take one shared atomic per decision.  Every decision issues its
// atomic (no branch around it): a rest decision adds to a scratch word of its
// lane past the histograms, which is never read.
template <int NC, bool ALLPOW2>
__global__ void k_idealgas_bin(IdealGasArgs ga, int64_t n, const float2 *__restrict__ pos,
                               const float2 *__restrict__ vel, unsigned long long *counts) {
    extern __shared__ uint32_t sh[];
    const int w = 2 * ga.vmax + 1, q1 = w * w + 1;
    const int center = ga.vmax * w + ga.vmax;
    uint32_t *scratch = sh + q1 * NC + (threadIdx.x & 31);   // rest decisions' atomics
    for (int b = threadIdx.x; b < q1 * NC; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    uint32_t rest[NC];   // rest-velocity counts kept in registers, added once per thread
#pragma unroll
    for (int k = 0; k < NC; ++k) rest[k] = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool act = j < n;
        float2 p = make_float2(1.f, 1.f), v = make_float2(0.f, 0.f);
        if (act) {
            p = pos[j];
            v = vel[j];
        }
        int32_t c0x = 0, c0y = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float dx = ga.dx[k], dt = ga.dt[k];
            const bool pow2 = ALLPOW2 || ga.pow2[k] != 0;
            const float inv = ga.inv_dx[k];
            if (k == 0 || dx != ga.dx[k - 1]) {
                const float qx = pow2 ? __fmul_rn(p.x, inv) : __fdiv_rn(p.x, dx);
                const float qy = pow2 ? __fmul_rn(p.y, inv) : __fdiv_rn(p.y, dx);
                c0x = ceil_small(qx) - 1;
                c0y = ceil_small(qy) - 1;
            }
            const float vx_ = ga.boost ? __fadd_rn(v.x, ga.ux[k]) : v.x;
            const float vy_ = ga.boost ? __fadd_rn(v.y, ga.uy[k]) : v.y;
            const float xn = __fadd_rn(p.x, __fmul_rn(vx_, dt));
            const float yn = __fadd_rn(p.y, __fmul_rn(vy_, dt));
            const float qx = pow2 ? __fmul_rn(xn, inv) : __fdiv_rn(xn, dx);
            const float qy = pow2 ? __fmul_rn(yn, inv) : __fdiv_rn(yn, dx);
            const int32_t vx = ceil_small(qx) - 1 - c0x;
            const int32_t vy = ceil_small(qy) - 1 - c0y;
            const bool at_rest = (vx | vy) == 0;
            rest[k] += (act && at_rest) ? 1u : 0u;
            // window index by unsigned range checks; the overflow bin past it
            const uint32_t ux = (uint32_t)(vx + ga.vmax), uy = (uint32_t)(vy + ga.vmax);
            const uint32_t bin = max(ux, uy) <= (uint32_t)(2 * ga.vmax) ? uy * (uint32_t)w + ux
                                                                        : (uint32_t)(w * w);
            atomicAdd((act && !at_rest) ? &sh[k * q1 + bin] : scratch, 1u);
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        uint32_t r = rest[k];
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((threadIdx.x & 31) == 0 && r) atomicAdd(&sh[k * q1 + center], r);
    }
    __syncthreads();
    for (int k = 0; k < NC; ++k) flush_hist(sh + k * q1, q1, counts + (size_t)k * q1);
}

// Non-interacting gas, every dx a power of two.  The pairs arrive ordered so
// that pairs sharing (dt, U) are adjacent: x' = fl(x + fl(v' dt)) is formed
// once per group, and the cell at every dx of the group is the cell at the
// smallest dx shifted right.  This is exact: dx_min = dx / 2^s and x / dx_min
// are exact in binary32, and with c = ceil(x / dx_min) - 1 (so c < x / dx_min
// <= c + 1) the cell ceil(x / dx) - 1 is floor(c / 2^s) (the multiples of 2^s
// are integers).  The decisions therefore equal the division form above bit
// for bit.  PPT particles per thread per loop trip (2: one 16-byte load of
// positions and one of velocities).  Rest decisions are counted in registers
// and send their atomic to the lane's scratch word, as in k_idealgas_bin.
// NS > 0: the pairs form a full grid, every (dt, U) group holding the shifts
// 0 ... NS-1 in order (grid_shifts); the shifts are then compile-time
// constants, so each particle's start cells are shifted once per distinct
// shift rather than once per pair, and the pairs at dx_min take no shift.
template <int NC, int PPT, int NS = 0>
__global__ void __launch_bounds__(256) k_idealgas_pow2(IdealGasArgs ga, int64_t n,
                                                       const float2 *__restrict__ pos,
                                                       const float2 *__restrict__ vel,
                                                       unsigned long long *counts) {
    extern __shared__ uint32_t sh[];
    const int w = 2 * ga.vmax + 1, q1 = w * w + 1;
    const int center = ga.vmax * w + ga.vmax;
    const uint32_t wmax = (uint32_t)(2 * ga.vmax);
    uint32_t *scratch = sh + q1 * NC + (threadIdx.x & 31);   // rest decisions' atomics
    for (int b = threadIdx.x; b < q1 * NC; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    uint32_t rest[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) rest[k] = 0u;
    const float inv = ga.inv_min;
    const int64_t ng = (n + PPT - 1) / PPT;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ng; base += stride) {
        const int64_t gi = base + threadIdx.x;
        const int64_t j0 = gi * PPT;
        float2 p[PPT], v[PPT];
        bool act[PPT];
        if (PPT == 2 && j0 + 1 < n) {
            const float4 pp = reinterpret_cast<const float4 *>(pos)[gi];
            const float4 vv = reinterpret_cast<const float4 *>(vel)[gi];
            p[0] = make_float2(pp.x, pp.y);
            p[PPT - 1] = make_float2(pp.z, pp.w);
            v[0] = make_float2(vv.x, vv.y);
            v[PPT - 1] = make_float2(vv.z, vv.w);
            act[0] = act[PPT - 1] = true;
        } else {
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                act[u] = gi < ng && j0 + u < n;
                p[u] = act[u] ? pos[j0 + u] : make_float2(1.f, 1.f);
                v[u] = act[u] ? vel[j0 + u] : make_float2(0.f, 0.f);
            }
        }
        int32_t bx[PPT], by[PPT], cx[PPT], cy[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            bx[u] = ceil_small(__fmul_rn(p[u].x, inv)) - 1;
            by[u] = ceil_small(__fmul_rn(p[u].y, inv)) - 1;
            cx[u] = cy[u] = 0;
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k == 0 || (NS ? k % NS == 0 : ga.first[k] != 0)) {
                const float dt = ga.dt[k];
#pragma unroll
                for (int u = 0; u < PPT; ++u) {
                    const float vx_ = ga.boost ? __fadd_rn(v[u].x, ga.ux[k]) : v[u].x;
                    const float vy_ = ga.boost ? __fadd_rn(v[u].y, ga.uy[k]) : v[u].y;
                    const float xn = __fadd_rn(p[u].x, __fmul_rn(vx_, dt));
                    const float yn = __fadd_rn(p[u].y, __fmul_rn(vy_, dt));
                    cx[u] = ceil_small(__fmul_rn(xn, inv)) - 1;
                    cy[u] = ceil_small(__fmul_rn(yn, inv)) - 1;
                }
            }
            const int sft = NS ? k % NS : ga.shift[k];
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                const int32_t dvx = (cx[u] >> sft) - (bx[u] >> sft);
                const int32_t dvy = (cy[u] >> sft) - (by[u] >> sft);
                const bool at_rest = (dvx | dvy) == 0;
                rest[k] += (act[u] && at_rest) ? 1u : 0u;
                const uint32_t ux = (uint32_t)(dvx + ga.vmax), uy = (uint32_t)(dvy + ga.vmax);
                const uint32_t bin = max(ux, uy) <= wmax ? uy * (uint32_t)w + ux : (uint32_t)(w * w);
                atomicAdd((act[u] && !at_rest) ? &sh[k * q1 + bin] : scratch, 1u);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        uint32_t r = rest[k];
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((threadIdx.x & 31) == 0 && r) atomicAdd(&sh[k * q1 + center], r);
    }
    __syncthreads();
    for (int k = 0; k < NC; ++k) flush_hist(sh + k * q1, q1, counts + (size_t)ga.out[k] * q1);
}

// Sum v over the block into out (added to, FP64); every thread calls it.
__device__ void block_sum_add(float v, float *red, double *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) atomicAdd(out, (double)t);
    }
    __syncthreads();
}

// Base cell of one axis of a state particle, on the lattice at rest or moved.
__device__ __forceinline__ int32_t state_base(const Geom &geo, const LatticeShift &sh, int a,
                                              int32_t origin, float cl) {
    return sh.on ? base_cell_moving(origin, cl, geo.inv_g, geo.lg[a], sh.K[a], sh.omb[a])
                 : base_cell(origin, cl, geo.inv_g, geo.lg[a]);
}

// Binning of the simulation state (sorted by MD cell) for the lags in `mask`:
// the lattice cell now versus the one stored at the lag's previous binning,
// which is then replaced.  Lag 0 may also write per-site outputs.  The MSD
// instantiation carries the optional per-lag sums, each on when its
// accumulator is set: with msd_acc every binned lag also adds the squared
// displacement since its previous binning, with vacf_acc the product of the
// velocity now and the one stored at that binning (Sec. IV-A).  Every load of an iteration is issued before any of its
// stores (a store followed by a load the compiler cannot prove independent
// stalls the thread), and the lag loop is unrolled over the compile-time
// maximum, predicated by the mask.
template <bool MSD, bool MOVE>
__global__ void k_bin_state(StateBinArgs sa) {
    extern __shared__ uint32_t sh[];
    __shared__ float red[32];
    const Geom &geo = sa.geo;
    const int w = 2 * geo.vmax + 1, q1 = w * w + 1;
    const int center = geo.vmax * w + geo.vmax;
    const bool msd = MSD && sa.msd_acc != nullptr;
    const bool vc = MSD && sa.vacf_acc != nullptr;
    for (int b = threadIdx.x; b < q1 * kMaxLags; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    float m2[kMaxLags][2], c2[kMaxLags][2];
#pragma unroll
    for (int l = 0; l < kMaxLags; ++l) m2[l][0] = m2[l][1] = c2[l][0] = c2[l][1] = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < sa.n; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool act = j < sa.n;
        uint32_t before[kMaxLags];
        float2 mp[kMaxLags], vp[kMaxLags];
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l) {
            const bool on = act && ((sa.mask >> l) & 1u);
            before[l] = on ? sa.lprev[l][j] : 0u;
            mp[l] = (on && msd) ? sa.mprev[l][j] : make_float2(0.f, 0.f);
            vp[l] = (on && vc) ? sa.vprev[l][j] : make_float2(0.f, 0.f);
        }
        const float2 vel = (act && vc) ? sa.vel[j] : make_float2(0.f, 0.f);
        int32_t lx = 0, ly = 0;
        float2 p = make_float2(0.f, 0.f);
        if (act) {
            const uint32_t c = sa.cell[j];
            p = sa.cl[j];
            const int32_t ccx = (int32_t)(c & 0xffffu), ccy = (int32_t)(c >> 16);
            const int32_t bx =
                MOVE ? base_cell_moving(ccx * geo.k, p.x, geo.inv_g, geo.lg[0], sa.shift.K[0], sa.shift.omb[0])
                     : base_cell(ccx * geo.k, p.x, geo.inv_g, geo.lg[0]);
            const int32_t by =
                MOVE ? base_cell_moving(ccy * geo.k, p.y, geo.inv_g, geo.lg[1], sa.shift.K[1], sa.shift.omb[1])
                     : base_cell(ccy * geo.k, p.y, geo.inv_g, geo.lg[1]);
            lx = lattice_of_base(bx, geo.ratio, sa.ratio_shift);
            ly = lattice_of_base(by, geo.ratio, sa.ratio_shift);
        }
        const uint32_t now = pack_cell(lx, ly);
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l) {
            if (!((sa.mask >> l) & 1u)) continue;
            int32_t bin = 0;
            if (act) {
                const int32_t vx = lattice_disp(lx - (int32_t)(before[l] & 0xffffu), geo.lat[0]);
                const int32_t vy = lattice_disp(ly - (int32_t)(before[l] >> 16), geo.lat[1]);
                bin = vel_index(vx, vy, geo.vmax);
                sa.lprev[l][j] = now;
                if (msd) {
                    const float ddx = p.x - mp[l].x, ddy = p.y - mp[l].y;
                    m2[l][0] += ddx * ddx;
                    m2[l][1] += ddy * ddy;
                    sa.mprev[l][j] = p;
                }
                if (vc) {
                    c2[l][0] = fmaf(vel.x, vp[l].x, c2[l][0]);
                    c2[l][1] = fmaf(vel.y, vp[l].y, c2[l][1]);
                    sa.vprev[l][j] = vel;
                }
                if (l == 0 && sa.site_n) {
                    const int64_t site = (int64_t)ly * geo.lat[0] + lx;
                    atomicAdd(&sa.site_n[site], 1u);
                    atomicAdd(&sa.site_counts[site * q1 + bin], 1u);
                }
            }
            hist_add(sh + l * q1, bin, center, act);
        }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < kMaxLags; ++l)
        if ((sa.mask >> l) & 1u) flush_hist(sh + l * q1, q1, sa.counts[l]);
    if (msd) {
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            if ((sa.mask >> l) & 1u) {
                block_sum_add(m2[l][0], red, sa.msd_acc + 2 * l);
                block_sum_add(m2[l][1], red, sa.msd_acc + 2 * l + 1);
            }
    }
    if (vc) {
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            if ((sa.mask >> l) & 1u) {
                block_sum_add(c2[l][0], red, sa.vacf_acc + 2 * l);
                block_sum_add(c2[l][1], red, sa.vacf_acc + 2 * l + 1);
            }
    }
}

// Binning of the state on the lattice at rest without displacement sums: the
// same decisions as k_bin_state, four consecutive particles per thread and
// loop trip with 16-byte loads (cell words, offsets, each lag's stored cells)
// and stores, every load of a trip issued before its first store.  K is the
// number of lags binned by the launch (the set bits of the mask, in order), so
// only their stored cells are loaded and kept in registers.  The rest velocity
// is counted in registers per lag and added to the block histogram once per
// thread.
template <int K>
__global__ void __launch_bounds__(256) k_bin_state_v(StateBinArgs sa) {
    extern __shared__ uint32_t sh[];   // K x (Q + 1): the k-th binned lag at k (Q + 1)
    const Geom &geo = sa.geo;
    const int w = 2 * geo.vmax + 1, q1 = w * w + 1;
    const int center = geo.vmax * w + geo.vmax;
    for (int b = threadIdx.x; b < q1 * K; b += blockDim.x) sh[b] = 0;
    int lag[K];
    {
        uint32_t m = sa.mask;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            lag[k] = __ffs(m) - 1;
            m &= m - 1u;
        }
    }
    const bool sites = sa.site_n != nullptr && lag[0] == 0;
    __syncthreads();
    uint32_t rest[K];
#pragma unroll
    for (int k = 0; k < K; ++k) rest[k] = 0u;
    const int64_t n = sa.n;
    const int64_t ng = (n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ng; base += stride) {
        const int64_t gi = base + threadIdx.x;
        const int64_t j0 = 4 * gi;
        const bool full = j0 + 3 < n;
        uint32_t c[4], bef[K][4];
        float2 p[4];
        if (full) {
            const uint4 cw = reinterpret_cast<const uint4 *>(sa.cell)[gi];
            const float4 pa = reinterpret_cast<const float4 *>(sa.cl)[2 * gi];
            const float4 pb = reinterpret_cast<const float4 *>(sa.cl)[2 * gi + 1];
            c[0] = cw.x; c[1] = cw.y; c[2] = cw.z; c[3] = cw.w;
            p[0] = make_float2(pa.x, pa.y);
            p[1] = make_float2(pa.z, pa.w);
            p[2] = make_float2(pb.x, pb.y);
            p[3] = make_float2(pb.z, pb.w);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const uint4 b4 = reinterpret_cast<const uint4 *>(sa.lprev[lag[k]])[gi];
                bef[k][0] = b4.x; bef[k][1] = b4.y; bef[k][2] = b4.z; bef[k][3] = b4.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool a = gi < ng && j0 + u < n;
                c[u] = a ? sa.cell[j0 + u] : 0u;
                p[u] = a ? sa.cl[j0 + u] : make_float2(1.f, 1.f);
#pragma unroll
                for (int k = 0; k < K; ++k) bef[k][u] = a ? sa.lprev[lag[k]][j0 + u] : 0u;
            }
        }
        uint32_t now[4];
        int32_t lx[4], ly[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t bx = base_cell((int32_t)(c[u] & 0xffffu) * geo.k, p[u].x, geo.inv_g, geo.lg[0]);
            const int32_t by = base_cell((int32_t)(c[u] >> 16) * geo.k, p[u].y, geo.inv_g, geo.lg[1]);
            lx[u] = lattice_of_base(bx, geo.ratio, sa.ratio_shift);
            ly[u] = lattice_of_base(by, geo.ratio, sa.ratio_shift);
            now[u] = pack_cell(lx[u], ly[u]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (full) {
                reinterpret_cast<uint4 *>(sa.lprev[lag[k]])[gi] = make_uint4(now[0], now[1], now[2], now[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (gi < ng && j0 + u < n) sa.lprev[lag[k]][j0 + u] = now[u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool a = full || (gi < ng && j0 + u < n);
                const int32_t vx = lattice_disp(lx[u] - (int32_t)(bef[k][u] & 0xffffu), geo.lat[0]);
                const int32_t vy = lattice_disp(ly[u] - (int32_t)(bef[k][u] >> 16), geo.lat[1]);
                const int32_t bin = vel_index(vx, vy, geo.vmax);
                if (k == 0 && sites && a) {
                    const int64_t site = (int64_t)ly[u] * geo.lat[0] + lx[u];
                    atomicAdd(&sa.site_n[site], 1u);
                    atomicAdd(&sa.site_counts[site * q1 + bin], 1u);
                }
                rest[k] += (a && bin == center) ? 1u : 0u;
                if (a && bin != center) atomicAdd(&sh[k * q1 + bin], 1u);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        uint32_t r = rest[k];
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((threadIdx.x & 31) == 0 && r) atomicAdd(&sh[k * q1 + center], r);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) flush_hist(sh + k * q1, q1, sa.counts[lag[k]]);
}

// Batched systems: one chunk (one system) per block iteration, so the block's
// histogram belongs to one system and is flushed into that system's totals.
__global__ void __launch_bounds__(kChunk) k_bin_state_batch(StateBinArgs sa) {
    extern __shared__ uint32_t sh[];
    const int w = 2 * sa.geo.vmax + 1, q1 = w * w + 1;
    const int center = sa.geo.vmax * w + sa.geo.vmax;
    const int64_t nchunks = sa.n / kChunk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        for (int b = threadIdx.x; b < q1 * kMaxLags; b += blockDim.x) sh[b] = 0;
        __syncthreads();
        const int sys = sa.batch.chunk_sys[ch];
        const Geom &geo = sa.batch.sys[sys].geo;
        const int64_t j = ch * kChunk + threadIdx.x;
        const uint32_t c = sa.cell[j];
        const bool act = c != kGhostCell;
        uint32_t before[kMaxLags];
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            before[l] = (act && ((sa.mask >> l) & 1u)) ? sa.lprev[l][j] : 0u;
        int32_t lx = 0, ly = 0;
        if (act) {
            const float2 p = sa.cl[j];
            const int32_t bx = base_cell((int32_t)(c & 0xffffu) * geo.k, p.x, geo.inv_g, geo.lg[0]);
            const int32_t by = base_cell((int32_t)(c >> 16) * geo.k, p.y, geo.inv_g, geo.lg[1]);
            lx = lattice_of_base(bx, geo.ratio, sa.ratio_shift);
            ly = lattice_of_base(by, geo.ratio, sa.ratio_shift);
        }
        const uint32_t now = pack_cell(lx, ly);
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l) {
            if (!((sa.mask >> l) & 1u)) continue;
            int32_t bin = 0;
            if (act) {
                const int32_t vx = lattice_disp(lx - (int32_t)(before[l] & 0xffffu), geo.lat[0]);
                const int32_t vy = lattice_disp(ly - (int32_t)(before[l] >> 16), geo.lat[1]);
                bin = vel_index(vx, vy, geo.vmax);
                sa.lprev[l][j] = now;
            }
            hist_add(sh + l * q1, bin, center, act);
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            if ((sa.mask >> l) & 1u)
                flush_hist(sh + l * q1, q1, sa.counts[l] + (size_t)sys * sa.nlags * q1);
        __syncthreads();
    }
}

// Lattice cell of every particle, stored as the starting point of every lag
// (with the position and velocity origins of the optional sums).
template <bool B>
__global__ void k_bin_seed(StateBinArgs sa) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < sa.n; j += stride) {
        const uint32_t c = sa.cell[j];
        if (B && c == kGhostCell) continue;
        const SysView sv = sys_view<B>(sa.geo, sa.batch, j);
        const Geom &geo = sv.geo;
        const float2 p = sa.cl[j];
        const int32_t ccx = (int32_t)(c & 0xffffu), ccy = (int32_t)(c >> 16);
        const int32_t bx = state_base(geo, sa.shift, 0, ccx * geo.k, p.x);
        const int32_t by = state_base(geo, sa.shift, 1, ccy * geo.k, p.y);
        const uint32_t now = pack_cell(lattice_of_base(bx, geo.ratio, sa.ratio_shift),
                                       lattice_of_base(by, geo.ratio, sa.ratio_shift));
        for (int l = 0; l < sa.nlags; ++l)
            if ((sa.mask >> l) & 1u) {
                sa.lprev[l][j] = now;
                if (sa.msd_acc) sa.mprev[l][j] = p;
                if (sa.vacf_acc) sa.vprev[l][j] = sa.vel[j];
            }
    }
}

// Collision operator of Eq. Xi.  One block per tile of TS consecutive sites
// of one lattice row y.
//  1. The tile's records of n_i(x, t) are contiguous in the site-major field:
//     they are read with 16-byte loads and stored negated into shared memory.
//  2. The needed n_i(x + v_i, t + dt) of velocity row v_y are the 2V+1
//     entries of that row group in the sites x0 - V .. x0 + TS - 1 + V of
//     lattice row y + v_y: one warp per velocity row, one lane per halo site
//     loads the 2V+1 contiguous entries, and entry k serves tile site lx - k
//     (a one-to-one map: it is added into shared memory without atomics;
//     lanes hit words Q apart, an odd stride, so the banks differ).
//  The first velocity row's loads are issued together with step 1's, so a
//  tile waits for memory once.  Xi leaves as one contiguous block of TS * Q
//  int32; one thread per site forms the mass and momentum sums.  V is a
//  template parameter, so every index division is by a constant.
__device__ __forceinline__ int32_t wrap_into(int32_t v, int32_t c) {
    while (v < 0) v += c;      // at most (V + TS) / c + 1 passes
    while (v >= c) v -= c;
    return v;
}

template <int V>
__host__ __device__ constexpr int coll_ts() {
    constexpr int q = (2 * V + 1) * (2 * V + 1);
    // 56 sites: 45 registers and five blocks per SM for V <= 3 (64 sites: 56
    // registers, four blocks, 12 % slower; 48 or 40 sites 2-3 % slower); TS x Q
    // int32 <= 48 KB
    return 12288 / q > 56 ? 56 : 12288 / q;
}

template <int V>
__global__ void __launch_bounds__(256, V <= 3 ? 5 : 1) k_collision(CollArgs ca) {
    constexpr int w = 2 * V + 1, q = w * w, q1 = q + 1;
    constexpr int TS = coll_ts<V>();
    constexpr int NV = ((TS * q1 + 6) / 4 + 255) / 256;     // 16-byte vectors per thread
    constexpr int NU = (TS + 2 * V + 31) / 32;               // halo sites per lane
    __shared__ int32_t xs[TS * q];
    const int32_t cx = ca.lat[0], cy = ca.lat[1];
    const int64_t cap = (int64_t)cx * cy * q1;                // words of a field
    const bool vec_ok = (reinterpret_cast<uintptr_t>(ca.prev) & 15) == 0;
    const int32_t tiles_x = (cx + TS - 1) / TS;
    const int64_t ntiles = (int64_t)tiles_x * cy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int32_t y = (int32_t)(tile / tiles_x);
        const int32_t x0 = (int32_t)(tile - (int64_t)y * tiles_x) * TS;
        const int32_t nx = min(TS, cx - x0);
        const int nl = nx + 2 * V;
        const int64_t s0 = (int64_t)y * cx + x0;
        // step 1 loads: words [a, e) of n_i(x, t) as 16-byte vectors from a0
        const int64_t a = s0 * q1, e = a + (int64_t)nx * q1, a0 = a & ~(int64_t)3;
        uint4 pv[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int64_t g = a0 + 4 * (int64_t)(threadIdx.x + u * 256);
            pv[u] = make_uint4(0u, 0u, 0u, 0u);
            if (g < e) {
                if (vec_ok && g + 4 <= cap) {
                    pv[u] = *reinterpret_cast<const uint4 *>(ca.prev + g);
                } else {
                    pv[u].x = ca.prev[g];
                    if (g + 1 < cap) pv[u].y = ca.prev[g + 1];
                    if (g + 2 < cap) pv[u].z = ca.prev[g + 2];
                    if (g + 3 < cap) pv[u].w = ca.prev[g + 3];
                }
            }
        }
        // step 2 loads of this warp's first velocity row
        uint32_t cv[NU][w];
        const uint32_t *rowbase = nullptr;
        if (warp < w) rowbase = ca.cur + (int64_t)wrap_into(y + warp - V, cy) * cx * q1 + warp * w;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int lx = lane + 32 * u;
            const bool on = warp < w && lx < nl;
            const uint32_t *src = on ? rowbase + (int64_t)wrap_into(x0 - V + lx, cx) * q1 : nullptr;
#pragma unroll
            for (int k = 0; k < w; ++k) cv[u][k] = on ? src[k] : 0u;
        }
        // step 1 stores
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int64_t g = a0 + 4 * (int64_t)(threadIdx.x + u * 256);
            const uint32_t wd[4] = {pv[u].x, pv[u].y, pv[u].z, pv[u].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (g + c < a || g + c >= e) continue;
                const int r = (int)(g + c - a);
                const int ls = r / q1, i = r - ls * q1;
                if (i < q) xs[ls * q + i] = -(int32_t)wd[c];
            }
        }
        __syncthreads();
        // step 2: first row from registers, further rows (V >= 4) loaded here
        for (int row = warp; row < w; row += nwarp) {
            if (row != warp) {
                const uint32_t *rb = ca.cur + (int64_t)wrap_into(y + row - V, cy) * cx * q1 + row * w;
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    const int lx = lane + 32 * u;
                    const uint32_t *src = lx < nl ? rb + (int64_t)wrap_into(x0 - V + lx, cx) * q1 : nullptr;
#pragma unroll
                    for (int k = 0; k < w; ++k) cv[u][k] = lx < nl ? src[k] : 0u;
                }
            }
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int lx = lane + 32 * u;
#pragma unroll
                for (int k = 0; k < w; ++k) {
                    const int ls = lx - k;
                    if (lx < nl && ls >= 0 && ls < nx) xs[ls * q + row * w + k] += (int32_t)cv[u][k];
                }
            }
        }
        __syncthreads();
        if (ca.xi) {
            int32_t *xo = ca.xi + s0 * q;
            for (int r = threadIdx.x; r < nx * q; r += blockDim.x) xo[r] = xs[r];
        }
        if (ca.dmass || ca.dmom) {
            for (int ls = threadIdx.x; ls < nx; ls += blockDim.x) {
                int32_t m = 0, jx = 0, jy = 0;
#pragma unroll
                for (int row = 0; row < w; ++row) {
                    int32_t rs = 0;
#pragma unroll
                    for (int k = 0; k < w; ++k) {
                        const int32_t x = xs[ls * q + row * w + k];
                        rs += x;
                        jx += (k - V) * x;
                    }
                    m += rs;
                    jy += (row - V) * rs;
                }
                if (ca.dmass) ca.dmass[s0 + ls] = m;
                if (ca.dmom) {
                    ca.dmom[2 * (s0 + ls)] = jx;
                    ca.dmom[2 * (s0 + ls) + 1] = jy;
                }
            }
        }
        __syncthreads();
    }
}

template <int V>
cudaError_t launch_collision_v(const CollArgs &ca, cudaStream_t s) {
    constexpr int TS = coll_ts<V>();
    const int64_t ntiles = (int64_t)((ca.lat[0] + TS - 1) / TS) * ca.lat[1];
    const int64_t cap = (int64_t)1 << 30;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_collision<V><<<grid < 1 ? 1 : grid, 256, 0, s>>>(ca);
    return cudaGetLastError();
}

}  // namespace

int hist_grid(int64_t n, int threads, int per_sm) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t need = (n + threads - 1) / threads;
    int64_t g = (int64_t)sms * per_sm;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_bin_snapshots(const LatticeArgs &la, int64_t n, const int32_t *prev,
                                 const int32_t *cur, unsigned long long *counts, uint32_t *ncell,
                                 uint32_t *field, cudaStream_t s) {
    const int threads = 256;
    const int q1 = (2 * la.vmax + 1) * (2 * la.vmax + 1) + 1;
    k_bin_snapshots<<<hist_grid(n, threads), threads, q1 * sizeof(uint32_t), s>>>(
        la, n, reinterpret_cast<const int2 *>(prev), reinterpret_cast<const int2 *>(cur), counts,
        ncell, field);
    return cudaGetLastError();
}

// NS of a pair list that forms a full grid -- every (dt, U) group holds the
// shifts 0 ... NS-1 in order -- for NS in 2..4, else 0 (runtime shifts).
int grid_shifts(const IdealGasArgs &ga) {
    int ns = 1;
    while (ns < ga.ncombo && !ga.first[ns]) ++ns;
    if (ns < 2 || ns > 4 || ga.ncombo % ns != 0) return 0;
    for (int k = 0; k < ga.ncombo; ++k)
        if (ga.shift[k] != k % ns || (ga.first[k] != 0) != (k % ns == 0)) return 0;
    return ns;
}

template <int NC>
cudaError_t launch_idealgas_nc(const IdealGasArgs &ga, int64_t n, const float *pos,
                               const float *vel, unsigned long long *counts, bool allpow2,
                               cudaStream_t s) {
    const int threads = 256;
    const int q1 = (2 * ga.vmax + 1) * (2 * ga.vmax + 1) + 1;
    const size_t smem = ((size_t)q1 * NC + 32) * sizeof(uint32_t);   // + one scratch word per lane
    const float2 *p2 = reinterpret_cast<const float2 *>(pos);
    const float2 *v2 = reinterpret_cast<const float2 *>(vel);
    void (*kern)(IdealGasArgs, int64_t, const float2 *, const float2 *, unsigned long long *);
    int64_t units = n;
    if (allpow2) {
        // two particles per thread when both arrays allow 16-byte loads
        const bool vec = ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(vel)) & 15) == 0;
        kern = vec ? k_idealgas_pow2<NC, 2> : k_idealgas_pow2<NC, 1>;
        const int ns = vec ? grid_shifts(ga) : 0;
        if constexpr (NC % 2 == 0) if (ns == 2) kern = k_idealgas_pow2<NC, 2, 2>;
        if constexpr (NC % 3 == 0) if (ns == 3) kern = k_idealgas_pow2<NC, 2, 3>;
        if constexpr (NC % 4 == 0) if (ns == 4) kern = k_idealgas_pow2<NC, 2, 4>;
        units = vec ? (n + 1) / 2 : n;
    } else {
        kern = k_idealgas_bin<NC, false>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<hist_grid(units, threads), threads, smem, s>>>(ga, n, p2, v2, counts);
    return cudaGetLastError();
}

cudaError_t launch_idealgas_bin(const IdealGasArgs &ga_in, int64_t n, const float *pos,
                                const float *vel, unsigned long long *counts, cudaStream_t s) {
    IdealGasArgs ga = ga_in;
    bool allpow2 = true;
    for (int k = 0; k < ga.ncombo; ++k) allpow2 = allpow2 && ga.pow2[k];
    for (int k = 0; k < ga.ncombo; ++k) ga.out[k] = k;
    if (allpow2) {
        // order the pairs by (dt, U), then by dx; record each pair's output row
        int ord[16];
        for (int k = 0; k < ga.ncombo; ++k) ord[k] = k;
        auto key_less = [&](int a, int b) {
            if (ga.dt[a] != ga.dt[b]) return ga.dt[a] < ga.dt[b];
            if (ga.boost && ga.ux[a] != ga.ux[b]) return ga.ux[a] < ga.ux[b];
            if (ga.boost && ga.uy[a] != ga.uy[b]) return ga.uy[a] < ga.uy[b];
            if (ga.dx[a] != ga.dx[b]) return ga.dx[a] < ga.dx[b];
            return a < b;
        };
        for (int i = 1; i < ga.ncombo; ++i)   // insertion sort of at most 16 pairs
            for (int j = i; j > 0 && key_less(ord[j], ord[j - 1]); --j) {
                const int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t;
            }
        float dxmin = ga.dx[0];
        for (int k = 1; k < ga.ncombo; ++k) dxmin = fminf(dxmin, ga.dx[k]);
        IdealGasArgs o = ga;
        for (int k = 0; k < ga.ncombo; ++k) {
            const int a = ord[k];
            o.dx[k] = ga.dx[a];
            o.dt[k] = ga.dt[a];
            o.inv_dx[k] = ga.inv_dx[a];
            o.pow2[k] = 1;
            o.ux[k] = ga.ux[a];
            o.uy[k] = ga.uy[a];
            o.out[k] = a;
            int sft = 0;   // dx_k / dx_min = 2^sft, both powers of two
            while (sft < 62 && std::ldexp((double)dxmin, sft) < (double)o.dx[k]) ++sft;
            o.shift[k] = sft;
            o.first[k] = k == 0 || o.dt[k] != o.dt[k - 1] ||
                         (ga.boost && (o.ux[k] != o.ux[k - 1] || o.uy[k] != o.uy[k - 1]));
        }
        o.inv_min = (float)(1.0 / (double)dxmin);
        ga = o;
    }
    switch (ga.ncombo) {
#define MDLG_IG_CASE(K) case K: return launch_idealgas_nc<K>(ga, n, pos, vel, counts, allpow2, s);
        MDLG_IG_CASE(1) MDLG_IG_CASE(2) MDLG_IG_CASE(3) MDLG_IG_CASE(4) MDLG_IG_CASE(5)
        MDLG_IG_CASE(6) MDLG_IG_CASE(7) MDLG_IG_CASE(8) MDLG_IG_CASE(9) MDLG_IG_CASE(10)
        MDLG_IG_CASE(11) MDLG_IG_CASE(12) MDLG_IG_CASE(13) MDLG_IG_CASE(14) MDLG_IG_CASE(15)
        MDLG_IG_CASE(16)
#undef MDLG_IG_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bin_state(const StateBinArgs &sa, cudaStream_t s) {
    const int q1 = (2 * sa.geo.vmax + 1) * (2 * sa.geo.vmax + 1) + 1;
    const size_t smem = (size_t)q1 * kMaxLags * sizeof(uint32_t);
    if (sa.batch.sys) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_bin_state_batch,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_bin_state_batch<<<hist_grid(sa.n, kChunk), kChunk, smem, s>>>(sa);
        return cudaGetLastError();
    }
    const int threads = 256;
    const bool msd = sa.msd_acc != nullptr || sa.vacf_acc != nullptr, move = sa.shift.on != 0;
    if (!msd && !move) {
        const int K = __builtin_popcount(sa.mask);
        void (*kv)(StateBinArgs) = nullptr;
        switch (K) {
            case 1: kv = k_bin_state_v<1>; break;
            case 2: kv = k_bin_state_v<2>; break;
            case 3: kv = k_bin_state_v<3>; break;
            case 4: kv = k_bin_state_v<4>; break;
            case 5: kv = k_bin_state_v<5>; break;
            case 6: kv = k_bin_state_v<6>; break;
            case 7: kv = k_bin_state_v<7>; break;
            case 8: kv = k_bin_state_v<8>; break;
            default: return cudaSuccess;
        }
        const size_t smv = (size_t)q1 * K * sizeof(uint32_t);
        if (smv > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv);
            if (e != cudaSuccess) return e;
        }
        kv<<<hist_grid((sa.n + 3) / 4, threads), threads, smv, s>>>(sa);
        return cudaGetLastError();
    }
    void (*kern)(StateBinArgs) = msd ? (move ? k_bin_state<true, true> : k_bin_state<true, false>)
                                     : (move ? k_bin_state<false, true> : k_bin_state<false, false>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // two waves of blocks per SM: fewer particles per thread (each one a
    // dependent load-store round) for twice the histogram flushes (6 % faster)
    kern<<<hist_grid(sa.n, threads, 16), threads, smem, s>>>(sa);
    return cudaGetLastError();
}

cudaError_t launch_collision(const CollArgs &ca, cudaStream_t s) {
    switch (ca.vmax) {
        case 1: return launch_collision_v<1>(ca, s);
        case 2: return launch_collision_v<2>(ca, s);
        case 3: return launch_collision_v<3>(ca, s);
        case 4: return launch_collision_v<4>(ca, s);
        case 5: return launch_collision_v<5>(ca, s);
        case 6: return launch_collision_v<6>(ca, s);
        case 7: return launch_collision_v<7>(ca, s);
        case 8: return launch_collision_v<8>(ca, s);
        case 9: return launch_collision_v<9>(ca, s);
        case 10: return launch_collision_v<10>(ca, s);
        case 11: return launch_collision_v<11>(ca, s);
        case 12: return launch_collision_v<12>(ca, s);
        case 13: return launch_collision_v<13>(ca, s);
        case 14: return launch_collision_v<14>(ca, s);
        case 15: return launch_collision_v<15>(ca, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bin_seed(const StateBinArgs &sa, cudaStream_t s) {
    const int threads = 256;
    if (sa.batch.sys) k_bin_seed<true><<<hist_grid(sa.n, threads), threads, 0, s>>>(sa);
    else k_bin_seed<false><<<hist_grid(sa.n, threads), threads, 0, s>>>(sa);
    return cudaGetLastError();
}

}  // namespace mdlg
