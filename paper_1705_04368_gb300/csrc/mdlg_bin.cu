// mdlg_bin.cu -- MDLG occupation-number kernels (Eq. MDni of arXiv:1705.04368).
//
// n_i(x,t) = sum_j Delta_x(x_j(t)) Delta_{x - v_i}(x_j(t - dt)): each particle
// contributes one count at its lattice cell at t, in the velocity given by its
// lattice displacement since t - dt.  All three kernels are grid-stride loops
// over particles with a block-private shared-memory histogram of the Q+1
// velocity bins, flushed once per block with 64-bit global atomics; optional
// per-site outputs (N(x,t), n_i(x,t)) are 32-bit global atomics.
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
// (no contraction into FMA): x' = fl(x + fl(v dt)), cell = ceil(fl(x / dx)) - 1.
// Multiplying by 1/dx equals dividing by dx when dx is a power of two.
__global__ void k_idealgas_bin(IdealGasArgs ga, int64_t n, const float2 *__restrict__ pos,
                               const float2 *__restrict__ vel, unsigned long long *counts) {
    extern __shared__ uint32_t sh[];
    const int w = 2 * ga.vmax + 1, q1 = w * w + 1;
    const int center = ga.vmax * w + ga.vmax;
    for (int b = threadIdx.x; b < q1 * ga.ncombo; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool act = j < n;
        float2 p = make_float2(1.f, 1.f), v = make_float2(0.f, 0.f);
        if (act) {
            p = pos[j];
            v = vel[j];
        }
        float last_dx = -1.f;
        int32_t c0x = 0, c0y = 0;
        for (int k = 0; k < ga.ncombo; ++k) {
            const float dx = ga.dx[k], dt = ga.dt[k];
            const bool pow2 = ga.pow2[k] != 0;
            const float inv = ga.inv_dx[k];
            if (dx != last_dx) {
                const float qx = pow2 ? __fmul_rn(p.x, inv) : __fdiv_rn(p.x, dx);
                const float qy = pow2 ? __fmul_rn(p.y, inv) : __fdiv_rn(p.y, dx);
                c0x = __float2int_ru(qx) - 1;
                c0y = __float2int_ru(qy) - 1;
                last_dx = dx;
            }
            const float xn = __fadd_rn(p.x, __fmul_rn(v.x, dt));
            const float yn = __fadd_rn(p.y, __fmul_rn(v.y, dt));
            const float qx = pow2 ? __fmul_rn(xn, inv) : __fdiv_rn(xn, dx);
            const float qy = pow2 ? __fmul_rn(yn, inv) : __fdiv_rn(yn, dx);
            const int32_t vx = __float2int_ru(qx) - 1 - c0x;
            const int32_t vy = __float2int_ru(qy) - 1 - c0y;
            hist_add(sh + k * q1, vel_index(vx, vy, ga.vmax), center, act);
        }
    }
    __syncthreads();
    for (int k = 0; k < ga.ncombo; ++k) flush_hist(sh + k * q1, q1, counts + (size_t)k * q1);
}

// Binning of the simulation state (sorted by MD cell) for the lags in `mask`:
// the lattice cell now versus the one stored at the lag's previous binning,
// which is then replaced.  Lag 0 may also write per-site outputs.  Every load
// of an iteration is issued before any of its stores (a store followed by a
// load the compiler cannot prove independent stalls the thread), and the lag
// loop is unrolled over the compile-time maximum, predicated by the mask.
__global__ void k_bin_state(StateBinArgs sa) {
    extern __shared__ uint32_t sh[];
    const Geom &geo = sa.geo;
    const int w = 2 * geo.vmax + 1, q1 = w * w + 1;
    const int center = geo.vmax * w + geo.vmax;
    for (int b = threadIdx.x; b < q1 * kMaxLags; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < sa.n; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool act = j < sa.n;
        uint32_t before[kMaxLags];
#pragma unroll
        for (int l = 0; l < kMaxLags; ++l)
            before[l] = (act && ((sa.mask >> l) & 1u)) ? sa.lprev[l][j] : 0u;
        int32_t lx = 0, ly = 0;
        if (act) {
            const uint32_t c = sa.cell[j];
            const float2 p = sa.cl[j];
            const int32_t ccx = (int32_t)(c & 0xffffu), ccy = (int32_t)(c >> 16);
            const int32_t bx = base_cell(ccx * geo.k, p.x, geo.inv_g, geo.lg[0]);
            const int32_t by = base_cell(ccy * geo.k, p.y, geo.inv_g, geo.lg[1]);
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

// Lattice cell of every particle, stored as the starting point of every lag.
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
        const int32_t bx = base_cell(ccx * geo.k, p.x, geo.inv_g, geo.lg[0]);
        const int32_t by = base_cell(ccy * geo.k, p.y, geo.inv_g, geo.lg[1]);
        const uint32_t now = pack_cell(lattice_of_base(bx, geo.ratio, sa.ratio_shift),
                                       lattice_of_base(by, geo.ratio, sa.ratio_shift));
        for (int l = 0; l < sa.nlags; ++l)
            if ((sa.mask >> l) & 1u) sa.lprev[l][j] = now;
    }
}

}  // namespace

int hist_grid(int64_t n, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t need = (n + threads - 1) / threads;
    int64_t g = (int64_t)sms * 8;
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

cudaError_t launch_idealgas_bin(const IdealGasArgs &ga, int64_t n, const float *pos,
                                const float *vel, unsigned long long *counts, cudaStream_t s) {
    const int threads = 256;
    const int q1 = (2 * ga.vmax + 1) * (2 * ga.vmax + 1) + 1;
    const size_t smem = (size_t)q1 * ga.ncombo * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_idealgas_bin,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_idealgas_bin<<<hist_grid(n, threads), threads, smem, s>>>(
        ga, n, reinterpret_cast<const float2 *>(pos), reinterpret_cast<const float2 *>(vel), counts);
    return cudaGetLastError();
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
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bin_state,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_bin_state<<<hist_grid(sa.n, threads), threads, smem, s>>>(sa);
    return cudaGetLastError();
}

cudaError_t launch_bin_seed(const StateBinArgs &sa, cudaStream_t s) {
    const int threads = 256;
    if (sa.batch.sys) k_bin_seed<true><<<hist_grid(sa.n, threads), threads, 0, s>>>(sa);
    else k_bin_seed<false><<<hist_grid(sa.n, threads), threads, 0, s>>>(sa);
    return cudaGetLastError();
}

}  // namespace mdlg
