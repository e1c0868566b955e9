// mdlg_adjoint.cu -- reverse-mode kernels for gradients of soft-binned MDLG
// occupations through the Lennard-Jones leapfrog trajectory.
//
// Loss.  The cell indicator of Sec. III is smoothed with a Gaussian of standard
// deviation s: u_c(x) = Phi((x - c dx)/s) - Phi((x - (c+1) dx)/s).  Over one
// interval [0, K] the soft occupations of Eq. MDni, averaged over particles,
//     ft_i = (1/N) sum_j prod_a k_a(v_ia),  k_a(v) = sum_c u_c(x_ja(K)) u_{c-v}(x_ja(0)),
// are combined with caller weights w_i into L = sum_i w_i ft_i.
//
// Adjoint of one leapfrog step (x_n, v_{n-1/2}) -> (x_{n+1}, v_{n+1/2}) with
// v_{n+1/2} = v_{n-1/2} + F(x_n) dt/m, x_{n+1} = x_n + v_{n+1/2} dt: given the
// adjoints (xb_{n+1}, vb_{n+1/2}),
//     w = vb_{n+1/2} + xb_{n+1} dt,   xb_n = xb_{n+1} + (dt/m) (dF/dx)^T w,
//     vb_{n-1/2} = w,                 theta_b += (dt/m) (dF/dtheta)^T w.
// For a pair force F_ij = f(q) d_ij (d_ij = x_i - x_j, q = |d|^2) the Jacobian
// block is J_ij = f I + 2 f'(q) d d^T, symmetric, and dF_i/dx_j = -J_ij, so
// ((dF/dx)^T w)_i = sum_j J_ij (w_i - w_j).
#include "mdlg_kernels.h"

namespace mdlg {

namespace {

constexpr int kAdjThreads = 128;
constexpr int kSoftMaxM = 8;      // cells searched each side of a point (width <= 0.875 dx)
constexpr int kSoftMaxV = 7;

__device__ __forceinline__ double ncdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752440); }
__device__ __forceinline__ double npdf(double z) { return 0.39894228040143267794 * exp(-0.5 * z * z); }

__device__ __forceinline__ int32_t cx_of(uint32_t cw) { return (int32_t)(cw & 0xffffu); }
__device__ __forceinline__ int32_t cy_of(uint32_t cw) { return (int32_t)(cw >> 16); }

// Soft loss, its per-bin values and its gradient for every particle.
__global__ void k_soft_loss(SoftArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n) return;
    const Geom &geo = a.geo;
    const uint32_t cw = a.cell[j];
    const float2 cl = a.cl[j];
    const int64_t o = a.pid[j];
    const double pa[2] = {(double)(cx_of(cw) * geo.k) * geo.g + (double)cl.x,
                          (double)(cy_of(cw) * geo.k) * geo.g + (double)cl.y};
    const double pb[2] = {a.x_start[2 * o], a.x_start[2 * o + 1]};
    const int V = a.vmax, W = 2 * V + 1, M = a.M;
    double k[2][2 * kSoftMaxV + 1], dka[2][2 * kSoftMaxV + 1], dkb[2][2 * kSoftMaxV + 1];
    for (int ax = 0; ax < 2; ++ax) {
        const double L = (double)geo.lg[ax] * geo.g;
        double d = pa[ax] - pb[ax];
        d -= L * rint(d / L);
        const double ta = pa[ax] / a.dx, tb = (pa[ax] - d) / a.dx, sw = a.width / a.dx;
        const double base = floor(ta);
        double ua[2 * kSoftMaxM + 1], dua[2 * kSoftMaxM + 1];
        for (int dc = -M; dc <= M; ++dc) {
            const double c = base + dc;
            const double z0 = (ta - c) / sw, z1 = (ta - c - 1.0) / sw;
            ua[dc + M] = ncdf(z0) - ncdf(z1);
            dua[dc + M] = (npdf(z0) - npdf(z1)) / sw;    // d/d(ta)
        }
        double ub[2 * kSoftMaxM + 2 * kSoftMaxV + 1], dub[2 * kSoftMaxM + 2 * kSoftMaxV + 1];
        for (int e = -M - V; e <= M + V; ++e) {         // cell base + e of the start point
            const double c = base + e;
            const double z0 = (tb - c) / sw, z1 = (tb - c - 1.0) / sw;
            ub[e + M + V] = ncdf(z0) - ncdf(z1);
            dub[e + M + V] = (npdf(z0) - npdf(z1)) / sw;
        }
        for (int v = -V; v <= V; ++v) {
            double s = 0.0, sa = 0.0, sb = 0.0;
            for (int dc = -M; dc <= M; ++dc) {
                const int e = dc - v + M + V;            // cell (base + dc) - v
                s += ua[dc + M] * ub[e];
                sa += dua[dc + M] * ub[e];
                sb += ua[dc + M] * dub[e];
            }
            k[ax][v + V] = s;
            dka[ax][v + V] = sa;
            dkb[ax][v + V] = sb;
        }
    }
    const double invn = 1.0 / (double)a.ntot;
    double ga[2] = {0.0, 0.0}, gb[2] = {0.0, 0.0}, lsum = 0.0;
    for (int vy = 0; vy < W; ++vy)
        for (int vx = 0; vx < W; ++vx) {
            const int i = vy * W + vx;
            const double kk = k[0][vx] * k[1][vy];
            if (a.fsum) atomicAdd(&a.fsum[i], kk * invn);
            const double wi = a.weights ? a.weights[i] : 0.0;
            lsum += wi * kk;
            ga[0] += wi * dka[0][vx] * k[1][vy];
            ga[1] += wi * k[0][vx] * dka[1][vy];
            gb[0] += wi * dkb[0][vx] * k[1][vy];
            gb[1] += wi * k[0][vx] * dkb[1][vy];
        }
    if (a.loss) atomicAdd(a.loss, lsum * invn);
    const double sc = invn / a.dx;                      // d/d(x) = (1/dx) d/d(tx)
    if (a.xb) a.xb[j] = make_float2((float)(ga[0] * sc), (float)(ga[1] * sc));
    if (a.gx_start) {
        a.gx_start[2 * o] = gb[0] * sc;
        a.gx_start[2 * o + 1] = gb[1] * sc;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

struct PairAdj {
    float gx, gy, te, ts;
};

// Jacobian-vector product and parameter derivatives of one pair.  Shifted
// force (potential 2): f -> f - F(rc)/r, f'(q) gains F(rc)/(2 q^(3/2)), and
// df/dsigma gains -(dF(rc)/dsigma)/r.
__device__ __forceinline__ void pair_adj(const AdjArgs &a, float dx, float dy, float2 wi,
                                         float2 wj, PairAdj &acc) {
    const float q = fmaf(dx, dx, dy * dy);
    if (!(q < a.rc2)) return;
    const float iq = 1.0f / q;
    const float sr2 = a.sig2 * iq;
    const float sr6 = sr2 * sr2 * sr2;
    float f = a.eps24 * iq * sr6 * (2.0f * sr6 - 1.0f);          // F_ij = f d
    float dfdq = a.eps24 * iq * iq * sr6 * (4.0f - 14.0f * sr6);  // f'(q)
    // df/dsigma = 24 eps (24 s^12 - 6 s^6) / (sigma q)
    float dfds = a.eps24 * a.inv_sigma * iq * sr6 * (24.0f * sr6 - 6.0f);
    if (a.potential == 2) {
        const float ir = rsqrtf(q);
        f -= a.fc * ir;
        dfdq += 0.5f * a.fc * ir * iq;
        dfds -= a.dfc_dsigma * ir;
    }
    const float wx = wi.x - wj.x, wy = wi.y - wj.y;
    const float ddw = fmaf(dx, wx, dy * wy);
    acc.gx = fmaf(f, wx, fmaf(2.0f * dfdq * ddw, dx, acc.gx));
    acc.gy = fmaf(f, wy, fmaf(2.0f * dfdq * ddw, dy, acc.gy));
    const float dwi = fmaf(dx, wi.x, dy * wi.y);
    acc.te = fmaf(f * a.inv_eps, dwi, acc.te);                     // df/deps = f / eps
    acc.ts = fmaf(dfds, dwi, acc.ts);
}

// One adjoint leapfrog step (or, with a_coef = 0, the initial half kick).
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_step(AdjArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < a.n;
    const Geom &geo = a.geo;
    const float D = a.ctl->dbound;      // bound at the end of the segment: covers every step
    const bool list_ok = a.nbr != nullptr && 2.0f * D <= a.list_skin;
    PairAdj acc = {0.f, 0.f, 0.f, 0.f};
    float2 w = make_float2(0.f, 0.f), xb = make_float2(0.f, 0.f);
    if (act) {
        xb = a.xb[i];
        const float2 wp = a.w_prev[i];
        w = make_float2(fmaf(a.a_coef, xb.x, wp.x), fmaf(a.a_coef, xb.y, wp.y));
        if (a.potential) {
            const uint32_t cw = a.cell[i];
            const int32_t cx = cx_of(cw), cy = cy_of(cw);
            const float2 p = a.x[i];
            const int cnt = list_ok ? a.ncount[i] : a.cap + 1;
            if (cnt <= a.cap) {
                const float sxm = (float)wrap_half((wrap_mod(cx - 1, geo.nc[0]) - cx) * geo.k, geo.lg[0]) * geo.g;
                const float sxp = (float)wrap_half((wrap_mod(cx + 1, geo.nc[0]) - cx) * geo.k, geo.lg[0]) * geo.g;
                const float sym = (float)wrap_half((wrap_mod(cy - 1, geo.nc[1]) - cy) * geo.k, geo.lg[1]) * geo.g;
                const float syp = (float)wrap_half((wrap_mod(cy + 1, geo.nc[1]) - cy) * geo.k, geo.lg[1]) * geo.g;
                for (int t = 0; t < cnt; ++t) {
                    const uint32_t ent = a.nbr[((int64_t)(t >> 2) * a.n + i) * 4 + (t & 3)];
                    const int32_t j = (int32_t)(ent & 0x0fffffffu);
                    const uint32_t ox = (ent >> 28) & 3u, oy = ent >> 30;
                    const float sx = ox == 0u ? sxm : (ox == 2u ? sxp : 0.0f);
                    const float sy = oy == 0u ? sym : (oy == 2u ? syp : 0.0f);
                    const float2 q = a.x[j];
                    const float2 xbj = a.xb[j], wpj = a.w_prev[j];
                    const float2 wj = make_float2(fmaf(a.a_coef, xbj.x, wpj.x), fmaf(a.a_coef, xbj.y, wpj.y));
                    pair_adj(a, (p.x - q.x) - sx, (p.y - q.y) - sy, w, wj, acc);
                }
            } else {
                const float Rf = ceilf((a.rc + 2.0f * D) / a.cell_w);
                const int R = (Rf >= 1.0f) ? (Rf < 65536.0f ? (int)Rf : 65536) : 1;
                int lox = -R, hix = R, loy = -R, hiy = R;
                if (2 * R + 1 > geo.nc[0]) { lox = -(geo.nc[0] >> 1); hix = lox + geo.nc[0] - 1; }
                if (2 * R + 1 > geo.nc[1]) { loy = -(geo.nc[1] >> 1); hiy = loy + geo.nc[1] - 1; }
                for (int oy = loy; oy <= hiy; ++oy) {
                    const int32_t ny = wrap_mod(cy + oy, geo.nc[1]);
                    const float ody = (float)wrap_half((ny - cy) * geo.k, geo.lg[1]) * geo.g;
                    for (int ox = lox; ox <= hix; ++ox) {
                        const int32_t nx = wrap_mod(cx + ox, geo.nc[0]);
                        const float odx = (float)wrap_half((nx - cx) * geo.k, geo.lg[0]) * geo.g;
                        const int32_t cn = ny * geo.nc[0] + nx;
                        const int32_t s = a.cell_start[cn], e = a.cell_start[cn + 1];
                        for (int32_t j = s; j < e; ++j) {
                            if (j == i) continue;
                            const float2 q = a.x[j];
                            const float2 xbj = a.xb[j], wpj = a.w_prev[j];
                            const float2 wj = make_float2(fmaf(a.a_coef, xbj.x, wpj.x),
                                                          fmaf(a.a_coef, xbj.y, wpj.y));
                            pair_adj(a, (p.x - q.x) - odx, (p.y - q.y) - ody, w, wj, acc);
                        }
                    }
                }
            }
        }
        a.xb_out[i] = make_float2(fmaf(a.b_coef, acc.gx, xb.x), fmaf(a.b_coef, acc.gy, xb.y));
        a.w_out[i] = w;
    }
    // parameter adjoints: FP64 from the per-particle FP32 sums
    double te = act ? (double)a.b_coef * (double)acc.te : 0.0;
    double ts = act ? (double)a.b_coef * (double)acc.ts : 0.0;
    te = warp_sum_d(te);
    ts = warp_sum_d(ts);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&a.theta[0], te);
        atomicAdd(&a.theta[1], ts);
    }
}

__global__ void k_gather2(int64_t n, const int32_t *pid, const float2 *src, float2 *dst) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[pid[j]];
}

__global__ void k_scatter2(int64_t n, const int32_t *pid, const float2 *src, float2 *dst) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[pid[j]] = src[j];
}

}  // namespace

cudaError_t launch_soft_loss(const SoftArgs &a, cudaStream_t s) {
    if (a.n < 1) return cudaSuccess;
    k_soft_loss<<<(unsigned)((a.n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const AdjArgs &a, cudaStream_t s) {
    if (a.n < 1) return cudaSuccess;
    k_adjoint_step<<<(unsigned)((a.n + kAdjThreads - 1) / kAdjThreads), kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_permute(int64_t n, const int32_t *pid, const float2 *src, float2 *dst,
                           bool to_original, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
    if (to_original) k_scatter2<<<g, 256, 0, s>>>(n, pid, src, dst);
    else k_gather2<<<g, 256, 0, s>>>(n, pid, src, dst);
    return cudaGetLastError();
}

}  // namespace mdlg
