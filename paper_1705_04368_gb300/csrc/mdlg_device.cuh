// mdlg_device.cuh -- device-side types and helpers shared by the MDLG kernels.
//
// State layout (device, structure of arrays, sorted by neighbour ("MD") cell):
//   cell[j]  int32   MD cell the particle was sorted into (row-major, x fastest)
//   cl[j]    float2  position relative to that cell's origin, in length units
//   vel[j]   float2  velocity (half-step velocity v_{n-1/2} between steps)
//   pid[j]   int32   original particle number
//   lprev[l][j] uint32 lattice cell of the particle at the last binning of
//            lag l, packed (c_y << 16) | c_x
//   mprev[l][j] float2 (mean-square displacement only) the particle's offset at
//            the last binning of lag l, re-expressed against its current MD
//            cell's origin at every re-sort, so cl - mprev is the displacement
// A cell's origin is an integer number of base cells g (g a power of two), so
// every position is "integer + binary32 offset": the base cell of a particle,
// and therefore its lattice cell, is exact integer arithmetic, and pair
// separations are differences of small offsets plus a small integer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mdlg {

constexpr int kMaxLags = 8;
constexpr int kMaxVmax = 15;

// Geometry of the base grid, the MD cells and the MDLG lattice.
struct Geom {
    int32_t lg[2];     // base cells per axis (L / g)
    int32_t nc[2];     // MD cells per axis; cell c spans base cells [c k, (c+1) k),
                       // the last one also takes the remainder lg - nc k
    int32_t k;         // base cells per MD cell
    float g;           // base grid spacing (power of two)
    float inv_g;       // 1 / g (exact)
    int32_t ratio;     // lattice spacing dx / g
    int32_t lat[2];    // lattice cells per axis
    int32_t vmax;      // window half-width V
};

// Wrap an integer base-cell difference into [-lg/2, lg/2).
__device__ __forceinline__ int32_t wrap_half(int32_t d, int32_t lg) {
    if (d >= (lg >> 1)) d -= lg;
    if (d < -(lg >> 1)) d += lg;
    return d;
}

__device__ __forceinline__ int32_t wrap_mod(int32_t d, int32_t m) {
    if (d < 0) d += m;
    if (d >= m) d -= m;
    return d;
}

// ceil(t) for |t| < 2^22 without a conversion instruction: t + 1.5 * 2^23
// rounded up lands on an integer in [2^23, 2^24), where binary32 spacing is 1,
// so the result is 1.5 * 2^23 + ceil(t) exactly; its bit pattern minus that of
// 1.5 * 2^23 is ceil(t).
__device__ __forceinline__ int32_t ceil_small(float t) {
    return __float_as_int(__fadd_ru(t, 12582912.0f)) - 0x4B400000;
}

// Base cell of a particle: the cell (b g, (b+1) g] that holds origin + cl.
// cl / g is exact (g a power of two), ceil(t) - 1 is the left-open rule.  A
// particle is within a few cells of its MD cell's origin, so one conditional
// wrap suffices; the clamp keeps any input (even a non-finite offset, which is
// flagged elsewhere) a valid index.
__device__ __forceinline__ int32_t base_cell(int32_t origin, float cl, float inv_g, int32_t lg) {
    const float lim = (float)lg;
    const float t = fminf(fmaxf(cl * inv_g, -lim + 1.0f), lim);   // NaN -> -lim + 1
    int32_t b = origin + ceil_small(t) - 1;
    b += b < 0 ? lg : 0;
    b -= b >= lg ? lg : 0;
    return b;
}

// Base cell of origin + cl + S on a lattice displaced by S = (K + b) g, K in
// [0, lg), b in [0, 1) a multiple of 2^-24 (omb = 1 - b, exact).  With a = cl/g
// (exact), k = floor(a) and f = a - k (exact), ceil(a + b) = k + j where
// j = 0 if f = b = 0, 2 if f > 1 - b, else 1: every decision is an exact
// comparison, so the cell of the real number x + S is found without rounding.
__device__ __forceinline__ int32_t base_cell_moving(int32_t origin, float cl, float inv_g,
                                                    int32_t lg, int32_t K, float omb) {
    const float a = cl * inv_g;
    const float k = floorf(a);
    const float f = a - k;
    const float j = (f == 0.0f && omb == 1.0f) ? 0.0f : (f > omb ? 2.0f : 1.0f);
    const float lim = (float)lg;
    const float t = fminf(fmaxf(k + j, -lim + 1.0f), lim + 1.0f);
    int32_t b = origin + K + (int32_t)t - 1;     // in [-lg, 3 lg)
    b += b < 0 ? lg : 0;
    b -= b >= lg ? lg : 0;
    b -= b >= lg ? lg : 0;
    return b;
}

// Lattice displacement of two cells in [0, C), reduced into (-C/2, C/2].
__device__ __forceinline__ int32_t lattice_disp(int32_t d, int32_t C) {
    d += d < 0 ? C : 0;               // [0, C)
    d -= d > (C >> 1) ? C : 0;        // (-C/2, C/2]
    return d;
}

// Velocity index of a lattice displacement (vx, vy); Q for outside the window.
__device__ __forceinline__ int32_t vel_index(int32_t vx, int32_t vy, int32_t vmax) {
    const int32_t w = 2 * vmax + 1;
    if (vx < -vmax || vx > vmax || vy < -vmax || vy > vmax) return w * w;
    return (vy + vmax) * w + (vx + vmax);
}

__device__ __forceinline__ uint32_t pack_cell(int32_t cx, int32_t cy) {
    return ((uint32_t)cy << 16) | (uint32_t)cx;
}

// Add one count to a block-shared histogram.  Most particles of a short
// coarse step land in the rest velocity, so the lanes that do are counted by
// one ballot and a single shared atomic; the rest add individually.
__device__ __forceinline__ void hist_add(uint32_t *sh, int32_t bin, int32_t center, bool active) {
    const unsigned full = 0xffffffffu;
    unsigned rest = __ballot_sync(full, active && bin == center);
    if (rest && (threadIdx.x & 31) == (unsigned)(__ffs(rest) - 1)) atomicAdd(&sh[center], (uint32_t)__popc(rest));
    if (active && bin != center) atomicAdd(&sh[bin], 1u);
}

}  // namespace mdlg
