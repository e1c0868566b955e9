// mdlg_kernels.h -- argument blocks and launchers of the MDLG kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mdlg_device.cuh"

namespace mdlg {

// ---- batches of independent systems ------------------------------------------
// A batch keeps every system's particles in one contiguous slot range padded to
// a multiple of kChunk slots; padding slots hold ghost particles (cell word
// kGhostCell) that take part in nothing.  Every chunk of kChunk slots belongs to
// one system, so a warp always works on one system and looks its geometry up.
// Each system owns the global cells [cell0, cell0 + ncells] (the last one holds
// its ghosts), so one counting sort orders all systems at once.
constexpr int kChunk = 128;
constexpr uint32_t kGhostCell = 0xffffffffu;

struct SysInfo {
    Geom geo;          // this system's lg, nc, lat (k, g, ratio, vmax as the batch's)
    int64_t p0;        // first slot
    int64_t q0;        // first particle in the caller's concatenated order
    int64_t n;         // particles (slots p0 .. p0+n-1; the rest of the range are ghosts)
    int64_t cell0;     // first global cell
    int32_t ncells;    // nc[0] * nc[1]; global cell cell0 + ncells is the ghost cell
    int32_t pad_;
};

struct Batch {
    const SysInfo *sys;          // null: a single system described by the kernel's Geom
    const uint16_t *chunk_sys;   // system of every kChunk-slot chunk
    long long *stats;            // nsys x 5 exact fixed-point sums of a statistics launch
    int32_t nsys;
};

// Geometry and cell range of the system that owns a slot.
struct SysView {
    Geom geo;
    int64_t cell0;
    int32_t ncells;
    int32_t sys;
};

template <bool B>
__device__ __forceinline__ SysView sys_view(const Geom &single, const Batch &b, int64_t slot) {
    SysView v;
    if (!B) {
        v.geo = single;
        v.cell0 = 0;
        v.ncells = single.nc[0] * single.nc[1];
        v.sys = 0;
    } else {
        const int s = b.chunk_sys[slot / kChunk];
        const SysInfo &si = b.sys[s];
        v.geo = si.geo;
        v.cell0 = si.cell0;
        v.ncells = si.ncells;
        v.sys = s;
    }
    return v;
}

// ---- binning ---------------------------------------------------------------
struct LatticeArgs {
    int32_t base[2];   // base cells per axis
    int32_t ratio;     // base cells per lattice cell
    int32_t shift;     // log2(ratio) if a power of two, else -1
    int32_t lat[2];    // lattice cells per axis
    int32_t vmax;
};

struct IdealGasArgs {
    int32_t ncombo;
    int32_t vmax;
    float dx[16], dt[16], inv_dx[16];
    int32_t pow2[16];
    int32_t boost;             // 1: velocities boosted by (ux[k], uy[k]) per pair
    float ux[16], uy[16];
    // every dx a power of two: the pairs are ordered so that pairs with the same
    // (dt, U) are adjacent, and each decision is a shift of the cell at dx_min
    int32_t out[16];           // counts row of pair k (the caller's order)
    int32_t shift[16];         // log2(dx_k / dx_min)
    int32_t first[16];         // 1: pair k is the first of its (dt, U) group
    float inv_min;             // 1 / dx_min (a power of two)
};

// Lattice displacement S = (K + b) g per axis of a moving lattice, K in [0, lg),
// b in [0, 1) a multiple of 2^-24, passed as 1 - b (exact in binary32).
struct LatticeShift {
    int32_t on;
    int32_t K[2];
    float omb[2];
};

struct StateBinArgs {
    Geom geo;
    int64_t n;
    int32_t ratio_shift;   // log2(ratio) or -1
    int32_t nlags;
    uint32_t mask;         // lags binned by this launch
    const uint32_t *cell;   // packed MD cell (c_x | c_y << 16)
    const float2 *cl;
    uint32_t *lprev[kMaxLags];
    unsigned long long *counts[kMaxLags];
    uint32_t *site_n;       // lag 0 per-site N(x,t), or null
    uint32_t *site_counts;  // lag 0 per-site n_i(x,t), or null
    Batch batch;            // batched: counts[l] point at system 0, system s at + s*nlags*q1
    LatticeShift shift;     // moving lattice (single systems)
    float2 *mprev[kMaxLags];  // per lag: offset at its previous binning, against the
                              // particle's current MD cell (mean-square displacement), or null
    double *msd_acc;        // nlags x 2 sums of squared displacements (added to)
    const float2 *vel;        // half-step velocities of the binned state
    float2 *vprev[kMaxLags];  // per lag: velocity at its previous binning (correlation), or null
    double *vacf_acc;         // nlags x 2 sums of velocity products (added to), or null
};

struct CollArgs {
    int32_t lat[2];
    int32_t vmax;
    const uint32_t *prev, *cur;   // C_y*C_x*(Q+1) occupation fields
    int32_t *xi;                  // C_y*C_x*Q, or null
    int32_t *dmass;               // C_y*C_x, or null
    int32_t *dmom;                // C_y*C_x*2, or null
};

int hist_grid(int64_t n, int threads, int per_sm = 8);   // blocks: per_sm per SM at most
cudaError_t launch_bin_snapshots(const LatticeArgs &la, int64_t n, const int32_t *prev,
                                 const int32_t *cur, unsigned long long *counts, uint32_t *ncell,
                                 uint32_t *field, cudaStream_t s);
cudaError_t launch_idealgas_bin(const IdealGasArgs &ga, int64_t n, const float *pos,
                                const float *vel, unsigned long long *counts, cudaStream_t s);
cudaError_t launch_bin_state(const StateBinArgs &sa, cudaStream_t s);
cudaError_t launch_bin_seed(const StateBinArgs &sa, cudaStream_t s);
cudaError_t launch_collision(const CollArgs &ca, cudaStream_t s);

// ---- molecular dynamics ------------------------------------------------------
// Device control block of one context (one allocation).
struct Control {
    float dbound;              // bound on any particle's distance outside its MD cell
    uint32_t vmax2_bits;       // max |v|^2 of the running step (float bits)
    uint32_t done;             // blocks finished in the running launch
    int32_t status;            // first device-side error (MDLG_E* value) or 0
    double stats[8];           // ke, pe, virial, px, py of the last stats launch
    unsigned long long vmax0_bits;   // max |v|^2 of the uploaded state (FP64 bits; >= 0)
    long long stats_acc[5];    // fixed-point sums of a running stats launch (zero at rest)
    uint32_t stale_steps;      // step launches that found the Verlet list out of date
};

// One MD step's displacement bound and largest speed, written by the last block
// of the step launch into host-mapped memory; the host paces the re-sorts from
// these (ring of kPaceRing slots indexed by step).
struct PaceSlot {
    int64_t step;              // MD step whose launch wrote the slot (-1: empty)
    float dbound;              // bound after that step (the next step's input positions)
    uint32_t vmax2_bits;       // largest |v|^2 of the step's half-step velocities (float bits)
};
constexpr int kPaceRing = 8;

enum StepMode : int32_t {
    kModeStep = 0,   // F(x_n); v_{n+1/2} = v_{n-1/2} + F dt/m; x_{n+1} = x_n + v dt
    kModeInit = 1,   // F(x_0); v_{-1/2} = v_0 - F dt/(2m)        (positions kept)
    kModeSync = 2,   // F(x_n); v_n = v_{n-1/2} + F dt/(2m) into sync buffers
};

struct StepArgs {
    Geom geo;
    int64_t n;
    const uint32_t *cell;       // packed MD cell (c_x | c_y << 16)
    const int32_t *cell_start;  // nc[0]*nc[1] + 1, by row-major cell number
    const float2 *cl_in;
    const float2 *v_in;
    float2 *cl_out;             // kModeStep
    float2 *v_out;              // kModeStep / kModeInit
    float2 *v_sync;             // kModeSync: v_n
    float2 *f_sync;             // kModeSync: F(x_n), or null
    float rc2, sig2, eps24, eps4, vshift;
    float dt, dt_m, half_dt_m, mass;
    float cell_w;               // k g: narrowest MD cell width
    float rc;
    float round_margin;         // per-step slack added to the displacement bound
    const uint32_t *nbr;        // Verlet list in batches of four (cap x n), or null
    const int32_t *ncount;      // entries per particle (cap + 1: overflowed)
    int32_t cap;                // list capacity per particle
    float list_skin;            // list radius - rc
    int32_t potential;          // 0 none, 1 LJ truncated-shifted, 2 LJ shifted-force
    float fc;                   // |F(rc)| (shifted-force subtracts it)
    int32_t stats;              // 1: FP64 reductions (Control::stats, or per system in a batch)
    Control *ctl;
    Batch batch;
    PaceSlot *pace;             // kModeStep: host-mapped ring for this step's bound, or null
    int64_t step;               // MD step of this launch (slot step % kPaceRing)
};

cudaError_t launch_step(const StepArgs &a, int mode, cudaStream_t s);

struct SortArgs {
    Geom geo;
    int64_t n;
    int32_t nlags;
    int64_t ncells;
    // current state
    const uint32_t *cell_in;
    const float2 *cl_in;
    const float2 *v_in;
    const int32_t *pid_in;
    const uint32_t *lprev_in[kMaxLags];
    // sorted state
    uint32_t *cell_out;
    float2 *cl_out;
    float2 *v_out;
    int32_t *pid_out;
    uint32_t *lprev_out[kMaxLags];
    const float2 *mprev_in[kMaxLags];   // mean-square displacement origins, or null
    float2 *mprev_out[kMaxLags];
    const float2 *vprev_in[kMaxLags];   // velocity-correlation origins, or null
    float2 *vprev_out[kMaxLags];
    int32_t *cell_start;     // ncells + 1
    // scratch
    uint32_t *key;           // n, packed new cell
    int32_t *slot;           // n
    int32_t *count;          // ncells
    unsigned long long *entry;  // n
    uint8_t *col;            // n: base column inside the new MD cell (lists on), or null
    int32_t *block_sums;     // scan partials
    Control *ctl;
    // Verlet list built from the sorted state (nbr null: none)
    uint32_t *nbr;
    int32_t *ncount;
    int32_t cap;
    float rl2;               // list radius squared
    Batch batch;
};

int64_t sort_scratch_blocks(int64_t ncells);
cudaError_t launch_sort(const SortArgs &a, cudaStream_t s);

// Upload conversion: FP64 positions -> (cell, cl) in original order (unsorted).
cudaError_t launch_pack(const Geom &geo, int64_t n, const double *x, const double *v,
                        uint32_t *cell, float2 *cl, float2 *vel, int32_t *pid, Control *ctl,
                        cudaStream_t s);
// Batched upload: slots of every system, ghosts in the padding (n = slot count).
cudaError_t launch_pack_batch(const Batch &b, int64_t slots, const double *x, const double *v,
                              uint32_t *cell, float2 *cl, float2 *vel, int32_t *pid, Control *ctl,
                              cudaStream_t s);
// Download conversion: sorted state -> FP64 arrays in original order.
cudaError_t launch_unpack(const Geom &geo, int64_t n, const uint32_t *cell, const float2 *cl,
                          const float2 *vsync, const float2 *fsync, const int32_t *pid,
                          double *x, double *v, double *f, cudaStream_t s,
                          const Batch *batch = nullptr);

// ---- adjoint ---------------------------------------------------------------
struct SoftArgs {
    Geom geo;
    int64_t n;                  // slots of the (single-system) state
    int64_t ntot;               // particles
    const uint32_t *cell;
    const float2 *cl;
    const int32_t *pid;
    const double *x_start;      // start positions, original order (n x 2)
    double dx, width;           // lattice spacing, smoothing s (length units)
    int32_t vmax, M;            // window half-width; cells searched each side
    const double *weights;      // Q loss weights, or null
    double *fsum;               // Q soft f_i (added to), or null
    double *loss;               // 1 (added to), or null
    float2 *xb;                 // dL/dx at the end, state order, or null
    double *gx_start;           // dL/dx at the start (direct term), original order, or null
};

struct AdjArgs {
    Geom geo;
    int64_t n;
    const uint32_t *cell;
    const int32_t *cell_start;
    const float2 *x;            // positions of the step being reversed
    const uint32_t *nbr;
    const int32_t *ncount;
    int32_t cap;
    float list_skin, rc, rc2, cell_w;
    float eps24, sig2, inv_eps, inv_sigma;
    float a_coef, b_coef;       // w = w_prev + a xb;  xb_out = xb + b (dF/dx)^T w
    const float2 *w_prev;
    const float2 *xb;
    float2 *w_out;
    float2 *xb_out;
    double *theta;              // [eps, sigma] adjoint accumulators (added to)
    Control *ctl;               // displacement bound at the end of the segment
    int32_t potential;          // 0 none, 1 truncated-shifted, 2 shifted-force
    float fc, dfc_dsigma;       // |F(rc)| and its sigma derivative (shifted force)
};

cudaError_t launch_soft_loss(const SoftArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_step(const AdjArgs &a, cudaStream_t s);
cudaError_t launch_permute(int64_t n, const int32_t *pid, const float2 *src, float2 *dst,
                           bool to_original, cudaStream_t s);

}  // namespace mdlg
