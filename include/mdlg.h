/*
 * mdlg.h -- C ABI of the GB300 MD + MDLG library.
 *
 * Method: M. R. Parsa and A. J. Wagner, "Lattice Gas with Molecular Dynamics
 * Collision Operator", arXiv:1705.04368.  The library integrates a periodic 2D
 * Lennard-Jones gas (Newton equations of Sec. III, potential of Sec. IV) and
 * coarse-grains it into the MDLG occupation numbers n_i(x,t) of Eq. MDni:
 * every particle is binned into a lattice cell at t - dt and at t, the cell
 * displacement is its lattice velocity v_i, and the counts are accumulated per
 * velocity (and optionally per lattice site) so that their average estimates
 * the equilibrium f_i of Eq. fieq.
 *
 * Conventions shared by every entry point
 *  - Return value: 0 (MDLG_OK) or a negative MDLG_E* code; no exception or
 *    abort crosses the ABI.  mdlg_strerror() names a code.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory; "host" pointers are ordinary host memory.  The caller owns every
 *    buffer it passes and the library never frees one of them.
 *  - Work is enqueued on the CUDA stream given at creation (or per call for
 *    the context-free entry points) and returns before it finishes, except
 *    where a function says it synchronizes.
 *  - Lattice cells are left-open, right-closed: coordinate x is in cell c iff
 *    c*dx < x <= (c+1)*dx (the cell indicator Delta_x of Sec. III).  The box
 *    is (0, L] per axis.
 *  - Lattice velocities are indexed i = (v_y + V)(2V+1) + (v_x + V) for
 *    |v_x|, |v_y| <= V; index Q = (2V+1)^2 counts every displacement outside
 *    that window.  Displacements are taken modulo the lattice size into
 *    (-C/2, C/2] (minimum image).
 */
#ifndef MDLG_H
#define MDLG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define MDLG_OK          0
#define MDLG_EINVAL     -1   /* an argument is out of range or inconsistent    */
#define MDLG_ENOMEM     -2   /* the allocator returned NULL                    */
#define MDLG_ECUDA      -3   /* a CUDA runtime call failed                     */
#define MDLG_EOVERFLOW  -4   /* a counter or index range was exceeded          */
#define MDLG_ENONFINITE -5   /* a non-finite position or velocity was found    */
#define MDLG_ETIMEOUT   -6   /* reserved: no entry point waits on the device with a
                                bound today, so none returns it                  */
#define MDLG_ENOTIMPL   -7   /* the entry point is declared but not built yet  */

/* ---- limits ------------------------------------------------------------- */
#define MDLG_MAX_LAGS   8    /* coarse time steps tracked concurrently         */
#define MDLG_MAX_VMAX   15   /* window half-width V                            */
#define MDLG_MAX_COMBOS 16   /* (dx, dt) pairs of one ideal-gas pass           */

/* ---- potentials --------------------------------------------------------- */
#define MDLG_POT_NONE   0    /* non-interacting gas (free flight)              */
#define MDLG_POT_LJ_TS  1    /* Lennard-Jones, truncated at rc, energy shifted */
#define MDLG_POT_LJ_SF  2    /* Lennard-Jones, shifted force: F(r) - F(rc) for r < rc,
                                continuous at rc (energy V - V(rc) + (r - rc) F(rc)) */

/* ---- per-site output modes (mdlg_params.site_mode, bit flags) ------------ */
#define MDLG_SITES_FIELD 1   /* keep n_i(x,t), N(x,t) of the latest interval   */
#define MDLG_SITES_ACCUM 2   /* accumulate sum_t n_i(x,t), sum_t N(x,t)        */
#define MDLG_SITES_XI    4   /* with MDLG_SITES_FIELD: also keep the previous
                                interval's n_i and form the collision operator
                                Xi_i(x) of Eq. Xi after every interval          */

/*
 * Parameters of one simulation (Sec. III: N particles, periodic box, pair
 * potential; Sec. III lattice spacing dx and coarse time step dt; Sec. IV:
 * Lennard-Jones eps, sigma, m).
 */
typedef struct {
    int32_t dim;          /* must be 2 (the paper's test case, Sec. IV)          */
    int64_t n;            /* particles, >= 1 (below 2^28 with a potential, and
                             for a batch its padded slot total too: Verlet-list
                             entries hold slot numbers in 28 bits)              */
    double  box[2];       /* periodic box L_x, L_y; integer multiples of dx       */
    int32_t potential;    /* MDLG_POT_LJ_TS, MDLG_POT_LJ_SF or MDLG_POT_NONE      */
    double  eps, sigma;   /* Lennard-Jones energy and length (Sec. IV)            */
    double  mass;         /* particle mass m                                     */
    double  rcut;         /* cutoff radius r_c (> 0)                              */
    double  dt;           /* MD time step (> 0)                                   */
    double  grid;         /* base grid g: a power of two; dx is a multiple of g   */
    double  skin;         /* minimum neighbour-cell skin beyond rcut (>= 0)        */
    int32_t sort_every;   /* MD steps between cell re-sorts; 0 picks them.  With
                             use_graphs: half the skin covered at 1.15 x the
                             fastest initial speed.  Otherwise the device paces
                             them: every step writes its displacement bound and
                             largest speed to pinned host memory, and mdlg_step
                             re-sorts before a step whose input bound, predicted
                             from the values of 3 steps earlier (1.1 x that
                             speed for the steps between, or for the steps since
                             a more recent re-sort), would exceed half the skin.  mdlg_step then keeps at most 3 steps
                             queued ahead of the device (it waits for the rest);
                             the schedule depends only on device values, so a
                             repeated or resumed run re-sorts at the same steps */
    double  dx;           /* lattice spacing Delta x (Sec. III)                   */
    int32_t nlags;        /* coarse time steps tracked, 1..MDLG_MAX_LAGS          */
    int32_t lag_steps[MDLG_MAX_LAGS]; /* Delta t of each, in MD steps (>= 1)      */
    int32_t vmax;         /* window half-width V, 1..MDLG_MAX_VMAX                */
    int32_t site_mode;    /* MDLG_SITES_* flags for lag 0; 0 = totals only         */
    int32_t stats_every;  /* MD steps between FP64 reductions; 0 = only on request */
    int32_t use_graphs;   /* 1: mdlg_step captures two periods of its launch schedule
                             (lcm of sort_every, the lags and stats_every) in a CUDA
                             graph and replays it; stretches shorter than that, and
                             schedules longer than 8192 steps, launch directly.
                             Ignored (direct launches) while the lattice moves.   */
    double  lattice_u[2]; /* lattice drift U (length / time), Sec. IV: the lattice
                             is displaced by -U t, i.e. every binning at MD step n
                             places a particle by x + S(n), S(n) = n * s1 modulo the
                             box, with the per-step shift s1 = U dt rounded to the
                             nearest multiple of grid * 2^-24 (the effective U is
                             reported by mdlg_stats).  The cell decision of x + S is
                             exact.  {0, 0}: the lattice is at rest.               */
    int32_t msd;          /* 1: accumulate, for every lag, the mean-square
                             displacement <dx_a^2> over the lag (Sec. IV-A)       */
    int32_t vacf;         /* 1: accumulate, for every lag, the velocity
                             correlation <v_a(t) v_a(t - Dt)> over the lag
                             (Sec. IV-A, Fig. VD(a)); see mdlg_stats_out.vacf  */
} mdlg_params;

/*
 * Device memory supplier.  alloc returns `bytes` of device memory aligned to
 * at least 256 bytes, or NULL; free releases it.  Passing NULL for the whole
 * struct makes the library use cudaMalloc / cudaFree.
 */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void  (*free)(void *ptr, void *user);
    void  *user;
} mdlg_allocator;

typedef struct mdlg_ctx mdlg_ctx;

/* FP64 observables of the most recent statistics step and the MDLG totals. */
typedef struct {
    int64_t step;                 /* MD steps taken so far                       */
    int64_t stats_step;           /* step the energies below refer to (-1: none) */
    double  kinetic;              /* sum m v^2 / 2 at that step                   */
    double  potential;            /* sum_{i<j} V(r_ij) - V(rc)                    */
    double  virial;               /* sum_{i<j} r_ij . F_ij                        */
    double  momentum[2];          /* sum m v                                      */
    double  temperature;          /* kinetic / (N - 1)  (2N - 2 degrees, k_B = 1) */
    double  pressure;             /* (kinetic + virial / 2) / (L_x L_y)           */
    int64_t intervals[MDLG_MAX_LAGS]; /* coarse intervals binned per lag          */
    int32_t status;               /* MDLG_OK or the first device-side error seen  */
    double  msd[MDLG_MAX_LAGS][2];/* params.msd: <dx_a^2> per lag and axis, the mean
                                     over particles and binned intervals of the
                                     squared displacement over the lag (0 if off) */
    double  lattice_u[2];         /* effective lattice drift: s1 / dt            */
    int64_t stale_steps;          /* step launches so far that found the Verlet list
                                     out of date (forces then came from the cell
                                     stencil: correct, slower); 0 when the re-sort
                                     schedule keeps up                           */
    int32_t sort_every;           /* MD steps between re-sorts: the fixed interval,
                                     or (device-paced schedule) the length of the
                                     last completed interval                     */
    double  vacf[MDLG_MAX_LAGS][2];/* params.vacf: <v_a(t) v_a(t - Dt)> per lag and
                                     axis, the mean over particles and binned
                                     intervals (0 if off).  v(t) is the leapfrog
                                     half-step velocity of the step that ends at
                                     t, (x(t) - x(t - dt)) / dt (at t = 0:
                                     v_0 - F(x_0) dt / 2m), so both ends of the
                                     correlation are sampled half a step early  */
} mdlg_stats_out;

/*
 * mdlg_create -- validate parameters, allocate device state, upload the
 * initial condition and enqueue the initial force evaluation.
 *   params    : see mdlg_params; MDLG_EINVAL on any inconsistency.
 *   x0, v0    : host, n x 2 FP64 positions in (0, L] and velocities (Sec. III
 *               initial condition x_i(0), v_i(0)); NULL -> MDLG_EINVAL.
 *   allocator : device memory supplier, or NULL for cudaMalloc.
 *   stream    : cudaStream_t (as void*) all work of the context is enqueued on;
 *               NULL is the legacy default stream.
 *   out       : receives the context.
 * The call copies x0 / v0 before it returns; it does not synchronize the
 * stream.  Errors: MDLG_EINVAL, MDLG_ENOMEM, MDLG_ECUDA, MDLG_ENONFINITE.
 */
int mdlg_create(const mdlg_params *params, const double *x0, const double *v0,
                const mdlg_allocator *allocator, void *stream, mdlg_ctx **out);

/*
 * mdlg_create_batch -- one context holding nsys independent systems that share
 * every parameter except the particle count and the box (an ensemble for the
 * averages of Eq. fieq, Sec. IV-A).  All systems advance together: each
 * kernel launch of mdlg_step covers every system, and each system's forces,
 * trajectory and counts are exactly those of a context made for it alone with
 * the same sort_every (set sort_every > 0 to compare).
 *   params : shared parameters; params->n and params->box are ignored;
 *            params->site_mode, params->msd and params->vacf must be 0
 *            and params->lattice_u {0, 0}.
 *   nsys   : systems, 1..65535.
 *   n      : host, nsys particle counts; each system is padded to a multiple
 *            of 128 slots, and the total of the padded counts must stay
 *            below 2^28 (the Verlet list indexes slots in 28 bits), else
 *            MDLG_EINVAL.
 *   box    : host, nsys x 2 box sides, each a multiple of params->dx.
 *   x0, v0 : host, (sum n) x 2 FP64 positions and velocities, system after
 *            system in the order of n.
 * mdlg_stats then reports all systems together (counts added, f_i over the
 * total particle number); mdlg_stats_system reports one.  mdlg_get_state
 * returns the concatenated state.  Errors as mdlg_create.
 */
int mdlg_create_batch(const mdlg_params *params, int32_t nsys, const int64_t *n,
                      const double *box, const double *x0, const double *v0,
                      const mdlg_allocator *allocator, void *stream, mdlg_ctx **out);

/*
 * mdlg_stats_system -- mdlg_stats for one system of a batch (0-based index);
 * MDLG_EINVAL for a context made by mdlg_create or an index out of range.
 */
int mdlg_stats_system(mdlg_ctx *ctx, int32_t system, mdlg_stats_out *out, uint64_t *counts,
                      double *fi);

/*
 * mdlg_step -- enqueue nsteps velocity-Verlet steps of the Newton equations
 * (Sec. III) with Lennard-Jones forces (Sec. IV).  After every MD step whose
 * count is a multiple of lag_steps[k], the particles are binned for lag k
 * (Eq. MDni) against their lattice cells lag_steps[k] steps earlier and the
 * counts are added to the lag's totals (Eq. fieq).  FP64 reductions run on
 * multiples of stats_every.  Asynchronous with a fixed re-sort interval;
 * with the device-paced schedule (sort_every = 0, no graphs) it returns once
 * the device has finished all but the last 3 steps.  Errors: MDLG_EINVAL,
 * MDLG_ECUDA.
 */
int mdlg_step(mdlg_ctx *ctx, int64_t nsteps);

/*
 * mdlg_stats -- synchronize the stream and report the FP64 observables of the
 * most recent statistics step (taking one now at the current step if none was
 * taken since the last step), the MDLG totals and the device status word.
 *   out    : host, filled in.
 *   counts : host, nlags x (Q+1) uint64 totals sum_{t,x} n_i(x,t), or NULL.
 *   fi     : host, nlags x (Q+1) FP64 estimates f_i / rho^eq
 *            = counts_i / (N * intervals) (Eq. fieq), or NULL.
 */
int mdlg_stats(mdlg_ctx *ctx, mdlg_stats_out *out, uint64_t *counts, double *fi);

/*
 * mdlg_get_state -- synchronize and copy the state in the original particle
 * order (host buffers, n x 2 each; any may be NULL):
 *   x : FP64 positions in (0, L] (exact value of the stored representation)
 *   v : FP64 velocities at the current integer step
 *   f : FP64 copy of the FP32 forces at the current positions
 */
int mdlg_get_state(mdlg_ctx *ctx, double *x, double *v, double *f);

/*
 * mdlg_get_sites -- synchronize and copy lag-0 per-site outputs (host; either
 * may be NULL).  site_counts: C_y*C_x*(Q+1) uint32, ncell: C_y*C_x uint32,
 * site-major with site = c_y*C_x + c_x.  They hold the latest interval
 * (MDLG_SITES_FIELD) or the sum over intervals (MDLG_SITES_ACCUM).
 * MDLG_EINVAL if site_mode is 0.
 */
int mdlg_get_sites(mdlg_ctx *ctx, uint32_t *site_counts, uint32_t *ncell);

/*
 * mdlg_get_collision -- synchronize and copy the MDLG collision operator of
 * the last two lag-0 intervals (site_mode MDLG_SITES_FIELD | MDLG_SITES_XI):
 * with t the time between them (Sec. III, Eq. Xi)
 *     Xi_i(x) = n_i(x + v_i, t + dt) - n_i(x, t)
 * for the (2V+1)^2 window velocities (the overflow entry has no destination
 * and is left out), and per site its mass and momentum sums
 *     dmass(x) = sum_i Xi_i(x),  dmom_a(x) = sum_i v_ia Xi_i(x)
 * (Eqs. masscons, momentumcons: the first vanishes when no move leaves the
 * window, the second in general does not).
 *   xi    : host, C_y*C_x*Q int32, site-major (site = c_y*C_x + c_x), or NULL.
 *   dmass : host, C_y*C_x int32, or NULL.
 *   dmom  : host, C_y*C_x*2 int32 (x, y per site), or NULL.
 * MDLG_EINVAL if the mode is off or fewer than two lag-0 intervals have been
 * binned since creation or the last mdlg_reset_counts.
 */
int mdlg_get_collision(mdlg_ctx *ctx, int32_t *xi, int32_t *dmass, int32_t *dmom);

/* mdlg_reset_counts -- enqueue zeroing of all MDLG totals and per-site outputs,
 * keeping the stored earlier lattice cells (to discard an equilibration). */
int mdlg_reset_counts(mdlg_ctx *ctx);

/*
 * mdlg_adjoint -- advance the context by nsteps MD steps (like mdlg_step) and
 * return the gradient of a soft-binned MDLG loss over that interval with
 * respect to eps, sigma and the state at its start.
 *
 * Loss: the cell indicator of Sec. III is smoothed with a Gaussian of standard
 * deviation `width` (length units): u_c(x) = Phi((x - c dx)/w) - Phi((x - (c+1) dx)/w).
 * The soft occupations of Eq. MDni between the start (t = 0) and the end
 * (t = nsteps), averaged over particles, are
 *     ftilde_i = (1/N) sum_j prod_a sum_c u_c(x_ja(end)) u_{c - v_ia}(x_ja(start))
 * on the (2V+1)^2 window (index as everywhere; no overflow entry), and
 *     loss = sum_i dloss_i ftilde_i.
 * Gradients are taken through the leapfrog trajectory by a hand-written
 * adjoint (Jacobian-vector products of the pair forces, FP32 per particle, FP64
 * accumulation of the eps and sigma adjoints), re-computing each segment of
 * ckpt_every steps from a checkpoint stored at its start.  x0 / v0 refer to the
 * positions and integer-step velocities at the start of the call.
 *   nsteps, ckpt_every : nsteps a multiple of ckpt_every; the context must have
 *                        been created with sort_every == ckpt_every and be at a
 *                        re-sort (true right after mdlg_create).
 *   width              : 0 < width <= 0.875 dx;  V (params.vmax) <= 7.
 *   dloss              : host, Q = (2V+1)^2 weights; NULL -> forward only
 *                        (ftilde and loss, no gradients).
 *   ftilde, loss       : host outputs (Q, 1), or NULL.
 *   grad_eps, grad_sigma : host, 1 each, or NULL.
 *   grad_x0, grad_v0   : host, n x 2 in the original particle order, or NULL.
 * The soft-binned loss uses the lattice at rest (lattice_u does not enter it).
 * Single systems only (MDLG_EINVAL for a batch).  Synchronizes.  Allocates its
 * checkpoints through the context's allocator for the duration of the call.
 */
int mdlg_adjoint(mdlg_ctx *ctx, int64_t nsteps, int32_t ckpt_every, double width,
                 const double *dloss, double *ftilde, double *loss, double *grad_eps,
                 double *grad_sigma, double *grad_x0, double *grad_v0);

/*
 * mdlg_profile -- per-kernel timing of the context's launches with CUDA events
 * on its stream (tracing aid; no counterpart in the paper).
 *   enable = 1 : clear the record and start recording every launch group;
 *   enable = 0 : stop, synchronize and report.
 * ms[k] / launches[k] (host, MDLG_PROF_KINDS entries each, may be NULL) receive
 * the summed device time and the number of kernel launches of each kind:
 * MDLG_PROF_STEP (force + velocity-Verlet), MDLG_PROF_SORT (cell re-sort,
 * all its kernels), MDLG_PROF_BIN (MDLG binning), MDLG_PROF_SYNC (statistics /
 * state download).  Recording adds two event records per launch group.
 */
#define MDLG_PROF_STEP  0
#define MDLG_PROF_SORT  1
#define MDLG_PROF_BIN   2
#define MDLG_PROF_SYNC  3
#define MDLG_PROF_KINDS 4
int mdlg_profile(mdlg_ctx *ctx, int enable, double *ms, int64_t *launches);

/*
 * Checkpoint / resume (no counterpart in the paper: long runs such as its 3e6-
 * step trajectories are restarted from one).  A checkpoint is the complete run
 * state of a context -- sorted particle state, every lag's stored lattice cells
 * (and displacement origins), the Verlet list of the last re-sort, the device
 * control block, MDLG totals, per-site fields and the host schedule (step, last
 * re-sort, binned intervals, the device-paced schedule's last three step slots)
 * -- so that a context restored from it continues bit for bit as the saved one
 * would have.
 *
 * mdlg_checkpoint_size -- bytes of this context's checkpoint (host out).
 * mdlg_save  -- synchronize and write the checkpoint into buf (host memory of at
 *               least that many bytes).
 * mdlg_load  -- restore a checkpoint into a context created with the same
 *               parameters (stats_every may differ, and use_graphs too when
 *               sort_every > 0: with sort_every = 0 it selects the schedule)
 *               and, for a
 *               batch, the same systems; the state it was created with is
 *               replaced.  Synchronizes.
 * Errors: MDLG_EINVAL (NULL arguments, buffer too small, not a checkpoint, or
 * made by a context of another shape or parameters), MDLG_ECUDA.
 */
int mdlg_checkpoint_size(mdlg_ctx *ctx, uint64_t *bytes);
int mdlg_save(mdlg_ctx *ctx, void *buf, uint64_t bytes);
int mdlg_load(mdlg_ctx *ctx, const void *buf, uint64_t bytes);

/* mdlg_destroy -- synchronize, release device state; NULL is ignored. */
void mdlg_destroy(mdlg_ctx *ctx);

/* mdlg_strerror -- static string naming an MDLG_E* code. */
const char *mdlg_strerror(int code);

/*
 * Lattice for the context-free binning entry point.  Positions are given as
 * integer base-cell indices: base cell k of an axis is (k g, (k+1) g], so a
 * particle in base cell k lies in lattice cell floor(k / ratio) with
 * ratio = dx / g.
 */
typedef struct {
    int32_t base[2];   /* base cells per axis, L / g (each a multiple of ratio)  */
    int32_t ratio;     /* dx / g, >= 1                                           */
    int32_t vmax;      /* window half-width V, 1..MDLG_MAX_VMAX                  */
} mdlg_lattice;

/*
 * mdlg_bin -- Eq. MDni for one pair of snapshots of the same n particles.
 *   idx_prev, idx_cur : device, n x 2 int32 base-cell indices (x, y) in
 *                       [0, base) at t - dt and at t.
 *   counts : device, Q+1 uint64 totals, ADDED to (zero them to start).
 *   ncell  : device, C_y*C_x uint32 N(x,t), added to, or NULL.
 *   field  : device, C_y*C_x*(Q+1) uint32 n_i(x,t), added to, or NULL.
 *   stream : cudaStream_t (as void*).
 * Errors: MDLG_EINVAL (bad lattice, n < 0, NULL counts), MDLG_ECUDA.
 * Out-of-range indices are wrapped modulo base (no fault, no error).
 */
int mdlg_bin(const mdlg_lattice *lat, int64_t n, const int32_t *idx_prev,
             const int32_t *idx_cur, uint64_t *counts, uint32_t *ncell,
             uint32_t *field, void *stream);

/*
 * mdlg_collision -- the collision operator of Eq. Xi from two occupation
 * fields of consecutive intervals (as mdlg_bin or mdlg_get_sites write them):
 *     Xi_i(x) = n_i(x + v_i, t + dt) - n_i(x, t),  window velocities only,
 * with x + v_i wrapped into the lattice, plus dmass(x) = sum_i Xi_i(x) and
 * dmom_a(x) = sum_i v_ia Xi_i(x).
 *   lat        : lattice (lat->base / lat->ratio cells per axis, lat->vmax).
 *   field_prev : device, C_y*C_x*(Q+1) uint32 n_i(x, t), site-major.
 *   field_cur  : device, the same for the next interval, n_i(x, t + dt).
 *   xi         : device, C_y*C_x*Q int32 (written), or NULL.
 *   dmass      : device, C_y*C_x int32 (written), or NULL.
 *   dmom       : device, C_y*C_x*2 int32 (written), or NULL.
 *   stream     : cudaStream_t (as void*).
 * Counts above 2^31 - 1 wrap.  Errors: MDLG_EINVAL (bad lattice, NULL field),
 * MDLG_ECUDA.
 */
int mdlg_collision(const mdlg_lattice *lat, const uint32_t *field_prev,
                   const uint32_t *field_cur, int32_t *xi, int32_t *dmass, int32_t *dmom,
                   void *stream);

/*
 * mdlg_idealgas_bin -- non-interacting gas of Sec. IV-A (ballistic limit):
 * stream every particle freely for each (dx_k, dt_k) pair and bin its start
 * and end points (Eq. MDni), all pairs in one pass over the particles.  The
 * cell decisions are taken in IEEE binary32:
 *   x' = fl(x + fl(v' dt_k)),  cell = ceil(fl(x / dx_k)) - 1 per axis,
 *   v_i = cell(x') - cell(x)  (x' is not wrapped; the box is a multiple of
 *   every dx_k and |v dt_k| < L/2 is assumed, as in the paper's regime),
 * where v' = v, or v' = fl(v + U_k) with a lattice drift U_k per pair (the
 * moving lattice of Sec. IV: the gas seen at mean velocity U_k).
 *   pos, vel : device, n x 2 float (x, y) pairs; positions in (0, L].
 *   dxs, dts : host, ncombo values each; 1 <= ncombo <= MDLG_MAX_COMBOS.
 *   us       : host, ncombo x 2 drifts (U_x, U_y), or NULL for none.
 *   counts   : device, ncombo x (Q+1) uint64, ADDED to.
 * Errors: MDLG_EINVAL, MDLG_ECUDA.
 */
int mdlg_idealgas_bin(int64_t n, const float *pos, const float *vel, int32_t ncombo,
                      const float *dxs, const float *dts, const float *us, int32_t vmax,
                      uint64_t *counts, void *stream);

/*
 * mdlg_forces_static -- Lennard-Jones forces and FP64 observables of one
 * configuration, computed without allocating any memory.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory where they need a force evaluation -- code inside a CUDA graph being
 * captured (an allocation there breaks the capture), frameworks whose memory
 * pool owns every allocation, or real-time loops that must not block in the
 * allocator.  It computes what a context computes at a statistics step
 * (pack, neighbour-cell sort, the step kernel's force/reduction mode with a
 * zero time step), with every intermediate array in one statically sized
 * device array of the library instead of allocated scratch.
 *   params : as for mdlg_create; only n, box, potential (MDLG_POT_LJ_TS or
 *            MDLG_POT_LJ_SF; anything else is MDLG_EINVAL), eps, sigma, mass,
 *            rcut, grid and skin are used.
 *   x, v   : device, n x 2 FP64 positions in (0, L] and velocities (inputs).
 *   f      : device, n x 2 FP64 forces F_i (output, original particle order).
 *   obs    : device, 5 FP64 (output): kinetic energy, potential energy,
 *            virial, momentum x, momentum y -- as in mdlg_stats_out.
 *   status : device, one int32 (output, may be NULL): 0, or MDLG_ENONFINITE if
 *            a position was outside the box or a value was not finite.
 *   stream : cudaStream_t (as void*); all work is enqueued there, nothing
 *            synchronizes.
 * Limits: n <= MDLG_STATIC_MAX_N and at most MDLG_STATIC_MAX_CELLS neighbour
 * cells (box area / (cell side)^2, cell side = grid * ceil((rcut+skin)/grid));
 * larger inputs return MDLG_EOVERFLOW before any GPU work.  The static array
 * (about 6 MB) exists on every GPU that loads the library and is held until
 * the process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current): make that first
 * call before any stream capture.  All calls on a device share the array and
 * it keeps the last call's contents; calls whose GPU work overlaps (other
 * streams, other host threads) race and corrupt each other: serialize them.
 * Errors: MDLG_EINVAL, MDLG_EOVERFLOW, MDLG_ECUDA.
 */
#define MDLG_STATIC_MAX_N     65536
#define MDLG_STATIC_MAX_CELLS 65536
int mdlg_forces_static(const mdlg_params *params, const double *x, const double *v, double *f,
                       double *obs, int32_t *status, void *stream);

/* ---- measurement probes --------------------------------------------------
 * The paper has no counterpart: these two kernels measure the denominators of
 * the roofline fractions reported beside the method's kernels.  The caller
 * times them (CUDA events on `stream`).
 *
 * mdlg_probe_fma -- `blocks` blocks of `threads` threads (a multiple of 32,
 *   at most 256); every thread runs 8 independent binary32 fused multiply-add
 *   chains of `iters` steps and stores their sum in out[block * threads + thread]
 *   (device, blocks x threads floats, caller-owned).  *flops (host, may be
 *   NULL) receives the floating-point operations launched, 2 per multiply-add.
 *   Errors: MDLG_EINVAL, MDLG_ECUDA.
 *
 * mdlg_probe_copy -- copies `bytes` (a multiple of 16) from src to dst (device,
 *   both 16-byte aligned, caller-owned, not overlapping) with 16-byte loads
 *   and stores.  Errors: MDLG_EINVAL, MDLG_ECUDA.
 */
int mdlg_probe_fma(int32_t blocks, int32_t threads, int64_t iters, float *out, double *flops,
                   void *stream);
int mdlg_probe_copy(const void *src, void *dst, int64_t bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MDLG_H */
