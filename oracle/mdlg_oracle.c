/*
 * mdlg_oracle.c -- plain, slow, FP64 CPU oracle for the MDLG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package entry's smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Paper: M. R. Parsa and A. J. Wagner, "Lattice Gas with Molecular Dynamics
 * Collision Operator" (arXiv:1705.04368).  Each function names the section /
 * equation it writes out.
 *
 * Conventions (readings of the paper, each fixed here and in the design notes):
 *  - positions live in the periodic box (0, L] per axis (left-open, right-closed
 *    like the cell indicator of Sec. III);
 *  - the lattice cell of coordinate x is ceil(x / dx) - 1, i.e. the cell c with
 *    c*dx < x <= (c+1)*dx  (cell indicator Delta_x, Sec. III);
 *  - the lattice displacement is taken modulo the lattice size into the range
 *    (-C/2, C/2]  (minimum image; the paper is silent on periodic images);
 *  - velocity index i = (v_y + V)(2V+1) + (v_x + V) for |v_a| <= V, and the
 *    extra index (2V+1)^2 collects every other displacement (overflow bin);
 *  - the pair force is the negative gradient of sum_{j != i} V(r_ij) with the
 *    Lennard-Jones V of Sec. IV, truncated at r_c, energy shifted by V(r_c);
 *    mass m enters as dv/dt = F/m (the Newton equations of Sec. III).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * Threads.  The default build is serial.  Built with -fopenmp (the timing
 * build of the benchmark's CPU baseline only), the per-particle loops below
 * run on several host threads: every particle's own sums keep their serial
 * order, only the global energy / virial sums and the histogram totals are
 * combined across threads.
 */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Periodic helpers                                                          */
/* ------------------------------------------------------------------------ */

/* Minimum-image separation component: d reduced into [-L/2, L/2]. */
static double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

/* Map a coordinate into the periodic interval (0, L]. */
static double wrap_open_closed(double x, double L)
{
    while (x <= 0.0) x += L;
    while (x > L) x -= L;
    return x;
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones pair interaction (Sec. IV, potential V(x))                  */
/* ------------------------------------------------------------------------ */

/* V(r) = 4 eps [ (sigma/r)^12 - (sigma/r)^6 ] */
static double lj_v(double r2, double eps, double sigma)
{
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* -(1/r) dV/dr = 24 eps [ 2 (sigma/r)^12 - (sigma/r)^6 ] / r^2 ; the force on
 * particle i from j is this scalar times (x_i - x_j). */
static double lj_fscalar_plain(double r2, double eps, double sigma)
{
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
}

/*
 * Shifted-force variant (g_sf = 1): the force magnitude is F(r) - F(rc) for
 * r < rc, so it falls continuously to zero at the cutoff; the matching energy
 * is V(r) - V(rc) + (r - rc) F(rc).  g_sf = 0: force truncated at rc, energy
 * shifted by V(rc).
 */
static int g_sf = 0;
static double g_rc = 0.0;

static double lj_fscalar(double r2, double eps, double sigma)
{
    double f = lj_fscalar_plain(r2, eps, sigma);
    if (g_sf) {
        double fc = lj_fscalar_plain(g_rc * g_rc, eps, sigma) * g_rc;   /* |F(rc)| */
        f -= fc / sqrt(r2);
    }
    return f;
}

/* pair energy relative to the cutoff: V(r) - V(rc) (+ (r - rc) F(rc) shifted force) */
static double lj_pair_energy(double r2, double eps, double sigma)
{
    double e = lj_v(r2, eps, sigma) - lj_v(g_rc * g_rc, eps, sigma);
    if (g_sf) e += (sqrt(r2) - g_rc) * lj_fscalar_plain(g_rc * g_rc, eps, sigma) * g_rc;
    return e;
}

/*
 * Error scale of one pair force evaluated in binary32: the magnitudes of its
 * terms -- the repulsive 2 s^12 and attractive s^6 parts of Sec. IV's force
 * (and the shifted-force constant) -- summed in absolute value.  Their
 * difference vanishes at r = 2^(1/6) sigma while the rounding error of each
 * term remains, so tolerances are stated against this sum, not against |F_ij|.
 */
static double lj_fterm_scale(double r2, double eps, double sigma)
{
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    double m = fabs(24.0 * eps * (2.0 * sr6 * sr6 + sr6)) / sqrt(r2);
    if (g_sf) m += fabs(lj_fscalar_plain(g_rc * g_rc, eps, sigma) * g_rc);
    return m;
}

/* Select the cutoff treatment for the following calls. */
void oracle_set_shifted_force(int sf) { g_sf = sf; }

/*
 * Direct O(N^2) forces: F_i = -d/dx_i sum_{j != i} V(|x_i - x_j|) over all
 * pairs with r < rc under minimum image (Newton equations of Sec. III with the
 * pair potential of Sec. IV).  Every pair is evaluated from both sides.
 *
 *   x      : n x 2 positions (row-major, x then y)
 *   f      : n x 2 output forces
 *   fscale : optional n output, sum_j of the pair-force term magnitudes
 *            (lj_fterm_scale): the per-particle scale relative force
 *            tolerances are stated against
 *   out    : optional [pe, virial] where pe = sum_{i<j} (V(r_ij) - V(rc)) and
 *            virial = sum_{i<j} r_ij . F_ij
 */
void oracle_lj_forces_direct(int64_t n, const double *x, const double *L,
                             double eps, double sigma, double rc,
                             double *f, double *fscale, double *out)
{
    double rc2 = rc * rc;
    double pe = 0.0, vir = 0.0;
    g_rc = rc;
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fs = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = min_image(x[2 * i] - x[2 * j], L[0]);
            double dy = min_image(x[2 * i + 1] - x[2 * j + 1], L[1]);
            double r2 = dx * dx + dy * dy;
            if (r2 >= rc2) continue;
            double s = lj_fscalar(r2, eps, sigma);
            fx += s * dx;
            fy += s * dy;
            fs += lj_fterm_scale(r2, eps, sigma);
            pe += 0.5 * lj_pair_energy(r2, eps, sigma);
            vir += 0.5 * s * r2;
        }
        f[2 * i] = fx;
        f[2 * i + 1] = fy;
        if (fscale) fscale[i] = fs;
    }
    if (out) { out[0] = pe; out[1] = vir; }
}

/*
 * Forces for a SAMPLE of particles only, each by the direct O(N) sum over all
 * other particles (same definition as above).  Lets tests check outputs of a
 * full-size system one particle at a time.
 */
void oracle_lj_forces_sample(int64_t n, const double *x, const double *L,
                             double eps, double sigma, double rc,
                             int64_t ns, const int64_t *which,
                             double *f, double *fscale)
{
    double rc2 = rc * rc;
    g_rc = rc;
    for (int64_t k = 0; k < ns; ++k) {
        int64_t i = which[k];
        double fx = 0.0, fy = 0.0, fs = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = min_image(x[2 * i] - x[2 * j], L[0]);
            double dy = min_image(x[2 * i + 1] - x[2 * j + 1], L[1]);
            double r2 = dx * dx + dy * dy;
            if (r2 >= rc2) continue;
            double s = lj_fscalar(r2, eps, sigma);
            fx += s * dx;
            fy += s * dy;
            fs += lj_fterm_scale(r2, eps, sigma);
        }
        f[2 * k] = fx;
        f[2 * k + 1] = fy;
        if (fscale) fscale[k] = fs;
    }
}

/*
 * The same forces found through a linked-cell list (cells of side >= rc), so
 * the oracle can integrate systems of 10^4 - 10^5 particles.  It visits exactly
 * the pairs with r < rc that the direct sum visits; only the summation order
 * differs.  Falls back to the direct sum when fewer than 3 cells fit per axis.
 */
void oracle_lj_forces_cells(int64_t n, const double *x, const double *L,
                            double eps, double sigma, double rc,
                            double *f, double *fscale, double *out)
{
    int64_t ncx = (int64_t)floor(L[0] / rc), ncy = (int64_t)floor(L[1] / rc);
    if (ncx < 3 || ncy < 3) {
        oracle_lj_forces_direct(n, x, L, eps, sigma, rc, f, fscale, out);
        return;
    }
    double hx = L[0] / (double)ncx, hy = L[1] / (double)ncy;
    int64_t ncell = ncx * ncy;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cy = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        double px = wrap_open_closed(x[2 * i], L[0]);
        double py = wrap_open_closed(x[2 * i + 1], L[1]);
        int64_t a = (int64_t)floor(px / hx), b = (int64_t)floor(py / hy);
        if (a >= ncx) a = ncx - 1;
        if (b >= ncy) b = ncy - 1;
        cx[i] = a; cy[i] = b;
        next[i] = head[b * ncx + a];
        head[b * ncx + a] = i;
    }
    double rc2 = rc * rc;
    double pe = 0.0, vir = 0.0;
    g_rc = rc;
#pragma omp parallel for schedule(static) reduction(+ : pe, vir)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fs = 0.0;
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int64_t a = (cx[i] + ox + ncx) % ncx, b = (cy[i] + oy + ncy) % ncy;
                for (int64_t j = head[b * ncx + a]; j >= 0; j = next[j]) {
                    if (j == i) continue;
                    double dx = min_image(x[2 * i] - x[2 * j], L[0]);
                    double dy = min_image(x[2 * i + 1] - x[2 * j + 1], L[1]);
                    double r2 = dx * dx + dy * dy;
                    if (r2 >= rc2) continue;
                    double s = lj_fscalar(r2, eps, sigma);
                    fx += s * dx;
                    fy += s * dy;
                    fs += lj_fterm_scale(r2, eps, sigma);
                    pe += 0.5 * lj_pair_energy(r2, eps, sigma);
                    vir += 0.5 * s * r2;
                }
            }
        f[2 * i] = fx;
        f[2 * i + 1] = fy;
        if (fscale) fscale[i] = fs;
    }
    if (out) { out[0] = pe; out[1] = vir; }
    free(head); free(next); free(cx); free(cy);
}

/*
 * Velocity-Verlet integration of the Newton equations (Sec. III) for nsteps:
 *   v <- v + F dt / (2m);  x <- x + v dt (wrapped into (0, L]);
 *   F <- F(x);             v <- v + F dt / (2m).
 * x, v are updated in place; f holds F(x) on entry and on exit (pass
 * have_force = 0 to have it computed first).  use_cells selects the cell-list
 * force routine.  out (optional) receives [pe, virial] of the final state.
 */
void oracle_vv(int64_t n, double *x, double *v, double *f, int have_force,
               const double *L, double mass, double eps, double sigma, double rc,
               double dt, int64_t nsteps, int use_cells, double *out)
{
    double tmp[2] = {0.0, 0.0};
    if (!have_force) {
        if (use_cells) oracle_lj_forces_cells(n, x, L, eps, sigma, rc, f, NULL, tmp);
        else oracle_lj_forces_direct(n, x, L, eps, sigma, rc, f, NULL, tmp);
    }
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 2; ++a) {
                v[2 * i + a] += 0.5 * dt * f[2 * i + a] / mass;
                x[2 * i + a] = wrap_open_closed(x[2 * i + a] + dt * v[2 * i + a], L[a]);
            }
        if (use_cells) oracle_lj_forces_cells(n, x, L, eps, sigma, rc, f, NULL, tmp);
        else oracle_lj_forces_direct(n, x, L, eps, sigma, rc, f, NULL, tmp);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 2; ++a)
                v[2 * i + a] += 0.5 * dt * f[2 * i + a] / mass;
    }
    if (out) { out[0] = tmp[0]; out[1] = tmp[1]; }
}

/* Free streaming x <- x + v dt of the non-interacting gas (ballistic limit of
 * Sec. IV-A), wrapped into (0, L]. */
void oracle_free_stream(int64_t n, double *x, const double *v, const double *L,
                        double dt, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 2; ++a)
                x[2 * i + a] = wrap_open_closed(x[2 * i + a] + dt * v[2 * i + a], L[a]);
}

/* ------------------------------------------------------------------------ */
/* MDLG occupation numbers (Sec. III, Eq. MDni)                              */
/* ------------------------------------------------------------------------ */

/* Cell indicator of Sec. III: the cell c with c*dx < x <= (c+1)*dx. */
static int64_t lattice_cell(double x, double dx)
{
    return (int64_t)ceil(x / dx) - 1;
}

/* Lattice displacement modulo C, reduced into (-C/2, C/2]. */
static int64_t lattice_disp(int64_t d, int64_t C)
{
    int64_t r = ((d % C) + C) % C;
    if (r > C / 2) r -= C;
    return r;
}

void oracle_mdlg_bin_shifted(int64_t n, const double *xprev, const double *xcur,
                             double dx, const int64_t *C, int vmax,
                             const double *s_prev, const double *s_cur,
                             uint64_t *counts, uint32_t *ncell, uint32_t *field,
                             int64_t *vsum);

/*
 * n_i(x,t) = sum_j Delta_x(x_j(t)) Delta_{x - v_i}(x_j(t - dt))   (Eq. MDni)
 * and N(x,t) = sum_j Delta_x(x_j(t))                               (Sec. III)
 *
 * Walks the particles one by one: the cell of each particle at t (site x) and
 * at t - dt (site x - v_i) give its lattice velocity v_i, and the particle adds
 * one to n_i at site x.
 *
 *   xprev, xcur : n x 2 positions at t - dt and t, each in (0, L]
 *   C[2]        : lattice cells per axis (L = C dx)
 *   vmax        : window half-width V; Q = (2V+1)^2 velocities + 1 overflow
 *   counts      : Q+1 totals over the lattice (added to)
 *   ncell       : optional C[0]*C[1] site counts N(x,t) (added to)
 *   field       : optional C[0]*C[1]*(Q+1) occupation numbers, site-major
 *                 (added to)
 *   vsum        : optional [sum_j v_jx, sum_j v_jy] over in-window particles
 */
void oracle_mdlg_bin(int64_t n, const double *xprev, const double *xcur,
                     double dx, const int64_t *C, int vmax,
                     uint64_t *counts, uint32_t *ncell, uint32_t *field,
                     int64_t *vsum)
{
    oracle_mdlg_bin_shifted(n, xprev, xcur, dx, C, vmax, NULL, NULL, counts, ncell, field, vsum);
}

/*
 * The same with a moving lattice (Sec. IV: a lattice displaced by -U dt gives
 * the distribution at mean velocity U): each snapshot is binned at x + S, S the
 * lattice displacement of its time (S_prev, S_cur; NULL = none), the sum taken
 * in FP64 and the cell then wrapped into the lattice.
 */
void oracle_mdlg_bin_shifted(int64_t n, const double *xprev, const double *xcur,
                             double dx, const int64_t *C, int vmax,
                             const double *s_prev, const double *s_cur,
                             uint64_t *counts, uint32_t *ncell, uint32_t *field,
                             int64_t *vsum)
{
    int64_t W = 2 * vmax + 1, Q = W * W;
    const double zero[2] = {0.0, 0.0};
    if (!s_prev) s_prev = zero;
    if (!s_cur) s_cur = zero;
    int64_t vs0 = 0, vs1 = 0;
    /* threaded only when no per-site output is requested (the totals are
     * integers: combining them across threads changes nothing) */
#pragma omp parallel for schedule(static) reduction(+ : counts[:Q + 1], vs0, vs1) if (!ncell && !field)
    for (int64_t j = 0; j < n; ++j) {
        int64_t c0x = lattice_cell(xprev[2 * j] + s_prev[0], dx);
        int64_t c0y = lattice_cell(xprev[2 * j + 1] + s_prev[1], dx);
        int64_t c1x = lattice_cell(xcur[2 * j] + s_cur[0], dx);
        int64_t c1y = lattice_cell(xcur[2 * j + 1] + s_cur[1], dx);
        c0x = ((c0x % C[0]) + C[0]) % C[0];
        c0y = ((c0y % C[1]) + C[1]) % C[1];
        c1x = ((c1x % C[0]) + C[0]) % C[0];
        c1y = ((c1y % C[1]) + C[1]) % C[1];
        int64_t vx = lattice_disp(c1x - c0x, C[0]);
        int64_t vy = lattice_disp(c1y - c0y, C[1]);
        int64_t i;
        if (vx < -vmax || vx > vmax || vy < -vmax || vy > vmax) {
            i = Q;
        } else {
            i = (vy + vmax) * W + (vx + vmax);
            vs0 += vx;
            vs1 += vy;
        }
        int64_t site = c1y * C[0] + c1x;
        counts[i] += 1;
        if (ncell) ncell[site] += 1;
        if (field) field[site * (Q + 1) + i] += 1;
    }
    if (vsum) { vsum[0] += vs0; vsum[1] += vs1; }
}

/*
 * Non-interacting gas streamed and binned in one pass (the ballistic case of
 * Sec. IV-A), for several (dx, dt) pairs.  The decision of which cell a point
 * falls in is taken in IEEE binary32, the precision the device path computes
 * in: x' = fl(x + fl(v dt)) (not wrapped), cell = ceil(fl(x / dx)) - 1 per
 * axis, lattice velocity = cell(x') - cell(x).  For |v dt| < L/2 this is the
 * periodic definition of Eq. MDni, with the site taken modulo C in integers.
 * With us (ncombo x 2, NULL = none) every velocity is first boosted by U:
 * v' = fl(v + U), the moving-lattice reading of Sec. IV.
 *
 *   pos, vel : n x 2 binary32 values, positions in (0, L]
 *   counts   : ncombo x (Q+1) totals (added to)
 */
void oracle_stream_bin_f32(int64_t n, const float *pos, const float *vel,
                           int ncombo, const float *dxs, const float *dts,
                           const float *us, int vmax, uint64_t *counts)
{
    int64_t W = 2 * vmax + 1, Q = W * W;
    for (int k = 0; k < ncombo; ++k) {
        volatile float dx = dxs[k], dt = dts[k];
        uint64_t *ck = counts + k * (Q + 1);
#pragma omp parallel for schedule(static) reduction(+ : ck[:Q + 1])
        for (int64_t j = 0; j < n; ++j) {
            int64_t c[2][2];
            for (int a = 0; a < 2; ++a) {
                volatile float x = pos[2 * j + a];
                /* moving lattice (Sec. IV): velocity boosted by U, one rounding */
                volatile float vb = us ? vel[2 * j + a] + us[2 * k + a] : vel[2 * j + a];
                volatile float d = vb * dt;                /* one rounding */
                volatile float xn = x + d;                 /* one rounding */
                volatile float q0 = x / dx, q1 = xn / dx;  /* one rounding each */
                c[a][0] = (int64_t)ceilf(q0) - 1;
                c[a][1] = (int64_t)ceilf(q1) - 1;
            }
            int64_t vx = c[0][1] - c[0][0], vy = c[1][1] - c[1][0];
            int64_t i = (vx < -vmax || vx > vmax || vy < -vmax || vy > vmax)
                            ? Q : (vy + vmax) * W + (vx + vmax);
            ck[i] += 1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 global reductions                                                    */
/* ------------------------------------------------------------------------ */

/* out = [kinetic energy sum m v^2 / 2, momentum_x, momentum_y] */
void oracle_kinetic(int64_t n, const double *v, double mass, double *out)
{
    double ke = 0.0, px = 0.0, py = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        ke += 0.5 * mass * (v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1]);
        px += mass * v[2 * i];
        py += mass * v[2 * i + 1];
    }
    out[0] = ke; out[1] = px; out[2] = py;
}

/* ------------------------------------------------------------------------ */
/* MDLG collision operator (Sec. III, Eq. Xi)                                */
/* ------------------------------------------------------------------------ */

/*
 * Xi_i(x) = n_i(x + v_i, t + dt) - n_i(x, t) for the (2V+1)^2 window velocities,
 * from the occupation fields of two consecutive intervals (site-major, Q+1
 * entries per site as oracle_mdlg_bin writes them).  xi: C[0]*C[1] x Q.
 */
void oracle_collision(const int64_t *C, int vmax, const uint32_t *field_prev,
                      const uint32_t *field_cur, int64_t *xi)
{
    int64_t W = 2 * vmax + 1, Q = W * W;
    for (int64_t sy = 0; sy < C[1]; ++sy)
        for (int64_t sx = 0; sx < C[0]; ++sx)
            for (int64_t i = 0; i < Q; ++i) {
                int64_t vx = i % W - vmax, vy = i / W - vmax;
                int64_t tx = ((sx + vx) % C[0] + C[0]) % C[0];
                int64_t ty = ((sy + vy) % C[1] + C[1]) % C[1];
                int64_t site = sy * C[0] + sx, dest = ty * C[0] + tx;
                xi[site * Q + i] = (int64_t)field_cur[dest * (Q + 1) + i] -
                                   (int64_t)field_prev[site * (Q + 1) + i];
            }
}

/* Mean over particles of the squared displacement per axis (minimum image),
 * <dx_a^2> of Sec. IV-A between two snapshots. */
void oracle_msd(int64_t n, const double *xprev, const double *xcur, const double *L,
                double *out)
{
    double sx = 0.0, sy = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double dx = min_image(xcur[2 * j] - xprev[2 * j], L[0]);
        double dy = min_image(xcur[2 * j + 1] - xprev[2 * j + 1], L[1]);
        sx += dx * dx;
        sy += dy * dy;
    }
    out[0] = n ? sx / (double)n : 0.0;
    out[1] = n ? sy / (double)n : 0.0;
}


/* Leapfrog half-step velocity of the step that ends at xcur (Sec. III,
 * velocity Verlet): v = (xcur - xprev) / dt, the displacement taken by minimum
 * image (one step moves far less than half the box). */
void oracle_half_velocity(int64_t n, const double *xprev, const double *xcur, const double *L,
                          double dt, double *vout)
{
    for (int64_t j = 0; j < n; ++j) {
        vout[2 * j] = min_image(xcur[2 * j] - xprev[2 * j], L[0]) / dt;
        vout[2 * j + 1] = min_image(xcur[2 * j + 1] - xprev[2 * j + 1], L[1]) / dt;
    }
}

/* Velocity correlation between two samples of the same particles (Sec. IV-A,
 * Fig. VD(a)): per axis, the mean over particles of v_a(now) v_a(before). */
void oracle_vacf(int64_t n, const double *vprev, const double *vcur, double *out)
{
    double sx = 0.0, sy = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        sx += vcur[2 * j] * vprev[2 * j];
        sy += vcur[2 * j + 1] * vprev[2 * j + 1];
    }
    out[0] = n ? sx / (double)n : 0.0;
    out[1] = n ? sy / (double)n : 0.0;
}
