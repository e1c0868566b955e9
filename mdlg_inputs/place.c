/*
 * place.c -- seeded random sequential placement of non-overlapping points.
 *
 * Input generation only (no arithmetic of the method).  Points are drawn one
 * at a time, uniform in the periodic box (0, Lx] x (0, Ly], and a draw is
 * repeated while it lies closer than dmin (minimum image) to a point already
 * placed.  The random stream is splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), so the result is a
 * pure function of (n, box, dmin, seed) on any machine.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, L]: L - L * u with u = k 2^-53, k in [0, 2^53) */
static double draw(uint64_t *s, double L)
{
    double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
    return L - L * u;
}

/* Returns 0 on success, -1 if some point needed more than max_tries draws,
 * -2 on allocation failure.  x receives n x 2 coordinates. */
int place_nonoverlap(int64_t n, double Lx, double Ly, double dmin, uint64_t seed,
                     int64_t max_tries, double *x)
{
    int64_t ncx = (int64_t)floor(Lx / dmin), ncy = (int64_t)floor(Ly / dmin);
    if (ncx < 1) ncx = 1;
    if (ncy < 1) ncy = 1;
    double hx = Lx / (double)ncx, hy = Ly / (double)ncy, d2 = dmin * dmin;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncx * ncy));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!head || !next) { free(head); free(next); return -2; }
    for (int64_t c = 0; c < ncx * ncy; ++c) head[c] = -1;
    uint64_t s = seed;
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; ++i) {
        int64_t tries = 0;
        for (;;) {
            if (++tries > max_tries) { rc = -1; break; }
            double px = draw(&s, Lx), py = draw(&s, Ly);
            int64_t cx = (int64_t)(px / hx), cy = (int64_t)(py / hy);
            if (cx >= ncx) cx = ncx - 1;
            if (cy >= ncy) cy = ncy - 1;
            int ok = 1;
            for (int oy = -1; oy <= 1 && ok; ++oy)
                for (int ox = -1; ox <= 1 && ok; ++ox) {
                    int64_t a = ((cx + ox) % ncx + ncx) % ncx;
                    int64_t b = ((cy + oy) % ncy + ncy) % ncy;
                    for (int64_t j = head[b * ncx + a]; j >= 0; j = next[j]) {
                        double dx = px - x[2 * j], dy = py - x[2 * j + 1];
                        dx -= Lx * nearbyint(dx / Lx);
                        dy -= Ly * nearbyint(dy / Ly);
                        if (dx * dx + dy * dy < d2) { ok = 0; break; }
                    }
                }
            if (!ok) continue;
            x[2 * i] = px;
            x[2 * i + 1] = py;
            next[i] = head[cy * ncx + cx];
            head[cy * ncx + cx] = i;
            break;
        }
    }
    free(head);
    free(next);
    return rc;
}
