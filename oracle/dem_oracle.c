/*
 * Plain FP64 CPU oracle for the DEM hot path of "Adaptive Coarse-Graining for
 * Large-Scale DEM Simulations" (Queteschiner, Lichtenegger, Schneiderbauer,
 * Pirker, CFD 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs use it.  It shares no code, header, constant
 * or table with the CUDA library.
 *
 * What it computes, in the paper's order and notation, without blocking,
 * fusion or reordering:
 *   - Newton's equations for translation and rotation (Sec. 2.1, Eqs. 1-2),
 *     advanced by velocity Verlet (the paper names no integrator; the
 *     velocity-dependent forces use the half-step velocities).
 *   - Normal contact force f_n = k_n delta_n - gamma_n d(delta_n)/dt (Eq. 3).
 *   - Tangential force f_t = k_t delta_t - gamma_t d(delta_t)/dt with a
 *     per-contact tangential overlap that is carried over the life of the
 *     contact (Eq. 4) and truncated so that |f_t| <= mu |f_n| (Eq. 5).
 *   - Non-linear damped Hertz coefficients k_n, gamma_n, k_t, gamma_t and
 *     beta(e) (Eq. 6).  E_eff, G_eff, R_eff, m_eff are used but not defined
 *     in the paper; the standard Hertz-Mindlin definitions are taken.
 *   - Gravity and a flat floor plane z = floor_z moving with a prescribed
 *     velocity (external forces, Sec. 2.1).
 *   - Contact detection by an O(N^2) all-pairs scan and, separately, by a
 *     cell list; both must give the same set.
 *
 * Sign readings (the paper prints magnitudes only):
 *   n = x_ij / |x_ij| points from j to i, delta = r_i + r_j - |x_ij| > 0 is a
 *   contact.  The force on i is (k_n delta - gamma_n v_n) n with
 *   v_n = (v_i - v_j) . n, and f_t = -k_t xi - gamma_t v_t, so that with
 *   beta <= 0 (e <= 1) both dashpots dissipate.
 *
 * Parameter block P (flat array of doubles):
 *   0 E   1 nu   2 e   3 mu   4 mu_wall   5 dt   6..8 g   9..11 lo
 *   12..14 hi   15..17 periodic flags   18 floor_on   19 floor_z
 *   20..22 floor velocity   23 clamp_fn (1: no tensile normal force)
 *   24 wall profile points (0: none)   25..26 wall axis (x, y)   27..42 profile (rho, z) pairs
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dem_oracle_common.h"

/* x_i - x_j with the minimum-image convention on periodic axes. */
static void geo_separation(const double *P, const double *xi, const double *xj, double *d)
{
    for (int a = 0; a < 3; ++a) {
        double s = xi[a] - xj[a];
        if (P[P_PER + a] != 0.0) {
            double L = P[P_HI + a] - P[P_LO + a];
            s -= L * floor(s / L + 0.5);
        }
        d[a] = s;
    }
}

static double geo_dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }


/* ------------------------------------------------------------------ pairs */


static int cmp_pair(const void *a, const void *b)
{
    const pair_t *p = (const pair_t *)a, *q = (const pair_t *)b;
    if (p->i != q->i) return p->i < q->i ? -1 : 1;
    if (p->j != q->j) return p->j < q->j ? -1 : 1;
    return 0;
}

static int near_pair(const double *P, const double *x, const double *r, double extra,
                     int64_t i, int64_t j)
{
    double d[3];
    geo_separation(P, x + 3 * i, x + 3 * j, d);
    double cut = r[i] + r[j] + extra;
    return sqrt(geo_dot3(d, d)) < cut;
}

/* All index pairs i < j with |x_ij| < r_i + r_j + extra, by brute force.
 * Returns the number found (the first `cap` are written, sorted by (i, j)). */
int64_t orc_pairs_brute(const double *P, int64_t n, const double *x, const double *r,
                        double extra, int64_t cap, int64_t *pi, int64_t *pj)
{
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (near_pair(P, x, r, extra, i, j)) {
                if (cnt < cap) { pi[cnt] = i; pj[cnt] = j; }
                ++cnt;
            }
    return cnt;
}

/* The same set through a uniform cell grid of width >= max(2 r) + extra.
 * Non-periodic axes clamp coordinates outside the box into the end cells. */
static pair_t *cell_pairs(const double *P, int64_t n, const double *x, const double *r,
                          double extra, int64_t *out_cnt)
{
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (r[i] > rmax) rmax = r[i];
    double h = 2.0 * rmax + extra;
    int64_t nc[3];
    double w[3];
    int brute = 0;
    for (int a = 0; a < 3; ++a) {
        double L = P[P_HI + a] - P[P_LO + a];
        nc[a] = (int64_t)floor(L / h);
        if (nc[a] < 1) nc[a] = 1;
        if (P[P_PER + a] != 0.0 && nc[a] < 3) brute = 1;
        w[a] = L / (double)nc[a];
    }
    int64_t cap = 16, cnt = 0;
    pair_t *out = (pair_t *)malloc(sizeof(pair_t) * cap);
    if (brute || n < 2) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j)
                if (near_pair(P, x, r, extra, i, j)) {
                    if (cnt == cap) { cap *= 2; out = (pair_t *)realloc(out, sizeof(pair_t) * cap); }
                    out[cnt].i = i; out[cnt].j = j; ++cnt;
                }
        *out_cnt = cnt;
        return out;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *cidx = (int64_t *)malloc(sizeof(int64_t) * 3 * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c3[3];
        for (int a = 0; a < 3; ++a) {
            double s = x[3 * i + a] - P[P_LO + a];
            if (P[P_PER + a] != 0.0) {
                double L = P[P_HI + a] - P[P_LO + a];
                s -= L * floor(s / L);
            }
            int64_t k = (int64_t)floor(s / w[a]);
            if (k < 0) k = 0;
            if (k >= nc[a]) k = nc[a] - 1;
            c3[a] = k;
            cidx[3 * i + a] = k;
        }
        int64_t c = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[c];
        head[c] = i;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t k3[3] = {cidx[3 * i] + dx, cidx[3 * i + 1] + dy, cidx[3 * i + 2] + dz};
                    int ok = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (k3[a] < 0 || k3[a] >= nc[a]) {
                            if (P[P_PER + a] != 0.0) k3[a] = (k3[a] + nc[a]) % nc[a];
                            else ok = 0;
                        }
                    }
                    if (!ok) continue;
                    int64_t c = (k3[2] * nc[1] + k3[1]) * nc[0] + k3[0];
                    for (int64_t j = head[c]; j >= 0; j = next[j]) {
                        if (j <= i) continue;
                        if (near_pair(P, x, r, extra, i, j)) {
                            if (cnt == cap) { cap *= 2; out = (pair_t *)realloc(out, sizeof(pair_t) * cap); }
                            out[cnt].i = i; out[cnt].j = j; ++cnt;
                        }
                    }
                }
    }
    free(head); free(next); free(cidx);
    qsort(out, (size_t)cnt, sizeof(pair_t), cmp_pair);
    *out_cnt = cnt;
    return out;
}

int64_t orc_pairs_cells(const double *P, int64_t n, const double *x, const double *r,
                        double extra, int64_t cap, int64_t *pi, int64_t *pj)
{
    int64_t cnt = 0;
    pair_t *p = cell_pairs(P, n, x, r, extra, &cnt);
    for (int64_t k = 0; k < cnt && k < cap; ++k) { pi[k] = p[k].i; pj[k] = p[k].j; }
    free(p);
    return cnt;
}


pair_t *orc_find_pairs(const double *P, int64_t n, const double *x, const double *r, double extra,
                       int use_cells, int64_t *out_cnt)
{
    if (use_cells) return cell_pairs(P, n, x, r, extra, out_cnt);
    int64_t pc = 16, np = 0;
    pair_t *pairs = (pair_t *)malloc(sizeof(pair_t) * pc);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (near_pair(P, x, r, extra, i, j)) {
                if (np == pc) { pc *= 2; pairs = (pair_t *)realloc(pairs, sizeof(pair_t) * pc); }
                pairs[np].i = i; pairs[np].j = j; ++np;
            }
    *out_cnt = np;
    return pairs;
}

/* The contact law, forces and integrator in double precision. */
#define OR_REAL 1
#include "dem_oracle_dyn.h"
