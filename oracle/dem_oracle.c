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
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define P_E 0
#define P_NU 1
#define P_REST 2
#define P_MU 3
#define P_MUW 4
#define P_DT 5
#define P_G 6
#define P_LO 9
#define P_HI 12
#define P_PER 15
#define P_FLOOR 18
#define P_FLOORZ 19
#define P_FLOORV 20
#define P_CLAMP 23

static const double PI = 3.14159265358979323846;

/* beta(e) of Eq. 6. */
double orc_beta(double e)
{
    double le = log(e);
    return le / sqrt(le * le + PI * PI);
}

/* Effective pair properties (standard Hertz-Mindlin forms; used but not
 * defined in Eq. 6).  Both bodies carry the same material (E, nu): the
 * coarse-grain rules of Sec. 2.2 keep E, nu, e, mu and rho per level, and the
 * floor is given the particle material.  A wall has infinite radius and mass. */
static void effective(const double *P, double ri, double rj, double mi, double mj,
                      int wall, double *Eeff, double *Geff, double *Reff, double *meff)
{
    double E = P[P_E], nu = P[P_NU];
    double invE = (1.0 - nu * nu) / E + (1.0 - nu * nu) / E;
    double invG = 2.0 * (2.0 - nu) * (1.0 + nu) / E + 2.0 * (2.0 - nu) * (1.0 + nu) / E;
    *Eeff = 1.0 / invE;
    *Geff = 1.0 / invG;
    if (wall) {
        *Reff = ri;
        *meff = mi;
    } else {
        *Reff = 1.0 / (1.0 / ri + 1.0 / rj);
        *meff = 1.0 / (1.0 / mi + 1.0 / mj);
    }
}

/* Eq. 6: out = {E_eff, G_eff, R_eff, m_eff, k_n, gamma_n, k_t, gamma_t}. */
void orc_pair_coeffs(const double *P, double ri, double rj, double mi, double mj,
                     double delta, int32_t wall, double *out)
{
    double Eeff, Geff, Reff, meff;
    effective(P, ri, rj, mi, mj, wall, &Eeff, &Geff, &Reff, &meff);
    double beta = orc_beta(P[P_REST]);
    double kn = 4.0 / 3.0 * Eeff * sqrt(Reff * delta);
    double gn = -beta * sqrt(5.0 * meff * kn);
    double kt = 8.0 * Geff * sqrt(Reff * delta);
    double gt = -beta * sqrt(10.0 / 3.0 * meff * kt);
    out[0] = Eeff; out[1] = Geff; out[2] = Reff; out[3] = meff;
    out[4] = kn; out[5] = gn; out[6] = kt; out[7] = gt;
}

/* x_i - x_j with the minimum-image convention on periodic axes. */
static void separation(const double *P, const double *xi, const double *xj, double *d)
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

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------ pairs */

typedef struct { int64_t i, j; } pair_t;

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
    separation(P, x + 3 * i, x + 3 * j, d);
    double cut = r[i] + r[j] + extra;
    return sqrt(dot3(d, d)) < cut;
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

/* ---------------------------------------------------------------- history */

/* One contact's tangential overlap, keyed by particle IDs (ia < ib), or by
 * (ia, -1) for the floor. */
typedef struct { int64_t a, b; double xi[3]; int32_t slip; } hrec_t;

static int cmp_hrec(const void *x, const void *y)
{
    const hrec_t *p = (const hrec_t *)x, *q = (const hrec_t *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

static const double *find_hist(int64_t nh, const int64_t *ha, const int64_t *hb,
                               const double *hxi, int64_t a, int64_t b)
{
    int64_t lo = 0, hi = nh - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ha[mid] == a && hb[mid] == b) return hxi + 3 * mid;
        if (ha[mid] < a || (ha[mid] == a && hb[mid] < b)) lo = mid + 1;
        else hi = mid - 1;
    }
    return NULL;
}

/* ----------------------------------------------------------- contact law */

/*
 * One contact, Eqs. 3-6.  Inputs are for body a (the lower particle ID) and
 * body b; n points from b to a, delta > 0.  xi is the stored tangential
 * overlap (updated in place), dt_hist the time over which the contact-point
 * velocity advances it (the step length; 0 for the start-up evaluation).
 * Outputs: force on a (fa) and the tangential force ft; returns 1 on slip.
 */
static int contact_law(const double *P, double ra, double rb, double ma, double mb,
                       int wall, double delta, const double *n,
                       const double *va, const double *vb, const double *wa, const double *wb,
                       double *xi, double dt_hist, double mu, double *fa, double *ft)
{
    double c[8];
    orc_pair_coeffs(P, ra, rb, ma, mb, delta, wall, c);
    double kn = c[4], gn = c[5], kt = c[6], gt = c[7];

    /* relative velocity of a w.r.t. b and of the contact points */
    double vr[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    double vn = dot3(vr, n);
    double rw[3];
    for (int k = 0; k < 3; ++k) rw[k] = ra * wa[k] + (wall ? 0.0 : rb * wb[k]);
    double rwxn[3];
    cross3(rw, n, rwxn);
    double vc[3] = {vr[0] - rwxn[0], vr[1] - rwxn[1], vr[2] - rwxn[2]};
    double vcn = dot3(vc, n);
    double vt[3] = {vc[0] - vcn * n[0], vc[1] - vcn * n[1], vc[2] - vcn * n[2]};

    /* Eq. 3 */
    double fnm = kn * delta - gn * vn;
    if (P[P_CLAMP] != 0.0 && fnm < 0.0) fnm = 0.0;
    double fn[3] = {fnm * n[0], fnm * n[1], fnm * n[2]};

    /* Eq. 4: keep the stored overlap in the current tangent plane (same
     * length), then advance it by the tangential contact-point motion */
    double xin = dot3(xi, n);
    double xr[3] = {xi[0] - xin * n[0], xi[1] - xin * n[1], xi[2] - xin * n[2]};
    double l0 = sqrt(dot3(xi, xi)), l1 = sqrt(dot3(xr, xr));
    if (l1 > 0.0) {
        double s = l0 / l1;
        for (int k = 0; k < 3; ++k) xi[k] = xr[k] * s;
    } else {
        xi[0] = xi[1] = xi[2] = 0.0;
    }
    for (int k = 0; k < 3; ++k) xi[k] += vt[k] * dt_hist;
    for (int k = 0; k < 3; ++k) ft[k] = -kt * xi[k] - gt * vt[k];

    /* Eq. 5: truncate so that |f_t| <= mu |f_n| (equality counts as stick) */
    double ftm = sqrt(dot3(ft, ft));
    double lim = mu * fabs(fnm);
    int slip = 0;
    if (ftm > lim) {
        double s = lim / ftm;
        for (int k = 0; k < 3; ++k) {
            ft[k] *= s;
            xi[k] = -(ft[k] + gt * vt[k]) / kt;
        }
        slip = 1;
    }
    for (int k = 0; k < 3; ++k) fa[k] = fn[k] + ft[k];
    return slip;
}

/*
 * Forces and torques on all particles at state (x, v, w) with history
 * (ha, hb, hxi; nh records sorted by (a, b)).  Writes F, T, and the new
 * history (sorted; at most `cap` records) with slip flags.  fabs_out (may be
 * NULL) receives per particle sum_j |F_ij| + |m g| (the scale of the forces
 * acting on it).  Returns the number of contacts, or -(count) if it exceeds
 * cap.
 */
int64_t orc_eval(const double *P, int64_t n, const double *x, const double *v,
                 const double *w, const double *r, const double *m, const int64_t *id,
                 int64_t nh, const int64_t *ha, const int64_t *hb, const double *hxi,
                 double dt_hist, int32_t use_cells, double *F, double *T,
                 int64_t cap, int64_t *ha_out, int64_t *hb_out, double *hxi_out,
                 int32_t *slip_out, double *fabs_out)
{
    pair_t *pairs = NULL;
    int64_t np = 0;
    if (use_cells) {
        pairs = cell_pairs(P, n, x, r, 0.0, &np);
    } else {
        int64_t pc = 16;
        pairs = (pair_t *)malloc(sizeof(pair_t) * pc);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j)
                if (near_pair(P, x, r, 0.0, i, j)) {
                    if (np == pc) { pc *= 2; pairs = (pair_t *)realloc(pairs, sizeof(pair_t) * pc); }
                    pairs[np].i = i; pairs[np].j = j; ++np;
                }
    }
    int64_t nrec_cap = np + n + 1;
    hrec_t *rec = (hrec_t *)malloc(sizeof(hrec_t) * nrec_cap);
    int64_t nrec = 0;

    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            F[3 * i + k] = m[i] * P[P_G + k];
            T[3 * i + k] = 0.0;
        }
        if (fabs_out) fabs_out[i] = m[i] * sqrt(dot3(P + P_G, P + P_G));
    }

    for (int64_t k = 0; k < np; ++k) {
        int64_t a = pairs[k].i, b = pairs[k].j;
        if (id[b] < id[a]) { int64_t t = a; a = b; b = t; }
        double d[3];
        separation(P, x + 3 * a, x + 3 * b, d);
        double dist = sqrt(dot3(d, d));
        double delta = r[a] + r[b] - dist;
        double nv[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double xi[3] = {0.0, 0.0, 0.0};
        const double *old = find_hist(nh, ha, hb, hxi, id[a], id[b]);
        if (old) { xi[0] = old[0]; xi[1] = old[1]; xi[2] = old[2]; }
        double fa[3], ft[3];
        int slip = contact_law(P, r[a], r[b], m[a], m[b], 0, delta, nv, v + 3 * a, v + 3 * b,
                               w + 3 * a, w + 3 * b, xi, dt_hist, P[P_MU], fa, ft);
        double ca[3] = {-r[a] * nv[0], -r[a] * nv[1], -r[a] * nv[2]};
        double cb[3] = {-r[b] * nv[0], -r[b] * nv[1], -r[b] * nv[2]};
        double ta[3], tb[3];
        cross3(ca, ft, ta);
        cross3(cb, ft, tb);
        for (int q = 0; q < 3; ++q) {
            F[3 * a + q] += fa[q];
            F[3 * b + q] -= fa[q];
            T[3 * a + q] += ta[q];
            T[3 * b + q] += tb[q];
        }
        if (fabs_out) {
            double fm = sqrt(dot3(fa, fa));
            fabs_out[a] += fm;
            fabs_out[b] += fm;
        }
        rec[nrec].a = id[a]; rec[nrec].b = id[b];
        memcpy(rec[nrec].xi, xi, sizeof(xi));
        rec[nrec].slip = slip;
        ++nrec;
    }
    free(pairs);

    if (P[P_FLOOR] != 0.0) {
        const double nz[3] = {0.0, 0.0, 1.0};
        const double zero3[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            double delta = r[i] - (x[3 * i + 2] - P[P_FLOORZ]);
            if (!(delta > 0.0)) continue;
            double xi[3] = {0.0, 0.0, 0.0};
            const double *old = find_hist(nh, ha, hb, hxi, id[i], -1);
            if (old) { xi[0] = old[0]; xi[1] = old[1]; xi[2] = old[2]; }
            double fa[3], ft[3];
            int slip = contact_law(P, r[i], 0.0, m[i], 0.0, 1, delta, nz, v + 3 * i, P + P_FLOORV,
                                   w + 3 * i, zero3, xi, dt_hist, P[P_MUW], fa, ft);
            double ca[3] = {-r[i] * nz[0], -r[i] * nz[1], -r[i] * nz[2]};
            double ta[3];
            cross3(ca, ft, ta);
            for (int q = 0; q < 3; ++q) {
                F[3 * i + q] += fa[q];
                T[3 * i + q] += ta[q];
            }
            if (fabs_out) fabs_out[i] += sqrt(dot3(fa, fa));
            rec[nrec].a = id[i]; rec[nrec].b = -1;
            memcpy(rec[nrec].xi, xi, sizeof(xi));
            rec[nrec].slip = slip;
            ++nrec;
        }
    }

    qsort(rec, (size_t)nrec, sizeof(hrec_t), cmp_hrec);
    for (int64_t k = 0; k < nrec && k < cap; ++k) {
        ha_out[k] = rec[k].a;
        hb_out[k] = rec[k].b;
        memcpy(hxi_out + 3 * k, rec[k].xi, 3 * sizeof(double));
        if (slip_out) slip_out[k] = rec[k].slip;
    }
    free(rec);
    return nrec <= cap ? nrec : -nrec;
}

/* ------------------------------------------------------------- integrator */

static void wrap_positions(const double *P, int64_t n, double *x)
{
    for (int a = 0; a < 3; ++a) {
        if (P[P_PER + a] == 0.0) continue;
        double lo = P[P_LO + a], L = P[P_HI + a] - P[P_LO + a];
        for (int64_t i = 0; i < n; ++i) {
            double s = x[3 * i + a] - lo;
            s -= L * floor(s / L);
            if (s >= L) s -= L;
            x[3 * i + a] = lo + s;
        }
    }
}

/*
 * Velocity Verlet (Eqs. 1-2 with I = 2/5 m r^2), nsteps steps of length dt.
 * State on entry: x^n, v^n, w^n and, when primed != 0, F^n, T^n and the
 * history of the evaluation at step n; when primed == 0 these are first
 * computed at (x^n, v^n, w^n) with the given history and no advance of it.
 * Per step:
 *   v^{n+1/2} = v^n + dt/2 F^n/m,   w^{n+1/2} = w^n + dt/2 T^n/I
 *   x^{n+1}   = x^n + dt v^{n+1/2}  (then wrapped on periodic axes)
 *   F^{n+1}, T^{n+1} from x^{n+1}, v^{n+1/2}, w^{n+1/2}, history advanced by dt
 *   v^{n+1}   = v^{n+1/2} + dt/2 F^{n+1}/m, and the same for w.
 * History arrays hold *nh records on entry and on return (capacity cap).
 * Returns 0, or -1 if the history capacity was exceeded.
 */
int32_t orc_run(const double *P, int64_t n, double *x, double *v, double *w,
                const double *r, const double *m, const int64_t *id,
                int64_t *nh, int64_t cap, int64_t *ha, int64_t *hb, double *hxi,
                int32_t *slip, double *F, double *T, int64_t nsteps, int32_t primed,
                int32_t use_cells)
{
    double dt = P[P_DT];
    int64_t *ta = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    int64_t *tb = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    double *tx = (double *)malloc(sizeof(double) * 3 * (cap > 0 ? cap : 1));
    int32_t rc = 0;
    if (!primed) {
        int64_t c = orc_eval(P, n, x, v, w, r, m, id, *nh, ha, hb, hxi, 0.0, use_cells, F, T,
                             cap, ta, tb, tx, slip, NULL);
        if (c < 0) { rc = -1; goto done; }
        memcpy(ha, ta, sizeof(int64_t) * c);
        memcpy(hb, tb, sizeof(int64_t) * c);
        memcpy(hxi, tx, sizeof(double) * 3 * c);
        *nh = c;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i) {
            double inv_m = 1.0 / m[i];
            double inv_I = 1.0 / (0.4 * m[i] * r[i] * r[i]);
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += 0.5 * dt * F[3 * i + k] * inv_m;
                w[3 * i + k] += 0.5 * dt * T[3 * i + k] * inv_I;
                x[3 * i + k] += dt * v[3 * i + k];
            }
        }
        wrap_positions(P, n, x);
        int64_t c = orc_eval(P, n, x, v, w, r, m, id, *nh, ha, hb, hxi, dt, use_cells, F, T,
                             cap, ta, tb, tx, slip, NULL);
        if (c < 0) { rc = -1; goto done; }
        memcpy(ha, ta, sizeof(int64_t) * c);
        memcpy(hb, tb, sizeof(int64_t) * c);
        memcpy(hxi, tx, sizeof(double) * 3 * c);
        *nh = c;
        for (int64_t i = 0; i < n; ++i) {
            double inv_m = 1.0 / m[i];
            double inv_I = 1.0 / (0.4 * m[i] * r[i] * r[i]);
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += 0.5 * dt * F[3 * i + k] * inv_m;
                w[3 * i + k] += 0.5 * dt * T[3 * i + k] * inv_I;
            }
        }
    }
done:
    free(ta); free(tb); free(tx);
    return rc;
}
