/*
 * Contact law (Eqs. 3-6), forces and velocity-Verlet integrator (Eqs. 1-2) of
 * the FP64 oracle, written once for a scalar type R and included twice:
 *   OR_REAL = 1: R = double, the oracle itself (functions orc_*).
 *   OR_REAL = 0: R = double complex, the same arithmetic for complex-step
 *                differentiation (functions orc_cs_*): a parameter p is given
 *                the value p + i h, and Im(result) / h is the derivative of the
 *                result with respect to p, exact up to rounding (Squire and
 *                Trapp, SIAM Rev. 40, 1998).  Every branch (contact, slip,
 *                sign) is decided on real parts, so the derivative is that of
 *                the forward map with the same contact and slip pattern.
 * Test infrastructure only.
 */
#if OR_REAL
typedef double R;
#define RE(x) (x)
#define RSQRT(x) sqrt(x)
#define RLOG(x) log(x)
#define FN(n) orc_##n
#else
#include <complex.h>
typedef double _Complex R;
#define RE(x) creal(x)
#define RSQRT(x) csqrt(x)
#define RLOG(x) clog(x)
#define FN(n) orc_cs_##n
#endif

/* |x| decided on the real part, analytic elsewhere */
static R FN(rabs)(R x) { return RE(x) < 0.0 ? -x : x; }

/* material of one system: E, e, mu (the differentiable parameters), nu */
typedef struct { R E, e, mu, mu_w; double nu; } FN(mat_t);

static FN(mat_t) FN(mat_from)(const double *P)
{
    FN(mat_t) M;
    M.E = P[P_E];
    M.e = P[P_REST];
    M.mu = P[P_MU];
    M.mu_w = P[P_MUW];
    M.nu = P[P_NU];
    return M;
}

/* beta(e) of Eq. 6 */
static R FN(beta_g)(R e)
{
    R le = RLOG(e);
    return le / RSQRT(le * le + ORC_PI * ORC_PI);
}

/* Effective pair properties (standard Hertz-Mindlin forms; used but not
 * defined in Eq. 6).  Both bodies carry the same material (E, nu): the
 * coarse-grain rules of Sec. 2.2 keep E, nu, e, mu and rho per level, and the
 * floor is given the particle material.  A wall has infinite radius and mass.
 * Then Eq. 6: out = {E_eff, G_eff, R_eff, m_eff, k_n, gamma_n, k_t, gamma_t}. */
static void FN(coeffs)(const FN(mat_t) *M, double ri, double rj, double mi, double mj, R delta, int wall,
                       R *out)
{
    R E = M->E;
    double nu = M->nu;
    R invE = (1.0 - nu * nu) / E + (1.0 - nu * nu) / E;
    R invG = 2.0 * (2.0 - nu) * (1.0 + nu) / E + 2.0 * (2.0 - nu) * (1.0 + nu) / E;
    R Eeff = 1.0 / invE;
    R Geff = 1.0 / invG;
    double Reff, meff;
    if (wall) {
        Reff = ri;
        meff = mi;
    } else {
        Reff = 1.0 / (1.0 / ri + 1.0 / rj);
        meff = 1.0 / (1.0 / mi + 1.0 / mj);
    }
    R beta = FN(beta_g)(M->e);
    R kn = 4.0 / 3.0 * Eeff * RSQRT(Reff * delta);
    R gn = -beta * RSQRT(5.0 * meff * kn);
    R kt = 8.0 * Geff * RSQRT(Reff * delta);
    R gt = -beta * RSQRT(10.0 / 3.0 * meff * kt);
    out[0] = Eeff; out[1] = Geff; out[2] = Reff; out[3] = meff;
    out[4] = kn; out[5] = gn; out[6] = kt; out[7] = gt;
}

/* x_i - x_j with the minimum-image convention on periodic axes */
static void FN(separation)(const double *P, const R *xi, const R *xj, R *d)
{
    for (int a = 0; a < 3; ++a) {
        R s = xi[a] - xj[a];
        if (P[P_PER + a] != 0.0) {
            double L = P[P_HI + a] - P[P_LO + a];
            s -= L * floor(RE(s) / L + 0.5);
        }
        d[a] = s;
    }
}

static R FN(dot3)(const R *a, const R *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void FN(cross3)(const R *a, const R *b, R *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---------------------------------------------------------------- history */

/* One contact's tangential overlap, keyed by particle IDs (ia < ib), or by
 * (ia, -1) for the floor. */
typedef struct { int64_t a, b; R xi[3]; int32_t slip; } FN(hrec_t);

static int FN(cmp_hrec)(const void *x, const void *y)
{
    const FN(hrec_t) *p = (const FN(hrec_t) *)x, *q = (const FN(hrec_t) *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

static const R *FN(find_hist)(int64_t nh, const int64_t *ha, const int64_t *hb, const R *hxi, int64_t a,
                              int64_t b)
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
static int FN(contact_law)(const double *P, const FN(mat_t) *M, double ra, double rb, double ma, double mb,
                           int wall, R delta, const R *n, const R *va, const R *vb, const R *wa, const R *wb,
                           R *xi, double dt_hist, R mu, R *fa, R *ft)
{
    R c[8];
    FN(coeffs)(M, ra, rb, ma, mb, delta, wall, c);
    R kn = c[4], gn = c[5], kt = c[6], gt = c[7];

    /* relative velocity of a w.r.t. b and of the contact points */
    R vr[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    R vn = FN(dot3)(vr, n);
    R rw[3];
    for (int k = 0; k < 3; ++k) rw[k] = ra * wa[k] + (wall ? 0.0 : rb * wb[k]);
    R rwxn[3];
    FN(cross3)(rw, n, rwxn);
    R vc[3] = {vr[0] - rwxn[0], vr[1] - rwxn[1], vr[2] - rwxn[2]};
    R vcn = FN(dot3)(vc, n);
    R vt[3] = {vc[0] - vcn * n[0], vc[1] - vcn * n[1], vc[2] - vcn * n[2]};

    /* Eq. 3 */
    R fnm = kn * delta - gn * vn;
    if (P[P_CLAMP] != 0.0 && RE(fnm) < 0.0) fnm = 0.0;
    R fn[3] = {fnm * n[0], fnm * n[1], fnm * n[2]};

    /* Eq. 4: keep the stored overlap in the current tangent plane (same
     * length), then advance it by the tangential contact-point motion */
    R xin = FN(dot3)(xi, n);
    R xr[3] = {xi[0] - xin * n[0], xi[1] - xin * n[1], xi[2] - xin * n[2]};
    R l0 = RSQRT(FN(dot3)(xi, xi)), l1 = RSQRT(FN(dot3)(xr, xr));
    if (RE(l1) > 0.0) {
        R s = l0 / l1;
        for (int k = 0; k < 3; ++k) xi[k] = xr[k] * s;
    } else {
        xi[0] = xi[1] = xi[2] = 0.0;
    }
    for (int k = 0; k < 3; ++k) xi[k] += vt[k] * dt_hist;
    for (int k = 0; k < 3; ++k) ft[k] = -kt * xi[k] - gt * vt[k];

    /* Eq. 5: truncate so that |f_t| <= mu |f_n| (equality counts as stick) */
    R ftm = RSQRT(FN(dot3)(ft, ft));
    R lim = mu * FN(rabs)(fnm);
    int slip = 0;
    if (RE(ftm) > RE(lim)) {
        R s = lim / ftm;
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
 * (ha, hb, hxi; nh records sorted by (a, b)) and the held external forces
 * fext (NULL: none; the coupling controllers' forces of Sec. 2.3, added to
 * gravity and the contact forces).  Writes F, T, and the new
 * history (sorted; at most `cap` records) with slip flags.  fabs_out (may be
 * NULL) receives per particle sum_j |F_ij| + |m g| (the scale of the forces
 * acting on it).  Returns the number of contacts, or -(count) if it exceeds
 * cap.
 */
static int64_t FN(eval_m)(const double *P, const FN(mat_t) *M, int64_t n, const R *x, const R *v, const R *w,
                          const double *r, const double *m, const int64_t *id, const double *fext, int64_t nh,
                          const int64_t *ha,
                          const int64_t *hb, const R *hxi, double dt_hist, int32_t use_cells, R *F, R *T,
                          int64_t cap, int64_t *ha_out, int64_t *hb_out, R *hxi_out, int32_t *slip_out,
                          double *fabs_out)
{
    pair_t *pairs = NULL;
    int64_t np = 0;
#if OR_REAL
    pairs = orc_find_pairs(P, n, x, r, 0.0, use_cells, &np);
#else
    {
        double *xr = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
        for (int64_t k = 0; k < 3 * n; ++k) xr[k] = creal(x[k]);
        pairs = orc_find_pairs(P, n, xr, r, 0.0, use_cells, &np);
        free(xr);
    }
#endif
    int64_t nrec_cap = np + (int64_t)ORC_MAXWP * n + n + 1;
    FN(hrec_t) *rec = (FN(hrec_t) *)malloc(sizeof(FN(hrec_t)) * nrec_cap);
    int64_t nrec = 0;

    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            F[3 * i + k] = m[i] * P[P_G + k];
            if (fext) F[3 * i + k] += fext[3 * i + k];   /* held external force (coupling controllers) */
            T[3 * i + k] = 0.0;
        }
        if (fabs_out) fabs_out[i] = m[i] * sqrt(P[P_G] * P[P_G] + P[P_G + 1] * P[P_G + 1] + P[P_G + 2] * P[P_G + 2]);
    }

    /* the contact law of every pair (independent of the others: run in parallel when the
     * oracle is compiled with OpenMP), then the sums over pairs in pair order (serial, so the
     * result does not depend on the thread count) */
    typedef struct { R fa[3], ta[3], tb[3], xi[3]; int slip; } FN(pres_t);
    FN(pres_t) *pres = (FN(pres_t) *)malloc(sizeof(FN(pres_t)) * (np > 0 ? np : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < np; ++k) {
        int64_t a = pairs[k].i, b = pairs[k].j;
        if (id[b] < id[a]) { int64_t t = a; a = b; b = t; }
        R d[3];
        FN(separation)(P, x + 3 * a, x + 3 * b, d);
        R dist = RSQRT(FN(dot3)(d, d));
        R delta = r[a] + r[b] - dist;
        R nv[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        R *xi = pres[k].xi;
        xi[0] = xi[1] = xi[2] = 0.0;
        const R *old = FN(find_hist)(nh, ha, hb, hxi, id[a], id[b]);
        if (old) { xi[0] = old[0]; xi[1] = old[1]; xi[2] = old[2]; }
        R ft[3];
        pres[k].slip = FN(contact_law)(P, M, r[a], r[b], m[a], m[b], 0, delta, nv, v + 3 * a, v + 3 * b, w + 3 * a,
                                       w + 3 * b, xi, dt_hist, M->mu, pres[k].fa, ft);
        R ca[3] = {-r[a] * nv[0], -r[a] * nv[1], -r[a] * nv[2]};
        R cb[3] = {-r[b] * nv[0], -r[b] * nv[1], -r[b] * nv[2]};
        FN(cross3)(ca, ft, pres[k].ta);
        FN(cross3)(cb, ft, pres[k].tb);
    }
    for (int64_t k = 0; k < np; ++k) {
        int64_t a = pairs[k].i, b = pairs[k].j;
        if (id[b] < id[a]) { int64_t t = a; a = b; b = t; }
        const R *fa = pres[k].fa;
        for (int q = 0; q < 3; ++q) {
            F[3 * a + q] += fa[q];
            F[3 * b + q] -= fa[q];
            T[3 * a + q] += pres[k].ta[q];
            T[3 * b + q] += pres[k].tb[q];
        }
        if (fabs_out) {
            double fm = sqrt(RE(fa[0]) * RE(fa[0]) + RE(fa[1]) * RE(fa[1]) + RE(fa[2]) * RE(fa[2]));
            fabs_out[a] += fm;
            fabs_out[b] += fm;
        }
        rec[nrec].a = id[a]; rec[nrec].b = id[b];
        memcpy(rec[nrec].xi, pres[k].xi, sizeof(pres[k].xi));
        rec[nrec].slip = pres[k].slip;
        ++nrec;
    }
    free(pres);
    free(pairs);

    if (P[P_FLOOR] != 0.0) {
        const R nz[3] = {0.0, 0.0, 1.0};
        const R zero3[3] = {0.0, 0.0, 0.0};
        const R fv[3] = {P[P_FLOORV], P[P_FLOORV + 1], P[P_FLOORV + 2]};
        for (int64_t i = 0; i < n; ++i) {
            R delta = r[i] - (x[3 * i + 2] - P[P_FLOORZ]);
            if (!(RE(delta) > 0.0)) continue;
            R xi[3] = {0.0, 0.0, 0.0};
            const R *old = FN(find_hist)(nh, ha, hb, hxi, id[i], -1);
            if (old) { xi[0] = old[0]; xi[1] = old[1]; xi[2] = old[2]; }
            R fa[3], ft[3];
            int slip = FN(contact_law)(P, M, r[i], 0.0, m[i], 0.0, 1, delta, nz, v + 3 * i, fv, w + 3 * i, zero3, xi,
                                       dt_hist, M->mu_w, fa, ft);
            R ca[3] = {-r[i] * nz[0], -r[i] * nz[1], -r[i] * nz[2]};
            R ta[3];
            FN(cross3)(ca, ft, ta);
            for (int q = 0; q < 3; ++q) {
                F[3 * i + q] += fa[q];
                T[3 * i + q] += ta[q];
            }
            if (fabs_out) fabs_out[i] += sqrt(RE(fa[0]) * RE(fa[0]) + RE(fa[1]) * RE(fa[1]) + RE(fa[2]) * RE(fa[2]));
            rec[nrec].a = id[i]; rec[nrec].b = -1;
            memcpy(rec[nrec].xi, xi, sizeof(xi));
            rec[nrec].slip = slip;
            ++nrec;
        }
    }

    /* Axisymmetric walls: the surface of revolution of the polyline (rho_k, z_k) about the
     * vertical axis through (P_WAX, P_WAY), one wall per segment (infinite radius and mass,
     * particle material, wall friction).  A particle touches segment k where its distance to
     * the segment, in its own azimuthal half-plane, is below its radius (end points included:
     * a free rim is an edge contact); n points from the contact point to the centre.  History
     * keyed (i, -2 - k). */
    const int nwp = (int)P[P_NWP];
    for (int64_t i = 0; nwp >= 2 && i < n; ++i) {
        const R ex = x[3 * i] - P[P_WAX], ey = x[3 * i + 1] - P[P_WAY];
        const R rho = RSQRT(ex * ex + ey * ey);
        R erx = 1.0, ery = 0.0;
        if (RE(rho) > 1e-12) { erx = ex / rho; ery = ey / rho; }
        const R z = x[3 * i + 2];
        for (int k = 0; k + 1 < nwp; ++k) {
            const double r0 = P[P_WP + 2 * k], z0 = P[P_WP + 2 * k + 1];
            const double dr = P[P_WP + 2 * k + 2] - r0, dz = P[P_WP + 2 * k + 3] - z0;
            R t = ((rho - r0) * dr + (z - z0) * dz) / (dr * dr + dz * dz);
            if (RE(t) < 0.0) t = 0.0;
            else if (RE(t) > 1.0) t = 1.0;
            const R drho = rho - (r0 + t * dr), dzz = z - (z0 + t * dz);
            const R dist = RSQRT(drho * drho + dzz * dzz);
            const R delta = r[i] - dist;
            if (!(RE(delta) > 0.0)) continue;
            const R nv[3] = {drho / dist * erx, drho / dist * ery, dzz / dist};
            const R zero3[3] = {0.0, 0.0, 0.0};
            R xi[3] = {0.0, 0.0, 0.0};
            const R *old = FN(find_hist)(nh, ha, hb, hxi, id[i], -2 - k);
            if (old) { xi[0] = old[0]; xi[1] = old[1]; xi[2] = old[2]; }
            R fa[3], ft[3];
            int slip = FN(contact_law)(P, M, r[i], 0.0, m[i], 0.0, 1, delta, nv, v + 3 * i, zero3, w + 3 * i, zero3,
                                       xi, dt_hist, M->mu_w, fa, ft);
            R ca[3] = {-r[i] * nv[0], -r[i] * nv[1], -r[i] * nv[2]};
            R ta[3];
            FN(cross3)(ca, ft, ta);
            for (int q = 0; q < 3; ++q) {
                F[3 * i + q] += fa[q];
                T[3 * i + q] += ta[q];
            }
            if (fabs_out) fabs_out[i] += sqrt(RE(fa[0]) * RE(fa[0]) + RE(fa[1]) * RE(fa[1]) + RE(fa[2]) * RE(fa[2]));
            rec[nrec].a = id[i]; rec[nrec].b = -2 - k;
            memcpy(rec[nrec].xi, xi, sizeof(xi));
            rec[nrec].slip = slip;
            ++nrec;
        }
    }

    qsort(rec, (size_t)nrec, sizeof(FN(hrec_t)), FN(cmp_hrec));
    for (int64_t k = 0; k < nrec && k < cap; ++k) {
        ha_out[k] = rec[k].a;
        hb_out[k] = rec[k].b;
        memcpy(hxi_out + 3 * k, rec[k].xi, 3 * sizeof(R));
        if (slip_out) slip_out[k] = rec[k].slip;
    }
    free(rec);
    return nrec <= cap ? nrec : -nrec;
}

/* ------------------------------------------------------------- integrator */

static void FN(wrap_positions)(const double *P, int64_t n, R *x)
{
    for (int a = 0; a < 3; ++a) {
        if (P[P_PER + a] == 0.0) continue;
        double lo = P[P_LO + a], L = P[P_HI + a] - P[P_LO + a];
        for (int64_t i = 0; i < n; ++i) {
            R s = x[3 * i + a] - lo;
            s -= L * floor(RE(s) / L);
            if (RE(s) >= L) s -= L;
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
static int32_t FN(run_m)(const double *P, const FN(mat_t) *M, int64_t n, R *x, R *v, R *w, const double *r,
                         const double *m, const int64_t *id, const double *fext, int64_t *nh, int64_t cap, int64_t *ha, int64_t *hb,
                         R *hxi, int32_t *slip, R *F, R *T, int64_t nsteps, int32_t primed, int32_t use_cells)
{
    double dt = P[P_DT];
    int64_t *ta = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    int64_t *tb = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    R *tx = (R *)malloc(sizeof(R) * 3 * (cap > 0 ? cap : 1));
    int32_t rc = 0;
    if (!primed) {
        int64_t c = FN(eval_m)(P, M, n, x, v, w, r, m, id, fext, *nh, ha, hb, hxi, 0.0, use_cells, F, T, cap, ta, tb, tx,
                               slip, NULL);
        if (c < 0) { rc = -1; goto done; }
        memcpy(ha, ta, sizeof(int64_t) * c);
        memcpy(hb, tb, sizeof(int64_t) * c);
        memcpy(hxi, tx, sizeof(R) * 3 * c);
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
        FN(wrap_positions)(P, n, x);
        int64_t c = FN(eval_m)(P, M, n, x, v, w, r, m, id, fext, *nh, ha, hb, hxi, dt, use_cells, F, T, cap, ta, tb, tx,
                               slip, NULL);
        if (c < 0) { rc = -1; goto done; }
        memcpy(ha, ta, sizeof(int64_t) * c);
        memcpy(hb, tb, sizeof(int64_t) * c);
        memcpy(hxi, tx, sizeof(R) * 3 * c);
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

#if OR_REAL
/* ----------------------------------------------------- public (double) API */

double orc_beta(double e) { return orc_beta_g(e); }

void orc_pair_coeffs(const double *P, double ri, double rj, double mi, double mj, double delta, int32_t wall,
                     double *out)
{
    orc_mat_t M = orc_mat_from(P);
    orc_coeffs(&M, ri, rj, mi, mj, delta, wall, out);
}

/* One contact of the contact law (Eqs. 3-6) for the coupling oracle: force on
 * a (fa) and tangential part (ft); xi is updated in place; returns 1 on slip. */
int orc_contact_pair(const double *P, double ra, double rb, double ma, double mb, int32_t wall, double delta,
                     const double *n, const double *va, const double *vb, const double *wa, const double *wb,
                     double *xi, double dt_hist, double *fa, double *ft)
{
    orc_mat_t M = orc_mat_from(P);
    return orc_contact_law(P, &M, ra, rb, ma, mb, wall, delta, n, va, vb, wa, wb, xi, dt_hist,
                           wall ? M.mu_w : M.mu, fa, ft);
}

int64_t orc_eval(const double *P, int64_t n, const double *x, const double *v, const double *w, const double *r,
                 const double *m, const int64_t *id, const double *fext, int64_t nh, const int64_t *ha,
                 const int64_t *hb,
                 const double *hxi, double dt_hist, int32_t use_cells, double *F, double *T, int64_t cap,
                 int64_t *ha_out, int64_t *hb_out, double *hxi_out, int32_t *slip_out, double *fabs_out)
{
    orc_mat_t M = orc_mat_from(P);
    return orc_eval_m(P, &M, n, x, v, w, r, m, id, fext, nh, ha, hb, hxi, dt_hist, use_cells, F, T, cap, ha_out, hb_out,
                      hxi_out, slip_out, fabs_out);
}

int32_t orc_run(const double *P, int64_t n, double *x, double *v, double *w, const double *r, const double *m,
                const int64_t *id, const double *fext, int64_t *nh, int64_t cap, int64_t *ha, int64_t *hb, double *hxi, int32_t *slip,
                double *F, double *T, int64_t nsteps, int32_t primed, int32_t use_cells)
{
    orc_mat_t M = orc_mat_from(P);
    return orc_run_m(P, &M, n, x, v, w, r, m, id, fext, nh, cap, ha, hb, hxi, slip, F, T, nsteps, primed, use_cells);
}
#else
/* ------------------------------------------------ complex-step derivative */

/*
 * Derivative of a rollout from (x0, v0, w0) with empty history with respect to
 * one material parameter (which = 0: E, 1: e, 2: mu; mu also sets the wall
 * friction when that is unset), by a complex step of size h.  On return x, v,
 * w, F, T hold the state at step nsteps (real parts) and dx, dv, dw, dF, dT
 * its derivative.  Returns 0, or -1 if the history capacity was exceeded.
 */
int32_t orc_cs_run_derivative(const double *P, int32_t which, double h, int64_t n, const double *x0,
                              const double *v0, const double *w0, const double *r, const double *m,
                              const int64_t *id, int64_t nsteps, int32_t use_cells, int64_t cap, double *x,
                              double *v, double *w, double *F, double *T, double *dx, double *dv, double *dw,
                              double *dF, double *dT)
{
    orc_cs_mat_t M = orc_cs_mat_from(P);
    if (which == 0) M.E += I * h;
    else if (which == 1) M.e += I * h;
    else if (which == 2) {
        int wall_follows = P[P_MUW] == P[P_MU];
        M.mu += I * h;
        if (wall_follows) M.mu_w += I * h;
    }
    size_t nb = sizeof(R) * 3 * (n > 0 ? n : 1);
    R *xc = (R *)malloc(nb), *vc = (R *)malloc(nb), *wc = (R *)malloc(nb), *Fc = (R *)malloc(nb),
      *Tc = (R *)malloc(nb);
    for (int64_t k = 0; k < 3 * n; ++k) { xc[k] = x0[k]; vc[k] = v0[k]; wc[k] = w0[k]; }
    int64_t *ha = (int64_t *)malloc(sizeof(int64_t) * cap), *hb = (int64_t *)malloc(sizeof(int64_t) * cap);
    R *hxi = (R *)malloc(sizeof(R) * 3 * cap);
    int32_t *slip = (int32_t *)malloc(sizeof(int32_t) * cap);
    int64_t nh = 0;
    int32_t rc = orc_cs_run_m(P, &M, n, xc, vc, wc, r, m, id, NULL, &nh, cap, ha, hb, hxi, slip, Fc, Tc, nsteps, 0,
                              use_cells);
    for (int64_t k = 0; k < 3 * n; ++k) {
        x[k] = creal(xc[k]); v[k] = creal(vc[k]); w[k] = creal(wc[k]); F[k] = creal(Fc[k]); T[k] = creal(Tc[k]);
        dx[k] = cimag(xc[k]) / h; dv[k] = cimag(vc[k]) / h; dw[k] = cimag(wc[k]) / h;
        dF[k] = cimag(Fc[k]) / h; dT[k] = cimag(Tc[k]) / h;
    }
    free(xc); free(vc); free(wc); free(Fc); free(Tc); free(ha); free(hb); free(hxi); free(slip);
    return rc;
}
#endif

#undef RE
#undef RSQRT
#undef RLOG
#undef FN
