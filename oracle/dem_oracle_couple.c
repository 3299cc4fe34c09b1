/*
 * FP64 oracle of the two-way volumetric coupling between a coarse-grain level
 * and an embedded fine level (Sec. 2.3 of Queteschiner et al. 2017).
 * TEST INFRASTRUCTURE ONLY (see dem_oracle.c).
 *
 * One call, in the paper's order and with the readings stated for the
 * library (the paper fixes neither cell sizes, bins, gains, fade shape nor the
 * random generator):
 *   1. boundary surface (feed faces split into square cells): mass of coarse
 *      particles whose centre entered the region through each cell since the
 *      previous call (integer mass units), their fine-scale diameter
 *      histogram (r / alpha), and the mass-weighted (Favre) velocity of coarse
 *      particles within one diameter of the face;
 *   2. transition layer (one hexahedral cell behind each surface cell) on both
 *      levels: volume fraction, Favre velocity, largest speed and the granular
 *      stress of Eq. 7 (1/2 r_ij f_ij over contacts, floor and axisymmetric-
 *      wall contacts with the branch vector from the contact point to the
 *      centre, plus m v'v', symmetrised);
 *   3. stress PI controller on the face-normal stress (setpoint coarse,
 *      process variable fine) and its force on fine particles, faded out
 *      linearly over 3/2 fine diameters and limited by the coarse cell's
 *      largest speed;
 *   4. fine-to-coarse P controller per correction cell (velocity or mass flow
 *      with the volume-fraction ratio capped at 4);
 *   5. simple sequential inhibition (Diggle et al. 1976) of fine particles per
 *      surface cell, in continuous space: radius uniform within a bin drawn
 *      from the entry histogram, centre uniform in the cell's insertion slab,
 *      from SplitMix64 random numbers on counters (a candidate overlapping a
 *      fine particle, an earlier insertion or one of the fine level's
 *      axisymmetric walls, or lying outside the vessel the walls enclose, is
 *      rejected);
 *   6. removal of fine particles that left through drain faces.
 *
 * Spec block CP (doubles): 0..2 lo, 3..5 hi, 6 feed bits, 7 drain bits,
 * 8 surface_cell, 9 layer, 10 corr_cell, 11 interval, 12 bins, 13 alpha,
 * 14 kp, 15 ki, 16 kv, 17 mode, 18 max_attempts, 19 velocity_below (correction
 * cells centred below this height take the velocity target; -inf: none; the seed
 * is passed separately), 20 mass_unit, 21 max_insert, 22 dt, 23 fine particle
 * density.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dem_oracle_common.h"

int orc_contact_pair(const double *P, double ra, double rb, double ma, double mb, int32_t wall, double delta,
                     const double *n, const double *va, const double *vb, const double *wa, const double *wb,
                     double *xi, double dt_hist, double *fa, double *ft);

typedef struct {
    int axis, side, b, c, nb, nc, off;
    double plane, wb, wc;
} cface_t;

typedef struct {
    double lo[3], hi[3];
    int nface;
    cface_t face[6];
    int S, ncr[3], C;
    double wcr[3];
} cgeo_t;

static void make_geo(const double *CP, cgeo_t *g)
{
    memset(g, 0, sizeof(*g));
    for (int a = 0; a < 3; ++a) { g->lo[a] = CP[a]; g->hi[a] = CP[3 + a]; }
    int feed = (int)CP[6], off = 0;
    for (int bit = 0; bit < 6; ++bit) {
        if (!((feed >> bit) & 1)) continue;
        cface_t *f = &g->face[g->nface++];
        f->axis = bit / 2;
        f->side = bit % 2;
        int o1 = (f->axis + 1) % 3, o2 = (f->axis + 2) % 3;
        f->b = o1 < o2 ? o1 : o2;
        f->c = o1 < o2 ? o2 : o1;
        f->plane = f->side == 0 ? g->lo[f->axis] : g->hi[f->axis];
        f->nb = (int)floor((g->hi[f->b] - g->lo[f->b]) / CP[8]);
        f->nc = (int)floor((g->hi[f->c] - g->lo[f->c]) / CP[8]);
        if (f->nb < 1) f->nb = 1;
        if (f->nc < 1) f->nc = 1;
        f->wb = (g->hi[f->b] - g->lo[f->b]) / f->nb;
        f->wc = (g->hi[f->c] - g->lo[f->c]) / f->nc;
        f->off = off;
        off += f->nb * f->nc;
    }
    g->S = off;
    g->C = 1;
    for (int a = 0; a < 3; ++a) {
        g->ncr[a] = (int)floor((g->hi[a] - g->lo[a]) / CP[10]);
        if (g->ncr[a] < 1) g->ncr[a] = 1;
        g->wcr[a] = (g->hi[a] - g->lo[a]) / g->ncr[a];
        g->C *= g->ncr[a];
    }
}

static int in_box(const cgeo_t *g, const double *x)
{
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= g->lo[a] && x[a] < g->hi[a])) return 0;
    return 1;
}

static int face_cell(const cgeo_t *g, const cface_t *f, double pb, double pc)
{
    if (pb < g->lo[f->b] || pb >= g->hi[f->b] || pc < g->lo[f->c] || pc >= g->hi[f->c]) return -1;
    int ib = (int)floor((pb - g->lo[f->b]) / f->wb), ic = (int)floor((pc - g->lo[f->c]) / f->wc);
    if (ib < 0) ib = 0;
    if (ib > f->nb - 1) ib = f->nb - 1;
    if (ic < 0) ic = 0;
    if (ic > f->nc - 1) ic = f->nc - 1;
    return f->off + ib + f->nb * ic;
}

static int layer_cell(const cgeo_t *g, double layer, const double *x, int *fk)
{
    if (!in_box(g, x)) return -1;
    for (int k = 0; k < g->nface; ++k) {
        const cface_t *f = &g->face[k];
        double s = f->side == 0 ? x[f->axis] - f->plane : f->plane - x[f->axis];
        if (s >= 0.0 && s < layer) {
            int c = face_cell(g, f, x[f->b], x[f->c]);
            if (c >= 0) { *fk = k; return c; }
        }
    }
    return -1;
}

static int corr_cell(const cgeo_t *g, const double *x)
{
    if (!in_box(g, x)) return -1;
    int i[3];
    for (int a = 0; a < 3; ++a) {
        i[a] = (int)floor((x[a] - g->lo[a]) / g->wcr[a]);
        if (i[a] < 0) i[a] = 0;
        if (i[a] > g->ncr[a] - 1) i[a] = g->ncr[a] - 1;
    }
    return (i[2] * g->ncr[1] + i[1]) * g->ncr[0] + i[0];
}

static void min_image_d(const double *P, double *d)
{
    for (int a = 0; a < 3; ++a)
        if (P[P_PER + a] != 0.0) {
            double L = P[P_HI + a] - P[P_LO + a];
            d[a] -= L * floor(d[a] / L + 0.5);
        }
}

/* Nearest point of wall segment k (the surface of revolution of the polyline
 * (rho_k, z_k) - (rho_k+1, z_k+1) about the vertical wall axis), seen in the
 * particle's azimuthal half-plane at distance rho from the axis and height z:
 * returns the offsets (a, b) = (rho, z) - nearest point.  Lengths in the
 * caller's frame: rs scales rho_k, zs the z_k, z0 is subtracted from them. */
static void seg_offset(const double *P, int k, double rho, double z, double rs, double z0, double *a, double *b)
{
    const double r0 = P[P_WP + 2 * k] / rs, zz0 = (P[P_WP + 2 * k + 1] - z0) / rs;
    const double dr = P[P_WP + 2 * k + 2] / rs - r0, dz = (P[P_WP + 2 * k + 3] - z0) / rs - zz0;
    double t = ((rho - r0) * dr + (z - zz0) * dz) / (dr * dr + dz * dz);
    if (t < 0.0) t = 0.0;
    else if (t > 1.0) t = 1.0;
    *a = rho - (r0 + t * dr);
    *b = z - (zz0 + t * dz);
}

/* The level's stored tangential overlap of contact (a, b) (a < b particle IDs; b = -1 the floor,
 * -2 - k wall segment k), from its history records sorted by (a, b); zero if it has none. */
static void stored_xi(int64_t nh, const int64_t *ha, const int64_t *hb, const double *hxi, int64_t a, int64_t b,
                      double *xi)
{
    int64_t lo = 0, hi = nh - 1;
    xi[0] = xi[1] = xi[2] = 0.0;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ha[mid] == a && hb[mid] == b) {
            xi[0] = hxi[3 * mid]; xi[1] = hxi[3 * mid + 1]; xi[2] = hxi[3 * mid + 2];
            return;
        }
        if (ha[mid] < a || (ha[mid] == a && hb[mid] < b)) lo = mid + 1;
        else hi = mid - 1;
    }
}

/* Eq. 7 contributions of the particles of one level to the transition cells.
 * lay[(cell)*20 + k]: 0 m, 1..3 m v, 4..9 m v v, 10 V, 11..16 contact stress. */
static void level_layer(const double *CP, const cgeo_t *g, const double *P, int64_t n, const double *x,
                        const double *v, const double *w, const double *r, const double *m, const int64_t *id,
                        int64_t nh, const int64_t *ha, const int64_t *hb, const double *hxi, double dt_hist,
                        double *lay, double *vmax)
{
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    int64_t np = 0;
    pair_t *pairs = orc_find_pairs(P, n, x, r, 0.0, 1, &np);
    int fk;
    for (int64_t i = 0; i < n; ++i) {
        int c = layer_cell(g, CP[9], x + 3 * i, &fk);
        if (c < 0) continue;
        double *A = lay + 20 * (size_t)c;
        A[0] += m[i];
        for (int a = 0; a < 3; ++a) A[1 + a] += m[i] * v[3 * i + a];
        for (int k = 0; k < 6; ++k) A[4 + k] += m[i] * v[3 * i + ij[k][0]] * v[3 * i + ij[k][1]];
        A[10] += 4.0 / 3.0 * ORC_PI * r[i] * r[i] * r[i];
        double sp = sqrt(v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
        if (sp > vmax[c]) vmax[c] = sp;
    }
    /* contacts: the pair force acts on both particles; each particle in a cell
     * adds 1/2 r_ij f_ij with r_ij = x_i - x_j and f_ij the force on i */
    for (int64_t k = 0; k < np; ++k) {
        int64_t a = pairs[k].i, b = pairs[k].j;
        if (id[b] < id[a]) { int64_t t = a; a = b; b = t; }    /* the history is kept in the lower ID's frame */
        double d[3] = {x[3 * a] - x[3 * b], x[3 * a + 1] - x[3 * b + 1], x[3 * a + 2] - x[3 * b + 2]};
        min_image_d(P, d);
        double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double nvec[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double xi[3], fa[3], ft[3];
        stored_xi(nh, ha, hb, hxi, id[a], id[b], xi);
        orc_contact_pair(P, r[a], r[b], m[a], m[b], 0, r[a] + r[b] - dist, nvec, v + 3 * a, v + 3 * b, w + 3 * a,
                         w + 3 * b, xi, dt_hist, fa, ft);
        int ca = layer_cell(g, CP[9], x + 3 * a, &fk), cb = layer_cell(g, CP[9], x + 3 * b, &fk);
        for (int q = 0; q < 6; ++q) {
            int s = ij[q][0], t = ij[q][1];
            double val = 0.25 * (d[s] * fa[t] + d[t] * fa[s]);   /* same for both ends */
            if (ca >= 0) lay[20 * (size_t)ca + 11 + q] += val;
            if (cb >= 0) lay[20 * (size_t)cb + 11 + q] += val;
        }
    }
    free(pairs);
    if (P[P_FLOOR] != 0.0) {
        const double nz[3] = {0, 0, 1}, zero3[3] = {0, 0, 0};
        for (int64_t i = 0; i < n; ++i) {
            double h = x[3 * i + 2] - P[P_FLOORZ];
            if (!(r[i] - h > 0)) continue;
            int c = layer_cell(g, CP[9], x + 3 * i, &fk);
            if (c < 0) continue;
            double xi[3], fa[3], ft[3];
            stored_xi(nh, ha, hb, hxi, id[i], -1, xi);
            orc_contact_pair(P, r[i], 0.0, m[i], 0.0, 1, r[i] - h, nz, v + 3 * i, P + P_FLOORV, w + 3 * i, zero3, xi,
                             dt_hist, fa, ft);
            double rv[3] = {0, 0, h};
            for (int q = 0; q < 6; ++q) {
                int s = ij[q][0], t = ij[q][1];
                lay[20 * (size_t)c + 11 + q] += 0.5 * (rv[s] * fa[t] + rv[t] * fa[s]);
            }
        }
    }
    const int nwp = (int)P[P_NWP];
    for (int64_t i = 0; nwp >= 2 && i < n; ++i) {
        int c = layer_cell(g, CP[9], x + 3 * i, &fk);
        if (c < 0) continue;
        const double ex = x[3 * i] - P[P_WAX], ey = x[3 * i + 1] - P[P_WAY];
        const double rho = sqrt(ex * ex + ey * ey);
        double erx = 1.0, ery = 0.0;
        if (rho > 1e-12) { erx = ex / rho; ery = ey / rho; }
        for (int k = 0; k + 1 < nwp; ++k) {
            double a, b;
            seg_offset(P, k, rho, x[3 * i + 2], 1.0, 0.0, &a, &b);
            const double dist = sqrt(a * a + b * b);
            if (!(r[i] - dist > 0.0)) continue;
            const double nv[3] = {a / dist * erx, a / dist * ery, b / dist}, zero3[3] = {0, 0, 0};
            double xi[3], fa[3], ft[3];
            stored_xi(nh, ha, hb, hxi, id[i], -2 - k, xi);
            orc_contact_pair(P, r[i], 0.0, m[i], 0.0, 1, r[i] - dist, nv, v + 3 * i, zero3, w + 3 * i, zero3, xi,
                             dt_hist, fa, ft);
            const double rv[3] = {dist * nv[0], dist * nv[1], dist * nv[2]};
            for (int q = 0; q < 6; ++q) {
                int s = ij[q][0], t = ij[q][1];
                lay[20 * (size_t)c + 11 + q] += 0.5 * (rv[s] * fa[t] + rv[t] * fa[s]);
            }
        }
    }
}

static void level_corr(const cgeo_t *g, int64_t n, const double *x, const double *v, const double *r,
                       const double *m, double *cor)
{
    for (int64_t i = 0; i < n; ++i) {
        int c = corr_cell(g, x + 3 * i);
        if (c < 0) continue;
        double *o = cor + 5 * (size_t)c;
        o[0] += m[i];
        for (int a = 0; a < 3; ++a) o[1 + a] += m[i] * v[3 * i + a];
        o[4] += 4.0 / 3.0 * ORC_PI * r[i] * r[i] * r[i];
    }
}

/* SplitMix64 (Steele, Lea and Flood 2014) */
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static uint64_t draw(uint64_t seed, int cell, int call, int attempt, int k)
{
    uint64_t ctr = (((uint64_t)cell * 1048576ull + (uint64_t)call) * 16777216ull + (uint64_t)attempt) * 8ull + (uint64_t)k;
    return splitmix64(seed ^ splitmix64(ctr));
}

static int64_t below(uint64_t u, int64_t n) { return (int64_t)(((u >> 32) * (uint64_t)n) >> 32); }

/* uniform in [0, 1) from the top 53 of 64 random bits */
static double unit(uint64_t u) { return (double)(u >> 11) * 0x1p-53; }

/*
 * One coupling call.  Inputs: spec CP and seed; the call number; both levels'
 * parameter blocks (Pc, Pf), states and contact histories (records sorted by
 * (a, b), as the dynamics keep them; the contact forces of Eq. 7 take the
 * stored overlap of each contact, advanced by dth_c / dth_f); the fine level's largest radius rmaxf
 * (the range of the radius histogram) and the borderline band (metres); the
 * coarse positions at the previous call by ID (prev, prev_ok; updated); the
 * carried mass per surface cell (carry; updated) and the controller integral
 * (integ; updated); dt_hist of the stress evaluation per level.
 * Outputs: cross[S] (mass units), hist[S*bins], fav[S*4], layout[2*S*11],
 * ctrl[S*3], corout[2*C*5], fext_c[nc*3], fext_f[nf*3], removed[nf],
 * inserted particles ins_x[S*max_insert*4] (centre and radius, metres),
 * ins_m[S*max_insert], nins[S], border[S].  Returns 0.
 */
int32_t orc_couple(const double *CP, uint64_t seed, int32_t call, const double *Pc, int64_t nc, const double *xc,
                   const double *vc, const double *wc, const double *rc, const double *mc, const int64_t *idc,
                   int64_t nhc, const int64_t *hac, const int64_t *hbc, const double *hxic,
                   const double *Pf, int64_t nf, const double *xf, const double *vf, const double *wf,
                   const double *rf, const double *mf, const int64_t *idf,
                   int64_t nhf, const int64_t *haf, const int64_t *hbf, const double *hxif, double rmaxf, double band,
                   double *prev, int32_t *prev_ok, int64_t *carry, double *integ, double dth_c,
                   double dth_f, uint64_t *cross, uint32_t *hist, double *fav, double *layout, double *ctrl,
                   double *corout, double *fext_c, double *fext_f, int32_t *removed, double *ins_x, double *ins_m,
                   int32_t *nins, int32_t *border)
{
    cgeo_t g;
    make_geo(CP, &g);
    const int S = g.S, C = g.C, bins = (int)CP[12], max_ins = (int)CP[21], max_att = (int)CP[18];
    const double alpha = CP[13], mass_unit = CP[20], dt = CP[22], Tc = CP[11] * dt, layer = CP[9];
    const double wbin = rmaxf / bins;    /* width of a radius bin [m] */
    memset(cross, 0, sizeof(uint64_t) * S);
    memset(hist, 0, sizeof(uint32_t) * S * bins);
    memset(fav, 0, sizeof(double) * S * 4);
    double *lay = (double *)calloc((size_t)2 * S * 20, sizeof(double));
    double *vmax = (double *)calloc((size_t)2 * S, sizeof(double));
    double *cor = (double *)calloc((size_t)2 * C * 5, sizeof(double));
    double L[3];
    for (int a = 0; a < 3; ++a) L[a] = Pc[P_HI + a] - Pc[P_LO + a];

    /* 1. coarse level: entries, histogram, Favre samples */
    for (int64_t i = 0; i < nc; ++i) {
        const double *x = xc + 3 * i;
        int64_t id = idc[i];
        const double *p = prev + 3 * id;
        if (prev_ok[id] && in_box(&g, x)) {
            double seg = 0.0;
            for (int k = 0; k < 3; ++k) seg = fmax(seg, fabs(x[k] - p[k]));
            double span = 0.25 * ((g.hi[0] - g.lo[0]) + (g.hi[1] - g.lo[1]) + (g.hi[2] - g.lo[2]));
            if (!in_box(&g, p) && seg < span) {
                double tbest = 2.0;
                int cbest = -1;
                for (int k = 0; k < g.nface; ++k) {
                    const cface_t *f = &g.face[k];
                    double p0 = p[f->axis], p1 = x[f->axis];
                    int enters = f->side == 0 ? (p0 < f->plane && p1 >= f->plane) : (p0 >= f->plane && p1 < f->plane);
                    if (!enters) continue;
                    double t = (f->plane - p0) / (p1 - p0);
                    int cc = face_cell(&g, f, p[f->b] + t * (x[f->b] - p[f->b]), p[f->c] + t * (x[f->c] - p[f->c]));
                    if (cc >= 0 && t < tbest) { tbest = t; cbest = cc; }
                }
                if (cbest >= 0) {
                    cross[cbest] += (uint64_t)llrint(mc[i] / mass_unit);
                    /* bin of the fine-scale radius r / alpha among bins equal bins over [0, r_max,fine) */
                    double fb = floor(rc[i] / alpha / wbin);
                    int b = fb < (double)(bins - 1) ? (int)fb : bins - 1;
                    hist[(size_t)cbest * bins + b] += 1;
                }
            }
        }
        for (int k = 0; k < g.nface; ++k) {
            const cface_t *f = &g.face[k];
            if (fabs(x[f->axis] - f->plane) >= 2.0 * rc[i]) continue;
            int cc = face_cell(&g, f, x[f->b], x[f->c]);
            if (cc < 0) continue;
            fav[4 * cc] += mc[i];
            for (int a = 0; a < 3; ++a) fav[4 * cc + 1 + a] += mc[i] * vc[3 * i + a];
            break;
        }
    }
    (void)L;

    /* 2. transition and correction cells on both levels */
    level_layer(CP, &g, Pc, nc, xc, vc, wc, rc, mc, idc, nhc, hac, hbc, hxic, dth_c, lay, vmax);
    level_layer(CP, &g, Pf, nf, xf, vf, wf, rf, mf, idf, nhf, haf, hbf, hxif, dth_f, lay + (size_t)S * 20, vmax + S);
    level_corr(&g, nc, xc, vc, rc, mc, cor);
    level_corr(&g, nf, xf, vf, rf, mf, cor + (size_t)C * 5);
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int i = 0; i < S; ++i) {
        int fk = 0;
        for (int k = 0; k < g.nface; ++k)
            if (i >= g.face[k].off && i < g.face[k].off + g.face[k].nb * g.face[k].nc) fk = k;
        const cface_t *f = &g.face[fk];
        double Vc = f->wb * f->wc * layer, saa[2];
        for (int lv = 0; lv < 2; ++lv) {
            const double *A = lay + 20 * ((size_t)lv * S + i);
            double *o = layout + 11 * ((size_t)lv * S + i);
            double M = A[0], vv[3] = {0, 0, 0};
            if (M > 0) for (int a = 0; a < 3; ++a) vv[a] = A[1 + a] / M;
            for (int k = 0; k < 6; ++k) o[k] = (A[11 + k] + A[4 + k] - M * vv[ij[k][0]] * vv[ij[k][1]]) / Vc;
            o[6] = A[10] / Vc;
            for (int a = 0; a < 3; ++a) o[7 + a] = vv[a];
            o[10] = vmax[lv * S + i];
            saa[lv] = o[f->axis];
        }
        /* 3. stress PI controller */
        double e = saa[0] - saa[1];
        integ[i] += e * Tc;
        ctrl[3 * i] = e;
        ctrl[3 * i + 1] = integ[i];
        ctrl[3 * i + 2] = CP[14] * e + CP[15] * integ[i];
    }
    /* 4. fine-to-coarse correction */
    double *dv = (double *)calloc((size_t)C * 3, sizeof(double));
    for (int i = 0; i < C; ++i) {
        const double *Ac = cor + 5 * (size_t)i, *Af = cor + 5 * ((size_t)C + i);
        double *oc = corout + 5 * (size_t)i, *of = corout + 5 * ((size_t)C + i);
        memcpy(oc, Ac, 5 * sizeof(double));
        memcpy(of, Af, 5 * sizeof(double));
        if (Ac[0] > 0 && Af[0] > 0) {
            double fac = 1.0;
            const int iz = i / (g.ncr[0] * g.ncr[1]);
            const double zc = g.lo[2] + (iz + 0.5) * g.wcr[2];
            if ((int)CP[17] == 1 && !(zc < CP[19])) fac = fmin(Af[4] / Ac[4], 4.0);
            for (int a = 0; a < 3; ++a) dv[3 * i + a] = Af[1 + a] / Af[0] * fac - Ac[1 + a] / Ac[0];
        }
    }
    for (int64_t i = 0; i < nc; ++i) {
        int c = corr_cell(&g, xc + 3 * i);
        for (int a = 0; a < 3; ++a) fext_c[3 * i + a] = c >= 0 ? CP[16] * mc[i] * dv[3 * c + a] / Tc : 0.0;
    }
    for (int64_t i = 0; i < nf; ++i) {
        int fk = 0;
        int c = layer_cell(&g, layer, xf + 3 * i, &fk);
        for (int a = 0; a < 3; ++a) fext_f[3 * i + a] = 0.0;
        if (c < 0) continue;
        const cface_t *f = &g.face[fk];
        double s = f->side == 0 ? xf[3 * i + f->axis] - f->plane : f->plane - xf[3 * i + f->axis];
        double wfade = fmax(0.0, 1.0 - s / (1.5 * 2.0 * rf[i]));
        double Fv[3] = {0, 0, 0};
        Fv[f->axis] = (f->side == 0 ? 1.0 : -1.0) * ctrl[3 * c + 2] * ORC_PI * rf[i] * rf[i] * wfade;
        double vm = vmax[c], acc[3], A2 = 0, VA = 0, V2 = 0;
        for (int a = 0; a < 3; ++a) {
            acc[a] = dt * Fv[a] / mf[i];
            A2 += acc[a] * acc[a];
            VA += vf[3 * i + a] * acc[a];
            V2 += vf[3 * i + a] * vf[3 * i + a];
        }
        double lam = 1.0;
        if (A2 > 0 && V2 + 2 * VA + A2 > vm * vm) {
            if (V2 >= vm * vm) lam = 0.0;
            else lam = fmin(1.0, (-VA + sqrt(VA * VA - A2 * (V2 - vm * vm))) / A2);
        }
        for (int a = 0; a < 3; ++a) fext_f[3 * i + a] = lam * Fv[a];
    }

    /* 5. simple sequential inhibition per surface cell, faces in order, cells in row order.
     * A candidate is decided by the smallest of its clearances: distance minus the sum of the
     * radii for the fine particles and the earlier insertions, distance minus the radius for
     * the walls; it is accepted when that is >= 0 (touching is allowed).  A decision whose
     * clearance lies within (-band, band) is recorded in border[cell] (first such attempt;
     * -1: none), where a grid representation of the same draws may decide otherwise. */
    for (int k = 0; k < g.nface; ++k) {
        const cface_t *f = &g.face[k];
        for (int local = 0; local < f->nb * f->nc; ++local) {
            int cell = f->off + local, ib = local % f->nb, ic = local / f->nb;
            int64_t quota = (int64_t)cross[cell] + carry[cell];
            uint64_t total = 0;
            for (int b = 0; b < bins; ++b) total += hist[(size_t)cell * bins + b];
            double M = fav[4 * cell], vn = 0.0;
            if (M > 0) vn = fav[4 * cell + 1 + f->axis] / M;
            int n_in = 0, fails = 0, attempt = 0;
            border[cell] = -1;
            double *mine = ins_x + (size_t)cell * max_ins * 4;
            double b0 = g.lo[f->b] + ib * f->wb, c0 = g.lo[f->c] + ic * f->wc;
            while (quota > 0 && total > 0 && fails < max_att && n_in < max_ins) {
                /* radius: a bin drawn with probability proportional to its count, then uniform in it */
                int64_t pick = below(draw(seed, cell, call, attempt, 0), (int64_t)total);
                int b = 0;
                while (pick >= (int64_t)hist[(size_t)cell * bins + b]) { pick -= hist[(size_t)cell * bins + b]; ++b; }
                double r = ((double)b + unit(draw(seed, cell, call, attempt, 1))) * wbin;
                /* centre: uniform over the cell's face shrunk by r, and along the inward normal over
                 * [r, r + depth] from the face, depth = max(2 r, |<v_n>| T_c) */
                double depth = fmax(2.0 * r, fabs(vn) * Tc);
                double sb = f->wb - 2.0 * r, sc = f->wc - 2.0 * r;
                if (!(r > 0.0) || sb < 0.0 || sc < 0.0) { ++attempt; ++fails; continue; }
                double nlo = f->side == 0 ? f->plane + r : f->plane - r - depth;
                double xc[3];
                xc[f->b] = (b0 + r) + unit(draw(seed, cell, call, attempt, 2)) * sb;
                xc[f->c] = (c0 + r) + unit(draw(seed, cell, call, attempt, 3)) * sc;
                xc[f->axis] = nlo + unit(draw(seed, cell, call, attempt, 4)) * depth;
                ++attempt;
                double clear = INFINITY;
                int inside = 1;
                /* the fine level's axisymmetric walls: clearance, and inside the vessel (a ray from
                 * the centre away from the axis crosses the non-horizontal segments, each closed
                 * below and open above, an odd number of times) */
                const int nwp = (int)Pf[P_NWP];
                if (nwp >= 2) {
                    const double ex = xc[0] - Pf[P_WAX], ey = xc[1] - Pf[P_WAY];
                    const double rho = sqrt(ex * ex + ey * ey), z = xc[2];
                    int crossings = 0;
                    for (int kk = 0; kk + 1 < nwp; ++kk) {
                        double a, bb;
                        seg_offset(Pf, kk, rho, z, 1.0, 0.0, &a, &bb);
                        clear = fmin(clear, sqrt(a * a + bb * bb) - r);
                        const double r0 = Pf[P_WP + 2 * kk], z0 = Pf[P_WP + 2 * kk + 1];
                        const double r1 = Pf[P_WP + 2 * kk + 2], z1 = Pf[P_WP + 2 * kk + 3];
                        if (z0 != z1 && (z >= z0) != (z >= z1) && r0 + (z - z0) * (r1 - r0) / (z1 - z0) > rho) ++crossings;
                    }
                    if (!(crossings & 1)) inside = 0;
                }
                for (int64_t j = 0; j < nf; ++j) {
                    double d[3] = {xc[0] - xf[3 * j], xc[1] - xf[3 * j + 1], xc[2] - xf[3 * j + 2]};
                    min_image_d(Pf, d);
                    clear = fmin(clear, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - (r + rf[j]));
                }
                for (int t = 0; t < n_in; ++t) {
                    double d[3] = {xc[0] - mine[4 * t], xc[1] - mine[4 * t + 1], xc[2] - mine[4 * t + 2]};
                    clear = fmin(clear, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - (r + mine[4 * t + 3]));
                }
                for (int kk = 0; kk < k; ++kk) {
                    const cface_t *o = &g.face[kk];
                    for (int oc = o->off; oc < o->off + o->nb * o->nc; ++oc) {
                        const double *other = ins_x + (size_t)oc * max_ins * 4;
                        for (int t = 0; t < nins[oc]; ++t) {
                            double d[3] = {xc[0] - other[4 * t], xc[1] - other[4 * t + 1], xc[2] - other[4 * t + 2]};
                            clear = fmin(clear, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - (r + other[4 * t + 3]));
                        }
                    }
                }
                if (inside && fabs(clear) < band && border[cell] < 0) border[cell] = attempt - 1;
                if (!inside || clear < 0.0) { ++fails; continue; }
                /* mass of a solid sphere of the fine density */
                double m = CP[23] * (4.0 / 3.0 * ORC_PI) * r * r * r;
                mine[4 * n_in] = xc[0]; mine[4 * n_in + 1] = xc[1]; mine[4 * n_in + 2] = xc[2]; mine[4 * n_in + 3] = r;
                ins_m[(size_t)cell * max_ins + n_in] = m;
                ++n_in;
                quota -= llrint(m / mass_unit);
            }
            nins[cell] = n_in;
            carry[cell] = quota;
        }
    }

    /* 6. removal through drain faces */
    int drain = (int)CP[7];
    for (int64_t i = 0; i < nf; ++i) {
        int gone = 0;
        for (int a = 0; a < 3; ++a) {
            if ((drain >> (2 * a)) & 1) gone |= xf[3 * i + a] < g.lo[a];
            if ((drain >> (2 * a + 1)) & 1) gone |= xf[3 * i + a] >= g.hi[a];
        }
        removed[i] = gone;
    }
    /* remember the coarse positions */
    for (int64_t i = 0; i < nc; ++i) {
        for (int a = 0; a < 3; ++a) prev[3 * idc[i] + a] = xc[3 * i + a];
        prev_ok[idc[i]] = 1;
    }
    free(lay);
    free(vmax);
    free(cor);
    free(dv);
    return 0;
}
