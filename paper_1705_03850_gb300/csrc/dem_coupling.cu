// Two-way volumetric coupling of a coarse-grain level and an embedded fine
// level (Sec. 2.3): boundary-surface measurement, transition-layer stress (Eq. 7)
// with a PI controller acting on the fine particles, fine-to-coarse P
// correction, insertion of fine particles by simple sequential inhibition, and
// removal through drain faces.  The interface and the readings of the paper are
// documented in include/dem.h (dem_coupling).
#include "dem.h"
#include "dem_contact.cuh"
#include "dem_ctx.h"
#include "dem_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace cgdem;

namespace {

constexpr int MAXBINS = 32;
constexpr int MAXCR = 256;     // correction cells per axis at most (integer thresholds per axis)

struct Face {
    int axis, side;      // side 0: the face at lo[axis] (inward normal +e_axis), 1: at hi[axis]
    int b, c;            // in-plane axes
    int nb, nc, off;     // cells along b and c, first cell index
    double plane, wb, wc;
    double iwb, iwc;     // 1 / wb, 1 / wc
};

struct Geo {
    double lo[3], hi[3];
    int nface;
    Face face[6];
    int S;               // surface cells (= transition cells)
    int ncr[3];
    double wcr[3], iwcr[3];   // correction cell widths and their reciprocals
    int C;               // correction cells
    double layer, alpha, Tc, dt, kp, ki, kv, mass_unit;
    int bins, mode, max_attempts, max_insert, drain;
    unsigned long long seed;
    int call;            // coupling interval counter (random-number counter)
    // the two levels' frames: x = lo + u q
    double loc[3], qc, lof[3], qf;
    double wbin;         // width of a radius bin: the fine level's largest radius / bins [m]
    int fresh_c, fresh_f;
    float cells_per_unit[2][3];  // correction cells per position unit (a first guess of the cell)
    int add;             // add the controller forces to the held ones instead of replacing them
    double vel_below;    // correction cells centred below this height take the velocity target
    // coarse positions (units) outside [ulo, uhi) take part in nothing but the position record:
    // the region grown by the largest coarse diameter and two units, rounded outwards
    long long ulo[3], uhi[3];
    // per level (0 coarse, 1 fine) and feed face: a box in that level's units, rounded outwards,
    // holding the face's transition layer; positions outside every such box lie in no layer cell
    long long lay_lo[2][6][3], lay_hi[2][6][3];
};

struct Acc {
    // surface cells
    unsigned long long* cross;   // entered mass [mass units]
    unsigned* hist;              // [S][MAXBINS]
    double* fav;                 // [S][4]: sum m, sum m v
    long long* carry;            // [S]
    int* nins;                   // [S]
    int4* ins;                   // [S][max_insert] inserted particles, fine units (r in w)
    double* insm;                // [S][max_insert] their masses [kg]
    // transition cells, level L = 0 coarse, 1 fine
    double* lay;                 // [2][S][20]: m, mv(3), mvv(6), V, contact stress(6), -, -, -
    unsigned* vmax;              // [2][S] largest speed (float bits)
    double* ctrl;                // [S][3]: e, I, u
    double* out;                 // [2][S][11]: sigma(6), phi, v(3), vmax
    // correction cells
    double* cor;                 // [2][C][5]: m, mv(3), V
    double* dv;                  // [C][3] velocity change asked of the coarse particles
    // coarse particles by ID: position at the previous call (integer units), validity
    int4* prev;                  // [idcap]
    int* prev_ok;
    // per level (0 coarse, 1 fine) and axis: the correction grid as integer thresholds in that
    // level's units: a position u lies in the region iff thr[0] <= u < thr[ncr], in cell i iff
    // thr[i] <= u < thr[i + 1] (the decisions of the double expressions, see cell_thresholds)
    long long* thr;              // [2][3][MAXCR + 1]
    int* removed;                // [1] fine particles removed at this call
    // rows of the particles inserted at this call, without a list build: the (existing slot,
    // new slot) pairs to append to existing rows, and [0] pairs, [1] fall back to a list
    // build, [2] particles appended at this call
    unsigned long long* pairs;   // [PAIRS_MAX]
    int* npairs;                 // [4]
};
constexpr int PAIRS_MAX = 4096;

// position in metres of integer coordinate u on axis a: lo + u q, rounded once (as the read-out)
__device__ __forceinline__ double posm(const double* lo, double q, int u, int a) { return __fma_rn((double)u, q, lo[a]); }

// correction cell of an integer position of level L from the integer thresholds (-1 outside)
__device__ __forceinline__ int corr_cell_u(const Geo& g, const long long* thr, int L, int4 P)
{
    int idx[3];
    for (int a = 0; a < 3; ++a) {
        const long long* T = thr + ((size_t)L * 3 + a) * (MAXCR + 1);
        const long long u = a == 0 ? P.x : a == 1 ? P.y : P.z;
        const int n = g.ncr[a];
        if (u < __ldg(T) || u >= __ldg(T + n)) return -1;
        int i = (int)((float)(u - __ldg(T)) * g.cells_per_unit[L][a]);
        i = min(max(i, 0), n - 1);
        while (i + 1 < n && u >= __ldg(T + i + 1)) ++i;
        while (i > 0 && u < __ldg(T + i)) --i;
        idx[a] = i;
    }
    return (idx[2] * g.ncr[1] + idx[1]) * g.ncr[0] + idx[0];
}

// inside the region by the integer thresholds (level L)
__device__ __forceinline__ bool inside_u(const Geo& g, const long long* thr, int L, long long ux, long long uy,
                                         long long uz)
{
    const long long u[3] = {ux, uy, uz};
    for (int a = 0; a < 3; ++a) {
        const long long* T = thr + ((size_t)L * 3 + a) * (MAXCR + 1);
        if (u[a] < __ldg(T) || u[a] >= __ldg(T + g.ncr[a])) return false;
    }
    return true;
}

__device__ __forceinline__ bool inside_box(const Geo& g, const double* x)
{
    return x[0] >= g.lo[0] && x[0] < g.hi[0] && x[1] >= g.lo[1] && x[1] < g.hi[1] && x[2] >= g.lo[2] &&
           x[2] < g.hi[2];
}

// floor(a / w) as the correctly rounded division gives it, from the product with the
// reciprocal (FP64 division is slow here); the division decides the rare cases where the
// product lies within 1e-6 of an integer
__device__ __forceinline__ double floor_div(double a, double w, double iw)
{
    const double t = a * iw, f = floor(t);
    if (t - f < 1e-6 || f + 1.0 - t < 1e-6) return floor(a / w);
    return f;
}

// surface / transition cell of an in-plane point of face f (-1 outside the face)
__device__ __forceinline__ int face_cell(const Face& f, double pb, double pc, const Geo& g)
{
    if (pb < g.lo[f.b] || pb >= g.hi[f.b] || pc < g.lo[f.c] || pc >= g.hi[f.c]) return -1;
    int ib = (int)floor_div(pb - g.lo[f.b], f.wb, f.iwb), ic = (int)floor_div(pc - g.lo[f.c], f.wc, f.iwc);
    ib = min(max(ib, 0), f.nb - 1);
    ic = min(max(ic, 0), f.nc - 1);
    return f.off + ib + f.nb * ic;
}

// false only if the integer position P of level L lies outside every face's layer box (then
// layer_cell is -1); true means: decide with layer_cell
__device__ __forceinline__ bool maybe_layer(const Geo& g, int L, int4 P)
{
    for (int k = 0; k < g.nface; ++k) {
        const long long* lo = g.lay_lo[L][k];
        const long long* hi = g.lay_hi[L][k];
        if (P.x >= lo[0] && P.x < hi[0] && P.y >= lo[1] && P.y < hi[1] && P.z >= lo[2] && P.z < hi[2]) return true;
    }
    return false;
}

// transition cell holding a point (first face in order wins at corners), or -1
__device__ __forceinline__ int layer_cell(const Geo& g, const double* x, int* fidx)
{
    if (!inside_box(g, x)) return -1;
    for (int k = 0; k < g.nface; ++k) {
        const Face& f = g.face[k];
        const double s = f.side == 0 ? x[f.axis] - f.plane : f.plane - x[f.axis];
        if (s >= 0.0 && s < g.layer) {
            const int c = face_cell(f, x[f.b], x[f.c], g);
            if (c >= 0) {
                *fidx = k;
                return c;
            }
        }
    }
    return -1;
}

// add (m, m v, V) of a particle to its correction cell.  With the whole warp active, the lanes
// form runs of equal cells (consecutive slots: Morton order keeps a cell's particles together);
// a segmented scan over the warp sums each run in float (at most 32 terms) and the run's last
// lane adds the sums to the cell's double accumulators, so a warp issues five atomics per run
// instead of five per particle
__device__ __forceinline__ void corr_add(double* cor, int cc, float m, const float4& V, float vol)
{
    const unsigned act = __activemask();
    const bool live = cc >= 0;
    float v[5] = {live ? m : 0.f, live ? m * V.x : 0.f, live ? m * V.y : 0.f, live ? m * V.z : 0.f, live ? vol : 0.f};
    if (act == 0xffffffffu) {
        const int lane = (int)threadIdx.x & 31;
        const int up = __shfl_up_sync(0xffffffffu, cc, 1);
        const int dn = __shfl_down_sync(0xffffffffu, cc, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || up != cc);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // this lane's run head
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float y = __shfl_up_sync(0xffffffffu, v[k], o);
                if (lane - o >= start) v[k] += y;
            }
        }
        if (live && (lane == 31 || dn != cc)) {
            double* o = cor + (size_t)cc * 5;
            for (int k = 0; k < 5; ++k) atomicAdd(o + k, (double)v[k]);
        }
        return;
    }
    if (!live) return;
    double* o = cor + (size_t)cc * 5;
    for (int k = 0; k < 5; ++k) atomicAdd(o + k, (double)v[k]);
}

__device__ __forceinline__ void atomic_max_f(unsigned* a, float v)
{
    if (v > 0.f) atomicMax(a, __float_as_uint(v));
}

// Eq. 7 accumulation of one particle into a transition cell: mass, momentum,
// m v v, volume, and the contact part 1/2 r_ij (x) f_ij over its contacts
// (floor contact: branch vector to the contact point, no 1/2), symmetrised.
// (not inlined: few particles lie in a transition cell, and inlining the contact law would
// give every thread of the per-particle passes its registers)
__device__ __noinline__ void layer_add(const Dev& d, const InstC& c, const InstD& D, int s, double* acc, unsigned* vmax,
                                       int fresh)
{
    const int cur = D.cur, lp = D.lp, ncap = d.ncap;
    const size_t plane = (size_t)d.Lmax * ncap;
    const int4 P = d.pos[cur][s];
    const float4 Vv = d.vel[cur][s], Wv = d.omg[cur][s];
    const double m = Wv.w, q = c.q;
    const double r = (double)P.w * q;
    const double v[3] = {Vv.x, Vv.y, Vv.z};
    atomicAdd(acc + 0, m);
    for (int a = 0; a < 3; ++a) atomicAdd(acc + 1 + a, m * v[a]);
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int k = 0; k < 6; ++k) atomicAdd(acc + 4 + k, m * v[ij[k][0]] * v[ij[k][1]]);
    atomicAdd(acc + 10, 4.0 / 3.0 * 3.14159265358979323846 * r * r * r);
    atomic_max_f(vmax, sqrtf(Vv.x * Vv.x + Vv.y * Vv.y + Vv.z * Vv.z));
    const Coef<float> cf{c.c_kn, c.c_kt, c.nbeta, c.gt_ratio, c.mu, c.mu_w, c.clamp_fn};
    const float dt_hist = fresh ? 0.f : c.dt;
    const unsigned hm = d.hmask[lp][s];
    double st[6] = {0, 0, 0, 0, 0, 0};
    const int ncnt = d.cnt[lp][s];
    // the contacts: the row's indices and positions in batches of four independent loads (a
    // walk entry by entry makes every entry a chain of dependent round trips)
    unsigned tm = 0u;
    for (int e0 = 0; e0 < ncnt; e0 += 4) {
        int jb[4];
        int4 Qb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) jb[k] = e0 + k < ncnt ? d.nbr[lp][(size_t)(e0 + k) * ncap + s] : s;
#pragma unroll
        for (int k = 0; k < 4; ++k) Qb[k] = d.pos[cur][jb[k]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int dx = min_image(P.x - Qb[k].x, c.per[0], c.ext[0], c.half[0]);
            const int dy = min_image(P.y - Qb[k].y, c.per[1], c.ext[1], c.half[1]);
            const int dz = P.z - Qb[k].z;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            const int S = P.w + Qb[k].w;
            if (e0 + k < ncnt && d2 < (long long)S * S) tm |= 1u << (e0 + k);
        }
    }
    for (unsigned rem = tm; rem; rem &= rem - 1u) {
        const int e = __ffs(rem) - 1;
        const int j = d.nbr[lp][(size_t)e * ncap + s];
        const int4 Q = d.pos[cur][j];
        const float4 Vj = d.vel[cur][j], Wj = d.omg[cur][j];
        const int dx = min_image(P.x - Q.x, c.per[0], c.ext[0], c.half[0]);
        const int dy = min_image(P.y - Q.y, c.per[1], c.ext[1], c.half[1]);
        const int dz = P.z - Q.z;
        const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
        const int S = P.w + Q.w;
        const long long S2 = (long long)S * S;
        const float d2f = (float)d2;
        const float inv = rsqrtf(d2f);
        const float dist = d2f * inv;
        const float delta = __fdividef((float)(S2 - d2), (float)S + dist) * (float)q;
        const Vec3<float> n = mk3((float)dx * inv, (float)dy * inv, (float)dz * inv);
        const float* h = d.hist[lp] + s + (size_t)e * ncap;
        Vec3<float> xi = ((hm >> e) & 1u) ? mk3(h[0], h[plane], h[2 * plane]) : mk3(0.f, 0.f, 0.f);
        Vec3<float> ft;
        bool slip;
        const Vec3<float> fa = contact_fwd<float, false>(cf, delta, n, (float)r, (float)((double)Q.w * q), (float)m,
                                                         Wj.w, mk3(Vv.x, Vv.y, Vv.z), mk3(Vj.x, Vj.y, Vj.z),
                                                         mk3(Wv.x, Wv.y, Wv.z), mk3(Wj.x, Wj.y, Wj.z), xi, dt_hist,
                                                         ft, slip);
        const double rv[3] = {dx * q, dy * q, dz * q}, f[3] = {fa.x, fa.y, fa.z};
        for (int k = 0; k < 6; ++k) {
            const int a = ij[k][0], b = ij[k][1];
            st[k] += 0.25 * (rv[a] * f[b] + rv[b] * f[a]);
        }
    }
    if (c.floor_on && P.w - P.z > 0) {
        const float4 hw = d.whist[lp][s];
        const bool wall_prev = (__float_as_uint(Vv.w) & WALL_BIT) != 0u;
        Vec3<float> xi = wall_prev ? mk3(hw.x, hw.y, hw.z) : mk3(0.f, 0.f, 0.f);
        Vec3<float> ft;
        bool slip;
        const Vec3<float> fa = contact_fwd<float, true>(cf, (float)((P.w - P.z) * q), mk3(0.f, 0.f, 1.f), (float)r, 0.f,
                                                        (float)m, 0.f, mk3(Vv.x, Vv.y, Vv.z),
                                                        mk3(c.floor_v[0], c.floor_v[1], c.floor_v[2]),
                                                        mk3(Wv.x, Wv.y, Wv.z), mk3(0.f, 0.f, 0.f), xi, dt_hist, ft, slip);
        const double rv[3] = {0.0, 0.0, (double)P.z * q}, f[3] = {fa.x, fa.y, fa.z};
        for (int k = 0; k < 6; ++k) {
            const int a = ij[k][0], b = ij[k][1];
            st[k] += 0.5 * (rv[a] * f[b] + rv[b] * f[a]);
        }
    }
    if (c.nwp >= 2) {   // axisymmetric walls: branch vector from the contact point to the centre
        const double ex = (double)P.x - c.wax, ey = (double)P.y - c.way, z = (double)P.z;
        const double rho = sqrt(ex * ex + ey * ey);
        float erx = 1.f, ery = 0.f;
        if (rho > 0.0) {
            erx = (float)(ex / rho);
            ery = (float)(ey / rho);
        }
        const float4 h0 = d.wseg[lp][s], h1 = d.wseg[lp][(size_t)ncap + s];
        for (int k = 0; k + 1 < c.nwp; ++k) {
            double a, b;
            wall_seg_offset(c, k, rho, z, a, b);
            const double dist = sqrt(a * a + b * b);
            const double dl = (double)P.w - dist;
            if (!(dl > 0.0)) continue;
            const float na = (float)(a / dist);
            const Vec3<float> n = mk3(na * erx, na * ery, (float)(b / dist));
            const unsigned tag = (unsigned)k + 1u;
            Vec3<float> xi = mk3(0.f, 0.f, 0.f);
            if (__float_as_uint(h0.w) == tag) xi = mk3(h0.x, h0.y, h0.z);
            else if (__float_as_uint(h1.w) == tag) xi = mk3(h1.x, h1.y, h1.z);
            Vec3<float> ft;
            bool slip;
            const Vec3<float> fa = contact_fwd<float, true>(cf, (float)(dl * q), n, (float)r, 0.f, (float)m, 0.f,
                                                            mk3(Vv.x, Vv.y, Vv.z), mk3(0.f, 0.f, 0.f),
                                                            mk3(Wv.x, Wv.y, Wv.z), mk3(0.f, 0.f, 0.f), xi, dt_hist,
                                                            ft, slip);
            const double rv[3] = {dist * q * n.x, dist * q * n.y, dist * q * n.z}, f[3] = {fa.x, fa.y, fa.z};
            for (int kk = 0; kk < 6; ++kk) {
                const int ia = ij[kk][0], ib = ij[kk][1];
                st[kk] += 0.5 * (rv[ia] * f[ib] + rv[ib] * f[ia]);
            }
        }
    }
    for (int k = 0; k < 6; ++k) atomicAdd(acc + 11 + k, st[k]);
}

// the live slots of a single-instance context (coupling contexts have one instance), two per
// thread and iteration, with both slots' position and velocity loaded before either is used;
// removed particles (below a wall's removal height) are skipped
template <typename Fn>
__device__ __forceinline__ void for_live(const Dev& d, Fn fn)
{
    const InstD D = d.id[0];
    const InstC& c = d.ic[0];
    const int4* __restrict__ pos = d.pos[D.cur];
    const float4* __restrict__ vel = d.vel[D.cur];
    const int end = c.slot0 + D.n;
    const int stride = (int)(gridDim.x * blockDim.x);
    for (int s0 = c.slot0 + (int)(blockIdx.x * blockDim.x + threadIdx.x); s0 < end; s0 += 2 * stride) {
        const int s1 = s0 + stride;
        const bool has1 = s1 < end;
        const int4 P0 = pos[s0];
        const float4 V0 = vel[s0];
        const int4 P1 = has1 ? pos[s1] : P0;
        const float4 V1 = has1 ? vel[s1] : V0;
        if (!(__float_as_uint(V0.w) & GONE_BIT)) fn(s0, c, D, P0, V0);
        if (has1 && !(__float_as_uint(V1.w) & GONE_BIT)) fn(s1, c, D, P1, V1);
    }
}

// one element of the per-call accumulators per thread (a thread per cell with a loop over its
// 90 words took 6-10 µs)
__global__ void k_cp_clear(Geo g, Acc a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.S * MAXBINS) a.hist[i] = 0u;
    if (i < 2 * g.S * 20) a.lay[i] = 0.0;
    if (i < 2 * g.C * 5) a.cor[i] = 0.0;
    if (i < 4 * g.S) a.fav[i] = 0.0;
    if (i < 2 * g.S) a.vmax[i] = 0u;
    if (i < g.S) {
        a.cross[i] = 0ull;
        a.nins[i] = 0;
    }
    if (i == 0) a.removed[0] = 0;
}
inline int clear_threads(int S, int C) { return std::max(std::max(S * MAXBINS, 2 * S * 20), 2 * C * 5); }

// coarse level: entries through the feed faces, Favre samples at the faces,
// transition and correction cells; remember the positions for the next call
__global__ void __launch_bounds__(TILE, 8) k_cp_coarse(Dev d, Geo g, Acc a, int record_only)
{
    for_live(d, [&](int s, const InstC& c, const InstD& D, const int4 P, const float4 V) {
        const unsigned id = __float_as_uint(V.w) & ID_MASK;
        const bool near = P.x >= g.ulo[0] && P.x < g.uhi[0] && P.y >= g.ulo[1] && P.y < g.uhi[1] &&
                          P.z >= g.ulo[2] && P.z < g.uhi[2];
        if (!record_only && near) {
            const double x[3] = {posm(g.loc, g.qc, P.x, 0), posm(g.loc, g.qc, P.y, 1), posm(g.loc, g.qc, P.z, 2)};
            const double r = (double)P.w * g.qc;
            const float mf = d.omg[D.cur][s].w;
            const double m = mf;
            // entry through a feed face since the previous call (inside now, outside then)
            if (a.prev_ok[id] && inside_u(g, a.thr, 0, P.x, P.y, P.z)) {
                const int4 pu = a.prev[id];
                if (!inside_u(g, a.thr, 0, pu.x, pu.y, pu.z)) {
                    const double p[3] = {posm(g.loc, g.qc, pu.x, 0), posm(g.loc, g.qc, pu.y, 1),
                                         posm(g.loc, g.qc, pu.z, 2)};
                    double seg = 0.0;
                    for (int k = 0; k < 3; ++k) seg = fmax(seg, fabs(x[k] - p[k]));
                    if (seg < 0.25 * (g.hi[0] - g.lo[0] + g.hi[1] - g.lo[1] + g.hi[2] - g.lo[2])) {
                        double tbest = 2.0;
                        int cbest = -1;
                        for (int k = 0; k < g.nface; ++k) {
                            const Face& f = g.face[k];
                            const double p0 = p[f.axis], p1 = x[f.axis];
                            const bool enters = f.side == 0 ? (p0 < f.plane && p1 >= f.plane) : (p0 >= f.plane && p1 < f.plane);
                            if (!enters) continue;
                            const double t = (f.plane - p0) / (p1 - p0);
                            const int cc = face_cell(f, p[f.b] + t * (x[f.b] - p[f.b]), p[f.c] + t * (x[f.c] - p[f.c]), g);
                            if (cc >= 0 && t < tbest) {
                                tbest = t;
                                cbest = cc;
                            }
                        }
                        if (cbest >= 0) {
                            atomicAdd(a.cross + cbest, (unsigned long long)llrint(m / g.mass_unit));
                            // bin of the fine-scale radius r / alpha among equal bins over [0, r_max,fine)
                            // (the last bin takes anything larger)
                            const double fb = floor(r / g.alpha / g.wbin);
                            const int b = fb < (double)(g.bins - 1) ? (int)fb : g.bins - 1;
                            atomicAdd(a.hist + (size_t)cbest * MAXBINS + b, 1u);
                        }
                    }
                }
            }
            // Favre sample at the faces: centres within one diameter of a feed face
            for (int k = 0; k < g.nface; ++k) {
                const Face& f = g.face[k];
                if (fabs(x[f.axis] - f.plane) >= 2.0 * r) continue;
                const int cc = face_cell(f, x[f.b], x[f.c], g);
                if (cc < 0) continue;
                atomicAdd(a.fav + 4 * cc, m);
                atomicAdd(a.fav + 4 * cc + 1, m * V.x);
                atomicAdd(a.fav + 4 * cc + 2, m * V.y);
                atomicAdd(a.fav + 4 * cc + 3, m * V.z);
                break;
            }
            int fk;
            const int lc = maybe_layer(g, 0, P) ? layer_cell(g, x, &fk) : -1;
            if (lc >= 0) layer_add(d, c, D, s, a.lay + (size_t)lc * 20, a.vmax + lc, g.fresh_c);
            const float rf = (float)r;
            corr_add(a.cor, corr_cell_u(g, a.thr, 0, P), mf, V, 4.18879020f * rf * rf * rf);
        }
        // the position record, kept only inside the grown region: a particle outside it cannot
        // be inside the region at the next call (that takes a move of more than a diameter in one
        // interval), and one that comes back crosses the band of the grown region first, where it
        // is recorded again; the far particles' scattered record writes took most of this pass
        if (near) {
            a.prev[id] = make_int4(P.x, P.y, P.z, 0);
            a.prev_ok[id] = 1;
        }
    });
}

// fine level: transition and correction cells, removal through drain faces
__global__ void __launch_bounds__(TILE, 8) k_cp_fine(Dev d, Geo g, Acc a)
{
    for_live(d, [&](int s, const InstC& c, const InstD& D, const int4 P, float4 V) {
        const float mf = d.omg[D.cur][s].w;     // loaded before the layer call (which may write memory)
        if (maybe_layer(g, 1, P)) {
            const double x[3] = {posm(g.lof, g.qf, P.x, 0), posm(g.lof, g.qf, P.y, 1), posm(g.lof, g.qf, P.z, 2)};
            int fk;
            const int lc = layer_cell(g, x, &fk);
            if (lc >= 0) layer_add(d, c, D, s, a.lay + ((size_t)g.S + lc) * 20, a.vmax + g.S + lc, g.fresh_f);
        }
        const float rf = (float)((double)P.w * g.qf);
        corr_add(a.cor + (size_t)g.C * 5, corr_cell_u(g, a.thr, 1, P), mf, V, 4.18879020f * rf * rf * rf);
        // drain faces: x < lo or x >= hi on their axes (the region bounds as integer thresholds)
        bool gone = false;
        for (int ax = 0; ax < 3; ++ax) {
            const long long* T = a.thr + ((size_t)3 + ax) * (MAXCR + 1);
            const long long u = ax == 0 ? P.x : ax == 1 ? P.y : P.z;
            if ((g.drain >> (2 * ax)) & 1) gone |= u < __ldg(T);
            if ((g.drain >> (2 * ax + 1)) & 1) gone |= u >= __ldg(T + g.ncr[ax]);
        }
        if (gone) {
            // marked and left in place with no radius until the next list build drops it (its
            // neighbours, further than a radius from its centre, can no longer touch it)
            V.w = __uint_as_float(__float_as_uint(V.w) | GONE_BIT);
            d.vel[D.cur][s] = V;
            d.pos[D.cur][s] = make_int4(P.x, P.y, P.z, 0);
            atomicAdd(a.removed, 1);
        }
    });
}

// per cell: finish the averages, update the controllers.  Threads 2i and 2i + 1 take surface
// cell i of the coarse and the fine level (Eq. 7 from the accumulated sums); the even one then
// updates the cell's PI controller from both.  Threads 2S + i take correction cell i.  The
// shared denominators are inverted once (FP64 division is slow on this part: one thread per
// cell doing every division in turn took 28-31 µs)
__global__ void k_cp_cells(Geo g, Acc a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ((2 * g.S + 31) & ~31)) {          // whole warps: the pair exchange below
        const int i = t >> 1, L = t & 1;
        double sig = 0.0;
        int axis = 0;
        if (i < g.S) {
            int fk = 0;
            for (int k = 0; k < g.nface; ++k)
                if (i >= g.face[k].off && i < g.face[k].off + g.face[k].nb * g.face[k].nc) fk = k;
            const Face& f = g.face[fk];
            axis = f.axis;
            const double iVc = 1.0 / (f.wb * f.wc * g.layer);
            const double* A = a.lay + ((size_t)L * g.S + i) * 20;
            double* o = a.out + ((size_t)L * g.S + i) * 11;
            const double M = A[0];
            double v[3] = {0, 0, 0};
            if (M > 0) {
                const double iM = 1.0 / M;
                for (int k = 0; k < 3; ++k) v[k] = A[1 + k] * iM;
            }
            const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
            for (int k = 0; k < 6; ++k) o[k] = (A[11 + k] + A[4 + k] - M * v[ij[k][0]] * v[ij[k][1]]) * iVc;
            o[6] = A[10] * iVc;
            for (int k = 0; k < 3; ++k) o[7 + k] = v[k];
            o[10] = __uint_as_float(a.vmax[L * g.S + i]);
            sig = o[axis];
        }
        const double sig_f = __shfl_xor_sync(0xffffffffu, sig, 1);
        if (i < g.S && L == 0) {
            double* ct = a.ctrl + 3 * (size_t)i;
            const double e = sig - sig_f;
            ct[0] = e;
            ct[1] += e * g.Tc;
            ct[2] = g.kp * e + g.ki * ct[1];
        }
        return;
    }
    const int i = t - ((2 * g.S + 31) & ~31);
    if (i < g.C) {
        const double* Ac = a.cor + (size_t)i * 5;
        const double* Af = a.cor + ((size_t)g.C + i) * 5;
        double* dv = a.dv + 3 * (size_t)i;
        dv[0] = dv[1] = dv[2] = 0.0;
        if (Ac[0] > 0 && Af[0] > 0) {
            double fac = 1.0;
            const int iz = i / (g.ncr[0] * g.ncr[1]);
            const double zc = g.lo[2] + (iz + 0.5) * g.wcr[2];
            if (g.mode == 1 && !(zc < g.vel_below)) fac = fmin(Af[4] / Ac[4], 4.0);
            const double iAf = 1.0 / Af[0], iAc = 1.0 / Ac[0];
            for (int k = 0; k < 3; ++k) dv[k] = Af[1 + k] * iAf * fac - Ac[1 + k] * iAc;
        }
    }
}
inline int cells_threads(int S, int C) { return ((2 * S + 31) & ~31) + C; }

__global__ void __launch_bounds__(TILE) k_cp_force_fine(Dev d, Geo g, Acc a)
{
    for_live(d, [&](int s, const InstC& c, const InstD& D, const int4 P, const float4 V) {
        // the held force first: a load with no dependence on the layer test below
        const float4 o = g.add ? d.fext[D.lp][s] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 F = make_float4(0.f, 0.f, 0.f, 0.f);
        int fk = 0;
        int lc = -1;
        double x[3] = {0.0, 0.0, 0.0};
        if (maybe_layer(g, 1, P)) {
            for (int k = 0; k < 3; ++k) x[k] = posm(g.lof, g.qf, k == 0 ? P.x : k == 1 ? P.y : P.z, k);
            lc = layer_cell(g, x, &fk);
        }
        if (lc >= 0) {
            const Face& f = g.face[fk];
            const double r = (double)P.w * g.qf, m = d.omg[D.cur][s].w;
            const double sdist = f.side == 0 ? x[f.axis] - f.plane : f.plane - x[f.axis];
            const double w = fmax(0.0, 1.0 - sdist / (1.5 * 2.0 * r));
            const double u = a.ctrl[3 * (size_t)lc + 2];
            double Fv[3] = {0, 0, 0};
            Fv[f.axis] = (f.side == 0 ? 1.0 : -1.0) * u * 3.14159265358979323846 * r * r * w;
            // keep the speed after one step below the coarse cell's largest speed
            const double vmax = __uint_as_float(a.vmax[lc]);
            const double vv[3] = {V.x, V.y, V.z};
            double acc[3], A2 = 0, VA = 0, V2 = 0;
            const double dtm = g.dt / m;        // one FP64 division (slow on this part), not three
            for (int k = 0; k < 3; ++k) {
                acc[k] = dtm * Fv[k];
                A2 += acc[k] * acc[k];
                VA += vv[k] * acc[k];
                V2 += vv[k] * vv[k];
            }
            double lam = 1.0;
            if (A2 > 0 && V2 + 2 * VA + A2 > vmax * vmax) {
                if (V2 >= vmax * vmax) lam = 0.0;
                else lam = fmin(1.0, (-VA + sqrt(VA * VA - A2 * (V2 - vmax * vmax))) / A2);
            }
            F = make_float4((float)(lam * Fv[0]), (float)(lam * Fv[1]), (float)(lam * Fv[2]), 0.f);
        }
        if (g.add) F = make_float4(o.x + F.x, o.y + F.y, o.z + F.z, 0.f);
        d.fext[D.lp][s] = F;
    });
}

__global__ void __launch_bounds__(TILE) k_cp_force_coarse(Dev d, Geo g, Acc a)
{
    for_live(d, [&](int s, const InstC& c, const InstD& D, const int4 P, const float4) {
        const float4 o = g.add ? d.fext[D.lp][s] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 F = make_float4(0.f, 0.f, 0.f, 0.f);
        const int cc = corr_cell_u(g, a.thr, 0, P);
        if (cc >= 0) {
            const double m = d.omg[D.cur][s].w, k = g.kv * m / g.Tc;
            const double* dv = a.dv + 3 * (size_t)cc;
            F = make_float4((float)(k * dv[0]), (float)(k * dv[1]), (float)(k * dv[2]), 0.f);
        }
        if (g.add) F = make_float4(o.x + F.x, o.y + F.y, o.z + F.z, 0.f);
        d.fext[D.lp][s] = F;
    });
}

// SplitMix64 (Steele, Lea and Flood 2014): finaliser of a Weyl sequence, used
// here on a counter built from (seed, cell, interval, attempt, draw)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ unsigned long long draw(const Geo& g, int cell, int attempt, int k)
{
    const unsigned long long ctr =
        (((unsigned long long)cell * 1048576ull + (unsigned long long)g.call) * 16777216ull + (unsigned long long)attempt) *
            8ull + (unsigned long long)k;
    return splitmix64(g.seed ^ splitmix64(ctr));
}

// uniform integer in [0, n) from 64 random bits (n < 2^32)
__device__ __forceinline__ long long below(unsigned long long u, long long n)
{
    return (long long)(((u >> 32) * (unsigned long long)n) >> 32);
}

// uniform in [0, 1) from the top 53 of 64 random bits
__device__ __forceinline__ double unit01(unsigned long long u) { return (double)(u >> 11) * 0x1p-53; }

__device__ __forceinline__ double sphere_mass(double rho, double r)
{
    return __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(rho, 4.0 / 3.0 * 3.14159265358979323846), r), r), r);
}

// false where a sphere of radius ru centred at u (units of q from the box origin) overlaps one
// of the instance's axisymmetric walls (the contact test of the step kernel) or lies on the far
// side of them from the axis: outside the vessel the walls enclose, i.e. where a ray from the
// centre away from the axis (in the (rho, z) half-plane) crosses the non-horizontal segments an
// even number of times (each segment spans its z range closed below, open above).  Called by a
// whole warp: lane k tests segment k, and warp votes combine the segments, so every lane gets
// the result of taking the segments one after another.
__device__ bool clear_of_walls(const InstC& c, const long long* u, long long ru, int lane)
{
    if (c.nwp < 2) return true;
    const double ex = (double)u[0] - c.wax, ey = (double)u[1] - c.way, z = (double)u[2];
    const double rho = sqrt(ex * ex + ey * ey), ru2 = (double)ru * (double)ru;
    bool hit = false, crosses = false;
    const int k = lane;
    if (k + 1 < c.nwp) {
        double a, b;
        wall_seg_offset(c, k, rho, z, a, b);
        hit = a * a + b * b < ru2;
        const double r0 = c.wp[2 * k], z0 = c.wp[2 * k + 1], r1 = c.wp[2 * k + 2], z1 = c.wp[2 * k + 3];
        crosses = z0 != z1 && (z >= z0) != (z >= z1) && r0 + (z - z0) * (r1 - r0) / (z1 - z0) > rho;
    }
    if (__any_sync(0xffffffffu, hit)) return false;
    return (__popc(__ballot_sync(0xffffffffu, crosses)) & 1) != 0;
}

// One block per surface cell of one face: simple sequential inhibition.  The attempts of a cell
// are taken in order, each against the insertions accepted before it; since most attempts fail
// in a dense packing, the block's INS_WARPS warps evaluate the next INS_WARPS attempts at once
// (the same draws: a function of the cell, the call and the attempt's index), against the
// insertions accepted so far, and the results are then taken in attempt order: failures count,
// the first success is accepted and the attempts after it are evaluated again in the next
// round (they have not seen it).  So the accepted set, the attempts used and the failures are
// those of taking the attempts one after another.  Within an attempt the warp's lanes share
// the clearance tests (a wall segment, a neighbour cell of the fine level's last list build, a
// stride of the earlier insertions each) and vote.
constexpr int INS_WARPS = 8;                 // attempts evaluated together

__global__ void __launch_bounds__(32 * INS_WARPS) k_cp_insert(Dev d, Geo g, Acc a, int fk, double rho)
{
    const Face& f = g.face[fk];
    const int lane = (int)threadIdx.x & 31, warp = (int)threadIdx.x >> 5;
    const int local = blockIdx.x;
    if (local >= f.nb * f.nc) return;       // the whole block leaves together
    const int cell = f.off + local;
    const int ib = local % f.nb, ic = local / f.nb;
    const InstC& c = d.ic[0];
    const InstD D = d.id[0];
    __shared__ int s_ok[INS_WARPS];          // 1: the warp's attempt is clear, -1: invalid radius
    __shared__ int4 s_u[INS_WARPS];
    __shared__ double s_r[INS_WARPS];
    long long quota = (long long)a.cross[cell] + a.carry[cell];
    unsigned total = 0;
    const unsigned* hist = a.hist + (size_t)cell * MAXBINS;
    for (int b = 0; b < g.bins; ++b) total += hist[b];
    int nins = 0, fails = 0, attempt = 0;
    const double M = a.fav[4 * cell];
    double vn = 0.0, vf[3] = {0, 0, 0};
    if (M > 0) {
        for (int k = 0; k < 3; ++k) vf[k] = a.fav[4 * cell + 1 + k] / M;
        vn = vf[f.axis];
    }
    // the length quantum is a power of two: dividing by it is multiplying by its reciprocal
    const double iqf = 1.0 / g.qf;
    int4* mine = a.ins + (size_t)cell * g.max_insert;
    double* mym = a.insm + (size_t)cell * g.max_insert;
    // the cell's extent on the face [m]
    const double b0 = __dadd_rn(g.lo[f.b], __dmul_rn((double)ib, f.wb));
    const double c0 = __dadd_rn(g.lo[f.c], __dmul_rn((double)ic, f.wc));
    const unsigned cbase = d.crange[c.code0].x;
    // every thread holds the same loop state; the loop ends for all of them at once
    while (quota > 0 && total > 0 && fails < g.max_attempts && nins < g.max_insert) {
        const int at = attempt + warp;      // this warp's attempt
        // radius: a bin drawn with probability proportional to its count, then uniform in it
        long long pick = below(draw(g, cell, at, 0), total);
        int b = 0;
        while (pick >= (long long)hist[b]) {
            pick -= hist[b];
            ++b;
        }
        const double r = __dmul_rn(__dadd_rn((double)b, unit01(draw(g, cell, at, 1))), g.wbin);
        // centre: uniform over the cell's face shrunk by r, and along the inward normal over
        // [r, r + depth] from the face, depth = max(2 r, |<v_n>| T_c); continuous values (the same
        // operations as a plain double evaluation), then rounded to the fine level's grid
        const double depth = fmax(2.0 * r, fabs(vn) * g.Tc);
        const double sb = __dsub_rn(f.wb, 2.0 * r), sc = __dsub_rn(f.wc, 2.0 * r);
        const long long ru = llrint(__dmul_rn(r, iqf));
        int verdict = -1;
        long long u[3] = {0, 0, 0};
        if (r > 0.0 && sb >= 0.0 && sc >= 0.0 && ru > 0) {
            const double nlo = f.side == 0 ? f.plane + r : f.plane - r - depth;
            double xc[3];
            xc[f.b] = __dadd_rn(__dadd_rn(b0, r), __dmul_rn(unit01(draw(g, cell, at, 2)), sb));
            xc[f.c] = __dadd_rn(__dadd_rn(c0, r), __dmul_rn(unit01(draw(g, cell, at, 3)), sc));
            xc[f.axis] = __dadd_rn(nlo, __dmul_rn(unit01(draw(g, cell, at, 4)), depth));
            for (int k = 0; k < 3; ++k) u[k] = llrint(__dmul_rn(__dsub_rn(xc[k], g.lof[k]), iqf));
            // inside the fine level's walls and clear of them, then no overlap with its particles
            // (cell lists of the last build) or earlier insertions
            bool ok = clear_of_walls(c, u, ru, lane);
            const int ru_i = (int)ru;
            if (ok) {
                bool hit = false;
                if (lane < 27) {
                    // lane = neighbour cell (dx, dy, dz) of the candidate's cell
                    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
                    const int cz = axis_cell(c, 2, (int)u[2]) + dz;
                    int cy = axis_cell(c, 1, (int)u[1]) + dy, cx = axis_cell(c, 0, (int)u[0]) + dx;
                    bool there = cz >= 0 && cz < c.nc[2];
                    if (cy < 0 || cy >= c.nc[1]) {
                        there = there && c.per[1];
                        cy = (cy + c.nc[1]) % c.nc[1];
                    }
                    if (cx < 0 || cx >= c.nc[0]) {
                        there = there && c.per[0];
                        cx = (cx + c.nc[0]) % c.nc[0];
                    }
                    if (there) {
                        const uint2 cr = d.crange[cell_code(d, c, cx, cy, cz)];
                        const int start = c.slot0 + (int)(cr.x - cbase);
                        for (int t = 0; t < (int)cr.y && !hit; ++t) {
                            const int j = d.fin[start + t];   // slot of this cell member
                            if (j - c.slot0 >= D.n) continue;
                            const int4 Q = d.pos[D.cur][j];
                            const long long ex = min_image((int)u[0] - Q.x, c.per[0], c.ext[0], c.half[0]);
                            const long long ey = min_image((int)u[1] - Q.y, c.per[1], c.ext[1], c.half[1]);
                            const long long ez = (long long)u[2] - Q.z;
                            const long long S = (long long)ru_i + Q.w;
                            hit = ex * ex + ey * ey + ez * ez < S * S;
                        }
                    }
                }
                // the fine level's particles inserted since its last list build (not in its cells)
                for (int j = c.slot0 + D.nbin + lane; j < c.slot0 + D.n && !hit; j += 32) {
                    if (__float_as_uint(d.vel[D.cur][j].w) & GONE_BIT) continue;
                    const int4 Q = d.pos[D.cur][j];
                    const long long ex = min_image((int)u[0] - Q.x, c.per[0], c.ext[0], c.half[0]);
                    const long long ey = min_image((int)u[1] - Q.y, c.per[1], c.ext[1], c.half[1]);
                    const long long ez = (long long)u[2] - Q.z;
                    const long long S = (long long)ru_i + Q.w;
                    hit = ex * ex + ey * ey + ez * ez < S * S;
                }
                // earlier insertions: this cell, and the cells of earlier faces
                for (int t = lane; t < nins && !hit; t += 32) {
                    const int4 o = mine[t];
                    const long long ex = u[0] - o.x, ey = u[1] - o.y, ez = u[2] - o.z;
                    const long long S = (long long)ru_i + o.w;
                    hit = ex * ex + ey * ey + ez * ez < S * S;
                }
                for (int k = 0; k < fk; ++k) {
                    const Face& o = g.face[k];
                    for (int oc = o.off + lane; oc < o.off + o.nb * o.nc && !hit; oc += 32) {
                        const int4* other = a.ins + (size_t)oc * g.max_insert;
                        for (int t = 0; t < a.nins[oc] && !hit; ++t) {
                            const long long ex = u[0] - other[t].x, ey = u[1] - other[t].y, ez = u[2] - other[t].z;
                            const long long S = (long long)ru_i + other[t].w;
                            hit = ex * ex + ey * ey + ez * ez < S * S;
                        }
                    }
                }
                ok = !__any_sync(0xffffffffu, hit);
            }
            verdict = ok ? 1 : 0;
        }
        if (lane == 0) {
            s_ok[warp] = verdict;
            s_u[warp] = make_int4((int)u[0], (int)u[1], (int)u[2], (int)ru);
            s_r[warp] = r;
        }
        __syncthreads();
        // the batch in attempt order (every thread alike)
        for (int w = 0; w < INS_WARPS; ++w) {
            if (!(quota > 0 && fails < g.max_attempts && nins < g.max_insert)) break;
            ++attempt;
            if (s_ok[w] != 1) {
                ++fails;
                continue;
            }
            const double m = sphere_mass(rho, s_r[w]);   // of the drawn radius (the grid radius differs by < q / 2)
            if (threadIdx.x == 0) {
                mine[nins] = s_u[w];
                mym[nins] = m;
            }
            ++nins;
            quota -= llrint(m / g.mass_unit);
            break;                                      // later attempts have not seen this insertion
        }
        __syncthreads();                                // the insertion is visible; s_* may be rewritten
    }
    if (threadIdx.x == 0) {
        a.nins[cell] = nins;
        a.carry[cell] = quota;
    }
}

// append the inserted particles (cell order) to the fine level's tail
__global__ void __launch_bounds__(1024) k_cp_append(Dev d, Geo g, Acc a, int* overflow)
{
    // one block: the total first (for the capacity check), then the cells in chunks of 1024,
    // each thread appending its cell's particles at the cell's offset from a block scan (one
    // thread walking the cells with a barrier per cell took 20 µs for 470 cells)
    __shared__ int wsum[32];
    __shared__ int stot;
    const InstC& c = d.ic[0];
    InstD& D = d.id[0];
    const int tid = (int)threadIdx.x, lane = tid & 31, w = tid >> 5;
    int loc = 0;
    for (int i = tid; i < g.S; i += 1024) loc += a.nins[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
    if (lane == 0) wsum[w] = loc;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int v = 0; v < 32; ++v) t += wsum[v];
        stot = t;
        a.npairs[0] = 0;
        a.npairs[1] = 0;
        a.npairs[2] = 0;
    }
    __syncthreads();
    const int tot = stot, n0 = D.n, nid0 = D.nid;
    if (n0 + tot > c.cap || nid0 + tot > c.cap) {
        if (tid == 0) {
            *overflow = 1;
            atomicOr(&d.g->status, ST_INSERT);
        }
        return;
    }
    int carry = 0;
    for (int base = 0; base < g.S; base += 1024) {
        const int i = base + tid;
        const int k = i < g.S ? a.nins[i] : 0;
        int inc = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        __syncthreads();                    // wsum of the previous chunk is read
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        int off = carry + inc - k, ctot = 0;
        for (int v = 0; v < 32; ++v) {
            if (v < w) off += wsum[v];
            ctot += wsum[v];
        }
        if (k > 0) {
            const double M = a.fav[4 * i];
            float v[3] = {0.f, 0.f, 0.f};
            if (M > 0)
                for (int q = 0; q < 3; ++q) v[q] = (float)(a.fav[4 * i + 1 + q] / M);
            for (int t = 0; t < k; ++t) {
                const int s = c.slot0 + n0 + off + t;
                const int id = nid0 + off + t;
                const int4 p = a.ins[(size_t)i * g.max_insert + t];
                d.pos[D.cur][s] = p;
                d.vel[D.cur][s] = make_float4(v[0], v[1], v[2], __uint_as_float((unsigned)id));
                d.omg[D.cur][s] = make_float4(0.f, 0.f, 0.f, (float)a.insm[(size_t)i * g.max_insert + t]);
                d.cnt[D.lp][s] = 0;
                d.hmask[D.lp][s] = 0u;
                d.whist[D.lp][s] = make_float4(0.f, 0.f, 0.f, 0.f);
                d.wseg[D.lp][s] = make_float4(0.f, 0.f, 0.f, 0.f);
                d.wseg[D.lp][d.ncap + s] = make_float4(0.f, 0.f, 0.f, 0.f);
                d.fext[D.lp][s] = make_float4(0.f, 0.f, 0.f, 0.f);
                d.slot_of_id[c.slot0 + id] = s;
            }
        }
        carry += ctot;
    }
    __syncthreads();                        // every thread has read D.n and D.nid
    if (tid == 0) {
        D.n = n0 + tot;
        D.nid = nid0 + tot;
        d.goff[0] = 0;                      // offsets of the user arrays (one instance)
        d.goff[1] = D.nid;
        a.npairs[2] = tot;                  // their rows are built next (k_cp_rows), no list build
    }
}

// Rows of the particles inserted at this call, built without a list build (one thread each).
// The exact test of the list build (|x_i - x_j| < r_i + r_j + skin, integer arithmetic) against
// every live particle that can be that close: those of the last build's cell lists within two
// cells (every particle has moved less than half the skin since, so a partner's cell of then is
// at most two cells away), and those inserted since, tested one by one.  The row is ordered as
// the list build orders rows (by d^2 - (r_i + r_j)^2, then ID); each partner that already had
// a row gets the new particle appended to it (k_cp_rows_append).  Lists stay valid: a pair
// left out was further apart than the skin now, and closing that gap needs the displacement
// bound that triggers the next build.  A row too long, or too many pairs, falls back to a list
// build.
constexpr int ROWS_T = 64;

__global__ void __launch_bounds__(ROWS_T) k_cp_rows(Dev d, Acc a)
{
    __shared__ float key[MAXL][ROWS_T];
    __shared__ int slot[MAXL][ROWS_T];
    const int tx = threadIdx.x;
    const InstC& c = d.ic[0];
    const InstD D = d.id[0];
    const int tot = a.npairs[2];
    const int t = blockIdx.x * ROWS_T + tx;
    if (t >= tot) return;
    const int n_old = D.n - tot;
    const int si = c.slot0 + n_old + t;
    const int cur = D.cur, lp = D.lp, Lmax = d.Lmax, ncap = d.ncap;
    const int4 p = d.pos[cur][si];
    const int per0 = c.per[0], per1 = c.per[1], ext0 = c.ext[0], ext1 = c.ext[1], hf0 = c.half[0], hf1 = c.half[1];
    const int skin = c.skin;
    int nc = 0;
    bool overflow = false;
    auto test = [&](int j) {
        if (j == si) return;
        if (__float_as_uint(d.vel[cur][j].w) & GONE_BIT) return;
        const int4 q = d.pos[cur][j];
        const int ddx = min_image(p.x - q.x, per0, ext0, hf0);
        const int ddy = min_image(p.y - q.y, per1, ext1, hf1);
        const long long ddz = (long long)p.z - q.z;
        const int cut = p.w + q.w + skin;
        if (abs(ddx) >= cut || abs(ddy) >= cut || ddz >= cut || ddz <= -cut) return;
        const long long d2 = (long long)ddx * ddx + (long long)ddy * ddy + ddz * ddz;
        if (d2 >= (long long)cut * cut) return;
        if (nc == Lmax) {
            overflow = true;
            return;
        }
        const long long S = (long long)p.w + q.w;
        key[nc][tx] = (float)(d2 - S * S);
        slot[nc][tx] = j;
        ++nc;
    };
    // the last build's cells within two cells per axis (each cell once on a short periodic axis)
    int cell0[3], ncell[3];
    const int cc[3] = {axis_cell(c, 0, p.x), axis_cell(c, 1, p.y), axis_cell(c, 2, p.z)};
    for (int ax = 0; ax < 3; ++ax) {
        if (c.per[ax] && c.nc[ax] <= 5) {
            cell0[ax] = 0;
            ncell[ax] = c.nc[ax];
        } else if (c.per[ax]) {
            cell0[ax] = cc[ax] - 2;
            ncell[ax] = 5;
        } else {
            cell0[ax] = max(cc[ax] - 2, 0);
            ncell[ax] = min(cc[ax] + 2, c.nc[ax] - 1) - cell0[ax] + 1;
        }
    }
    const unsigned cbase = d.crange[c.code0].x;
    for (int iz = 0; iz < ncell[2]; ++iz)
        for (int iy = 0; iy < ncell[1]; ++iy)
            for (int ix = 0; ix < ncell[0]; ++ix) {
                const int cx = (cell0[0] + ix + c.nc[0]) % c.nc[0], cy = (cell0[1] + iy + c.nc[1]) % c.nc[1];
                const int cz = cell0[2] + iz;
                const uint2 cr = d.crange[cell_code(d, c, cx, cy, cz)];
                const int start = c.slot0 + (int)(cr.x - cbase);
                for (int m = 0; m < (int)cr.y; ++m) test(d.fin[start + m]);
            }
    // the particles inserted since the last build (this call's included)
    for (int j = c.slot0 + D.nbin; j < c.slot0 + D.n; ++j) test(j);
    // order: (d^2 - (r_i + r_j)^2, ID), as the list build
    for (int i = 1; i < nc; ++i) {
        const float kk = key[i][tx];
        const int m = slot[i][tx];
        const unsigned idm = __float_as_uint(d.vel[cur][m].w) & ID_MASK;
        int j = i - 1;
        while (j >= 0 && (key[j][tx] > kk ||
                          (key[j][tx] == kk && (__float_as_uint(d.vel[cur][slot[j][tx]].w) & ID_MASK) > idm))) {
            key[j + 1][tx] = key[j][tx];
            slot[j + 1][tx] = slot[j][tx];
            --j;
        }
        key[j + 1][tx] = kk;
        slot[j + 1][tx] = m;
    }
    int* row = d.nbr[lp] + si;
    for (int e = 0; e < nc; ++e) {
        const int j = slot[e][tx];
        row[(size_t)e * ncap] = j;
        if (j < c.slot0 + n_old) {         // a partner with a row of its own: append to it
            const int k = atomicAdd(&a.npairs[0], 1);
            if (k < PAIRS_MAX) a.pairs[k] = ((unsigned long long)(unsigned)j << 32) | (unsigned)si;
            else overflow = true;
        }
    }
    d.cnt[lp][si] = nc;
    d.hmask[lp][si] = 0u;
    if (overflow) atomicExch(&a.npairs[1], 1);
}

// Append the inserted particles to their partners' rows, in (partner, new slot) order (the
// pairs sorted first, so the rows do not depend on the order the pairs were found in); fall
// back to a list build if a row would overflow or the pairs did not fit.  Then the tiles
// fused steps walk grow to cover the new slots.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_cp_rows_append(Dev d, Acc a)
{
    __shared__ unsigned long long key[PAIRS_MAX];
    __shared__ int fallback;
    InstD& D = d.id[0];
    const InstC& c = d.ic[0];
    const int P = a.npairs[0];
    if (threadIdx.x == 0) fallback = a.npairs[1] != 0 || P > PAIRS_MAX;
    __syncthreads();
    if (!fallback && P > 0) {
        int n2 = 1;
        while (n2 < P) n2 <<= 1;
        for (int k = threadIdx.x; k < n2; k += blockDim.x) key[k] = k < P ? a.pairs[k] : ~0ull;
        __syncthreads();
        // bitonic sort of n2 keys
        for (int size = 2; size <= n2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = threadIdx.x; k < n2; k += blockDim.x) {
                    const int l = k ^ stride;
                    if (l > k) {
                        const bool up = (k & size) == 0;
                        const unsigned long long x = key[k], y = key[l];
                        if ((x > y) == up) {
                            key[k] = y;
                            key[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        const int lp = D.lp, ncap = d.ncap, Lmax = d.Lmax;
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const unsigned j = (unsigned)(key[k] >> 32);
            if (k > 0 && (unsigned)(key[k - 1] >> 32) == j) continue;   // not the first of its run
            int r = 1;
            while (k + r < P && (unsigned)(key[k + r] >> 32) == j) ++r;
            const int c0 = d.cnt[lp][j];
            if (c0 + r > Lmax) {
                fallback = 1;
                continue;
            }
            for (int t = 0; t < r; ++t) d.nbr[lp][(size_t)(c0 + t) * ncap + j] = (int)(unsigned)key[k + t];
            d.cnt[lp][j] = c0 + r;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (fallback && D.flag == 0) {
            D.flag = 1;                      // the rows are rebuilt from the positions
            atomicOr(&d.g->any, 1u);
        }
        // the tiles holding live slots (one instance): fused steps walk them
        const int t0 = c.slot0 / TILE, nl = 2 * ((D.n + 2 * TILE - 1) / (2 * TILE));
        if (nl > d.g->nlive) {
            for (int i = d.g->nlive; i < nl; ++i) d.live_tiles[i] = t0 + i;
            d.g->nlive = nl;
        }
    }
}

}  // namespace

struct dem_coupler {
    dem_ctx* c = nullptr;
    dem_ctx* f = nullptr;
    dem_coupling spec{};
    Geo g{};
    Acc a{};
    int* overflow = nullptr;
    int calls = 0;
    double rho_f = 0.0;
    cudaEvent_t ready = nullptr;   // orders the fine level's stream after the coarse level's
    cudaEvent_t done = nullptr;    // orders the coarse level's stream after the coupling kernels
};

namespace {

size_t coupler_layout(dem_coupler* cp, char* base)
{
    struct L {
        size_t t = 0;
        size_t take(size_t b)
        {
            size_t o = t;
            t += (b + 255) & ~size_t(255);
            return o;
        }
    } L;
    const size_t S = cp->g.S, C = cp->g.C, MI = cp->g.max_insert, ncap = (size_t)cp->c->ncap;
    size_t o_cross = L.take(S * 8), o_hist = L.take(S * MAXBINS * 4), o_fav = L.take(S * 32), o_carry = L.take(S * 8),
           o_nins = L.take(S * 4), o_ins = L.take(S * MI * 16), o_insm = L.take(S * MI * 8), o_lay = L.take(2 * S * 160),
           o_vmax = L.take(2 * S * 4), o_ctrl = L.take(S * 24), o_out = L.take(2 * S * 88), o_cor = L.take(2 * C * 40),
           o_dv = L.take(C * 24), o_prev = L.take(ncap * 16), o_pok = L.take(ncap * 4), o_rem = L.take(16),
           o_ovf = L.take(16), o_thr = L.take(2 * 3 * (MAXCR + 1) * 8), o_pairs = L.take(PAIRS_MAX * 8),
           o_np = L.take(16);
    if (base) {
        Acc& a = cp->a;
        a.cross = (unsigned long long*)(base + o_cross);
        a.hist = (unsigned*)(base + o_hist);
        a.fav = (double*)(base + o_fav);
        a.carry = (long long*)(base + o_carry);
        a.nins = (int*)(base + o_nins);
        a.ins = (int4*)(base + o_ins);
        a.insm = (double*)(base + o_insm);
        a.lay = (double*)(base + o_lay);
        a.vmax = (unsigned*)(base + o_vmax);
        a.ctrl = (double*)(base + o_ctrl);
        a.out = (double*)(base + o_out);
        a.cor = (double*)(base + o_cor);
        a.dv = (double*)(base + o_dv);
        a.prev = (int4*)(base + o_prev);
        a.prev_ok = (int*)(base + o_pok);
        a.thr = (long long*)(base + o_thr);
        a.removed = (int*)(base + o_rem);
        a.pairs = (unsigned long long*)(base + o_pairs);
        a.npairs = (int*)(base + o_np);
        cp->overflow = (int*)(base + o_ovf);
    }
    return L.t;
}

dem_status plan_geo(dem_ctx* coarse, dem_ctx* fine, const dem_coupling* sp, Geo& g, std::string& err)
{
    if (!coarse || !fine || !sp) { err = "null argument"; return DEM_ERR_ARG; }
    if (coarse->B != 1 || fine->B != 1) { err = "coupling needs single-instance contexts"; return DEM_ERR_ARG; }
    if (sp->interval < 1 || sp->bins < 1 || sp->bins > MAXBINS || !(sp->alpha > 0) || !(sp->surface_cell > 0) ||
        !(sp->layer > 0) || !(sp->corr_cell > 0) || !(sp->mass_unit > 0) || sp->max_insert < 1 || sp->max_attempts < 1 ||
        sp->feed_faces <= 0 || sp->feed_faces >= 64) {
        err = "coupling spec: interval, bins (1..32), alpha, cell sizes, layer, mass_unit, max_insert, max_attempts and "
              "feed_faces must be positive";
        return DEM_ERR_ARG;
    }
    memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = sp->lo[a];
        g.hi[a] = sp->hi[a];
        if (!(g.hi[a] > g.lo[a])) { err = "empty fine region"; return DEM_ERR_ARG; }
        g.loc[a] = coarse->hl[0].lo[a];
        g.lof[a] = fine->hl[0].lo[a];
    }
    g.qc = coarse->hl[0].q;
    g.qf = fine->hl[0].q;
    int off = 0;
    for (int bit = 0; bit < 6; ++bit) {
        if (!((sp->feed_faces >> bit) & 1)) continue;
        Face& f = g.face[g.nface++];
        f.axis = bit / 2;
        f.side = bit % 2;
        f.b = (f.axis + 1) % 3;
        f.c = (f.axis + 2) % 3;
        if (f.b > f.c) std::swap(f.b, f.c);
        f.plane = f.side == 0 ? g.lo[f.axis] : g.hi[f.axis];
        f.nb = std::max(1, (int)std::floor((g.hi[f.b] - g.lo[f.b]) / sp->surface_cell));
        f.nc = std::max(1, (int)std::floor((g.hi[f.c] - g.lo[f.c]) / sp->surface_cell));
        f.wb = (g.hi[f.b] - g.lo[f.b]) / f.nb;
        f.wc = (g.hi[f.c] - g.lo[f.c]) / f.nc;
        f.iwb = 1.0 / f.wb;
        f.iwc = 1.0 / f.wc;
        f.off = off;
        off += f.nb * f.nc;
    }
    g.S = off;
    g.C = 1;
    for (int a = 0; a < 3; ++a) {
        g.ncr[a] = std::max(1, (int)std::floor((g.hi[a] - g.lo[a]) / sp->corr_cell));
        if (g.ncr[a] > MAXCR) {
            err = "more than 256 correction cells along an axis";
            return DEM_ERR_ARG;
        }
        g.wcr[a] = (g.hi[a] - g.lo[a]) / g.ncr[a];
        g.iwcr[a] = 1.0 / g.wcr[a];
        g.C *= g.ncr[a];
    }
    g.layer = sp->layer;
    g.alpha = sp->alpha;
    g.dt = fine->ic[0].dt;
    g.Tc = sp->interval * (double)fine->ic[0].dt;
    g.kp = sp->kp;
    g.ki = sp->ki;
    g.kv = sp->kv;
    g.mass_unit = sp->mass_unit;
    g.bins = sp->bins;
    g.mode = sp->mode;
    g.max_attempts = sp->max_attempts;
    g.max_insert = sp->max_insert;
    g.drain = sp->drain_faces;
    g.seed = sp->seed;
    g.add = sp->add_forces ? 1 : 0;
    g.vel_below = (sp->velocity_below_on && !std::isnan(sp->velocity_below)) ? sp->velocity_below : -INFINITY;
    // a coarse particle outside the region grown by one largest diameter (Favre samples reach
    // a diameter beyond the faces) touches no cell: bounds in coarse units, rounded outwards
    for (int L = 0; L < 2; ++L)
        for (int a = 0; a < 3; ++a) g.cells_per_unit[L][a] = (float)((L == 0 ? g.qc : g.qf) / g.wcr[a]);
    const double grow = 2.0 * coarse->rmax[0];
    for (int a = 0; a < 3; ++a) {
        g.ulo[a] = (long long)std::floor((g.lo[a] - grow - g.loc[a]) / g.qc) - 2;
        g.uhi[a] = (long long)std::ceil((g.hi[a] + grow - g.loc[a]) / g.qc) + 2;
    }
    // layer boxes: the region's extent across the face and [plane, plane + layer) inwards, in
    // each level's units, widened by two units on every side (a box too large costs time only)
    for (int L = 0; L < 2; ++L) {
        const double* lo0 = L == 0 ? g.loc : g.lof;
        const double q = L == 0 ? g.qc : g.qf;
        for (int k = 0; k < g.nface; ++k) {
            const Face& f = g.face[k];
            for (int a = 0; a < 3; ++a) {
                double lo = g.lo[a], hi = g.hi[a];
                if (a == f.axis) {
                    lo = f.side == 0 ? f.plane : f.plane - g.layer;
                    hi = f.side == 0 ? f.plane + g.layer : f.plane;
                }
                g.lay_lo[L][k][a] = (long long)std::floor((lo - lo0[a]) / q) - 2;
                g.lay_hi[L][k][a] = (long long)std::ceil((hi - lo0[a]) / q) + 2;
            }
        }
    }
    return DEM_OK;
}

// The correction grid as integer thresholds per level and axis (layout of Acc::thr).  A level's
// position in metres is lo + u q rounded once (as the kernels and the read-out form it); a
// position is in the region when lo_r <= x < hi_r and in cell floor_div(x - lo_r, w, 1/w) (clamped).
// Both decisions are monotone in u, so each is a threshold on u: the smallest u where it holds,
// found from the estimate by evaluating the same double expressions.
double floor_div_host(double a, double w, double iw)
{
    const double t = a * iw, f = std::floor(t);
    if (t - f < 1e-6 || f + 1.0 - t < 1e-6) return std::floor(a / w);
    return f;
}

template <typename Pred>
bool first_true(Pred pred, double estimate, long long& out)
{
    long long u = (long long)std::floor(estimate) - 4;
    for (int i = 0; i < 64 && pred(u); ++i) u -= 64;
    if (pred(u)) return false;
    for (int i = 0; i < 4096; ++i, ++u)
        if (pred(u)) {
            out = u;
            return true;
        }
    return false;
}

bool cell_thresholds(const Geo& g, std::vector<long long>& thr)
{
    thr.assign((size_t)2 * 3 * (MAXCR + 1), 0);
    for (int L = 0; L < 2; ++L) {
        const double* lo0 = L == 0 ? g.loc : g.lof;
        const double q = L == 0 ? g.qc : g.qf;
        for (int a = 0; a < 3; ++a) {
            long long* T = thr.data() + ((size_t)L * 3 + a) * (MAXCR + 1);
            auto x = [&](long long u) { return std::fma((double)u, q, lo0[a]); };
            const int n = g.ncr[a];
            bool ok = first_true([&](long long u) { return x(u) >= g.lo[a]; }, (g.lo[a] - lo0[a]) / q, T[0]) &&
                      first_true([&](long long u) { return x(u) >= g.hi[a]; }, (g.hi[a] - lo0[a]) / q, T[n]);
            for (int k = 1; k < n && ok; ++k)
                ok = first_true([&](long long u) { return floor_div_host(x(u) - g.lo[a], g.wcr[a], g.iwcr[a]) >= k; },
                                (g.lo[a] + k * g.wcr[a] - lo0[a]) / q, T[k]);
            if (!ok) return false;
        }
    }
    return true;
}

}  // namespace

extern "C" {

dem_status dem_coupler_workspace(dem_ctx* coarse, dem_ctx* fine, const dem_coupling* spec, int64_t* bytes)
{
    if (!bytes) return DEM_ERR_ARG;
    dem_coupler tmp;
    std::string err;
    dem_status st = plan_geo(coarse, fine, spec, tmp.g, err);
    if (st) {
        set_thread_error(err);
        return st;
    }
    tmp.c = coarse;
    tmp.f = fine;
    *bytes = (int64_t)coupler_layout(&tmp, nullptr);
    return DEM_OK;
}

dem_status dem_coupler_create(dem_ctx* coarse, dem_ctx* fine, const dem_coupling* spec, void* ws, int64_t bytes,
                              dem_coupler** out)
{
    if (!out) return DEM_ERR_ARG;
    *out = nullptr;
    dem_coupler* cp = new dem_coupler();
    std::string err;
    dem_status st = plan_geo(coarse, fine, spec, cp->g, err);
    if (st) {
        set_thread_error(err);
        delete cp;
        return st;
    }
    cp->c = coarse;
    cp->f = fine;
    cp->spec = *spec;
    const size_t need = coupler_layout(cp, nullptr);
    if (!ws || (size_t)bytes < need || ((uintptr_t)ws & 255)) {
        set_thread_error("coupler workspace missing, too small or not 256-byte aligned");
        delete cp;
        return DEM_ERR_ARG;
    }
    coupler_layout(cp, (char*)ws);
    if (cudaEventCreateWithFlags(&cp->ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cp->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (cp->ready) cudaEventDestroy(cp->ready);
        set_thread_error("could not create the coupler's CUDA events");
        delete cp;
        return DEM_ERR_CUDA;
    }
    cp->rho_f = fine->hl[0].rho;
    // radius bins: equal widths over [0, r_max) of the fine level
    cp->g.wbin = fine->rmax[0] / cp->g.bins;
    cudaStream_t s = fine->stream;
    dem_ctx* ctx = fine;
    CU(cudaMemsetAsync(ws, 0, need, s));
    {
        std::vector<long long> thr;
        if (!cell_thresholds(cp->g, thr)) {
            set_thread_error("correction grid thresholds not found");
            cudaEventDestroy(cp->ready);
            cudaEventDestroy(cp->done);
            delete cp;
            return DEM_ERR_ARG;
        }
        CU(cudaMemcpyAsync(cp->a.thr, thr.data(), thr.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));
    }
    // enable the external force on both levels
    for (dem_ctx* x : {coarse, fine}) {
        int one = 1;
        ctx = x;
        CU(cudaMemcpyAsync((char*)x->dev.id + offsetof(InstD, fext), &one, sizeof(int), cudaMemcpyHostToDevice,
                           x->stream));
        CU(cudaStreamSynchronize(x->stream));
    }
    ctx = fine;
    CU(cudaStreamSynchronize(s));
    // first sample of the coarse positions
    cp->g.call = 0;
    cudaStreamSynchronize(coarse->stream);
    k_cp_coarse<<<coarse->grid_rb, TILE, 0, s>>>(coarse->dev, cp->g, cp->a, 1);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
    *out = cp;
    return DEM_OK;
}

dem_status dem_couple(dem_coupler* cp)
{
    NvtxRange nvtx_range("dem_couple");
    if (!cp) return DEM_ERR_ARG;
    dem_ctx* ctx = cp->f;
    dem_ctx* coarse = cp->c;
    if (coarse->status) return check_status(coarse);
    if (ctx->status) return check_status(ctx);
    // both levels must be current and their lists valid; work on the fine level's stream,
    // after everything queued on the coarse level's (an event, no host wait)
    dem_status st = launch_rebuild(coarse, coarse->stream);
    if (st) return st;
    if ((st = launch_rebuild(ctx, ctx->stream))) return st;
    cudaStream_t s = ctx->stream;
    if (coarse->stream != s) {
        CU(cudaEventRecord(cp->ready, coarse->stream));
        CU(cudaStreamWaitEvent(s, cp->ready, 0));
    }
    Geo g = cp->g;
    g.call = ++cp->calls;
    g.fresh_c = coarse->fresh ? 1 : 0;
    g.fresh_f = ctx->fresh ? 1 : 0;
    k_cp_clear<<<(clear_threads(g.S, g.C) + 255) / 256, 256, 0, s>>>(g, cp->a);
    k_cp_coarse<<<coarse->grid_rb, TILE, 0, s>>>(coarse->dev, g, cp->a, 0);
    k_cp_fine<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, g, cp->a);
    k_cp_cells<<<(cells_threads(g.S, g.C) + 255) / 256, 256, 0, s>>>(g, cp->a);
    k_cp_force_fine<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, g, cp->a);
    k_cp_force_coarse<<<coarse->grid_rb, TILE, 0, s>>>(coarse->dev, g, cp->a);
    for (int fk = 0; fk < g.nface; ++fk)
        k_cp_insert<<<g.face[fk].nb * g.face[fk].nc, 32 * INS_WARPS, 0, s>>>(ctx->dev, g, cp->a, fk, cp->rho_f);
    CU(cudaMemsetAsync(cp->overflow, 0, sizeof(int), s));
    k_cp_append<<<1, 1024, 0, s>>>(ctx->dev, g, cp->a, cp->overflow);
    k_cp_rows<<<(g.S * g.max_insert + ROWS_T - 1) / ROWS_T, ROWS_T, 0, s>>>(ctx->dev, cp->a);
    k_cp_rows_append<<<1, 1024, 0, s>>>(ctx->dev, cp->a);
    CU(cudaGetLastError());
    // the coarse level's later work (its next steps) waits for the coupling kernels, which read
    // its state and write its held forces and corrected velocities (an event, no host wait)
    if (coarse->stream != s) {
        CU(cudaEventRecord(cp->done, s));
        CU(cudaStreamWaitEvent(coarse->stream, cp->done, 0));
    }
    // no host wait: the device updated the count and the offsets (k_cp_append) and reports an
    // overflow in the status word; the host copy of the count is refreshed when next needed
    ctx->count_stale = true;
    return DEM_OK;
}

dem_status dem_coupler_read(dem_coupler* cp, int32_t field, double* dst, int64_t n)
{
    if (!cp || !dst) return DEM_ERR_ARG;
    dem_ctx* ctx = cp->f;
    const Geo& g = cp->g;
    const size_t S = g.S, C = g.C;
    CU(cudaStreamSynchronize(ctx->stream));
    auto get = [&](const void* src, size_t bytes, void* h) -> dem_status {
        CU(cudaMemcpy(h, src, bytes, cudaMemcpyDeviceToHost));
        return DEM_OK;
    };
    std::vector<double> tmp;
    std::vector<long long> li(S);
    std::vector<unsigned long long> lu(S);
    std::vector<int> ii(S);
    std::vector<unsigned> hu;
    size_t need = 0;
    switch (field) {
    case DEM_CPL_SIZES: need = 4; break;
    case DEM_CPL_SURFACE_MASS: case DEM_CPL_SURFACE_CARRY: case DEM_CPL_SURFACE_INSERTED: need = S; break;
    case DEM_CPL_SURFACE_VEL: need = 3 * S; break;
    case DEM_CPL_SURFACE_HIST: need = S * g.bins; break;
    case DEM_CPL_LAYER_STRESS: need = 12 * S; break;
    case DEM_CPL_LAYER_PHI: case DEM_CPL_LAYER_VMAX: need = 2 * S; break;
    case DEM_CPL_LAYER_VEL: need = 6 * S; break;
    case DEM_CPL_LAYER_CTRL: need = 3 * S; break;
    case DEM_CPL_CORR_PHI: need = 2 * C; break;
    case DEM_CPL_CORR_VEL: need = 6 * C; break;
    default: return fail(ctx, DEM_ERR_ARG, "unknown coupler field");
    }
    if ((size_t)n != need) return fail(ctx, DEM_ERR_ARG, "wrong element count for the coupler field");
    dem_status st = DEM_OK;
    switch (field) {
    case DEM_CPL_SIZES: dst[0] = (double)S; dst[1] = (double)S; dst[2] = (double)C; dst[3] = cp->calls; break;
    case DEM_CPL_SURFACE_MASS:
        st = get(cp->a.cross, S * 8, lu.data());
        for (size_t i = 0; i < S; ++i) dst[i] = (double)lu[i] * g.mass_unit;
        break;
    case DEM_CPL_SURFACE_CARRY:
        st = get(cp->a.carry, S * 8, li.data());
        for (size_t i = 0; i < S; ++i) dst[i] = (double)li[i] * g.mass_unit;
        break;
    case DEM_CPL_SURFACE_INSERTED:
        st = get(cp->a.nins, S * 4, ii.data());
        for (size_t i = 0; i < S; ++i) dst[i] = ii[i];
        break;
    case DEM_CPL_SURFACE_VEL:
        tmp.resize(4 * S);
        st = get(cp->a.fav, S * 32, tmp.data());
        for (size_t i = 0; i < S; ++i)
            for (int k = 0; k < 3; ++k) dst[3 * i + k] = tmp[4 * i] > 0 ? tmp[4 * i + 1 + k] / tmp[4 * i] : 0.0;
        break;
    case DEM_CPL_SURFACE_HIST:
        hu.resize(S * MAXBINS);
        st = get(cp->a.hist, S * MAXBINS * 4, hu.data());
        for (size_t i = 0; i < S; ++i)
            for (int b = 0; b < g.bins; ++b) dst[i * g.bins + b] = hu[i * MAXBINS + b];
        break;
    default:
        if (field >= DEM_CPL_LAYER_STRESS && field <= DEM_CPL_LAYER_VMAX) {
            tmp.resize(2 * S * 11);
            st = get(cp->a.out, 2 * S * 88, tmp.data());
            for (size_t L = 0; L < 2; ++L)
                for (size_t i = 0; i < S; ++i) {
                    const double* o = &tmp[(L * S + i) * 11];
                    if (field == DEM_CPL_LAYER_STRESS) for (int k = 0; k < 6; ++k) dst[(i * 2 + L) * 6 + k] = o[k];
                    if (field == DEM_CPL_LAYER_PHI) dst[i * 2 + L] = o[6];
                    if (field == DEM_CPL_LAYER_VEL) for (int k = 0; k < 3; ++k) dst[(i * 2 + L) * 3 + k] = o[7 + k];
                    if (field == DEM_CPL_LAYER_VMAX) dst[i * 2 + L] = o[10];
                }
        } else if (field == DEM_CPL_LAYER_CTRL) {
            st = get(cp->a.ctrl, S * 24, dst);
        } else {
            tmp.resize(2 * C * 5);
            st = get(cp->a.cor, 2 * C * 40, tmp.data());
            for (size_t L = 0; L < 2; ++L)
                for (size_t i = 0; i < C; ++i) {
                    const double* o = &tmp[(L * C + i) * 5];
                    const double V = g.wcr[0] * g.wcr[1] * g.wcr[2];
                    if (field == DEM_CPL_CORR_PHI) dst[i * 2 + L] = o[4] / V;
                    if (field == DEM_CPL_CORR_VEL)
                        for (int k = 0; k < 3; ++k) dst[(i * 2 + L) * 3 + k] = o[0] > 0 ? o[1 + k] / o[0] : 0.0;
                }
        }
    }
    return st;
}

dem_status dem_coupler_destroy(dem_coupler* cp)
{
    if (!cp) return DEM_ERR_ARG;
    if (cp->ready) cudaEventDestroy(cp->ready);
    if (cp->done) cudaEventDestroy(cp->done);
    delete cp;   // touches neither context (they may already be gone)
    return DEM_OK;
}

dem_status dem_clear_external_force(dem_ctx* ctx)
{
    if (!ctx) return DEM_ERR_ARG;
    CU(cudaMemsetAsync(ctx->dev.fext[0], 0, sizeof(float4) * (size_t)ctx->ncap, ctx->stream));
    CU(cudaMemsetAsync(ctx->dev.fext[1], 0, sizeof(float4) * (size_t)ctx->ncap, ctx->stream));
    return DEM_OK;
}

dem_status dem_counts(dem_ctx* ctx, int64_t* live, int64_t* ids)
{
    if (!ctx || !live || !ids) return DEM_ERR_ARG;
    if (dem_status st = refresh_count(ctx)) return st;
    std::vector<InstD> D(ctx->B);
    CU(cudaMemcpyAsync(D.data(), ctx->dev.id, sizeof(InstD) * ctx->B, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->B; ++k) {
        live[k] = D[k].n;
        ids[k] = D[k].nid;
    }
    return DEM_OK;
}

}  // extern "C"
