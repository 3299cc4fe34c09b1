// Contact law of one particle pair (Eqs. 3-6) and its reverse-mode derivative,
// as __host__ __device__ templates: float with fast intrinsics on the GPU, any
// floating type on the host (the host instantiation in double is what the CPU
// tests differentiate numerically to check the hand-written derivative).
#pragma once

#ifndef __CUDACC__
#include <cmath>
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace cgdem {

#define HD __host__ __device__ __forceinline__

template <typename T>
struct Vec3 {
    T x, y, z;
};
template <typename T> HD Vec3<T> mk3(T x, T y, T z) { return {x, y, z}; }
template <typename T> HD Vec3<T> operator+(Vec3<T> a, Vec3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T> HD Vec3<T> operator-(Vec3<T> a, Vec3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T> HD Vec3<T> operator-(Vec3<T> a) { return {-a.x, -a.y, -a.z}; }
template <typename T> HD Vec3<T> operator*(T s, Vec3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T> HD T dot(Vec3<T> a, Vec3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> HD Vec3<T> cross(Vec3<T> a, Vec3<T> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// 1/sqrt, division and individually rounded product / sum
HD float rsq(float x)
{
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / std::sqrt(x);
#endif
}
HD double rsq(double x)
{
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / std::sqrt(x);
#endif
}
HD float fdiv(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
HD double fdiv(double a, double b) { return a / b; }
HD float rn_mul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
HD float rn_add(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
HD double rn_mul(double a, double b) { return a * b; }
HD double rn_add(double a, double b) { return a + b; }

// per-system coefficients of Eq. 6 (constant factors) and friction
template <typename T>
struct Coef {
    T c_kn;       // 4/3 E_eff
    T c_kt;       // 8 G_eff
    T nbeta;      // -beta(e) >= 0
    T gt_ratio;   // gamma_t / gamma_n = sqrt(2 c_kt / (3 c_kn))
    T mu;         // particle-particle friction
    T mu_w;       // particle-wall friction
    int clamp_fn; // drop tensile normal forces
};

// One contact seen from body a (n from b to a, delta > 0 in metres): Eq. 6
// coefficients, Eq. 3 normal force, Eq. 4 tangential force with the stored
// overlap xi kept in the tangent plane at its length and advanced by the
// tangential contact-point motion, Eq. 5 truncation.  Returns the force on a;
// ft receives the tangential part.  Every operation is either symmetric in
// (a, b) or odd under exchanging them (r_a w_a + r_b w_b is rounded term by
// term), so with sign-symmetric rounding body b obtains exactly the negated
// force and overlap.
template <typename T, bool WALL>
HD Vec3<T> contact_fwd(const Coef<T>& c, T delta, Vec3<T> n, T ra, T rb, T ma, T mb, Vec3<T> va, Vec3<T> vb,
                       Vec3<T> wa, Vec3<T> wb, Vec3<T>& xi, T dt_hist, Vec3<T>& ft, bool& slip)
{
    T R, meff;
    if (WALL) {
        R = ra;
        meff = ma;
    } else {
        R = fdiv(ra * rb, ra + rb);
        meff = fdiv(ma * mb, ma + mb);
    }
    const T Rd = R * delta;
    const T sRd = Rd * rsq(Rd);                 // sqrt(R_eff delta), Rd > 0
    const T kn = c.c_kn * sRd;
    const T kt = c.c_kt * sRd;
    const T x5 = T(5) * meff * kn;
    const T gn = c.nbeta * (x5 * rsq(x5));      // -beta sqrt(5 m_eff k_n)
    const T gt = gn * c.gt_ratio;               // -beta sqrt(10/3 m_eff k_t)
    const Vec3<T> vr = va - vb;
    const T vn = dot(vr, n);
    const Vec3<T> rw = WALL ? ra * wa
                            : mk3(rn_add(rn_mul(ra, wa.x), rn_mul(rb, wb.x)), rn_add(rn_mul(ra, wa.y), rn_mul(rb, wb.y)),
                                  rn_add(rn_mul(ra, wa.z), rn_mul(rb, wb.z)));
    const Vec3<T> vc = vr - cross(rw, n);
    const Vec3<T> vt = vc - dot(vc, n) * n;
    T fnm = kn * delta - gn * vn;
    if (c.clamp_fn && fnm < T(0)) fnm = T(0);
    // keep xi in the tangent plane at its previous length (|xr| <= |xi|)
    const T xin = dot(xi, n);
    const Vec3<T> xr = xi - xin * n;
    const T l0 = dot(xi, xi), l1 = dot(xr, xr);
    xi = l1 > T(0) ? rsq(fdiv(l1, l0)) * xr : mk3(T(0), T(0), T(0));
    xi = xi + dt_hist * vt;
    ft = (-kt) * xi - gt * vt;
    const T ft2 = dot(ft, ft);
    const T lim = (WALL ? c.mu_w : c.mu) * (fnm < T(0) ? -fnm : fnm);
    slip = ft2 > lim * lim;
    if (slip) {
        ft = (lim * rsq(ft2)) * ft;
        xi = fdiv(T(-1), kt) * (ft + gt * vt);
    }
    return fnm * n + ft;
}

// Adjoint seeds and results of one contact seen from body a.
template <typename T>
struct PairGrad {
    Vec3<T> r;        // d/d(x_a - x_b)   (for a wall: d/d x_a)
    Vec3<T> va, vb;   // d/d v_a, d/d v_b
    Vec3<T> wa, wb;   // d/d w_a, d/d w_b
    Vec3<T> xi;       // d/d (stored overlap before the step)
    T c_kn, c_kt, nbeta, mu;
};

// Reverse-mode derivative of
//   L = G . f_a - H . (n x f_t) + xibar . xi'
// through contact_fwd (recomputed here), with G = Fbar_a - Fbar_b and
// H = r_a Tbar_a + r_b Tbar_b (for a wall: G = Fbar_a, H = r_a Tbar_a).  The
// contact and slip pattern is the one the forward evaluation takes.  dist is
// |x_a - x_b|, delta = r_a + r_b - dist (for a wall dist is the height above it
// and n is fixed).
template <typename T, bool WALL>
HD void contact_vjp(const Coef<T>& c, T delta, Vec3<T> n, T dist, T ra, T rb, T ma, T mb, Vec3<T> va, Vec3<T> vb,
                    Vec3<T> wa, Vec3<T> wb, Vec3<T> xi_old, T dt_hist, Vec3<T> G, Vec3<T> H, Vec3<T> xibar,
                    PairGrad<T>& g)
{
    const Vec3<T> z3 = mk3(T(0), T(0), T(0));
    // ---- forward recomputation
    T R, meff;
    if (WALL) {
        R = ra;
        meff = ma;
    } else {
        R = fdiv(ra * rb, ra + rb);
        meff = fdiv(ma * mb, ma + mb);
    }
    const T Rd = R * delta;
    const T sRd = Rd * rsq(Rd);
    const T kn = c.c_kn * sRd;
    const T kt = c.c_kt * sRd;
    const T x5 = T(5) * meff * kn;
    const T sX = x5 * rsq(x5);
    const T gn = c.nbeta * sX;
    const T gt = gn * c.gt_ratio;
    const Vec3<T> vr = va - vb;
    const T vn = dot(vr, n);
    const Vec3<T> rw = WALL ? ra * wa
                            : mk3(rn_add(rn_mul(ra, wa.x), rn_mul(rb, wb.x)), rn_add(rn_mul(ra, wa.y), rn_mul(rb, wb.y)),
                                  rn_add(rn_mul(ra, wa.z), rn_mul(rb, wb.z)));
    const Vec3<T> cwn = cross(rw, n);
    const Vec3<T> vc = vr - cwn;
    const T vcn = dot(vc, n);
    const Vec3<T> vt = vc - vcn * n;
    T fnm = kn * delta - gn * vn;
    bool clamped = false;
    if (c.clamp_fn && fnm < T(0)) {
        fnm = T(0);
        clamped = true;
    }
    const T xin = dot(xi_old, n);
    const Vec3<T> xr = xi_old - xin * n;
    const T l0 = dot(xi_old, xi_old), l1 = dot(xr, xr);
    T s = T(0);
    Vec3<T> xir = z3;
    if (l1 > T(0)) {
        s = rsq(fdiv(l1, l0));
        xir = s * xr;
    }
    const Vec3<T> xi1 = xir + dt_hist * vt;
    const Vec3<T> fts = (-kt) * xi1 - gt * vt;
    const T ft2 = dot(fts, fts);
    const T mu = WALL ? c.mu_w : c.mu;
    const T afn = fnm < T(0) ? -fnm : fnm;
    const T lim = mu * afn;
    const bool slip = ft2 > lim * lim;
    Vec3<T> ft = fts, xin_new = xi1, u = z3;
    T N = T(0);
    if (slip) {
        N = ft2 * rsq(ft2);
        u = fdiv(T(1), N) * fts;
        ft = lim * u;
        xin_new = fdiv(T(-1), kt) * (ft + gt * vt);
    }

    // ---- reverse sweep
    T fnm_b = dot(G, n);
    Vec3<T> n_b = fnm * G - cross(ft, H);
    Vec3<T> ft_b = G - cross(H, n);
    T kt_b = T(0), gt_b = T(0), mu_b = T(0);
    Vec3<T> vt_b = z3, fts_b, xi1_b;
    if (slip) {
        const T ikt = fdiv(T(1), kt);
        ft_b = ft_b - ikt * xibar;
        gt_b = -ikt * dot(xibar, vt);
        vt_b = (-gt * ikt) * xibar;
        kt_b = -ikt * dot(xibar, xin_new);
        const T lim_b = dot(ft_b, u);
        fts_b = (lim / N) * (ft_b - lim_b * u);
        mu_b = lim_b * afn;
        fnm_b = fnm_b + lim_b * mu * (fnm < T(0) ? T(-1) : T(1));
        xi1_b = (-kt) * fts_b;
    } else {
        fts_b = ft_b;
        xi1_b = xibar - kt * fts_b;
    }
    kt_b = kt_b - dot(xi1, fts_b);
    gt_b = gt_b - dot(vt, fts_b);
    vt_b = vt_b - gt * fts_b;
    // xi1 = xir + dt_hist vt
    const Vec3<T> xir_b = xi1_b;
    vt_b = vt_b + dt_hist * xi1_b;
    // xir = s xr
    Vec3<T> xi_old_b = z3;
    if (l1 > T(0)) {
        Vec3<T> xr_b = s * xir_b;
        const T s_b = dot(xir_b, xr);
        const T l0_b = s_b * s / (T(2) * l0);
        const T l1_b = -s_b * s / (T(2) * l1);
        xi_old_b = (T(2) * l0_b) * xi_old;
        xr_b = xr_b + (T(2) * l1_b) * xr;
        const T xrbn = dot(xr_b, n);
        xi_old_b = xi_old_b + xr_b - xrbn * n;
        n_b = n_b - (xin * xr_b + xrbn * xi_old);
    }
    // vt = vc - (vc . n) n
    const T vtbn = dot(vt_b, n);
    const Vec3<T> vc_b = vt_b - vtbn * n;
    n_b = n_b - (vcn * vt_b + vtbn * vc);
    // vc = vr - rw x n
    Vec3<T> vr_b = vc_b;
    const Vec3<T> cwn_b = -vc_b;
    const Vec3<T> rw_b = cross(n, cwn_b);
    n_b = n_b + cross(cwn_b, rw);
    // fnm = kn delta - gn vn
    if (clamped) fnm_b = T(0);
    T kn_b = fnm_b * delta;
    T delta_b = fnm_b * kn;
    T gn_b = -fnm_b * vn;
    const T vn_b = -fnm_b * gn;
    vr_b = vr_b + vn_b * n;
    n_b = n_b + vn_b * vr;
    // gt = gn ratio; gn = nbeta sqrt(5 meff kn)
    gn_b = gn_b + gt_b * c.gt_ratio;
    const T nbeta_b = gn_b * sX;
    kn_b = kn_b + gn_b * c.nbeta * (T(5) * meff) / (T(2) * sX);
    // kn = c_kn sRd, kt = c_kt sRd, sRd = sqrt(R delta)
    const T sRd_b = kn_b * c.c_kn + kt_b * c.c_kt;
    delta_b = delta_b + sRd_b * R / (T(2) * sRd);
    // delta = r_a + r_b - dist, and n = (x_a - x_b) / dist
    const T dist_b = -delta_b;
    if (WALL) {
        g.r = dist_b * n;
    } else {
        g.r = (fdiv(T(1), dist)) * (n_b - dot(n_b, n) * n) + dist_b * n;
    }
    g.va = vr_b;
    g.vb = -vr_b;
    g.wa = ra * rw_b;
    g.wb = WALL ? z3 : rb * rw_b;
    g.xi = xi_old_b;
    g.c_kn = kn_b * sRd;
    g.c_kt = kt_b * sRd;
    g.nbeta = nbeta_b;
    g.mu = mu_b;
}

#undef HD

}  // namespace cgdem
