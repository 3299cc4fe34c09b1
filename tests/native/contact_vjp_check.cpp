// Checks the hand-written reverse-mode derivative of the contact law
// (contact_vjp in dem_contact.cuh) against central differences of the same
// law (contact_fwd), both instantiated in double on the host.  Prints one line
// per case: "<case> <max relative error>".
#include <cmath>
#include <cstdio>
#include <random>

#include "dem_contact.cuh"

using namespace cgdem;
using V = Vec3<double>;

struct In {
    V r;            // x_a - x_b (pair) or (0, 0, height) (wall)
    V va, vb, wa, wb, xi;
    double ckn, ckt, nbeta, mu;
};

static const int NIN = 3 * 6 + 4;
static double& comp(In& in, int k)
{
    V* vs[6] = {&in.r, &in.va, &in.vb, &in.wa, &in.wb, &in.xi};
    if (k < 18) {
        V* v = vs[k / 3];
        return k % 3 == 0 ? v->x : k % 3 == 1 ? v->y : v->z;
    }
    double* ps[4] = {&in.ckn, &in.ckt, &in.nbeta, &in.mu};
    return *ps[k - 18];
}

template <bool WALL>
static double loss(In in, double ra, double rb, double ma, double mb, double dt, V G, V H, V xib, bool* slip_out)
{
    Coef<double> c{in.ckn, in.ckt, in.nbeta, std::sqrt(2.0 * in.ckt / (3.0 * in.ckn)), in.mu, in.mu, 0};
    double dist, delta;
    V n;
    if (WALL) {
        dist = in.r.z;
        n = mk3(0.0, 0.0, 1.0);
        delta = ra - dist;
    } else {
        dist = std::sqrt(dot(in.r, in.r));
        n = (1.0 / dist) * in.r;
        delta = ra + rb - dist;
    }
    V xi = in.xi, ft;
    bool slip;
    V fa = contact_fwd<double, WALL>(c, delta, n, ra, rb, ma, mb, in.va, in.vb, in.wa, in.wb, xi, dt, ft, slip);
    if (slip_out) *slip_out = slip;
    return dot(G, fa) - dot(H, cross(n, ft)) + dot(xib, xi);
}

template <bool WALL>
static double check(std::mt19937_64& rng, bool want_slip, int* got_slip)
{
    std::normal_distribution<double> N(0.0, 1.0);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    const double ra = 1.0e-3 * (0.9 + 0.2 * U(rng)), rb = 1.0e-3 * (0.9 + 0.2 * U(rng));
    const double ma = 1.0e-5 * (0.8 + 0.4 * U(rng)), mb = 1.0e-5 * (0.8 + 0.4 * U(rng));
    const double dt = 1e-6;
    In in;
    const double overlap = 5e-6 * (0.2 + U(rng));
    if (WALL) {
        in.r = mk3(0.0, 0.0, ra - overlap);
    } else {
        V dir = mk3(N(rng), N(rng), N(rng));
        dir = (1.0 / std::sqrt(dot(dir, dir))) * dir;
        in.r = (ra + rb - overlap) * dir;
    }
    in.va = mk3(0.05 * N(rng), 0.05 * N(rng), 0.05 * N(rng));
    in.vb = mk3(0.05 * N(rng), 0.05 * N(rng), 0.05 * N(rng));
    in.wa = mk3(20 * N(rng), 20 * N(rng), 20 * N(rng));
    in.wb = mk3(20 * N(rng), 20 * N(rng), 20 * N(rng));
    in.xi = mk3(1e-7 * N(rng), 1e-7 * N(rng), 1e-7 * N(rng));
    in.ckn = 7.1e6;
    in.ckt = 9.1e6;
    in.nbeta = 0.2;
    in.mu = want_slip ? 0.02 : 5.0;
    const V G = mk3(N(rng), N(rng), N(rng)), H = mk3(1e-3 * N(rng), 1e-3 * N(rng), 1e-3 * N(rng));
    const V xib = mk3(1e5 * N(rng), 1e5 * N(rng), 1e5 * N(rng));

    bool slip;
    loss<WALL>(in, ra, rb, ma, mb, dt, G, H, xib, &slip);
    *got_slip = slip ? 1 : 0;
    // analytic
    Coef<double> c{in.ckn, in.ckt, in.nbeta, std::sqrt(2.0 * in.ckt / (3.0 * in.ckn)), in.mu, in.mu, 0};
    double dist, delta;
    V n;
    if (WALL) {
        dist = in.r.z;
        n = mk3(0.0, 0.0, 1.0);
        delta = ra - dist;
    } else {
        dist = std::sqrt(dot(in.r, in.r));
        n = (1.0 / dist) * in.r;
        delta = ra + rb - dist;
    }
    PairGrad<double> g;
    contact_vjp<double, WALL>(c, delta, n, dist, ra, rb, ma, mb, in.va, in.vb, in.wa, in.wb, in.xi, dt, G, H, xib, g);
    // the gradient of gt_ratio is folded into c_kn and c_kt by the chain rule
    // here, because the forward computes gt_ratio from them
    In ga;
    ga.r = g.r; ga.va = g.va; ga.vb = g.vb; ga.wa = g.wa; ga.wb = g.wb; ga.xi = g.xi;
    ga.ckn = g.c_kn; ga.ckt = g.c_kt; ga.nbeta = g.nbeta; ga.mu = g.mu;
    // fourth-order central differences, compared per vector group against the
    // size of that group's gradient
    auto L = [&](const In& q) { return loss<WALL>(q, ra, rb, ma, mb, dt, G, H, xib, nullptr); };
    double worst = 0.0;
    for (int grp = 0; grp < 10; ++grp) {
        if (WALL && (grp == 2 || grp == 4)) continue;                 // v_b, w_b: absent for a wall
        if (grp == 6 || grp == 7) continue;                          // c_kn, c_kt: checked together below
        const int k0 = grp < 6 ? 3 * grp : 18 + (grp - 6);
        const int nk = grp < 6 ? 3 : 1;
        double size = 0.0;
        for (int q = 0; q < nk; ++q) size += comp(in, k0 + q) * comp(in, k0 + q);
        size = std::sqrt(size);
        double h = grp == 0 ? 1e-11 : 1e-4 * size;
        double err2 = 0.0, an2 = 0.0;
        for (int q = 0; q < nk; ++q) {
            const int k = k0 + q;
            if (WALL && grp == 0 && q < 2) continue;                // only the height matters for a wall
            In p1 = in, m1 = in, p2 = in, m2 = in;
            comp(p1, k) += h; comp(m1, k) -= h; comp(p2, k) += 2 * h; comp(m2, k) -= 2 * h;
            const double fd = (8.0 * (L(p1) - L(m1)) - (L(p2) - L(m2))) / (12.0 * h);
            const double an = comp(ga, k);
            err2 += (fd - an) * (fd - an);
            an2 += an * an;
        }
        if (an2 > 0) worst = std::fmax(worst, std::sqrt(err2 / an2));
    }
    {
        // c_kn and c_kt move together with E (their ratio, hence gt_ratio, fixed)
        auto scaled = [&](double f) {
            In q = in;
            q.ckn *= f;
            q.ckt *= f;
            return loss<WALL>(q, ra, rb, ma, mb, dt, G, H, xib, nullptr);
        };
        const double eps = 1e-6;
        const double fd = (scaled(1 + eps) - scaled(1 - eps)) / (2 * eps);
        const double an = g.c_kn * in.ckn + g.c_kt * in.ckt;
        worst = std::fmax(worst, std::fabs(fd - an) / (std::fabs(fd) + std::fabs(an) + 1e-300));
    }
    return worst;
}

int main()
{
    std::mt19937_64 rng(12345);
    double w[4] = {0, 0, 0, 0};
    int slips[4] = {0, 0, 0, 0};
    for (int t = 0; t < 200; ++t) {
        int s;
        w[0] = std::fmax(w[0], check<false>(rng, false, &s)); slips[0] += s;
        w[1] = std::fmax(w[1], check<false>(rng, true, &s)); slips[1] += s;
        w[2] = std::fmax(w[2], check<true>(rng, false, &s)); slips[2] += s;
        w[3] = std::fmax(w[3], check<true>(rng, true, &s)); slips[3] += s;
    }
    std::printf("pair_stick %.3e %d\npair_slip %.3e %d\nwall_stick %.3e %d\nwall_slip %.3e %d\n", w[0], slips[0], w[1],
                slips[1], w[2], slips[2], w[3], slips[3]);
    return 0;
}
