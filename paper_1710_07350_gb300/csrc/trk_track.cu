// Fused FP64 tracking kernel, per-turn moment partials, moment finalisation and
// stable loss compaction.
//
// Design (GB300, FP64-pipe bound): one launch pushes a tile of particles
// through many consecutive elements and turns with the 6 coordinates held in
// registers (the paper's particle accessor keeps one read/write per coordinate
// per element kernel, Sec. 2.1; here it is one per launch).  Element records
// are read warp-uniformly.  Square roots and divisions of the exact drift and
// the slope/canonical conversions are replaced, for the small arguments that
// occur in practice, by truncated binomial series that agree with the exact
// expressions to FP64 rounding (the exact path runs otherwise); aperture tests
// compare integer bit patterns (the ellipse takes its exact FP64 test only
// outside an inner box), so they cost almost no FP64 instructions.
#include <cmath>

#include "trk_device.cuh"
#include "trk_internal.cuh"

namespace trk {
namespace {

// The P particles a thread owns, advanced in lock-step through every element so
// that their independent FP64 chains interleave (the pipe's latency is long
// compared with one particle's dependent drift-kick chain).
template <int P>
struct Tile {
    double x[P], xp[P], y[P], yp[P], l[P], d[P];
};

template <int P>
__device__ __forceinline__ double tget(const Tile<P> &q, int p, int j) {
    double r = q.x[p];
    r = (j == 1) ? q.xp[p] : r;
    r = (j == 2) ? q.y[p] : r;
    r = (j == 3) ? q.yp[p] : r;
    r = (j == 4) ? q.l[p] : r;
    r = (j == 5) ? q.d[p] : r;
    return r;
}

// ---------------------------------------------------------------- map ----
// x_i <- C_i + R x + T x x + U x x x from the input vector (simultaneous).
// The six rows are independent sums; they are stepped through together (term k
// of every row that has one, then term k + 1), so that their FMA chains
// interleave and one particle's latency is the longest row, not the sum of all
// rows (which is what bounds a lightly occupied GPU).
template <int P>
__device__ __forceinline__ void v_map(Tile<P> &q, const DevElem *__restrict__ E, const DevTerm *__restrict__ terms,
                                      uint32_t rows, bool &dirty) {
    const uint32_t flags = __ldg(&E->flags);
    const int4 rbv = __ldg(reinterpret_cast<const int4 *>(E->rb));
    const int16_t *rb = reinterpret_cast<const int16_t *>(&rbv);
    const double2 *t = reinterpret_cast<const double2 *>(terms + __ldg(&E->term0));
    // +0 known only at run time (a map's p[] is zero): monomial products are
    // fma(m, x_j, z0), rounded as m * x_j but issued at the DFMA rate (taken per
    // element: the kernel-wide zero measured 3-10 % slower on map rings)
    const double z0 = __ldg(&E->p[0]) * 0.0;
    double acc[6][P];
    int len[6], n = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        len[r] = ((rows >> r) & 1u) ? rb[r + 1] - rb[r] : 0;   // rows outside `rows` are not evaluated
        n = len[r] > n ? len[r] : n;
#pragma unroll
        for (int p = 0; p < P; ++p) acc[r][p] = ((flags >> r) & 1u) ? tget(q, p, r) : 0.0;
    }
    for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (k >= len[r]) continue;
            const double2 tv = __ldg(t + rb[r] + k);
            const int code = (int)(unsigned)(__double_as_longlong(tv.y) & 0xffffffffll);
            const int deg = code & 3, j = (code >> 2) & 7, jk = (code >> 5) & 7, jl = (code >> 8) & 7;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                double m = 1.0;
                if (deg >= 1) m = tget(q, p, j);
                if (deg >= 2) m = fma(m, tget(q, p, jk), z0);
                if (deg >= 3) m = fma(m, tget(q, p, jl), z0);
                acc[r][p] = fma(tv.x, m, acc[r][p]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        q.x[p] = acc[0][p];
        q.xp[p] = acc[1][p];
        q.y[p] = acc[2][p];
        q.yp[p] = acc[3][p];
        q.l[p] = acc[4][p];
        q.d[p] = acc[5][p];
    }
    if (flags & 64u) dirty = true;
}

// -------------------------------------------------------- exact drift ----
// x += L x', y += L y', l += L (sqrt(1 + v) - 1), v = x'^2 + y'^2; for v < 2^-14
// sqrt(1+v) - 1 = v/2 - v^2/8 + v^3/16 - 5 v^4/128 to FP64 rounding.
template <int P>
__device__ __forceinline__ void v_edrift(Tile<P> &q, double L, double z0) {
    // z0 = run-time +0: products issued as FMAs (as in v_map)
    double g[P];
    bool need = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double v = fma(q.xp[p], q.xp[p], fma(q.yp[p], q.yp[p], z0));
        g[p] = fma(v, fma(v, fma(v, fma(v, -0.0390625, 0.0625), -0.125), 0.5), z0);
        need |= !series_ok(v);
        q.x[p] = fma(L, q.xp[p], q.x[p]);
        q.y[p] = fma(L, q.yp[p], q.y[p]);
    }
    if (need) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double v = fma(q.xp[p], q.xp[p], q.yp[p] * q.yp[p]);
            if (!series_ok(v)) g[p] = edrift_exact_g(v);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) q.l[p] = fma(L, g[p], q.l[p]);
}

// ------------------------------------------------ kick-drift multipole ----
// Inside a kick-drift element the momenta are carried scaled by the particle's
// total momentum, qx = px/(1+delta) (delta is constant through the element).
// Exact-Hamiltonian drift: pz/(1+delta) = sqrt(1 - u), u = qx^2 + qy^2, so
//   x += h qx (1 + g),  y += h qy (1 + g),  l += h g,
//   g = (1 - u)^(-1/2) - 1 = u/2 + 3u^2/8 + 5u^3/16 + ...  (u < 2^-14; the
// first dropped term is then below 4e-18), or rsqrt(1 - u) - 1 otherwise.
__device__ __noinline__ double drift_g_exact(double u) { return rsqrt(1.0 - u) - 1.0; }

// With hh = h/2 and hq = 3h/8 given, the two-term series is taken as
//   c = hq u + hh,  h g = c u,  h (1 + g) = c u + h
// (three FMAs and no multiply).  A = c, B = u, or A = h, B = g on the longer
// series and exact branches, and then t = A B + h, l += A B.
template <int P>
__device__ __forceinline__ void v_drift(double (&x)[P], double (&y)[P], double (&l)[P], const double (&qx)[P],
                                        const double (&qy)[P], double h, double hh, double hq, double z0) {
    double A[P], B[P];
    bool need = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double u = fma(qx[p], qx[p], fma(qy[p], qy[p], z0));
        A[p] = fma(hq, u, hh);
        B[p] = u;
        need |= !quad_ok(u);
    }
    if (need) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double u = B[p];
            if (!quad_ok(u)) {
                A[p] = h;
                B[p] = series_ok(u) ? u * fma(u, fma(u, 0.3125, 0.375), 0.5) : drift_g_exact(u);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double t = fma(A[p], B[p], h);
        x[p] = fma(t, qx[p], x[p]);
        y[p] = fma(t, qy[p], y[p]);
        l[p] = fma(A[p], B[p], l[p]);
    }
}

// Kicks on the scaled momenta: quadrupole qx -= (K1 h/(1+delta)) x, qy += ...;
// sextupole qx -= hb (x^2 - y^2), qy += b x y with hb = K2 h/(2(1+delta)), b = 2 hb.
template <int P, uint32_t FL>
__device__ __forceinline__ void v_kick(const double (&x)[P], const double (&y)[P], double (&qx)[P], double (&qy)[P],
                                       const double (&a)[P], const double (&hb)[P], const double (&b)[P],
                                       double z0) {
    if (FL & 1u) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            qx[p] = fma(-a[p], x[p], qx[p]);
            qy[p] = fma(a[p], y[p], qy[p]);
        }
    }
    if (FL & 2u) {
        // two products and three FMAs: w = x^2 - y^2 = fma(x, x, -y^2)
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double w = fma(x[p], x[p], -fma(y[p], y[p], z0));
            qx[p] = fma(-hb[p], w, qx[p]);
            qy[p] = fma(fma(b[p], y[p], z0), x[p], qy[p]);
        }
    }
}

// Slopes -> scaled canonical momenta: qx = x' (1 + x'^2 + y'^2)^(-1/2).
template <int P>
__device__ __forceinline__ void v_to_canonical(Tile<P> &q) {
    double c[P];
    bool need = false;
    // (1 + v)^(-1/2) = 1 - v/2 + 3v^2/8 - 5v^3/16 + ...
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double v = fma(q.xp[p], q.xp[p], q.yp[p] * q.yp[p]);
        c[p] = fma(v, fma(v, 0.375, -0.5), 1.0);
        need |= !quad_ok(v);
    }
    if (need) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double v = fma(q.xp[p], q.xp[p], q.yp[p] * q.yp[p]);
            if (!quad_ok(v))
                c[p] = series_ok(v) ? fma(v, fma(v, fma(v, -0.3125, 0.375), -0.5), 1.0) : rsqrt_exact(1.0 + v);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        q.xp[p] = c[p] * q.xp[p];
        q.yp[p] = c[p] * q.yp[p];
    }
}

// Scaled canonical momenta -> slopes: x' = qx (1 - u)^(-1/2) = qx (1 + g).
__device__ __forceinline__ double2 slopes_of(double qx, double qy) {
    const double u = fma(qx, qx, qy * qy);
    double g = u * fma(u, 0.375, 0.5);
    if (!quad_ok(u)) g = series_ok(u) ? u * fma(u, fma(u, 0.3125, 0.375), 0.5) : drift_g_exact(u);
    return make_double2(fma(qx, g, qx), fma(qy, g, qy));
}

template <int P>
__device__ __forceinline__ void v_to_slopes(Tile<P> &q) {
    double g[P];
    bool need = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double u = fma(q.xp[p], q.xp[p], q.yp[p] * q.yp[p]);
        g[p] = u * fma(u, 0.375, 0.5);
        need |= !quad_ok(u);
    }
    if (need) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const double u = fma(q.xp[p], q.xp[p], q.yp[p] * q.yp[p]);
            if (!quad_ok(u)) g[p] = series_ok(u) ? u * fma(u, fma(u, 0.3125, 0.375), 0.5) : drift_g_exact(u);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        q.xp[p] = fma(q.xp[p], g[p], q.xp[p]);
        q.yp[p] = fma(q.yp[p], g[p], q.yp[p]);
    }
}

// n steps of the 4th-order Yoshida scheme D K D K D K D with adjacent drifts of
// consecutive steps merged, on the scaled canonical momenta (q.xp, q.yp hold
// qx, qy here).  FL: bit 0 quadrupole kick, bit 1 sextupole kick (one
// instantiation each, so that only the strengths in use occupy registers).
template <int P, uint32_t FL>
__device__ __forceinline__ void v_kick_drift_t(Tile<P> &q, const double (&iP)[P], const DevElem *__restrict__ E) {
    const int n = __ldg(&E->n);
    const double d1 = __ldg(&E->p[0]), d2 = __ldg(&E->p[1]), dm = __ldg(&E->p[2]);
    const double d1h = __ldg(&E->p[7]), d1q = __ldg(&E->p[8]), d2h = __ldg(&E->p[9]), d2q = __ldg(&E->p[10]),
                 dmq = __ldg(&E->p[11]);
    // z0 = +0 known only at run time: products (and doublings) are written
    // fma(a, b, z0), which rounds as a * b (adding +0 to a rounded product is
    // exact but for the sign of an exact zero) and issues as an FMA, faster than
    // a multiply or an add on this GPU's FP64 pipe.  Taken from the element (the
    // kernel-wide zero measured 2.7 % slower on the kick-drift ring)
    const double z0 = d1 * 0.0;
    double a1[P], a0[P], hb1[P], hb0[P], b1[P], b0[P];
    if (FL & 1u) {
        const double A1 = __ldg(&E->p[3]), A0 = __ldg(&E->p[4]);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            a1[p] = fma(A1, iP[p], z0);
            a0[p] = fma(A0, iP[p], z0);
        }
    }
    if (FL & 2u) {
        const double H1 = __ldg(&E->p[5]), H0 = __ldg(&E->p[6]);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            hb1[p] = fma(H1, iP[p], z0);
            hb0[p] = fma(H0, iP[p], z0);
            b1[p] = fma(2.0, hb1[p], z0);
            b0[p] = fma(2.0, hb0[p], z0);
        }
    }
    v_drift<P>(q.x, q.y, q.l, q.xp, q.yp, d1, d1h, d1q, z0);
    for (int s = 0; s < n; ++s) {
        v_kick<P, FL>(q.x, q.y, q.xp, q.yp, a1, hb1, b1, z0);
        v_drift<P>(q.x, q.y, q.l, q.xp, q.yp, d2, d2h, d2q, z0);
        v_kick<P, FL>(q.x, q.y, q.xp, q.yp, a0, hb0, b0, z0);
        v_drift<P>(q.x, q.y, q.l, q.xp, q.yp, d2, d2h, d2q, z0);
        v_kick<P, FL>(q.x, q.y, q.xp, q.yp, a1, hb1, b1, z0);
        const bool mid = s + 1 < n;   // merged drift dm = 2 d1, so dm / 2 = d1
        v_drift<P>(q.x, q.y, q.l, q.xp, q.yp, mid ? dm : d1, mid ? d1 : d1h, mid ? dmq : d1q, z0);
    }
}

// Kick-drift element; leaves the tile in the canonical representation.
template <int P>
__device__ __forceinline__ void v_kick_drift(Tile<P> &q, double (&iP)[P], bool &dirty, bool &canon,
                                             const DevElem *__restrict__ E) {
    if (dirty) {
#pragma unroll
        for (int p = 0; p < P; ++p) iP[p] = 1.0 / (1.0 + q.d[p]);
        dirty = false;
    }
    if (!canon) {
        v_to_canonical<P>(q);
        canon = true;
    }
    switch (__ldg(&E->flags) & 3u) {
    case 1u: v_kick_drift_t<P, 1u>(q, iP, E); break;
    case 2u: v_kick_drift_t<P, 2u>(q, iP, E); break;
    case 3u: v_kick_drift_t<P, 3u>(q, iP, E); break;
    default: v_kick_drift_t<P, 0u>(q, iP, E); break;
    }
}

// Thin sextupole (Table 1 THINSEXT): x' -= (K2L/2)(x^2 - y^2), y' += K2L x y.
template <int P>
__device__ __forceinline__ void v_thin_sext(Tile<P> &q, const DevElem *__restrict__ E, double z0) {
    const double k = __ldg(&E->p[0]), hk = __ldg(&E->p[1]);   // z0: run-time +0 (as in v_map)
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double t = fma(q.x[p], q.x[p], -fma(q.y[p], q.y[p], z0));
        q.xp[p] = fma(-hk, t, q.xp[p]);
        q.yp[p] = fma(k, fma(q.x[p], q.y[p], z0), q.yp[p]);
    }
}

// Sector dipole, hard edge (Table 1 CSBEND without fringe fields or
// radiation): the particle enters at radius rho + x with canonical radial and
// tangential momenta px, pz and moves on a circle of radius rho p_h centred at
// (rho + x - rho pz, rho px) until the exit face at angle theta, after turning
// by alpha = theta + beta, beta = atan2(px, pz) + asin(S / p_h),
// S = (1 + x/rho - pz) sin(theta) - px cos(theta).  Exit: x = |P| - rho,
// px = px cos(beta) - pz sin(beta), y += py rho alpha, l += rho (1+delta) alpha - L.
template <int P>
__device__ __forceinline__ void v_sbend(Tile<P> &q, const DevElem *__restrict__ E) {
    const double L = __ldg(&E->p[0]), th = __ldg(&E->p[1]), rho = __ldg(&E->p[2]), h = __ldg(&E->p[3]);
    const double st = __ldg(&E->p[4]), ct = __ldg(&E->p[5]);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double d1 = 1.0 + q.d[p];
        const double ir = rsqrt(fma(q.xp[p], q.xp[p], fma(q.yp[p], q.yp[p], 1.0)));
        const double pz = d1 * ir, px = q.xp[p] * pz, py = q.yp[p] * pz;
        const double ph = sqrt(fma(d1, d1, -py * py));
        const double S = fma(fma(q.x[p], h, 1.0) - pz, st, -px * ct);
        const double beta = atan2(px, pz) + asin(S / ph);
        const double alpha = th + beta;
        double sa, ca, sb, cb;
        sincos(alpha, &sa, &ca);
        sincos(beta, &sb, &cb);
        const double Px = fma(rho, fma(pz, ca, px * sa), fma(-rho, pz, rho + q.x[p]));
        const double Py = fma(rho, fma(pz, sa, -px * ca), rho * px);
        const double pxf = fma(px, cb, -pz * sb);
        const double ipzf = rsqrt(fma(d1, d1, -fma(pxf, pxf, py * py)));
        q.x[p] = sqrt(fma(Px, Px, Py * Py)) - rho;
        q.xp[p] = pxf * ipzf;
        q.y[p] = fma(py * rho, alpha, q.y[p]);
        q.yp[p] = py * ipzf;
        q.l[p] = fma(rho * d1, alpha, q.l[p] - L);
    }
}

// cos(phi + x) for |x| >= 2^-4 (or NaN), out of line: it runs only for the
// particles that need it.
__device__ __noinline__ double rf_cos_exact(double phi, double x) { return cos(phi + x); }

// cos(phi + x) = cos(phi) C(x) - sin(phi) S(x) with the Taylor series of
// C = cos and S = sin at 0 (Abramowitz & Stegun 4.3.65-66) through x^8 and x^9:
// for |x| < 2^-4 the first dropped terms are below 3e-19, far under the
// rounding of the result, so this is cos(phi + x) to FP64 rounding at about
// half the instructions of a general cosine.  The test is an integer compare
// of |x|'s high word (2^-4 = 0x3FB00000; NaN fails it).
// z0 is a run-time +0: the products are written fma(a, b, z0), rounded as a * b
// but issued at the DFMA rate (as in the maps).
__device__ __forceinline__ double rf_cos(double cphi, double sphi, double phi, double x, double z0) {
    const double x2 = fma(x, x, z0);
    const double C = fma(x2, fma(x2, fma(x2, fma(x2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
    const double S = fma(x, fma(x2, fma(x2, fma(x2, fma(x2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0), z0);
    double c = fma(cphi, C, fma(-sphi, S, z0));
    if ((__double2hiint(x) & 0x7fffffff) >= 0x3FB00000) c = rf_cos_exact(phi, x);
    return c;
}

// Thin RF: P = (1+delta) p0, P' = P + V cos(phi + k l), delta' = P'/p0' - 1,
// slopes scaled by P/P'.
template <int P>
__device__ __forceinline__ void v_rfca(Tile<P> &q, const DevElem *__restrict__ E, double p0, double ip01,
                                       double z0, bool &dirty) {
    const double V = __ldg(&E->p[0]), phi = __ldg(&E->p[1]), k = __ldg(&E->p[2]);
    const double cphi = __ldg(&E->p[4]), sphi = __ldg(&E->p[5]);
    // z0: run-time +0 (see rf_cos)
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double Pp = fma(q.d[p], p0, p0);   // (1 + delta) p0 in one rounding
        const double P1 = fma(V, rf_cos(cphi, sphi, phi, fma(k, q.l[p], z0), z0), Pp);
        // s = Pp / P1 through Newton's iteration for the reciprocal, r <- r + r (1 - P1 r),
        // which squares the relative error 1 - P1 r at every step, seeded with 1/p0'
        // (P1 = (1 + delta') p0': the seed's error is -delta').  Three steps from
        // |1 - P1 r| <= 2^-8 leave the rounding of the last step; s = Pp r is then
        // within two units of rounding of the quotient.  A particle further off the
        // reference momentum (or a NaN) takes the division.
        double s;
        const double e0 = fma(-P1, ip01, 1.0);
        if (((unsigned long long)__double_as_longlong(e0) << 1) <= (0x3F70000000000000ull << 1)) {
            double r = fma(ip01, e0, ip01);
            r = fma(r, fma(-P1, r, 1.0), r);
            r = fma(r, fma(-P1, r, 1.0), r);
            s = fma(Pp, r, z0);
        } else {
            s = Pp / P1;
        }
        q.xp[p] = fma(q.xp[p], s, z0);
        q.yp[p] = fma(q.yp[p], s, z0);
        q.d[p] = -e0;   // P1 / p0' - 1: the rounding of P1 ip01 - 1 is minus that of 1 - P1 ip01
    }
    dirty = true;
}

// Wake voltage at l: linear interpolation between bin centres, clamped.
// c0 = -(lmin idl + 1/2), once per thread: u = l idl + c0 = (l - lmin) / dl - 1/2
// in one FMA (a rounding of c0 and one of u, against the oracle's difference,
// quotient and subtraction).
__device__ __forceinline__ double wake_volt(double l, double c0, double idl, bool flat,
                                            const double *__restrict__ V, int nb) {
    if (flat) return __ldg(V);
    const double u = fma(l, idl, c0);
    // k = floor(u) by one conversion (saturating at the int range) and integer
    // bounds tests; NaN (exponent all ones, mantissa non-zero) takes bin 0's
    // voltage, as a negative u does
    if (((unsigned long long)__double_as_longlong(u) << 1) > 0xFFE0000000000000ull) return __ldg(V);
    const int k = __double2int_rd(u);
    if (k < 0) return __ldg(V);
    if (k >= nb - 1) return __ldg(V + nb - 1);
    // the differences as fma(a, -1, b): one rounding, the same as b - a
    const double f = fma((double)k, -1.0, u);
    const double v0 = __ldg(V + k), v1 = __ldg(V + k + 1);
    return fma(f, fma(v0, -1.0, v1), v0);
}

// -------------------------------------------------------- block sums ----
// Sum 28 per-thread values over the block; the totals land in tot[0..27].
__device__ __forceinline__ void block_sum28(double (&v)[kMomentsN], double *sh, double *tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kMomentsN; ++q) {
        double s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        v[q] = s;
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kMomentsN; ++q) sh[w * kMomentsN + q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < kMomentsN) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += sh[j * kMomentsN + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
}

template <int P>
__device__ __forceinline__ void tile_moments(const Tile<P> &q, const bool (&alive)[P], double *sh, double *tot,
                                             double *K, double *out) {
    double v[kMomentsN];
#pragma unroll
    for (int i = 0; i < kMomentsN; ++i) v[i] = 0.0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!alive[p]) continue;
        const double d[6] = {q.x[p] - K[0], q.xp[p] - K[1], q.y[p] - K[2],
                             q.yp[p] - K[3], q.l[p] - K[4], q.d[p] - K[5]};
        v[0] += 1.0;
        int m = 7;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            v[1 + j] += d[j];
#pragma unroll
            for (int k = j; k < 6; ++k) {
                v[m] = fma(d[j], d[k], v[m]);
                ++m;
            }
        }
    }
    block_sum28(v, sh, tot);
    if (threadIdx.x == 0) {
        const double n = tot[0];
        out[0] = n;
        if (n > 0.0) {
            const double in = 1.0 / n;
            double s1[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                s1[j] = tot[1 + j];
                out[1 + j] = K[j] + s1[j] * in;
            }
            int m = 7;
#pragma unroll
            for (int j = 0; j < 6; ++j)
#pragma unroll
                for (int k = j; k < 6; ++k, ++m) out[m] = tot[m] - s1[j] * s1[k] * in;
#pragma unroll
            for (int j = 0; j < 6; ++j)
                if (isfinite(out[1 + j])) K[j] = out[1 + j];
        } else {
#pragma unroll
            for (int j = 1; j < kMomentsN; ++j) out[j] = 0.0;
        }
    }
    __syncthreads();
}

// Initial moment shift: the tile's mean (keeps the shifted sums well conditioned).
template <int P>
__device__ __forceinline__ void tile_mean(const Tile<P> &q, const bool (&alive)[P], double *sh, double *tot,
                                          double *K) {
    double v[kMomentsN];
#pragma unroll
    for (int i = 0; i < kMomentsN; ++i) v[i] = 0.0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!alive[p]) continue;
        v[0] += 1.0;
        v[1] += q.x[p]; v[2] += q.xp[p]; v[3] += q.y[p];
        v[4] += q.yp[p]; v[5] += q.l[p]; v[6] += q.d[p];
    }
    block_sum28(v, sh, tot);
    if (threadIdx.x < 6) {
        // A particle that is about to be lost may be non-finite: fall back to 0.
        const double m = tot[0] > 0.0 ? tot[1 + threadIdx.x] / tot[0] : 0.0;
        K[threadIdx.x] = isfinite(m) ? m : 0.0;
    }
    __syncthreads();
}

constexpr int kMaxBlock = 512;

template <int P>
__device__ __forceinline__ void store_particle(const TrackArgs &a, int64_t i, const Tile<P> &q, int p) {
    a.coords[i] = q.x[p];
    a.coords[a.pitch + i] = q.xp[p];
    a.coords[2 * a.pitch + i] = q.y[p];
    a.coords[3 * a.pitch + i] = q.yp[p];
    a.coords[4 * a.pitch + i] = q.l[p];
    a.coords[5 * a.pitch + i] = q.d[p];
}

// Kick of collective element `which` (0 or 1) of the group on key slot
// a.kick_slot: the transverse slope kicks first (V_x / P, V_y / P with
// P = p0 (1 + delta)), then the energy kick delta += V(l) / p0.
template <int P>
__device__ __forceinline__ void wake_kick(const TrackArgs &a, Tile<P> &q, const bool (&alive)[P], double p0,
                                          const double *V, const double *Vx, int nbins, int which) {
    const uint64_t kmin = a.win->key[2 * a.kick_slot];
    const double lmin = dkey_inv(kmin);
    const double idl = a.win->idl[2 * a.kick_slot + which];   // 1/dl from the histogram pass, 0 when flat
    const bool flat = !(idl > 0.0);
    const double c0 = -fma(lmin, idl, 0.5);
    const double ip0 = a.ip0c;
    if (Vx) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!alive[p]) continue;
            const double iP = ip0 / (1.0 + q.d[p]);
            q.xp[p] = fma(wake_volt(q.l[p], c0, idl, flat, Vx, nbins), iP, q.xp[p]);
            q.yp[p] = fma(wake_volt(q.l[p], c0, idl, flat, Vx + nbins, nbins), iP, q.yp[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (alive[p]) q.d[p] = fma(wake_volt(q.l[p], c0, idl, flat, V, nbins), ip0, q.d[p]);
}

// Check the aperture of every alive particle after element e; a particle that
// is lost is written out at once (coordinates at the loss point and the loss
// record) and its registers are zeroed so that it keeps taking the fast paths.
template <int P>
__device__ __forceinline__ void apply_aperture(const TrackArgs &a, const LatticeView &L, Tile<P> &q,
                                               bool (&alive)[P], int64_t base, int turn, int e, int &lost_here,
                                               bool canon) {
    if (L.ap_type == TRK_APERTURE_NONE) return;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (alive[p] && !inside(q.x[p], q.y[p], L)) {
            const int64_t i = base + (int64_t)p * blockDim.x + threadIdx.x;
            if (canon) {
                // the record holds slopes whatever the representation in registers
                const double2 sl = slopes_of(q.xp[p], q.yp[p]);
                q.xp[p] = sl.x;
                q.yp[p] = sl.y;
            }
            store_particle<P>(a, i, q, p);
            a.loss_turn[i] = turn;
            a.loss_elem[i] = e;
            alive[p] = false;
            q.x[p] = q.xp[p] = q.y[p] = q.yp[p] = q.l[p] = q.d[p] = 0.0;
            ++lost_here;
        }
    }
}

struct TrackShared {
    double sh[(kMaxBlock / 32) * kMomentsN];
    double tot[kMomentsN];
    double K[6];
    unsigned long long mm[2];
    int cnt;
};

// One tile of one bunch: load, track a.n_turns turns through [a.e0, a.e1),
// per-turn moment partials, optional l window, store, alive count.
template <int P>
__device__ __forceinline__ void track_tile(const TrackArgs &a, const int tile, TrackShared &S) {
    double *sh = S.sh, *tot = S.tot, *K = S.K;
    unsigned long long *mm = S.mm;
    int &cnt = S.cnt;
    const int64_t n_alive = a.st->n_alive;
    const int T = blockDim.x * P;
    const int64_t base = (int64_t)tile * T;
    if (base >= n_alive) return;  // whole block beyond the alive range

    // +0 known only at run time: the element products fma(a, b, z0) round as
    // a * b (but for the sign of an exact zero, which no loss test or later
    // non-zero value depends on) and issue at the DFMA rate
    const double z0 = a.zero;
    Tile<P> q;
    bool alive[P];
    double iP[P];
    bool dirty = true;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int64_t i = base + (int64_t)p * blockDim.x + threadIdx.x;
        alive[p] = false;
        iP[p] = 1.0;
        q.x[p] = q.xp[p] = q.y[p] = q.yp[p] = q.l[p] = q.d[p] = 0.0;
        if (i < n_alive && a.loss_turn[i] < 0) {
            alive[p] = true;
            q.x[p] = a.coords[i];
            q.xp[p] = a.coords[a.pitch + i];
            q.y[p] = a.coords[2 * a.pitch + i];
            q.yp[p] = a.coords[3 * a.pitch + i];
            q.l[p] = a.coords[4 * a.pitch + i];
            q.d[p] = a.coords[5 * a.pitch + i];
        }
    }
    if (threadIdx.x == 0) cnt = 0;
    if (a.do_moments) tile_mean<P>(q, alive, sh, tot, K);

    const LatticeView &L = a.lat;
    const DevElem *__restrict__ elems = L.elems;
    int lost_here = 0;
    // Between consecutive kick-drift and exact-drift elements the tile keeps the
    // scaled canonical momenta qx = px/(1+delta) in q.xp, q.yp (x, y and l are
    // the same in both representations); slopes are restored for every other
    // element, the moments, loss records and the final store.
    bool canon = false;
    double p0 = a.p0c;  // reference momentum, identical in every thread
    int n_rf = 0;       // RF cavities passed (for the host's reciprocals)
    for (int t = 0; t < a.n_turns; ++t) {
        const int turn = a.turn_abs0 + t;
        if (a.kick_wake >= 0) {
            // Kicks of the collective element(s) that precede this segment, in
            // lattice order, each followed by the aperture test.
            wake_kick<P>(a, q, alive, p0, a.wake_V, a.wake_Vx, a.wake_nbins, 0);
            dirty = true;
            apply_aperture<P>(a, L, q, alive, base, turn, a.kick_wake, lost_here, canon);
            if (a.kick_wake2 >= 0) {
                wake_kick<P>(a, q, alive, p0, a.wake_V2, a.wake_Vx2, a.wake_nbins2, 1);
                apply_aperture<P>(a, L, q, alive, base, turn, a.kick_wake2, lost_here, canon);
            }
        }
        int type_next = a.e0 < a.e1 ? __ldg(&elems[a.e0].type) : 0;
        for (int e = a.e0; e < a.e1; ++e) {
            const DevElem *E = elems + e;
            const int type = type_next;   // loaded one element ahead
            if (e + 1 < a.e1) type_next = __ldg(&elems[e + 1].type);
            if (canon && type != TRK_EDRIFT && type != TRK_KQUAD && type != TRK_KSEXT) {
                v_to_slopes<P>(q);
                canon = false;
            }
            switch (type) {
            case TRK_MAP: v_map<P>(q, E, L.terms, L.row_mask, dirty); break;
            case TRK_EDRIFT:
                // x += L x', y += L y', l += L (sqrt(1 + x'^2 + y'^2) - 1); in scaled canonical
                // momenta x' = qx (1 + g) and sqrt(1 + x'^2 + y'^2) = 1 + g: the drift of the integrator
                if (canon)
                    v_drift<P>(q.x, q.y, q.l, q.xp, q.yp, __ldg(&E->p[0]), __ldg(&E->p[1]), __ldg(&E->p[2]),
                               __ldg(&E->p[0]) * 0.0);
                else
                    v_edrift<P>(q, __ldg(&E->p[0]), z0);
                break;
            case TRK_KQUAD:
            case TRK_KSEXT: v_kick_drift<P>(q, iP, dirty, canon, E); break;
            case TRK_THINSEXT: v_thin_sext<P>(q, E, z0); break;
            case TRK_SBEND: v_sbend<P>(q, E); break;
            case TRK_RFCA: {
                const double p01 = p0 + __ldg(&E->p[3]);
                // the host's reciprocal when it has one for this cavity (single-turn segments)
                const double ip01 = n_rf < a.n_rf_ip ? a.rf_ip[n_rf] : 1.0 / p01;
                ++n_rf;
                v_rfca<P>(q, E, p0, ip01, z0, dirty);
                p0 = p01;
                break;
            }
            default: break;
            }
            apply_aperture<P>(a, L, q, alive, base, turn, e, lost_here, canon);
        }
        if (a.do_moments && canon) {
            v_to_slopes<P>(q);
            canon = false;
        }
        if (a.do_moments)
            tile_moments<P>(q, alive, sh, tot, K,
                            a.partials + ((size_t)(a.local_turn0 + t) * a.n_tiles + tile) * kMomentsN);
    }

    if (a.minmax_slot >= 0) {
        // l window of the next wake over the alive particles.
        unsigned long long kmin = ~0ull, kmax = 0ull;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!alive[p]) continue;
            const unsigned long long k = dkey(q.l[p]);
            kmin = k < kmin ? k : kmin;
            kmax = k > kmax ? k : kmax;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a1 = __shfl_xor_sync(0xffffffffu, kmin, o);
            const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, kmax, o);
            kmin = a1 < kmin ? a1 : kmin;
            kmax = b1 > kmax ? b1 : kmax;
        }
        if (threadIdx.x == 0) {
            mm[0] = ~0ull;
            mm[1] = 0ull;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[0], kmin);
            atomicMax(&mm[1], kmax);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicMin((unsigned long long *)&a.win->key[2 * a.minmax_slot], mm[0]);
            atomicMax((unsigned long long *)&a.win->key[2 * a.minmax_slot + 1], mm[1]);
        }
    }

    if (canon) v_to_slopes<P>(q);
    int na = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!alive[p]) continue;
        const int64_t i = base + (int64_t)p * blockDim.x + threadIdx.x;
        store_particle<P>(a, i, q, p);
        ++na;
    }
    if (a.tile_alive) {
        na = __reduce_add_sync(0xffffffffu, na);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicAdd(&cnt, na);
        __syncthreads();
        if (threadIdx.x == 0) a.tile_alive[tile] = cnt;
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_track(TrackArgs a) {
    __shared__ TrackShared S;
    track_tile<P>(a, blockIdx.x, S);
}

// Batched form: block b tracks tile items[b].y of variant items[b].x with the
// arguments args[variant * n_chunks + chunk].
template <int P>
__global__ void __launch_bounds__(256) k_track_batch(const TrackArgs *__restrict__ args,
                                                      const int2 *__restrict__ items, int n_chunks, int chunk) {
    __shared__ TrackShared S;
    const int2 it = items[blockIdx.x];
    track_tile<P>(args[(size_t)it.x * n_chunks + chunk], it.y, S);
}

// ---------------------------------------------------- moments finalise ----
// Chan et al. pairwise merge of (n, mean, M2) partials in a fixed order.
struct Acc {
    double n, m[6], M[21];
};

__device__ __forceinline__ void acc_merge(Acc &a, const Acc &b) {
    if (b.n == 0.0) return;
    if (a.n == 0.0) {
        a = b;
        return;
    }
    const double n = a.n + b.n;
    const double fb = b.n / n, fab = a.n * b.n / n;
    double d[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        d[j] = b.m[j] - a.m[j];
        a.m[j] = fma(d[j], fb, a.m[j]);
    }
    int q = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int k = j; k < 6; ++k, ++q) a.M[q] = a.M[q] + b.M[q] + d[j] * d[k] * fab;
    a.n = n;
}

constexpr int kFinThreads = 128;

__device__ __forceinline__ void finalize_turn(const double *__restrict__ partials, int n_tiles, const BunchState *st,
                                              int tile, double *__restrict__ out, int t, Acc *sh) {
    const int64_t n_alive = st->n_alive;
    const int n_act = (int)((n_alive + tile - 1) / tile);
    Acc a;
    a.n = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) a.m[j] = 0.0;
#pragma unroll
    for (int q = 0; q < 21; ++q) a.M[q] = 0.0;
    for (int j = threadIdx.x; j < n_act; j += kFinThreads) {
        const double *p = partials + ((size_t)t * n_tiles + j) * kMomentsN;
        Acc b;
        b.n = p[0];
#pragma unroll
        for (int k = 0; k < 6; ++k) b.m[k] = p[1 + k];
#pragma unroll
        for (int q = 0; q < 21; ++q) b.M[q] = p[7 + q];
        acc_merge(a, b);
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = kFinThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            Acc x = sh[threadIdx.x];
            acc_merge(x, sh[threadIdx.x + s]);
            sh[threadIdx.x] = x;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const Acc &r = sh[0];
        double *o = out + (size_t)t * kMomentsN;
        o[0] = r.n;
        const double in = r.n > 0.0 ? 1.0 / r.n : 0.0;
        for (int j = 0; j < 6; ++j) o[1 + j] = r.n > 0.0 ? r.m[j] : 0.0;
        for (int q = 0; q < 21; ++q) o[7 + q] = r.M[q] * in;
    }
}

__global__ void __launch_bounds__(kFinThreads) k_moments_finalize(const double *__restrict__ partials, int n_tiles,
                                                                   const BunchState *st, int tile,
                                                                   double *__restrict__ out) {
    __shared__ Acc sh[kFinThreads];
    finalize_turn(partials, n_tiles, st, tile, out, blockIdx.x, sh);
}

// Batched: block (t, v) finalises turn t of variant v's chunk.
__global__ void __launch_bounds__(kFinThreads) k_moments_finalize_batch(const TrackArgs *__restrict__ args,
                                                                         int n_chunks, int chunk) {
    __shared__ Acc sh[kFinThreads];
    const TrackArgs &a = args[(size_t)blockIdx.y * n_chunks + chunk];
    if (!a.do_moments || (int)blockIdx.x >= a.n_turns) return;
    finalize_turn(a.partials, a.n_tiles, a.st, a.tile, a.mom_out, blockIdx.x, sh);
}

// ------------------------------------------------------------ compaction ----
constexpr int kScanThreads = 1024;

__device__ __forceinline__ void scan_tiles(const int32_t *__restrict__ tile_alive, int64_t *__restrict__ tile_off,
                                           int tile, BunchState *st, int64_t *wsum) {
    const int64_t n_alive = st->n_alive;
    const int n_act = (int)((n_alive + tile - 1) / tile);
    const int per = (n_act + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per, e = min(b + per, n_act);
    int64_t s = 0;
    for (int j = b; j < e; ++j) s += tile_alive[j];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t v = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int64_t off = inc - s + (w > 0 ? wsum[w - 1] : 0);
    for (int j = b; j < e; ++j) {
        tile_off[j] = off;
        off += tile_alive[j];
    }
    if (threadIdx.x == kScanThreads - 1) st->n_alive_next = off;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *__restrict__ tile_alive,
                                                              int64_t *__restrict__ tile_off, int tile,
                                                              BunchState *st) {
    __shared__ int64_t wsum[kScanThreads / 32];
    scan_tiles(tile_alive, tile_off, tile, st, wsum);
}

// Stable partition of one tile into the compaction buffers: alive particles to
// [tile_off, ...), lost ones after all survivors, in slot order.
__device__ __forceinline__ void scatter_tile(const CompactArgs &c, int tile, int *wcnt) {
    const BunchState *st = c.st;
    const int64_t n_alive = st->n_alive, n_next = st->n_alive_next;
    if (n_next == n_alive) return;  // nothing lost in this chunk
    const int T = blockDim.x;
    const int64_t base = (int64_t)tile * T;
    if (base >= n_alive) return;
    const int64_t i = base + threadIdx.x;
    const bool valid = i < n_alive;
    const bool al = valid && c.lt[i] < 0;
    const unsigned bal = __ballot_sync(0xffffffffu, al);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int j = 0; j < w; ++j) before += wcnt[j];
    const int rank = before + __popc(bal & ((1u << lane) - 1u));
    if (!valid) return;
    const int64_t toff = c.tile_off[tile];
    const int64_t dst = al ? toff + rank : n_next + (base - toff) + (threadIdx.x - rank);
    const int64_t pitch = c.pitch;
#pragma unroll
    for (int k = 0; k < 6; ++k) c.cb[k * pitch + dst] = c.coords[k * pitch + i];
    c.ib[dst] = c.ids[i];
    c.ltb[dst] = c.lt[i];
    c.leb[dst] = c.le[i];
}

__global__ void k_scatter(CompactArgs c) {
    __shared__ int wcnt[32];
    scatter_tile(c, blockIdx.x, wcnt);
}

__global__ void k_copyback(CompactArgs c) {
    const BunchState *st = c.st;
    const int64_t n_alive = st->n_alive;
    if (st->n_alive_next == n_alive) return;
    const int64_t pitch = c.pitch;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_alive;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) c.coords[k * pitch + i] = c.cb[k * pitch + i];
        c.ids[i] = c.ib[i];
        c.lt[i] = c.ltb[i];
        c.le[i] = c.leb[i];
    }
}

// Batched compaction: one scan block per variant; scatter and copy-back per
// (variant, tile) item; one commit thread per variant.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles_batch(const CompactArgs *__restrict__ cs) {
    __shared__ int64_t wsum[kScanThreads / 32];
    const CompactArgs &c = cs[blockIdx.x];
    scan_tiles(c.tile_alive, c.tile_off, c.tile, c.st, wsum);
}

__global__ void k_scatter_batch(const CompactArgs *__restrict__ cs, const int2 *__restrict__ items) {
    __shared__ int wcnt[32];
    const int2 it = items[blockIdx.x];
    scatter_tile(cs[it.x], it.y, wcnt);
}

__global__ void k_copyback_batch(const CompactArgs *__restrict__ cs, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.x];
    const CompactArgs &c = cs[it.x];
    const BunchState *st = c.st;
    const int64_t n_alive = st->n_alive;
    if (st->n_alive_next == n_alive) return;
    const int64_t i = (int64_t)it.y * blockDim.x + threadIdx.x;
    if (i >= n_alive) return;
    const int64_t pitch = c.pitch;
#pragma unroll
    for (int k = 0; k < 6; ++k) c.coords[k * pitch + i] = c.cb[k * pitch + i];
    c.ids[i] = c.ib[i];
    c.lt[i] = c.ltb[i];
    c.le[i] = c.leb[i];
}

__global__ void k_commit_batch(const CompactArgs *__restrict__ cs, int n_var) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n_var) cs[v].st->n_alive = cs[v].st->n_alive_next;
}

__global__ void k_commit(BunchState *st) { st->n_alive = st->n_alive_next; }

__global__ void k_init_bunch(BunchState *st, int32_t *lt, int32_t *le, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        lt[i] = -1;
        le[i] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->n_alive = n;
        st->n_alive_next = n;
        st->error = 0;
        for (int s = 0; s < 2; ++s) {
            st->win.key[2 * s] = ~0ull;
            st->win.key[2 * s + 1] = 0ull;
        }
    }
}

}  // namespace

cudaError_t launch_track(const TrackArgs &a, int block, int per_thread, int n_tiles, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    if (per_thread == 4)
        k_track<4><<<n_tiles, block, 0, s>>>(a);
    else if (per_thread == 2)
        k_track<2><<<n_tiles, block, 0, s>>>(a);
    else
        k_track<1><<<n_tiles, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_moments_finalize(const double *partials, int n_tiles, int n_turns, const BunchState *st, int tile,
                                    double *out, cudaStream_t s) {
    if (n_turns <= 0) return cudaSuccess;
    k_moments_finalize<<<n_turns, kFinThreads, 0, s>>>(partials, n_tiles, st, tile, out);
    return cudaGetLastError();
}

cudaError_t launch_compact(const CompactArgs &c, int n_tiles, cudaStream_t s) {
    k_scan_tiles<<<1, kScanThreads, 0, s>>>(c.tile_alive, c.tile_off, c.tile, c.st);
    k_scatter<<<n_tiles, c.tile, 0, s>>>(c);
    const int64_t n = (int64_t)n_tiles * c.tile;
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_copyback<<<grid, 256, 0, s>>>(c);
    k_commit<<<1, 1, 0, s>>>(c.st);
    return cudaGetLastError();
}

cudaError_t launch_batch_chunk(const TrackArgs *args, const CompactArgs *cargs, const int2 *items, int n_items,
                               int n_var, int n_chunks, int chunk, int block, int per_thread, int tile,
                               int max_turns, bool moments, cudaStream_t s) {
    if (n_items > 0) {
        if (per_thread == 4)
            k_track_batch<4><<<n_items, block, 0, s>>>(args, items, n_chunks, chunk);
        else if (per_thread == 2)
            k_track_batch<2><<<n_items, block, 0, s>>>(args, items, n_chunks, chunk);
        else
            k_track_batch<1><<<n_items, block, 0, s>>>(args, items, n_chunks, chunk);
    }
    if (moments && max_turns > 0)
        k_moments_finalize_batch<<<dim3(max_turns, n_var), kFinThreads, 0, s>>>(args, n_chunks, chunk);
    k_scan_tiles_batch<<<n_var, kScanThreads, 0, s>>>(cargs);
    if (n_items > 0) {
        k_scatter_batch<<<n_items, tile, 0, s>>>(cargs, items);
        k_copyback_batch<<<n_items, tile, 0, s>>>(cargs, items);
    }
    k_commit_batch<<<(n_var + 127) / 128, 128, 0, s>>>(cargs, n_var);
    return cudaGetLastError();
}

cudaError_t launch_init_bunch(BunchState *st, int32_t *lt, int32_t *le, int64_t n, cudaStream_t s) {
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    k_init_bunch<<<grid, 256, 0, s>>>(st, lt, le, n);
    return cudaGetLastError();
}

}  // namespace trk
