/*
 * trk_oracle.c -- plain, slow, single-threaded FP64 CPU tracker.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py load this library.  It shares
 * no code, header or table with the product library and is compiled with
 * -O2 -ffp-contract=off so every operation rounds exactly as written.
 *
 * What it computes (GPU acceleration of Elegant, arXiv:1710.07350):
 *   - the element-by-element particle loop of the paper's CPU listings
 *     (Sec. 2.1, exactDrift over double **part), kept array-of-structs;
 *   - transport maps up to third order (Sec. 1; Table 1 track_particles M1-M3):
 *       x_i <- C_i + sum_j R_ij x_j + sum_{j<=k} T_ijk x_j x_k
 *                  + sum_{j<=k<=l} U_ijkl x_j x_k x_l     (simultaneous update);
 *   - exact drift EDRIFT (Sec. 2.1 listings, path-length deviation stored);
 *   - kick-drift thick quadrupole / sextupole (Table 1 multipole_tracking2,
 *     Sec. 3 "canonical kick ... 4th order symplectic integration"):
 *     n steps of the 4th-order Yoshida scheme D K D K D K D, exact-Hamiltonian
 *     drifts, canonical momenta converted from / to slopes at entry / exit;
 *   - thin sextupole kick, thin RF cavity (Table 1 simple_rf_cavity, beta = 1);
 *   - global aperture after every element with particle loss (Sec. 2.5, Table 1
 *     limit_amplitudes / RCOL / ECOL); lost particles keep their coordinates
 *     at the loss point and the (turn, element) of the loss;
 *   - per-turn beam moments (Sec. 2.4, accumulate_beam_sums; compensated sums as
 *     the paper's USE_KAHAN option): n, 6 means, 21 central second moments;
 *   - longitudinal wake (Sec. 2.2-2.3, Table 1 WAKE): min/max of l, histogram,
 *     direct O(N^2) causal convolution with W(s) = W0/sqrt(max(s, s_c)),
 *     linearly interpolated energy kick;
 *   - transverse dipole wake on the same bins (Table 1 TRWAKE, the transverse
 *     half of RFCW): per-bin sums of x and y, convolution with
 *     W_T(s) = W0T/sqrt(max(s, s_c)), interpolated kicks on x' and y';
 *   - sector dipole (Table 1 CSBEND without gradient, fringe fields or
 *     radiation): the exact motion in a uniform vertical field, a circle of
 *     radius rho p_h in the horizontal plane (p_h = sqrt((1+delta)^2 - py^2)),
 *     followed to the exit face at angle theta;
 *   - longitudinal space charge (Table 1 LSCDRIFT) on the same histogram as a
 *     line density, either in the long-wavelength limit (impedance proportional
 *     to i k: smoothed by repeated 1-2-1 passes, differentiated, energy kick
 *     delta += K L (d lambda / d l)(l) / p0c) or with the impedance of a round,
 *     transversely uniform beam of radius r_b,
 *       Z(k) = i Z0 / (pi k r_b^2) (1 - xi K1(xi)),  xi = |k| r_b / gamma,
 *     applied by discrete Fourier transforms of the zero-padded line density.
 *
 * Coordinates: (x, x', y, y', l, delta), l the path-length deviation [m].
 * Lattice description: one row per element in three flat arrays
 *   ei[4*e + 0..3]  = type, order (MAP) or smoothing passes (LSC), n_kicks (KQUAD/KSEXT),
 *                     nbins (WAKE, LSC)
 *   ed[20*e + ...]  = see ED_* below
 *   em[504*e + ...] = C[6], R[36] (row-major), T[6*21], U[6*56] (MAP only)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_MAP = 1, O_EDRIFT = 2, O_KQUAD = 3, O_KSEXT = 4, O_THINSEXT = 5, O_RFCA = 6, O_WAKE = 7, O_LSC = 8,
       O_SBEND = 9 };
enum { O_AP_NONE = 0, O_AP_RECT = 1, O_AP_ELLIPSE = 2 };
enum { ED_LENGTH = 0, ED_K1 = 1, ED_K2 = 2, ED_VOLT = 3, ED_PHASE = 4, ED_FREQ = 5,
       ED_W0 = 6, ED_SC = 7, ED_CHARGE = 8, ED_K2L = 9, ED_W0T = 10, ED_KLSC = 11, ED_ANGLE = 12,
       ED_RB = 13, ED_MC2 = 14, ED_F0 = 15, ED_F1 = 16, ED_N = 20 };
#define EM_N 504
#define C_LIGHT 299792458.0
#define O_PI 3.14159265358979323846
#define O_EULER 0.57721566490153286061   /* Euler's constant */
#define O_Z0 376.730313412               /* impedance of free space mu0 c [Ohm], CODATA 2018 */

/* ---------------------------------------------------------------- maps ---- */

/* Dense plain definition of a polynomial map of order 1..3.  Monomial order:
 * (j,k) j<=k and (j,k,l) j<=k<=l, lexicographic. */
static void apply_map(double *z, const double *m, int order)
{
    const double *C = m, *R = m + 6, *T = m + 42, *U = m + 168;
    double in[6], out[6];
    memcpy(in, z, sizeof in);
    for (int i = 0; i < 6; ++i) {
        double acc = C[i];
        for (int j = 0; j < 6; ++j)
            acc += R[6 * i + j] * in[j];
        if (order >= 2) {
            int q = 0;
            for (int j = 0; j < 6; ++j)
                for (int k = j; k < 6; ++k, ++q)
                    acc += T[21 * i + q] * in[j] * in[k];
        }
        if (order >= 3) {
            int q = 0;
            for (int j = 0; j < 6; ++j)
                for (int k = j; k < 6; ++k)
                    for (int l = k; l < 6; ++l, ++q)
                        acc += U[56 * i + q] * in[j] * in[k] * in[l];
        }
        out[i] = acc;
    }
    memcpy(z, out, sizeof out);
}

/* ------------------------------------------------------- exact drift ---- */

/* The path-length deviation L (sqrt(1 + v) - 1), v = x'^2 + y'^2, is evaluated
 * as L v / (sqrt(1 + v) + 1): the same quantity without the cancellation that
 * would quantise an increment of ~1e-10 m to the 2.2e-16 spacing of doubles
 * near 1. */
static void exact_drift(double *z, double L)
{
    double xp = z[1], yp = z[3];
    double v = xp * xp + yp * yp;
    z[0] += L * xp;
    z[2] += L * yp;
    z[4] += L * (v / (sqrt(1.0 + v) + 1.0));
}

/* ------------------------------------------------ kick-drift multipoles ---- */

/* l += h (P/pz - 1), written as h (px^2 + py^2) / (pz (P + pz)) (since
 * P^2 - pz^2 = px^2 + py^2) to keep the small increment free of cancellation. */
static void drift_canonical(double *c, double h)
{
    double P = 1.0 + c[5];
    double p2 = c[1] * c[1] + c[3] * c[3];
    double pz = sqrt(P * P - p2);
    c[0] += h * c[1] / pz;
    c[2] += h * c[3] / pz;
    c[4] += h * (p2 / (pz * (P + pz)));
}

static void kick_canonical(double *c, double h, double k1, double k2)
{
    double x = c[0], y = c[2];
    if (k1 != 0.0) {
        c[1] -= k1 * h * x;
        c[3] += k1 * h * y;
    }
    if (k2 != 0.0) {
        c[1] -= 0.5 * k2 * h * (x * x - y * y);
        c[3] += k2 * h * x * y;
    }
}

/* 4th-order Yoshida: w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1 (= -2^(1/3) w1);
 * one step D(w1/2) K(w1) D((w0+w1)/2) K(w0) D((w0+w1)/2) K(w1) D(w1/2). */
static void thick_multipole(double *z, double L, double k1, double k2, int n)
{
    double w1 = 1.0 / (2.0 - cbrt(2.0));
    double w0 = 1.0 - 2.0 * w1;
    double h = L / n;
    double c[6];
    double P = 1.0 + z[5];
    double r = sqrt(1.0 + z[1] * z[1] + z[3] * z[3]);
    c[0] = z[0]; c[1] = P * z[1] / r;
    c[2] = z[2]; c[3] = P * z[3] / r;
    c[4] = z[4]; c[5] = z[5];
    for (int s = 0; s < n; ++s) {
        drift_canonical(c, 0.5 * w1 * h);
        kick_canonical(c, w1 * h, k1, k2);
        drift_canonical(c, 0.5 * (w0 + w1) * h);
        kick_canonical(c, w0 * h, k1, k2);
        drift_canonical(c, 0.5 * (w0 + w1) * h);
        kick_canonical(c, w1 * h, k1, k2);
        drift_canonical(c, 0.5 * w1 * h);
    }
    double pz = sqrt(P * P - c[1] * c[1] - c[3] * c[3]);
    z[0] = c[0]; z[1] = c[1] / pz;
    z[2] = c[2]; z[3] = c[3] / pz;
    z[4] = c[4];
}

static void thin_sext(double *z, double k2l)
{
    double x = z[0], y = z[2];
    z[1] -= 0.5 * k2l * (x * x - y * y);
    z[3] += k2l * x * y;
}

/* ------------------------------------------------------------------ RF ---- */

static void rfca(double *z, double volt, double phi, double k, double p0c, double p0c1)
{
    double P = (1.0 + z[5]) * p0c;
    double P1 = P + volt * cos(phi + k * z[4]);
    double s = P / P1;
    z[1] *= s;
    z[3] *= s;
    z[5] = P1 / p0c1 - 1.0;
}

/* ------------------------------------------------------------ aperture ---- */

/* Returns 1 if the particle is inside (edge counts as inside; NaN is outside).
 * *margin receives an estimate of the distance to the edge [m]. */
static int aperture_ok(const double *z, int type, double a, double b, double *margin)
{
    double x = z[0], y = z[2];
    if (type == O_AP_RECT) {
        double mx = a - fabs(x), my = b - fabs(y);
        *margin = mx < my ? mx : my;
        return fabs(x) <= a && fabs(y) <= b;
    }
    /* ellipse */
    double u = x / a, v = y / b;
    double rho = u * u + v * v;
    double gx = 2.0 * x / (a * a), gy = 2.0 * y / (b * b);
    double g = sqrt(gx * gx + gy * gy);
    *margin = g > 0.0 ? (1.0 - rho) / g : (a < b ? a : b);
    return rho <= 1.0;
}

/* ------------------------------------------------------------- moments ---- */

/* Neumaier's improved Kahan-Babuska summation. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* out[28] = n, 6 means, 21 population central second moments (j<=k),
 * two-pass over the alive particles.  No alive particle: all zero. */
void o_moments(const double *x, const uint8_t *alive, int64_t n, double *out)
{
    memset(out, 0, 28 * sizeof(double));
    int64_t na = 0;
    nsum s1[6];
    memset(s1, 0, sizeof s1);
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        ++na;
        for (int j = 0; j < 6; ++j) nsum_add(&s1[j], x[6 * i + j]);
    }
    out[0] = (double)na;
    if (na == 0) return;
    double m[6];
    for (int j = 0; j < 6; ++j) m[j] = nsum_get(&s1[j]) / (double)na;
    nsum s2[21];
    memset(s2, 0, sizeof s2);
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        double d[6];
        for (int j = 0; j < 6; ++j) d[j] = x[6 * i + j] - m[j];
        int q = 0;
        for (int j = 0; j < 6; ++j)
            for (int k = j; k < 6; ++k, ++q) nsum_add(&s2[q], d[j] * d[k]);
    }
    for (int j = 0; j < 6; ++j) out[1 + j] = m[j];
    for (int q = 0; q < 21; ++q) out[7 + q] = nsum_get(&s2[q]) / (double)na;
}

/* ---------------------------------------------------------- sector bend ---- */

/* Sector dipole of length L (along the reference arc) and angle theta, hard
 * edge: rho = L/theta, the reference circle centred at the origin, the
 * particle entering at radius rho + x with radial momentum px and tangential
 * momentum pz (canonical, in units of the reference momentum).  Its orbit is a
 * circle of radius rho p_h centred at C = (rho + x - rho pz, rho px); it leaves
 * through the ray at angle theta after turning by alpha = theta + beta with
 *   pz sin(beta) - px cos(beta) = (1 + x/rho - pz) sin(theta) - px cos(theta)
 * (the branch through beta = 0 for the reference particle).  Then
 *   x_f = |P_exit| - rho,  px_f = px cos(beta) - pz sin(beta),
 *   y_f = y + py rho alpha,  l += rho (1 + delta) alpha - L,
 * and slopes are restored with pz_f = sqrt((1+delta)^2 - px_f^2 - py^2).
 * theta == 0 is the exact drift. */
static void sbend(double *z, double L, double theta)
{
    if (theta == 0.0) {
        exact_drift(z, L);
        return;
    }
    const double rho = L / theta;
    const double d1 = 1.0 + z[5];
    const double r = sqrt(1.0 + z[1] * z[1] + z[3] * z[3]);
    const double px = z[1] * d1 / r, py = z[3] * d1 / r, pz = d1 / r;
    const double ph = sqrt(d1 * d1 - py * py);
    const double S = (1.0 + z[0] / rho - pz) * sin(theta) - px * cos(theta);
    const double beta = atan2(px, pz) + asin(S / ph);
    const double alpha = theta + beta;
    const double Cx = rho + z[0] - rho * pz, Cy = rho * px;
    const double Px = Cx + rho * (pz * cos(alpha) + px * sin(alpha));
    const double Py = Cy + rho * (pz * sin(alpha) - px * cos(alpha));
    const double pxf = px * cos(beta) - pz * sin(beta);
    const double pzf = sqrt(d1 * d1 - pxf * pxf - py * py);
    z[0] = sqrt(Px * Px + Py * Py) - rho;
    z[1] = pxf / pzf;
    z[2] = z[2] + py * rho * alpha;
    z[3] = py / pzf;
    z[4] = z[4] + (rho * d1 * alpha - L);
}

/* The sector bend alone on one particle (for the tests). */
void o_sbend(double *z, double L, double theta) { sbend(z, L, theta); }

/* ---------------------------------------------------------------- wake ---- */

/* A10 + A11: window [min l, max l] over alive particles, nb equal bins,
 * bin = clamp(floor((l - lmin)/dl), 0, nb-1).  If max == min, dl = 0 and every
 * particle is in bin 0.  Returns the number of alive particles. */
int64_t o_wake_hist(const double *x, const uint8_t *alive, int64_t n, int nb,
                    double *lmin_out, double *dl_out, int64_t *hist)
{
    double lmin = INFINITY, lmax = -INFINITY;
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        double l = x[6 * i + 4];
        if (l < lmin) lmin = l;
        if (l > lmax) lmax = l;
        ++na;
    }
    memset(hist, 0, (size_t)nb * sizeof(int64_t));
    if (na == 0) { *lmin_out = 0.0; *dl_out = 0.0; return 0; }
    double dl = (lmax - lmin) / nb;
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        int64_t b = 0;
        if (dl > 0.0) {
            b = (int64_t)floor((x[6 * i + 4] - lmin) / dl);
            if (b < 0) b = 0;
            if (b > nb - 1) b = nb - 1;
        }
        ++hist[b];
    }
    *lmin_out = lmin;
    *dl_out = dl;
    return na;
}

/* A12: V_k = -q_m sum_{j<=k} h_j W((k-j) dl),  W(s) = W0/sqrt(max(s, s_c)).
 * Direct O(nb^2), compensated sums. */
void o_wake_conv(const int64_t *hist, int nb, double dl, double w0, double sc, double qm, double *V)
{
    for (int k = 0; k < nb; ++k) {
        nsum acc = {0.0, 0.0};
        for (int j = 0; j <= k; ++j) {
            if (hist[j] == 0) continue;
            double s = (double)(k - j) * dl;
            double w = w0 / sqrt(s > sc ? s : sc);
            nsum_add(&acc, (double)hist[j] * w);
        }
        V[k] = -qm * nsum_get(&acc);
    }
}

/* Voltage seen at l: linear interpolation between bin centres, clamped to the
 * end bins.  dl == 0: V[0]. */
double o_wake_interp(const double *V, int nb, double lmin, double dl, double l)
{
    if (!(dl > 0.0)) return V[0];
    double u = (l - lmin) / dl - 0.5;
    double k0 = floor(u);
    if (k0 < 0.0) return V[0];
    if (k0 >= (double)(nb - 1)) return V[nb - 1];
    int k = (int)k0;
    double f = u - k0;
    return (1.0 - f) * V[k] + f * V[k + 1];
}

/* A13: delta += V(l)/p0c for every alive particle. */
void o_wake_kick(double *x, const uint8_t *alive, int64_t n, const double *V, int nb,
                 double lmin, double dl, double p0c)
{
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        x[6 * i + 5] += o_wake_interp(V, nb, lmin, dl, x[6 * i + 4]) / p0c;
    }
}

/* Transverse dipole sums on the bins of o_wake_hist: D[k] = sum of coordinate
 * c (0 = x, 2 = y) over the alive particles of bin k whose coordinate is finite
 * (a non-finite offset carries no dipole moment), compensated sums in particle
 * order. */
void o_wake_dipole(const double *x, const uint8_t *alive, int64_t n, int nb, double lmin, double dl, int c,
                   double *D)
{
    nsum *acc = (nsum *)calloc((size_t)nb, sizeof(nsum));
    for (int64_t i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        int64_t b = 0;
        if (dl > 0.0) {
            b = (int64_t)floor((x[6 * i + 4] - lmin) / dl);
            if (b < 0) b = 0;
            if (b > nb - 1) b = nb - 1;
        }
        if (isfinite(x[6 * i + c])) nsum_add(&acc[b], x[6 * i + c]);
    }
    for (int k = 0; k < nb; ++k) D[k] = nsum_get(&acc[k]);
    free(acc);
}

/* Transverse voltage: V_k = +q_m sum_{j<=k} D_j W_T((k-j) dl),
 * W_T(s) = W0T/sqrt(max(s, s_c)): a leading offset deflects the particles
 * behind it towards the same side.  Direct O(nb^2), compensated sums. */
void o_wake_conv_t(const double *D, int nb, double dl, double w0t, double sc, double qm, double *V)
{
    for (int k = 0; k < nb; ++k) {
        nsum acc = {0.0, 0.0};
        for (int j = 0; j <= k; ++j) {
            if (D[j] == 0.0) continue;
            double s = (double)(k - j) * dl;
            double w = w0t / sqrt(s > sc ? s : sc);
            nsum_add(&acc, D[j] * w);
        }
        V[k] = qm * nsum_get(&acc);
    }
}

/* Whole wake element; n_total sets the macro-particle charge q_m = Q/n_total.
 * With w0t != 0 the transverse kicks x' += Vx(l)/(p0c (1 + delta)),
 * y' += Vy(l)/(p0c (1 + delta)) come first (delta before the energy kick); all
 * voltages are computed from the particles entering the element.
 * hist_out / V_out / Vx_out / Vy_out (nb entries each) may be NULL. */
void o_wake2(double *x, const uint8_t *alive, int64_t n, int64_t n_total, int nb, double w0, double w0t,
             double sc, double charge, double p0c, int64_t *hist_out, double *V_out, double *Vx_out,
             double *Vy_out)
{
    int64_t *h = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
    double *V = (double *)calloc((size_t)nb, sizeof(double));
    double *Vx = (double *)calloc((size_t)nb, sizeof(double));
    double *Vy = (double *)calloc((size_t)nb, sizeof(double));
    double *D = (double *)malloc((size_t)nb * sizeof(double));
    double lmin, dl;
    int64_t na = o_wake_hist(x, alive, n, nb, &lmin, &dl, h);
    if (na > 0) {
        const double qm = charge / (double)n_total;
        o_wake_conv(h, nb, dl, w0, sc, qm, V);
        if (w0t != 0.0) {
            o_wake_dipole(x, alive, n, nb, lmin, dl, 0, D);
            o_wake_conv_t(D, nb, dl, w0t, sc, qm, Vx);
            o_wake_dipole(x, alive, n, nb, lmin, dl, 2, D);
            o_wake_conv_t(D, nb, dl, w0t, sc, qm, Vy);
            for (int64_t i = 0; i < n; ++i) {
                if (!alive[i]) continue;
                double *z = x + 6 * i;
                const double P = p0c * (1.0 + z[5]);
                z[1] += o_wake_interp(Vx, nb, lmin, dl, z[4]) / P;
                z[3] += o_wake_interp(Vy, nb, lmin, dl, z[4]) / P;
            }
        }
        o_wake_kick(x, alive, n, V, nb, lmin, dl, p0c);
    }
    if (hist_out) memcpy(hist_out, h, (size_t)nb * sizeof(int64_t));
    if (V_out) memcpy(V_out, V, (size_t)nb * sizeof(double));
    if (Vx_out) memcpy(Vx_out, Vx, (size_t)nb * sizeof(double));
    if (Vy_out) memcpy(Vy_out, Vy, (size_t)nb * sizeof(double));
    free(h);
    free(V);
    free(Vx);
    free(Vy);
    free(D);
}

/* The longitudinal wake alone (w0t = 0). */
void o_wake(double *x, const uint8_t *alive, int64_t n, int64_t n_total, int nb,
            double w0, double sc, double charge, double p0c, int64_t *hist_out, double *V_out)
{
    o_wake2(x, alive, n, n_total, nb, w0, 0.0, sc, charge, p0c, hist_out, V_out, NULL, NULL);
}

/* --------------------------------------------------- space charge ---- */

/* Field of the long-wavelength space charge on the bins of o_wake_hist:
 * lambda_k = q_m h_k / dl (C/m); `passes` times lambda_k <- (lambda_{k-1} +
 * 2 lambda_k + lambda_{k+1}) / 4 with the end bins repeated outside; then
 * d_k = (lambda_{k+1} - lambda_{k-1}) / (2 dl) inside, one-sided differences
 * at the two ends; V_k = KL d_k (V).  dl == 0 or nb == 1: V = 0. */
void o_lsc_field(const int64_t *hist, int nb, double dl, double qm, double KL, int passes, double *V)
{
    if (!(dl > 0.0) || nb < 2) {
        memset(V, 0, (size_t)nb * sizeof(double));
        return;
    }
    double *a = (double *)malloc((size_t)nb * sizeof(double));
    double *b = (double *)malloc((size_t)nb * sizeof(double));
    for (int k = 0; k < nb; ++k) a[k] = qm * (double)hist[k] / dl;
    for (int p = 0; p < passes; ++p) {
        for (int k = 0; k < nb; ++k) {
            double lo = a[k > 0 ? k - 1 : 0], hi = a[k < nb - 1 ? k + 1 : nb - 1];
            b[k] = (lo + 2.0 * a[k] + hi) / 4.0;
        }
        double *t = a;
        a = b;
        b = t;
    }
    for (int k = 0; k < nb; ++k) {
        double d;
        if (k == 0) d = (a[1] - a[0]) / dl;
        else if (k == nb - 1) d = (a[nb - 1] - a[nb - 2]) / dl;
        else d = (a[k + 1] - a[k - 1]) / (2.0 * dl);
        V[k] = KL * d;
    }
    free(a);
    free(b);
}

/* Whole space-charge element (a thin kick of effective length L);
 * hist_out / V_out may be NULL. */
void o_lsc(double *x, const uint8_t *alive, int64_t n, int64_t n_total, int nb, double KL, int passes,
           double charge, double p0c, int64_t *hist_out, double *V_out)
{
    int64_t *h = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
    double *V = (double *)calloc((size_t)nb, sizeof(double));
    double lmin, dl;
    int64_t na = o_wake_hist(x, alive, n, nb, &lmin, &dl, h);
    if (na > 0) {
        o_lsc_field(h, nb, dl, charge / (double)n_total, KL, passes, V);
        o_wake_kick(x, alive, n, V, nb, lmin, dl, p0c);
    }
    if (hist_out) memcpy(hist_out, h, (size_t)nb * sizeof(int64_t));
    if (V_out) memcpy(V_out, V, (size_t)nb * sizeof(double));
    free(h);
    free(V);
}

/* Bracket of the round-beam space-charge impedance, B(x) = 1 - x K1(x), x >= 0.
 * x <= 2: the power series of K1 (Abramowitz & Stegun 9.6.11, n = 1),
 *   x K1(x) = 1 + x ln(x/2) I1(x) - (x^2/4) S,
 *   I1(x) = (x/2) sum_k y^k / (k! (k+1)!),  S = sum_k (psi(k+1) + psi(k+2)) y^k / (k! (k+1)!),
 *   y = x^2/4, psi(k+1) = -gamma_E + H_k (H_k the harmonic numbers),
 * so B = -x ln(x/2) I1(x) + y S with no cancellation at small x.
 * x > 2: the integral K1(x) = int_0^inf exp(-x cosh t) cosh t dt (A&S 9.6.24) by the
 * trapezoidal rule with step 1/16, exp(-x) taken out (cosh t - 1 = 2 sinh^2(t/2));
 * for this entire integrand the rule's error falls like exp(-pi^2 / h), far below
 * double rounding.  Terms are added until one is below 1e-18 of the sum. */
double o_lsc_bracket(double x)
{
    if (!(x > 0.0)) return 0.0;
    if (x <= 2.0) {
        const double y = 0.25 * x * x;
        double term = 1.0, H = 0.0, si = 0.0, ss = 0.0;
        for (int k = 0; k < 40; ++k) {
            if (k > 0) {
                term = term * y / ((double)k * (double)(k + 1));
                H += 1.0 / (double)k;
            }
            const double psi = (H - O_EULER) + (H + 1.0 / (double)(k + 1) - O_EULER);
            si += term;
            ss += psi * term;
        }
        const double I1 = 0.5 * x * si;
        return -x * log(0.5 * x) * I1 + y * ss;
    }
    const double h = 1.0 / 16.0;
    double sum = 0.5;   /* t = 0 at half weight: exp(0) cosh(0) / 2 */
    for (int j = 1; j < 100000; ++j) {
        const double t = (double)j * h;
        const double sh = sinh(0.5 * t);
        const double f = exp(-x * (2.0 * sh * sh)) * cosh(t);
        sum += f;
        if (f < 1e-18 * sum) break;
    }
    return 1.0 - x * exp(-x) * (h * sum);
}

/* Cosine taper of the space-charge filter at f = |m'| / (N/2), a fraction of the
 * Nyquist frequency: 1 up to f0, (1 + cos(pi (f - f0) / (f1 - f0))) / 2 between,
 * 0 from f1 on; f1 <= 0: no filter. */
static double o_lsc_taper(double f, double f0, double f1)
{
    if (!(f1 > 0.0) || f <= f0) return 1.0;
    if (f >= f1) return 0.0;
    return 0.5 * (1.0 + cos(O_PI * (f - f0) / (f1 - f0)));
}

/* Impedance kick on a periodic line density lam[0..N) of bin width dl:
 *   Lambda_m = sum_k lam_k exp(-2 pi i m k / N),
 *   kappa_m = 2 pi m' / (N dl),  m' = m (m < N/2), m - N (m > N/2),
 *   Z_m = i sgn(m') Z0 / (pi |kappa_m| r_b^2) B(|kappa_m| r_b / gamma) taper(|m'| / (N/2)),
 *         Z_0 = 0 and, for even N, Z_{N/2} = 0 (no mean field; the Nyquist term has no sign),
 *   V_k = L c Re[(1/N) sum_m Z_m Lambda_m exp(+2 pi i m k / N)]   (V), all k < N.
 * With lambda in C/m, Z in Ohm/m and c in m/s, Z c lambda is a field in V/m.  Direct
 * transforms, phases from a table of 2 pi j / N (the index m k reduced modulo N),
 * compensated sums. */
void o_lsc_imp_apply(const double *lam, int N, double dl, double L, double rb, double gamma, double f0,
                     double f1, double *V)
{
    double *cs = (double *)malloc((size_t)N * sizeof(double));
    double *sn = (double *)malloc((size_t)N * sizeof(double));
    double *Zr = (double *)malloc((size_t)N * sizeof(double));
    double *Zi = (double *)malloc((size_t)N * sizeof(double));
    for (int j = 0; j < N; ++j) {
        cs[j] = cos(2.0 * O_PI * (double)j / (double)N);
        sn[j] = sin(2.0 * O_PI * (double)j / (double)N);
    }
    for (int m = 0; m < N; ++m) {
        /* Lambda_m */
        nsum re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int k = 0; k < N; ++k) {
            const int j = (int)(((int64_t)m * k) % N);
            nsum_add(&re, lam[k] * cs[j]);
            nsum_add(&im, -lam[k] * sn[j]);
        }
        const double Lr = nsum_get(&re), Li = nsum_get(&im);
        const int mp = 2 * m < N ? m : m - N;
        if (mp == 0 || 2 * m == N) {
            Zr[m] = Zi[m] = 0.0;
            continue;
        }
        const double kap = 2.0 * O_PI * fabs((double)mp) / ((double)N * dl);
        const double z = O_Z0 / (O_PI * kap * rb * rb) * o_lsc_bracket(kap * rb / gamma) *
                         o_lsc_taper(fabs((double)mp) / (0.5 * (double)N), f0, f1);
        const double zs = mp > 0 ? z : -z;   /* Z_m = i zs */
        Zr[m] = -zs * Li;                     /* (Lr + i Li) (i zs) */
        Zi[m] = zs * Lr;
    }
    for (int k = 0; k < N; ++k) {
        nsum acc = {0.0, 0.0};
        for (int m = 0; m < N; ++m) {
            const int j = (int)(((int64_t)m * k) % N);
            nsum_add(&acc, Zr[m] * cs[j]);    /* Re[(Zr + i Zi)(cos + i sin)] */
            nsum_add(&acc, -Zi[m] * sn[j]);
        }
        V[k] = L * C_LIGHT * (nsum_get(&acc) / (double)N);
    }
    free(cs);
    free(sn);
    free(Zr);
    free(Zi);
}

/* Impedance field on the bins of o_wake_hist: lambda_k = q_m h_k / dl, zero-padded
 * to N = 2 nb so that the periodic transform adds no field from a wrapped image of
 * the bunch; V_k for k < nb.  dl == 0 or nb == 1: V = 0. */
void o_lsc_imp_field(const int64_t *hist, int nb, double dl, double qm, double L, double rb, double gamma,
                     double f0, double f1, double *V)
{
    if (!(dl > 0.0) || nb < 2) {
        memset(V, 0, (size_t)nb * sizeof(double));
        return;
    }
    const int N = 2 * nb;
    double *lam = (double *)calloc((size_t)N, sizeof(double));
    double *W = (double *)malloc((size_t)N * sizeof(double));
    for (int k = 0; k < nb; ++k) lam[k] = qm * (double)hist[k] / dl;
    o_lsc_imp_apply(lam, N, dl, L, rb, gamma, f0, f1, W);
    memcpy(V, W, (size_t)nb * sizeof(double));
    free(lam);
    free(W);
}

/* Whole impedance space-charge element (a thin kick of effective length L) for a
 * particle of rest energy mc2 [eV]: gamma = sqrt(1 + (p0c / mc2)^2). */
void o_lsc_imp(double *x, const uint8_t *alive, int64_t n, int64_t n_total, int nb, double L, double rb,
               double mc2, double f0, double f1, double charge, double p0c, int64_t *hist_out, double *V_out)
{
    int64_t *h = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
    double *V = (double *)calloc((size_t)nb, sizeof(double));
    double lmin, dl;
    int64_t na = o_wake_hist(x, alive, n, nb, &lmin, &dl, h);
    if (na > 0) {
        const double r = p0c / mc2;
        o_lsc_imp_field(h, nb, dl, charge / (double)n_total, L, rb, sqrt(1.0 + r * r), f0, f1, V);
        o_wake_kick(x, alive, n, V, nb, lmin, dl, p0c);
    }
    if (hist_out) memcpy(hist_out, h, (size_t)nb * sizeof(int64_t));
    if (V_out) memcpy(V_out, V, (size_t)nb * sizeof(double));
    free(h);
    free(V);
}

/* ------------------------------------------------------------ tracking ---- */

/*
 * Track n particles (x: n x 6, AoS) for n_turns turns through ne elements.
 *   alive[i]      in/out, 1 = alive; lost particles are skipped.
 *   loss_turn[i]  out, absolute turn (turn0 + t) of the loss, -1 if alive
 *   loss_elem[i]  out, element index of the loss, -1 if alive
 *   margin[i]     in/out, running minimum of |distance to the aperture edge|
 *                 over all element exits checked so far (pass +inf initially)
 *   moments       out [n_turns][28] after each turn, or NULL
 *   p0c           in/out reference momentum [eV]
 *   n_total       particle count that sets the wake macro-charge
 * Returns the number of alive particles at the end.
 */
int64_t o_track(int ne, const int32_t *ei, const double *ed, const double *em,
                int ap_type, double ap_a, double ap_b,
                double *x, int64_t n, int64_t n_total, int n_turns, int turn0,
                uint8_t *alive, int32_t *loss_turn, int32_t *loss_elem, double *margin,
                double *moments, double *p0c)
{
    for (int t = 0; t < n_turns; ++t) {
        for (int e = 0; e < ne; ++e) {
            const int32_t *iv = ei + 4 * e;
            const double *dv = ed + ED_N * e;
            int type = iv[0];
            if (type == O_WAKE) {
                o_wake2(x, alive, n, n_total, iv[3], dv[ED_W0], dv[ED_W0T], dv[ED_SC], dv[ED_CHARGE], *p0c, NULL,
                        NULL, NULL, NULL);
            } else if (type == O_LSC && dv[ED_RB] > 0.0) {
                o_lsc_imp(x, alive, n, n_total, iv[3], dv[ED_LENGTH], dv[ED_RB], dv[ED_MC2], dv[ED_F0],
                          dv[ED_F1], dv[ED_CHARGE], *p0c, NULL, NULL);
            } else if (type == O_LSC) {
                o_lsc(x, alive, n, n_total, iv[3], dv[ED_KLSC] * dv[ED_LENGTH], iv[1], dv[ED_CHARGE], *p0c, NULL,
                      NULL);
            } else if (type == O_RFCA) {
                double phi = dv[ED_PHASE] * O_PI / 180.0;
                double k = 2.0 * O_PI * dv[ED_FREQ] / C_LIGHT;
                double p1 = *p0c + dv[ED_VOLT] * cos(phi);
                for (int64_t i = 0; i < n; ++i)
                    if (alive[i]) rfca(x + 6 * i, dv[ED_VOLT], phi, k, *p0c, p1);
                *p0c = p1;
            } else {
                for (int64_t i = 0; i < n; ++i) {
                    if (!alive[i]) continue;
                    double *z = x + 6 * i;
                    switch (type) {
                    case O_MAP: apply_map(z, em + (size_t)EM_N * e, iv[1]); break;
                    case O_EDRIFT: exact_drift(z, dv[ED_LENGTH]); break;
                    case O_KQUAD:
                    case O_KSEXT: thick_multipole(z, dv[ED_LENGTH], dv[ED_K1], dv[ED_K2], iv[2]); break;
                    case O_THINSEXT: thin_sext(z, dv[ED_K2L]); break;
                    case O_SBEND: sbend(z, dv[ED_LENGTH], dv[ED_ANGLE]); break;
                    default: break;
                    }
                }
            }
            if (ap_type != O_AP_NONE) {
                for (int64_t i = 0; i < n; ++i) {
                    if (!alive[i]) continue;
                    double m;
                    int ok = aperture_ok(x + 6 * i, ap_type, ap_a, ap_b, &m);
                    double am = fabs(m);
                    if (!(am >= margin[i])) margin[i] = am; /* NaN margin also recorded */
                    if (!ok) {
                        alive[i] = 0;
                        loss_turn[i] = turn0 + t;
                        loss_elem[i] = e;
                    }
                }
            }
        }
        if (moments) o_moments(x, alive, n, moments + 28 * (size_t)t);
    }
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) na += alive[i] ? 1 : 0;
    return na;
}
