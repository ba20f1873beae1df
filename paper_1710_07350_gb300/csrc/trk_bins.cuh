// Histogram bin index shared by the wake histograms (trk_wake.cu, trk_static.cu):
// the oracle's floor((l - lmin) / dl) bit for bit, without a division per particle.
#pragma once

#include <cmath>

namespace trk {
namespace {

// floor(a / dl) with the correctly rounded division, kept out of line: the
// histogram takes it only for quotients within a few units of rounding of an
// integer (and for NaN).
__device__ __noinline__ double floor_div_exact(double a, double dl) { return floor(__ddiv_rn(a, dl)); }

constexpr int kBinFracBits = 44;

// Bin of l: floor of the correctly rounded (l - lmin) / dl, clamped to the bins,
// without a division in the common case.  q = (l - lmin) * rdl (rdl = 1/dl rounded)
// is within 3 units of rounding of the rounded quotient, which is at most
// nbins + 1 < 2^17; scaled by 2^44 (rdl_s = rdl 2^44, an exact power-of-two
// scaling) and truncated to an integer, its top bits are floor(q) and its low 44
// bits q's fraction.  When the fraction is farther than m units (m 2^-44 >=
// (nbins + 2) 2^-49) from 0 and from 1, floor(q) is the floor of the rounded
// quotient; otherwise, and for NaN, the division decides.  Only the subtraction,
// one multiply and one conversion use the FP64 pipe.  Bit for bit the oracle's bin.
__device__ __forceinline__ int bin_of(double l, double lmin, double dl, double rdl_s, long long m, int nbins) {
    if (!(dl > 0.0)) return 0;
    const double a = __dsub_rn(l, lmin);
    const long long t = __double2ll_rd(__dmul_rn(a, rdl_s));
    const long long fr = t & ((1ll << kBinFracBits) - 1);
    if (t >= 0 && fr > m && fr < (1ll << kBinFracBits) - m) {
        const long long c = t >> kBinFracBits;
        return c > nbins - 1 ? nbins - 1 : (int)c;
    }
    const double u = floor_div_exact(a, dl);
    if (!(u >= 0.0)) return 0;
    if (u > (double)(nbins - 1)) return nbins - 1;
    return (int)u;
}

// Per-launch constants of bin_of; a scaled reciprocal that is not finite (dl
// below 2^-980) sends every particle to the division.
__device__ __forceinline__ void bin_consts(double dl, int nbins, double &rdl_s, long long &m) {
    rdl_s = dl > 0.0 ? (1.0 / dl) * 0x1p44 : 0.0;
    m = rdl_s < INFINITY ? (long long)((nbins + 2 + 31) / 32) + 1 : (1ll << 62);
}

// Integer estimate of the bin: L = trunc(l 2^F) from l's bit pattern (|L| <
// 2^62 for every l of the window, F = 62 - e with max(|lmin|, |lmax|) < 2^e),
// D = L - Lmin, D' = D >> s (s makes Lmax - Lmin fit 32 bits) and
// Q = D' R with R = trunc(2^(G + s - F) / dl) normalised into [2^31, 2^32):
// one 32 x 32 -> 64-bit product estimates (l - lmin) / dl in units of 2^-G of
// a bin.  In those units the truncations of L, Lmin and D cost below 3 R <
// 2^34, R's truncation below D' < 2^32, the rounding of R's quotient below
// 2^11, and the oracle's rounded difference and quotient are within 2^-52
// relative of the exact quotient, below 2^(G - 36) for up to 2^16 bins; so
// where Q's fraction is more than m = 2^35 + 2^(G - 35) units from 0 and from
// 1, floor(Q 2^-G) is the oracle's bin.  G must lie in [40, 63] (windows far
// narrower than 2^-30 of their magnitude leave it below and take the division).
struct BinFast {
    int F, s, G;
    uint32_t R;
    long long lmin_fix;
    unsigned long long m;
    bool on;
};

// trunc(l 2^F) from the bit pattern; `ok` false for inf/NaN or a value that
// does not fit (never for l inside the window the constants were made for).
__device__ __forceinline__ long long fix_of(double l, int F, bool &ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(l);
    const int ex = (int)((b >> 52) & 0x7FF);
    ok = ex != 0x7FF;
    unsigned long long mant = b & ((1ull << 52) - 1);
    int e = ex - 1075;                        // l = mant 2^e (with the hidden bit)
    if (ex) mant |= 1ull << 52;
    else e = -1074;
    const int sh = e + F;
    long long v;
    if (sh >= 0) {
        if (sh > 9) ok = false;               // 53 + 9 bits: no room left below 2^62
        v = (long long)(mant << (sh > 9 ? 0 : sh));
    } else {
        v = sh <= -64 ? 0 : (long long)(mant >> -sh);
    }
    return (b >> 63) ? -v : v;
}

// The constants of one window (computed once per block).
__device__ __forceinline__ BinFast bin_fast_consts(double lmin, double lmax, double dl, int nbins) {
    BinFast c;
    c.on = false;
    c.F = c.s = c.G = 0;
    c.R = 0;
    c.lmin_fix = 0;
    c.m = 0;
    if (!(dl > 0.0) || nbins > 65536) return c;
    const double big = fmax(fabs(lmin), fabs(lmax));
    if (!(big > 0.0) || !isfinite(big)) return c;
    int eb;
    frexp(big, &eb);                          // big < 2^eb
    c.F = 62 - eb;                            // |l| 2^F < 2^62
    bool ok0, ok1;
    c.lmin_fix = fix_of(lmin, c.F, ok0);
    const long long lmax_fix = fix_of(lmax, c.F, ok1);
    if (!ok0 || !ok1 || lmax_fix < c.lmin_fix) return c;
    const unsigned long long dmax = (unsigned long long)(lmax_fix - c.lmin_fix);
    const int bits = 64 - __clzll((long long)dmax);
    c.s = bits > 32 ? bits - 32 : 0;          // D' = D >> s < 2^32
    const double A = ldexp(1.0, c.s - c.F) / dl;
    if (!(A > 0.0) || !isfinite(A)) return c;
    int ea;
    const double fa = frexp(A, &ea);          // A = fa 2^ea, fa in [0.5, 1)
    c.G = 32 - ea;                            // R = fa 2^32 in [2^31, 2^32)
    if (c.G < 40 || c.G > 63) return c;
    c.R = (uint32_t)ldexp(fa, 32);
    c.m = (1ull << 35) + (1ull << (c.G - 35));
    c.on = true;
    return c;
}

// The oracle's bin of l: the integer estimate where it decides, else bin_of.
__device__ __forceinline__ int bin_of_fast(double l, const BinFast &c, double lmin, double dl, double rdl_s,
                                           long long m_exact, int nbins) {
    if (c.on) {
        bool ok;
        const long long L = fix_of(l, c.F, ok);
        const long long D = L - c.lmin_fix;
        if (ok && D >= 0) {
            const unsigned long long dp = (unsigned long long)D >> c.s;
            if ((dp >> 32) == 0) {
                const unsigned long long Q = (unsigned long long)(uint32_t)dp * (unsigned long long)c.R;
                const unsigned long long k = Q >> c.G;
                const unsigned long long fr = Q & ((1ull << c.G) - 1);
                if (k < (unsigned long long)nbins && fr > c.m && fr < (1ull << c.G) - c.m) return (int)k;
            }
        }
    }
    return bin_of(l, lmin, dl, rdl_s, m_exact, nbins);
}

}  // namespace
}  // namespace trk
