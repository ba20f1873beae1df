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

}  // namespace
}  // namespace trk
