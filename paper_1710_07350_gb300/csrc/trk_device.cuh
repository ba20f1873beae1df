// Per-particle device helpers shared by the tracking kernels (trk_track.cu) and
// the lane-parallel dynamic-aperture kernel (trk_da.cu), so that both take every
// branch and round every operation the same way.
#pragma once

#include <cmath>

#include "trk_internal.cuh"

namespace trk {
namespace {

// Series are used below 2^-14: the first dropped binomial term is then below
// 4e-18 relative.  v >= 0 (a sum of squares) or NaN, so the test is an integer
// compare of the high word (NaN fails it and takes the exact branch).
constexpr int kSeriesMaxHi = 0x3F100000;  // high word of 2^-14
// Below 2^-19 the cubic terms of the series are also below 2e-18 and dropped.
constexpr int kQuadMaxHi = 0x3EC00000;    // high word of 2^-19

__device__ __forceinline__ bool series_ok(double v) { return __double2hiint(v) < kSeriesMaxHi; }
__device__ __forceinline__ bool quad_ok(double v) { return __double2hiint(v) < kQuadMaxHi; }

// Exact fallbacks for arguments outside the series range.  They are kept out of
// line so that the compiler cannot if-convert them into the hot path (where they
// would execute for every particle); they run only when a particle needs them.
__device__ __noinline__ double rsqrt_exact(double s) { return rsqrt(s); }

__device__ __noinline__ double edrift_exact_g(double v) { return v / (sqrt(1.0 + v) + 1.0); }

__device__ __noinline__ bool ellipse_exact(double x, double y, double a, double b) {
    const double u = __ddiv_rn(x, a), v = __ddiv_rn(y, b);
    return __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)) <= 1.0;
}

// |x| as an unsigned integer: the bit pattern shifted left by one, so the sign
// bit drops out and every NaN, whatever its sign, compares above every finite
// value.  (A sign mask would not do: the compiler may turn it into a
// floating-point absolute value, which keeps the sign of a NaN on this GPU, so a
// NaN produced with its sign bit set compared as negative and stayed inside.)
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) << 1;
}

// Aperture test (Sec. 2.5 limit_amplitudes, RCOL, ECOL).  The rectangle is an
// integer compare of the abs_key of x, y with those of a, b (NaN is outside); the
// ellipse accepts the inner box |x| <= 0.7 a, |y| <= 0.7 b the same way
// ((0.7)^2 + (0.7)^2 < 1) and otherwise takes the exact test, rounded as
// (x/a)^2 + (y/b)^2 <= 1 in IEEE double.
__device__ __forceinline__ bool inside(double x, double y, const LatticeView &L) {
    if (L.ap_type == TRK_APERTURE_RECT) return (abs_key(x) <= L.ap_a_key) & (abs_key(y) <= L.ap_b_key);
    if (L.ap_type == TRK_APERTURE_ELLIPSE) {
        if ((abs_key(x) <= L.ap_ia_key) & (abs_key(y) <= L.ap_ib_key)) return true;
        return ellipse_exact(x, y, L.ap_a, L.ap_b);
    }
    return true;
}

// Exact drift on slopes (Table 1 EDRIFT): l += L (sqrt(1 + v) - 1), v = x'^2 + y'^2,
// as v (1/2 - v/8 + v^2/16 - 5 v^3/128) for v < 2^-14, the exact form otherwise.
__device__ __forceinline__ double edrift_g(double v) {
    double g = v * fma(v, fma(v, fma(v, -0.0390625, 0.0625), -0.125), 0.5);
    if (!series_ok(v)) g = edrift_exact_g(v);
    return g;
}

}  // namespace
}  // namespace trk
