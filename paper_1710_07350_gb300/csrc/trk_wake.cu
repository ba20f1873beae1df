// Wake path (Sec. 2.2 histogram, Sec. 2.3 convolution; Table 1 WAKE, TRWAKE):
// l-window by min/max over alive particles, privatised shared-memory histogram
// with an exact bin index, causal convolution with the wake function, and (in
// the tracking kernel) the interpolated energy kick.  With a transverse
// strength the same pass sums x and y per bin (the dipole moments), in 64-bit
// fixed point so that the sums do not depend on the order of the atomics, and
// two more convolutions give the transverse voltages for the slope kicks.
// Longitudinal space charge (Table 1 LSCDRIFT) uses the same window and counts:
// either a smoothed derivative of the line density (long-wavelength limit) or
// the round-beam impedance applied with radix-2 transforms in shared memory.
#include <cmath>

#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kHistThreads = 512;
constexpr int kSmemBins = 8192;      // sub-histograms in shared memory up to this many bins
constexpr int kSubHists = 2;         // per block (one per half of the warps)
constexpr int kConvOut = 16;         // outputs per convolution block
constexpr int kConvThreads = 256;

__global__ void k_wake_reset(BunchState *st, int slot, uint32_t *hist, unsigned long long *dip, int nbins) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x) {
        hist[i] = 0u;
        if (dip) dip[i] = dip[nbins + i] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->lkey[2 * slot] = ~0ull;
        st->lkey[2 * slot + 1] = 0ull;
    }
}

__global__ void k_wake_minmax(const double *__restrict__ coords, int64_t pitch, const int32_t *__restrict__ lt,
                              BunchState *st, int slot) {
    __shared__ unsigned long long mm[2];
    const int64_t n = st->n_alive;
    unsigned long long kmin = ~0ull, kmax = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (lt[i] >= 0) continue;
        const unsigned long long k = dkey(coords[4 * pitch + i]);
        kmin = k < kmin ? k : kmin;
        kmax = k > kmax ? k : kmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
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
        atomicMin((unsigned long long *)&st->lkey[2 * slot], mm[0]);
        atomicMax((unsigned long long *)&st->lkey[2 * slot + 1], mm[1]);
    }
}

// Bin index exactly as floor((l - lmin) / dl) in IEEE double, clamped.
__device__ __forceinline__ int bin_of(double l, double lmin, double dl, int nbins) {
    if (!(dl > 0.0)) return 0;
    const double u = floor(__ddiv_rn(__dsub_rn(l, lmin), dl));
    if (!(u >= 0.0)) return 0;
    if (u > (double)(nbins - 1)) return nbins - 1;
    return (int)u;
}

// A finite offset in fixed point (round to nearest); a non-finite one carries no
// dipole moment.
__device__ __forceinline__ unsigned long long dipole_units(double x) {
    return isfinite(x) ? (unsigned long long)__double2ll_rn(x * kDipoleScale) : 0ull;
}

__global__ void __launch_bounds__(kHistThreads) k_wake_hist(const double *__restrict__ coords, int64_t pitch,
                                                             const int32_t *__restrict__ lt, const BunchState *st,
                                                             int slot, int nbins, double w0, double sc,
                                                             uint32_t *__restrict__ hist, double *__restrict__ wfun,
                                                             double w0t, unsigned long long *__restrict__ dip,
                                                             double *__restrict__ wfun_t, int use_smem) {
    extern __shared__ __align__(8) unsigned char smem_raw[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw);
    const int64_t n = st->n_alive;
    const uint64_t kmin = st->lkey[2 * slot], kmax = st->lkey[2 * slot + 1];
    const bool any = kmin <= kmax;
    const double lmin = any ? dkey_inv(kmin) : 0.0;
    const double lmax = any ? dkey_inv(kmax) : 0.0;
    const double dl = (lmax - lmin) / nbins;
    // wake function samples W(m dl) = w0 / sqrt(max(m dl, s_c))
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nbins; m += gridDim.x * blockDim.x) {
        const double s = (double)m * dl;
        const double r = sqrt(s > sc ? s : sc);
        wfun[m] = w0 / r;
        if (dip) wfun_t[m] = w0t / r;
    }
    if (!any) return;
    const bool smem = use_smem != 0;
    // shared memory: kSubHists count sub-histograms (an even number of uint32
    // arrays, so the next byte is 8-aligned), then the transverse x and y sums
    unsigned long long *shd = reinterpret_cast<unsigned long long *>(smem_raw + kSubHists * nbins * sizeof(uint32_t));
    if (smem) {
        for (int i = threadIdx.x; i < kSubHists * nbins; i += blockDim.x) sh[i] = 0u;
        if (dip)
            for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) shd[i] = 0ull;
        __syncthreads();
    }
    uint32_t *mine = sh + ((threadIdx.x >> 5) % kSubHists) * nbins;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (lt[i] >= 0) continue;
        const int b = bin_of(coords[4 * pitch + i], lmin, dl, nbins);
        if (smem)
            atomicAdd(mine + b, 1u);
        else
            atomicAdd(hist + b, 1u);
        if (dip) {
            const unsigned long long ux = dipole_units(coords[i]), uy = dipole_units(coords[2 * pitch + i]);
            if (smem) {
                atomicAdd(shd + b, ux);
                atomicAdd(shd + nbins + b, uy);
            } else {
                atomicAdd(dip + b, ux);
                atomicAdd(dip + nbins + b, uy);
            }
        }
    }
    if (smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
            uint32_t c = 0;
#pragma unroll
            for (int s = 0; s < kSubHists; ++s) c += sh[s * nbins + b];
            if (c) {
                atomicAdd(hist + b, c);
                if (dip) {
                    atomicAdd(dip + b, shd[b]);
                    atomicAdd(dip + nbins + b, shd[nbins + b]);
                }
            }
        }
    }
}

// V_k = -q_m sum_{j <= k} h_j W((k - j) dl); a block owns kConvOut outputs and
// its threads split the source bins.
__global__ void __launch_bounds__(kConvThreads) k_wake_conv(const uint32_t *__restrict__ hist,
                                                             const double *__restrict__ wfun, int nbins, double qm,
                                                             double *__restrict__ V) {
    __shared__ double sh[(kConvThreads / 32) * kConvOut];
    const int k0 = blockIdx.x * kConvOut;
    const int kend = min(k0 + kConvOut, nbins);
    double acc[kConvOut];
#pragma unroll
    for (int i = 0; i < kConvOut; ++i) acc[i] = 0.0;
    for (int j = threadIdx.x; j < kend; j += blockDim.x) {
        const uint32_t hj = __ldg(hist + j);
        if (hj == 0u) continue;
        const double h = (double)hj;
#pragma unroll
        for (int i = 0; i < kConvOut; ++i) {
            const int k = k0 + i;
            if (k >= j && k < kend) acc[i] = fma(h, __ldg(wfun + (k - j)), acc[i]);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kConvOut; ++i) {
        double s = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[w * kConvOut + i] = s;
    }
    __syncthreads();
    if (threadIdx.x < kConvOut && k0 + threadIdx.x < kend) {
        double s = 0.0;
        for (int j = 0; j < kConvThreads / 32; ++j) s += sh[j * kConvOut + threadIdx.x];
        V[k0 + threadIdx.x] = -qm * s;
    }
}

// V_c[k] = q_m sum_{j <= k} D_c[j] W_T((k - j) dl), D in fixed point; blocks of
// kConvOut outputs per coordinate (blockIdx.y = coordinate).
__global__ void __launch_bounds__(kConvThreads) k_wake_conv_t(const unsigned long long *__restrict__ dip,
                                                               const double *__restrict__ wfun_t, int nbins,
                                                               double qm, double *__restrict__ V) {
    __shared__ double sh[(kConvThreads / 32) * kConvOut];
    const unsigned long long *D = dip + (size_t)blockIdx.y * nbins;
    const int k0 = blockIdx.x * kConvOut;
    const int kend = min(k0 + kConvOut, nbins);
    double acc[kConvOut];
#pragma unroll
    for (int i = 0; i < kConvOut; ++i) acc[i] = 0.0;
    for (int j = threadIdx.x; j < kend; j += blockDim.x) {
        const long long dj = (long long)__ldg(D + j);
        if (dj == 0) continue;
        const double d = (double)dj * (1.0 / kDipoleScale);
#pragma unroll
        for (int i = 0; i < kConvOut; ++i) {
            const int k = k0 + i;
            if (k >= j && k < kend) acc[i] = fma(d, __ldg(wfun_t + (k - j)), acc[i]);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kConvOut; ++i) {
        double s = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[w * kConvOut + i] = s;
    }
    __syncthreads();
    if (threadIdx.x < kConvOut && k0 + threadIdx.x < kend) {
        double s = 0.0;
        for (int j = 0; j < kConvThreads / 32; ++j) s += sh[j * kConvOut + threadIdx.x];
        V[(size_t)blockIdx.y * nbins + k0 + threadIdx.x] = qm * s;
    }
}

// One block: line density, `passes` 1-2-1 smoothing passes, central
// difference; every operation rounded as written (no contraction), so the field
// is the oracle's on identical counts.
__global__ void __launch_bounds__(1024) k_lsc_field(const uint32_t *__restrict__ hist, const BunchState *st, int slot,
                                                    int nbins, double qm, double KL, int passes, double *a, double *b,
                                                    double *__restrict__ V) {
    const uint64_t kmin = st->lkey[2 * slot], kmax = st->lkey[2 * slot + 1];
    const bool any = kmin <= kmax;
    const double lmin = any ? dkey_inv(kmin) : 0.0;
    const double lmax = any ? dkey_inv(kmax) : 0.0;
    const double dl = (lmax - lmin) / nbins;
    if (!any || !(dl > 0.0) || nbins < 2) {
        for (int k = threadIdx.x; k < nbins; k += blockDim.x) V[k] = 0.0;
        return;
    }
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) a[k] = __ddiv_rn(__dmul_rn(qm, (double)hist[k]), dl);
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
            const double lo = a[k > 0 ? k - 1 : 0], hi = a[k < nbins - 1 ? k + 1 : nbins - 1];
            b[k] = __dmul_rn(__dadd_rn(__dadd_rn(lo, __dmul_rn(2.0, a[k])), hi), 0.25);
        }
        __syncthreads();
        double *t = a;
        a = b;
        b = t;
    }
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
        double d;
        if (k == 0) d = __ddiv_rn(__dsub_rn(a[1], a[0]), dl);
        else if (k == nbins - 1) d = __ddiv_rn(__dsub_rn(a[nbins - 1], a[nbins - 2]), dl);
        else d = __ddiv_rn(__dsub_rn(a[k + 1], a[k - 1]), __dmul_rn(2.0, dl));
        V[k] = __dmul_rn(KL, d);
    }
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kZ0 = 376.730313412;          // mu0 c [Ohm], CODATA 2018
constexpr double kEulerGamma = 0.57721566490153286061;
constexpr double kClight = 299792458.0;

// 1 - x K1(x), x >= 0.  Up to x = 2 from the ascending series of K1 and I1
// (Abramowitz & Stegun 9.6.11 and 9.6.10, order 1), written so that nothing
// cancels at small x:  1 - x K1 = -x ln(x/2) I1(x) + (x^2/4) sum_k c_k t_k with
// t_k = (x^2/4)^k / (k! (k+1)!) and c_k = psi(k+1) + psi(k+2) = 2 H_k + 1/(k+1)
// - 2 gamma_E; I1 = (x/2) sum_k t_k.  Above 2 from K1(x) = int_0^inf exp(-x cosh t)
// cosh t dt (A&S 9.6.24) by the trapezoidal rule, step 1/16 (exponentially
// accurate for this entire integrand), with exp(-x) factored out.
__device__ double lsc_bracket(double x) {
    if (!(x > 0.0)) return 0.0;
    if (x <= 2.0) {
        const double q = 0.25 * x * x;
        double t = 1.0, harm = 0.0, sum_t = 1.0, sum_ct = 1.0 - 2.0 * kEulerGamma;
        for (int k = 1; k < 40; ++k) {
            t *= q / ((double)k * (double)(k + 1));
            harm += 1.0 / (double)k;
            sum_t += t;
            sum_ct += (2.0 * harm + 1.0 / (double)(k + 1) - 2.0 * kEulerGamma) * t;
        }
        return q * sum_ct - x * log(0.5 * x) * (0.5 * x * sum_t);
    }
    const double h = 0.0625;
    double acc = 0.5;
    for (int j = 1; j < 100000; ++j) {   // cosh t - 1 = 2 sinh^2(t/2), t = j h
        const double sh = sinh(0.5 * (double)j * h);
        const double f = exp(-2.0 * x * sh * sh) * cosh((double)j * h);
        acc += f;
        if (f < 1e-18 * acc) break;
    }
    return 1.0 - x * exp(-x) * (h * acc);
}

// Cosine taper at f (fraction of Nyquist): 1 to f0, 0 from f1, f1 <= 0: none.
__device__ double lsc_taper(double f, double f0, double f1) {
    if (!(f1 > 0.0) || f <= f0) return 1.0;
    if (f >= f1) return 0.0;
    return 0.5 * (1.0 + cospi((f - f0) / (f1 - f0)));
}

// In-place radix-2 decimation-in-time transform of N = 2^logn complex values in
// shared memory: input in bit-reversed order, output in natural order,
// X_m = sum_k x_k exp(sign 2 pi i m k / N).  Twiddles from sincospi of exact
// dyadic arguments.  All threads of the block call it.
__device__ void fft_radix2(double *re, double *im, int logn, double sign) {
    const int N = 1 << logn;
    for (int st = 0; st < logn; ++st) {
        const int half = 1 << st;
        for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
            const int pos = i & (half - 1);
            const int a = ((i >> st) << (st + 1)) | pos;
            const int b = a + half;
            double sn, cs;
            sincospi(sign * (double)pos / (double)half, &sn, &cs);
            const double br = re[b], bi = im[b];
            const double tr = cs * br - sn * bi, ti = cs * bi + sn * br;
            const double ar = re[a], ai = im[a];
            re[a] = ar + tr;
            im[a] = ai + ti;
            re[b] = ar - tr;
            im[b] = ai - ti;
        }
        __syncthreads();
    }
}

// Impedance space-charge field (TRK_LSC with r_b > 0): lambda_k = q_m h_k / dl on
// the nbins bins, zero-padded to N = 2 nbins, forward transform, times
// Z_m = i sgn(m') Z0 / (pi kappa r_b^2) (1 - xi K1(xi)) taper (kappa = 2 pi |m'| / (N dl),
// xi = kappa r_b / gamma, m' the signed frequency index, 0 at m = 0 and at Nyquist),
// inverse transform, V_k = L c Re(.) / N for k < nbins.  One block; 16 N bytes of
// dynamic shared memory.
__global__ void __launch_bounds__(1024) k_lsc_imp(const uint32_t *__restrict__ hist, const BunchState *st, int slot,
                                                  int nbins, int logn, double qm, double L, double rb, double gamma,
                                                  double f0, double f1, double *__restrict__ V) {
    extern __shared__ double sm[];
    const int N = 1 << logn;
    double *re = sm, *im = sm + N;
    const uint64_t kmin = st->lkey[2 * slot], kmax = st->lkey[2 * slot + 1];
    const bool any = kmin <= kmax;
    const double lmin = any ? dkey_inv(kmin) : 0.0;
    const double lmax = any ? dkey_inv(kmax) : 0.0;
    const double dl = (lmax - lmin) / nbins;
    if (!any || !(dl > 0.0) || nbins < 2) {
        for (int k = threadIdx.x; k < nbins; k += blockDim.x) V[k] = 0.0;
        return;
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int j = (int)(__brev((unsigned)k) >> (32 - logn));
        re[j] = k < nbins ? __ddiv_rn(__dmul_rn(qm, (double)hist[k]), dl) : 0.0;
        im[j] = 0.0;
    }
    __syncthreads();
    fft_radix2(re, im, logn, -1.0);
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        const int mp = 2 * m < N ? m : m - N;
        double zs = 0.0;
        if (mp != 0 && 2 * m != N) {
            const double am = (double)(mp > 0 ? mp : -mp);
            const double kap = 2.0 * kPi * am / ((double)N * dl);
            const double z = kZ0 / (kPi * kap * rb * rb) * lsc_bracket(kap * rb / gamma) *
                             lsc_taper(am / (0.5 * (double)N), f0, f1);
            zs = mp > 0 ? z : -z;
        }
        const double a = re[m], b = im[m];
        re[m] = -zs * b;   // (a + i b)(i zs)
        im[m] = zs * a;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {   // back to bit-reversed order
        const int j = (int)(__brev((unsigned)k) >> (32 - logn));
        if (k < j) {
            const double tr = re[k], ti = im[k];
            re[k] = re[j];
            im[k] = im[j];
            re[j] = tr;
            im[j] = ti;
        }
    }
    __syncthreads();
    fft_radix2(re, im, logn, 1.0);
    const double scale = L * kClight;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) V[k] = scale * (re[k] / (double)N);
}

int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_wake_reset(BunchState *st, int slot, uint32_t *hist, unsigned long long *dip, int nbins,
                              cudaStream_t s) {
    k_wake_reset<<<grid_for(nbins, 256, 64), 256, 0, s>>>(st, slot, hist, dip, nbins);
    return cudaGetLastError();
}

cudaError_t launch_wake_minmax(const double *coords, int64_t pitch, const int32_t *lt, BunchState *st, int slot,
                               int64_t n_max, cudaStream_t s) {
    k_wake_minmax<<<grid_for(n_max, 256, 152 * 8), 256, 0, s>>>(coords, pitch, lt, st, slot);
    return cudaGetLastError();
}

cudaError_t launch_wake_hist(const double *coords, int64_t pitch, const int32_t *lt, BunchState *st, int slot,
                             int nbins, double w0, double sc, uint32_t *hist, double *wfun, double w0t,
                             unsigned long long *dip, double *wfun_t, int64_t n_max, cudaStream_t s) {
    // privatised sub-histograms up to kSmemBins bins, with the transverse sums up
    // to kSmemBins / 2 (96 KB per block at most); global atomics above
    const bool smem_ok = nbins <= kSmemBins && (!dip || nbins <= kSmemBins / 2);
    const size_t smem = smem_ok ? (size_t)kSubHists * nbins * sizeof(uint32_t) +
                                      (dip ? (size_t)2 * nbins * sizeof(unsigned long long) : 0)
                                : 0;
    static bool attr = false;
    if (!attr) {
        const int most = kSubHists * (kSmemBins / 2) * (int)sizeof(uint32_t) +
                         2 * (kSmemBins / 2) * (int)sizeof(unsigned long long);
        const int plain = kSubHists * kSmemBins * (int)sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(k_wake_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             most > plain ? most : plain);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int g = grid_for(n_max, kHistThreads, 152 * 2);
    const int gw = (nbins + kHistThreads - 1) / kHistThreads;
    if (g < gw) g = gw;
    k_wake_hist<<<g, kHistThreads, smem, s>>>(coords, pitch, lt, st, slot, nbins, w0, sc, hist, wfun, w0t, dip,
                                              wfun_t, smem_ok ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_lsc_field(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double KL,
                             int passes, double *a, double *b, double *V, cudaStream_t s) {
    k_lsc_field<<<1, 1024, 0, s>>>(hist, st, slot, nbins, qm, KL, passes, a, b, V);
    return cudaGetLastError();
}

cudaError_t launch_lsc_imp(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double L,
                           double rb, double gamma, double f0, double f1, double *V, cudaStream_t s) {
    if (nbins < 1 || nbins > kLscImpMaxBins || (nbins & (nbins - 1)) != 0) return cudaErrorInvalidValue;
    int logn = 1;
    while ((1 << logn) < 2 * nbins) ++logn;
    const size_t smem = (size_t)2 * (size_t)(1 << logn) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_lsc_imp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(2 * 2 * kLscImpMaxBins * sizeof(double)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_lsc_imp<<<1, 1024, smem, s>>>(hist, st, slot, nbins, logn, qm, L, rb, gamma, f0, f1, V);
    return cudaGetLastError();
}

cudaError_t launch_wake_conv_t(const unsigned long long *dip, const double *wfun_t, int nbins, double qm, double *V,
                               cudaStream_t s) {
    k_wake_conv_t<<<dim3((nbins + kConvOut - 1) / kConvOut, 2), kConvThreads, 0, s>>>(dip, wfun_t, nbins, qm, V);
    return cudaGetLastError();
}

cudaError_t launch_wake_conv(const uint32_t *hist, const double *wfun, int nbins, double qm, double *V,
                             cudaStream_t s) {
    k_wake_conv<<<(nbins + kConvOut - 1) / kConvOut, kConvThreads, 0, s>>>(hist, wfun, nbins, qm, V);
    return cudaGetLastError();
}

}  // namespace trk
