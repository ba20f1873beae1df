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

#include <cooperative_groups.h>

#include "trk_bins.cuh"
#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kHistThreads = 512;
constexpr int kSmemBins = 8192;      // sub-histograms in shared memory up to this many bins
constexpr int kHistUnroll = 4;      // particles per thread and step of the histogram
constexpr int kSubHists = 2;         // per block (one per half of the warps)
constexpr int kConvOut = 16;         // outputs per convolution block
constexpr int kConvThreads = 256;
constexpr int kLscThreads = 512;     // threads per CTA of the space-charge transform
constexpr int kLscClusterMinN = 1024; // transforms of at least this many points run on a cluster of 8 CTAs

namespace cg = cooperative_groups;

__global__ void k_wake_reset(BunchState *st, int slot, uint32_t *hist, unsigned long long *dip, int nbins,
                             int reset_keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x) {
        hist[i] = 0u;
        if (dip) dip[i] = dip[nbins + i] = 0ull;
    }
    if (reset_keys && blockIdx.x == 0 && threadIdx.x == 0) {
        st->win.key[2 * slot] = ~0ull;
        st->win.key[2 * slot + 1] = 0ull;
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
        atomicMin((unsigned long long *)&st->win.key[2 * slot], mm[0]);
        atomicMax((unsigned long long *)&st->win.key[2 * slot + 1], mm[1]);
    }
}

// A finite offset in fixed point (round to nearest); a non-finite one carries no
// dipole moment.
__device__ __forceinline__ unsigned long long dipole_units(double x) {
    return isfinite(x) ? (unsigned long long)__double2ll_rn(x * kDipoleScale) : 0ull;
}

// kDip: the transverse sums are taken (dip != NULL).
template <bool kDip>
__global__ void __launch_bounds__(kHistThreads, 2) k_wake_hist(const double *__restrict__ coords, int64_t pitch,
                                                             const int32_t *__restrict__ lt, const BunchState *st,
                                                             WakeWindow *win, int slot, int which, int nbins,
                                                             double w0, double sc,
                                                             uint32_t *__restrict__ hist, double *__restrict__ wfun,
                                                             double w0t, unsigned long long *__restrict__ dip,
                                                             double *__restrict__ wfun_t, int use_smem) {
    extern __shared__ __align__(8) unsigned char smem_raw[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw);
    const int64_t n = st->n_alive;
    const uint64_t kmin = win->key[2 * slot], kmax = win->key[2 * slot + 1];
    const bool any = kmin <= kmax;
    const double lmin = any ? dkey_inv(kmin) : 0.0;
    const double lmax = any ? dkey_inv(kmax) : 0.0;
    // the window's constants, once per block (a chain of divisions: computed by
    // every thread they kept the FP64 pipe busy for a third of the pass)
    __shared__ double s_dl, s_rdl;
    __shared__ long long s_m;
    __shared__ BinFast s_bf;
    if (threadIdx.x == 0) {
        const double d = (lmax - lmin) / nbins;
        s_dl = d;
        bin_consts(d, nbins, s_rdl, s_m);
        s_bf = bin_fast_consts(lmin, lmax, d, nbins);
        // 1/dl for the kick (0: no window or zero width, every particle takes bin 0's voltage)
        if (blockIdx.x == 0) win->idl[2 * slot + which] = (any && d > 0.0) ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const double dl = s_dl, rdl_s = s_rdl;
    const long long bin_m = s_m;
    const BinFast bf = s_bf;
    // wake function samples W(m dl) = w0 / sqrt(max(m dl, s_c))
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nbins; m += gridDim.x * blockDim.x) {
        const double s = (double)m * dl;
        const double r = sqrt(s > sc ? s : sc);
        wfun[m] = w0 / r;
        if (kDip) wfun_t[m] = w0t / r;
    }
    if (!any) return;
    const bool smem = use_smem != 0;
    // shared memory: kSubHists count sub-histograms (an even number of uint32
    // arrays, so the next byte is 8-aligned), then the transverse x and y sums
    unsigned long long *shd = reinterpret_cast<unsigned long long *>(smem_raw + kSubHists * nbins * sizeof(uint32_t));
    if (smem) {
        for (int i = threadIdx.x; i < kSubHists * nbins; i += blockDim.x) sh[i] = 0u;
        if (kDip)
            for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) shd[i] = 0ull;
        __syncthreads();
    }
    uint32_t *mine = sh + ((threadIdx.x >> 5) % kSubHists) * nbins;
    auto add = [&](double l, double x, double y) {
        const int b = bin_of_fast(l, bf, lmin, dl, rdl_s, bin_m, nbins);
        if (smem)
            atomicAdd(mine + b, 1u);
        else
            atomicAdd(hist + b, 1u);
        if (kDip) {
            const unsigned long long ux = dipole_units(x), uy = dipole_units(y);
            if (smem) {
                atomicAdd(shd + b, ux);
                atomicAdd(shd + nbins + b, uy);
            } else {
                atomicAdd(dip + b, ux);
                atomicAdd(dip + nbins + b, uy);
            }
        }
    };
    // U particles per thread and step, their loads issued together (the
    // counts are integers: the order of the additions does not matter)
    constexpr int U = kDip ? kHistUnroll / 2 : kHistUnroll;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < n; i += U * stride) {
        int32_t lv[U];
        double l[U], x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            lv[u] = lt[i + u * stride];
            l[u] = coords[4 * pitch + i + u * stride];
            x[u] = kDip ? coords[i + u * stride] : 0.0;
            y[u] = kDip ? coords[2 * pitch + i + u * stride] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (lv[u] < 0) add(l[u], x[u], y[u]);
    }
    for (; i < n; i += stride)
        if (lt[i] < 0) add(coords[4 * pitch + i], kDip ? coords[i] : 0.0, kDip ? coords[2 * pitch + i] : 0.0);
    if (smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
            uint32_t c = 0;
#pragma unroll
            for (int s = 0; s < kSubHists; ++s) c += sh[s * nbins + b];
            if (c) {
                atomicAdd(hist + b, c);
                if (kDip) {
                    atomicAdd(dip + b, shd[b]);
                    atomicAdd(dip + nbins + b, shd[nbins + b]);
                }
            }
        }
    }
}

// Sum over the block of every thread's kConvOut partial sums: the partials go to
// shared memory, then 16 lanes per output add 16 of them each and fold the 16
// results with four shuffles (20 adds per thread instead of five shuffle steps
// for each of the kConvOut sums).  Returns output t >> 4's sum in lanes with
// (t & 15) == 0.
static_assert(kConvThreads == 256 && kConvOut == 16, "reduction layout");
__device__ __forceinline__ double conv_block_sum(const double (&acc)[kConvOut], double *red) {
#pragma unroll
    for (int i = 0; i < kConvOut; ++i) red[i * kConvThreads + threadIdx.x] = acc[i];
    __syncthreads();
    const int o = threadIdx.x >> 4, p = threadIdx.x & 15;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kConvThreads / 16; ++q) s += red[o * kConvThreads + p + 16 * q];
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

// Output chunk c (kConvOut outputs) costs in proportion to c + 1, so block b
// takes chunks b and C - 1 - b (C chunks): every block does the same work.
__device__ __forceinline__ int conv_chunk(int pass, int nbins) {
    const int C = (nbins + kConvOut - 1) / kConvOut;
    const int c = pass == 0 ? (int)blockIdx.x : C - 1 - (int)blockIdx.x;
    return pass == 1 && c <= (int)blockIdx.x ? -1 : c;   // -1: no second chunk
}

int conv_blocks(int nbins) { return ((nbins + kConvOut - 1) / kConvOut + 1) / 2; }

// V_k = -q_m sum_{j <= k} h_j W((k - j) dl); a chunk of kConvOut outputs per
// pass, its source bins split over the block's threads.
__global__ void __launch_bounds__(kConvThreads) k_wake_conv(const uint32_t *__restrict__ hist,
                                                             const double *__restrict__ wfun, int nbins, double qm,
                                                             double *__restrict__ V) {
    __shared__ double red[kConvThreads * kConvOut];
    for (int pass = 0; pass < 2; ++pass) {
        const int c = conv_chunk(pass, nbins);
        if (c < 0) break;
        const int k0 = c * kConvOut;
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
        const double s = conv_block_sum(acc, red);
        const int o = threadIdx.x >> 4;
        if ((threadIdx.x & 15) == 0 && k0 + o < kend) V[k0 + o] = -qm * s;
        __syncthreads();   // red is reused by the second chunk
    }
}

// V_c[k] = q_m sum_{j <= k} D_c[j] W_T((k - j) dl), D in fixed point; chunks
// as k_wake_conv per coordinate (blockIdx.y = coordinate).
__global__ void __launch_bounds__(kConvThreads) k_wake_conv_t(const unsigned long long *__restrict__ dip,
                                                               const double *__restrict__ wfun_t, int nbins,
                                                               double qm, double *__restrict__ V) {
    __shared__ double red[kConvThreads * kConvOut];
    const unsigned long long *D = dip + (size_t)blockIdx.y * nbins;
    for (int pass = 0; pass < 2; ++pass) {
        const int c = conv_chunk(pass, nbins);
        if (c < 0) break;
        const int k0 = c * kConvOut;
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
        const double s = conv_block_sum(acc, red);
        const int o = threadIdx.x >> 4;
        if ((threadIdx.x & 15) == 0 && k0 + o < kend) V[(size_t)blockIdx.y * nbins + k0 + o] = qm * s;
        __syncthreads();
    }
}

// One block: line density, `passes` 1-2-1 smoothing passes, central
// difference; every operation rounded as written (no contraction), so the field
// is the oracle's on identical counts.
__global__ void __launch_bounds__(1024) k_lsc_field(const uint32_t *__restrict__ hist, const BunchState *st, int slot,
                                                    int nbins, double qm, double KL, int passes, double *a, double *b,
                                                    double *__restrict__ V) {
    const uint64_t kmin = st->win.key[2 * slot], kmax = st->win.key[2 * slot + 1];
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
// - 2 gamma_E; I1 = (x/2) sum_k t_k; terms stop below 1e-18 of the sum.  Above 2
// from K1(x) = int_0^inf exp(-x cosh t) cosh t dt (A&S 9.6.24) by the trapezoidal
// rule, step 1/8, exp(-x) factored out: sum_j exp(-x e_j) c_j with the node values
// e_j = cosh t_j - 1 = 2 sinh^2(t_j / 2), c_j = cosh t_j (t_j = j / 8) shared by all
// x (`nodes`, 2 kLscNodes doubles); for this entire integrand the rule's error
// stays at double rounding for every x > 2 at that step (checked against an
// independent K1 to x = 80).  Above x = 45, x K1(x) < 1e-18 and 1 - x K1 rounds to 1.
// The quadrature's nodes are split over a group of lanes (lsc_bracket_group).
constexpr int kLscNodes = 48;   // t up to 6: exp(-2 e_j) c_j < 1e-150 there
constexpr int kLscLanes = 8;    // lanes that share one impedance value's quadrature

// The series branch (x <= 2) of the bracket.
__device__ double lsc_series(double x) {
    const double q = 0.25 * x * x;
    double t = 1.0, harm = 0.0, sum_t = 1.0, sum_ct = 1.0 - 2.0 * kEulerGamma;
    for (int k = 1; k < 40; ++k) {
        t *= q / ((double)k * (double)(k + 1));
        harm += 1.0 / (double)k;
        sum_t += t;
        sum_ct += (2.0 * harm + 1.0 / (double)(k + 1) - 2.0 * kEulerGamma) * t;
        if (t < 1e-18 * sum_t) break;
    }
    return q * sum_ct - x * log(0.5 * x) * (0.5 * x * sum_t);
}

// The bracket evaluated by a group of kLscLanes lanes (lane j of the group, lane
// mask gm; every lane of the group calls it with the same x and gets the value):
// lane 0 takes the series, or the lanes split the quadrature nodes and add their
// partial sums with shuffles.
__device__ double lsc_bracket_group(double x, const double *nodes, int j, unsigned gm) {
    if (!(x > 0.0)) return 0.0;
    double acc;
    if (x <= 2.0) {
        acc = j == 0 ? lsc_series(x) : 0.0;
    } else {
        if (x > 45.0) return 1.0;
        acc = j == 0 ? 0.5 : 0.0;
        for (int k = 1 + j; k < kLscNodes; k += kLscLanes) acc += exp(-x * nodes[2 * k]) * nodes[2 * k + 1];
    }
#pragma unroll
    for (int o = kLscLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gm, acc, o);
    return x <= 2.0 ? acc : 1.0 - x * exp(-x) * (0.125 * acc);
}

// Cosine taper at f (fraction of Nyquist): 1 to f0, 0 from f1, f1 <= 0: none.
__device__ double lsc_taper(double f, double f0, double f1) {
    if (!(f1 > 0.0) || f <= f0) return 1.0;
    if (f >= f1) return 0.0;
    return 0.5 * (1.0 + cospi((f - f0) / (f1 - f0)));
}

// Bin width of slot `slot`'s window (the wake's): dl > 0 when the field is defined.
__device__ __forceinline__ double lsc_dl(const BunchState *st, int slot, int nbins) {
    const uint64_t kmin = st->win.key[2 * slot], kmax = st->win.key[2 * slot + 1];
    if (kmin > kmax) return 0.0;
    return (dkey_inv(kmax) - dkey_inv(kmin)) / nbins;
}

// Impedance and twiddle tables of one impedance space-charge pass, spread over the
// whole GPU, kLscLanes lanes per impedance value (the bracket's quadrature is the
// costly part): Z_m = i zs[m] for m = 0 .. N/2
// (zs[N - m] = -zs[m]; m = 0 and the Nyquist term carry no field),
// zs[m] = Z0 / (pi kappa r_b^2) (1 - xi K1(xi)) taper(m / (N/2)), kappa = 2 pi m / (N dl),
// xi = kappa r_b / gamma; tw[2j], tw[2j+1] = cos, sin of 2 pi j / N for j < N/2.
__global__ void k_lsc_tables(const BunchState *st, int slot, int nbins, int logn, double rb, double gamma, double f0,
                             double f1, double *__restrict__ zs, double *__restrict__ tw) {
    __shared__ double nodes[2 * kLscNodes];
    const int N = 1 << logn;
    const double dl = lsc_dl(st, slot, nbins);
    if (!(dl > 0.0) || nbins < 2) return;   // the transform kernel writes V = 0
    for (int j = threadIdx.x; j < kLscNodes; j += blockDim.x) {
        const double sh = sinh(0.0625 * (double)j);
        nodes[2 * j] = 2.0 * sh * sh;
        nodes[2 * j + 1] = cosh(0.125 * (double)j);
    }
    __syncthreads();
    // groups of kLscLanes consecutive lanes; the stride is a multiple of kLscLanes,
    // so a group stays together through the loop
    const int nz = N / 2 + 1;
    const unsigned gm = 0xFFu << ((threadIdx.x & 31) & ~(kLscLanes - 1));
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nz * kLscLanes; t += gridDim.x * blockDim.x) {
        const int i = t / kLscLanes, j = t % kLscLanes;
        if (i == 0 || 2 * i == N) {
            if (j == 0) zs[i] = 0.0;
            continue;
        }
        const double kap = 2.0 * kPi * (double)i / ((double)N * dl);
        const double B = lsc_bracket_group(kap * rb / gamma, nodes, j, gm);
        if (j == 0) zs[i] = kZ0 / (kPi * kap * rb * rb) * B * lsc_taper((double)i / (0.5 * (double)N), f0, f1);
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N / 2; j += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)j / (double)N, &sn, &cs);
        tw[2 * j] = cs;
        tw[2 * j + 1] = sn;
    }
}

// One radix-2 butterfly stage inside a CTA's own P points (all pairs local):
// decimation in time (forward, w applied to the second input) or in frequency
// (inverse, w applied to the difference).  x interleaved (re, im).
__device__ __forceinline__ void local_stage(double *x, const double *tws, int P, int s, int logn, bool dit,
                                            double wsign) {
    const int half = 1 << s;
    for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        const int pos = t & (half - 1);
        const int a = ((t >> s) << (s + 1)) | pos;
        const int b = a + half;
        const int j = pos << (logn - 1 - s);
        const double wr = tws[2 * j], wi = wsign * tws[2 * j + 1];
        const double ar = x[2 * a], ai = x[2 * a + 1], br = x[2 * b], bi = x[2 * b + 1];
        if (dit) {
            const double tr = wr * br - wi * bi, ti = wr * bi + wi * br;
            x[2 * a] = ar + tr;
            x[2 * a + 1] = ai + ti;
            x[2 * b] = ar - tr;
            x[2 * b + 1] = ai - ti;
        } else {
            const double dr = ar - br, di = ai - bi;
            x[2 * a] = ar + br;
            x[2 * a + 1] = ai + bi;
            x[2 * b] = wr * dr - wi * di;
            x[2 * b + 1] = wr * di + wi * dr;
        }
    }
    __syncthreads();
}

// Impedance space-charge field (TRK_LSC with r_b > 0) on a cluster of C CTAs
// (C = 1 or 8), each holding P = N / C of the N = 2 nbins points in shared memory:
// lambda_k = q_m h_k / dl zero-padded to N, loaded in bit-reversed order; forward
// transform by decimation in time (natural-order spectrum); times i zs[m];
// inverse by decimation in frequency (bit-reversed output, so no permutation
// pass); V_k = scale Re(.) with scale = L c / N, for k < nbins.  Stages whose
// butterflies span CTAs read the partner CTA's points through distributed shared
// memory into a second buffer, between cluster barriers; every CTA passes the
// same barriers (the stage loops depend on N and C only, and the degenerate exit
// is taken by all CTAs before the first barrier).
__global__ void __launch_bounds__(kLscThreads) k_lsc_fft(const uint32_t *__restrict__ hist, const BunchState *st,
                                                          int slot, int nbins, int logn, int logc, double qm,
                                                          double scale, const double *__restrict__ zs,
                                                          const double *__restrict__ tw, double *__restrict__ V) {
    extern __shared__ double sm[];
    const int N = 1 << logn, P = N >> logc, logp = logn - logc;
    cg::cluster_group cl = cg::this_cluster();
    const int c = logc > 0 ? (int)cl.block_rank() : 0;
    const double dl = lsc_dl(st, slot, nbins);
    if (!(dl > 0.0) || nbins < 2) {
        if (c == 0)
            for (int k = threadIdx.x; k < nbins; k += blockDim.x) V[k] = 0.0;
        return;
    }
    double *cur = sm, *nxt = sm + 2 * P, *tws = sm + 4 * P;
    for (int j = threadIdx.x; j < N; j += blockDim.x) tws[j] = tw[j];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int k = (int)(__brev((unsigned)(c * P + i)) >> (32 - logn));
        cur[2 * i] = k < nbins ? __ddiv_rn(__dmul_rn(qm, (double)hist[k]), dl) : 0.0;
        cur[2 * i + 1] = 0.0;
    }
    __syncthreads();
    // forward, decimation in time
    for (int s = 0; s < logn; ++s) {
        if (s < logp) {
            local_stage(cur, tws, P, s, logn, true, -1.0);
            continue;
        }
        const int half = 1 << s;
        cl.sync();
        const double *rem = cl.map_shared_rank(cur, c ^ (half >> logp));
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int g = c * P + i;
            const int j = (g & (half - 1)) << (logn - 1 - s);
            const double wr = tws[2 * j], wi = -tws[2 * j + 1];
            const double pr = rem[2 * i], pi = rem[2 * i + 1], orr = cur[2 * i], oi = cur[2 * i + 1];
            if (g & half) {   // second input: partner - w * own
                nxt[2 * i] = pr - (wr * orr - wi * oi);
                nxt[2 * i + 1] = pi - (wr * oi + wi * orr);
            } else {          // first input: own + w * partner
                nxt[2 * i] = orr + (wr * pr - wi * pi);
                nxt[2 * i + 1] = oi + (wr * pi + wi * pr);
            }
        }
        cl.sync();
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    // impedance: (a + i b)(i z) = -z b + i z a
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int m = c * P + i;
        const double z = 2 * m <= N ? zs[m] : -zs[N - m];
        const double a = cur[2 * i], b = cur[2 * i + 1];
        cur[2 * i] = -z * b;
        cur[2 * i + 1] = z * a;
    }
    __syncthreads();
    // inverse, decimation in frequency
    for (int s = logn - 1; s >= 0; --s) {
        if (s < logp) {
            local_stage(cur, tws, P, s, logn, false, 1.0);
            continue;
        }
        const int half = 1 << s;
        cl.sync();
        const double *rem = cl.map_shared_rank(cur, c ^ (half >> logp));
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int g = c * P + i;
            const int j = (g & (half - 1)) << (logn - 1 - s);
            const double wr = tws[2 * j], wi = tws[2 * j + 1];
            const double pr = rem[2 * i], pi = rem[2 * i + 1], orr = cur[2 * i], oi = cur[2 * i + 1];
            if (g & half) {   // second input: (partner - own) w
                const double dr = pr - orr, di = pi - oi;
                nxt[2 * i] = wr * dr - wi * di;
                nxt[2 * i + 1] = wr * di + wi * dr;
            } else {          // first input: own + partner
                nxt[2 * i] = orr + pr;
                nxt[2 * i + 1] = oi + pi;
            }
        }
        cl.sync();
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int k = (int)(__brev((unsigned)(c * P + i)) >> (32 - logn));
        if (k < nbins) V[k] = scale * cur[2 * i];
    }
}

int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_wake_reset(BunchState *st, int slot, uint32_t *hist, unsigned long long *dip, int nbins,
                              bool reset_keys, cudaStream_t s) {
    k_wake_reset<<<grid_for(nbins, 256, 64), 256, 0, s>>>(st, slot, hist, dip, nbins, reset_keys ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_wake_minmax(const double *coords, int64_t pitch, const int32_t *lt, BunchState *st, int slot,
                               int64_t n_max, cudaStream_t s) {
    k_wake_minmax<<<grid_for(n_max, 256, 152 * 8), 256, 0, s>>>(coords, pitch, lt, st, slot);
    return cudaGetLastError();
}

cudaError_t launch_wake_hist(const double *coords, int64_t pitch, const int32_t *lt, const BunchState *st,
                             WakeWindow *win, int slot, int which,
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
        cudaError_t e = cudaFuncSetAttribute(k_wake_hist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             most > plain ? most : plain);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_wake_hist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     most > plain ? most : plain);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int g = grid_for(n_max, kHistThreads, 152 * 2);
    const int gw = (nbins + kHistThreads - 1) / kHistThreads;
    if (g < gw) g = gw;
    if (dip)
        k_wake_hist<true><<<g, kHistThreads, smem, s>>>(coords, pitch, lt, st, win, slot, which, nbins, w0, sc, hist,
                                                        wfun, w0t, dip, wfun_t, smem_ok ? 1 : 0);
    else
        k_wake_hist<false><<<g, kHistThreads, smem, s>>>(coords, pitch, lt, st, win, slot, which, nbins, w0, sc, hist,
                                                         wfun, w0t, dip, wfun_t, smem_ok ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_lsc_field(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double KL,
                             int passes, double *a, double *b, double *V, cudaStream_t s) {
    k_lsc_field<<<1, 1024, 0, s>>>(hist, st, slot, nbins, qm, KL, passes, a, b, V);
    return cudaGetLastError();
}

cudaError_t launch_lsc_imp(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double L,
                           double rb, double gamma, double f0, double f1, double *scratch, double *V, cudaStream_t s) {
    if (nbins < 1 || nbins > kLscImpMaxBins || (nbins & (nbins - 1)) != 0) return cudaErrorInvalidValue;
    int logn = 1;
    while ((1 << logn) < 2 * nbins) ++logn;
    const int N = 1 << logn;
    const int logc = N >= kLscClusterMinN ? 3 : 0;
    const int P = N >> logc;
    double *zs = scratch, *tw = scratch + (N / 2 + 1);    // N/2 + 1 and N doubles
    const size_t smem = ((size_t)4 * P + (size_t)N) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        const int most = (int)((4 * (2 * kLscImpMaxBins) / 8 + 2 * kLscImpMaxBins) * sizeof(double));
        const int small = (int)((4 + 1) * (kLscClusterMinN - 1) * sizeof(double));
        cudaError_t e = cudaFuncSetAttribute(k_lsc_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             most > small ? most : small);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int tb = 128;   // a multiple of kLscLanes
    int grid = ((N / 2 + 1) * kLscLanes + tb - 1) / tb;
    if (grid > 152 * 4) grid = 152 * 4;
    k_lsc_tables<<<grid, tb, 0, s>>>(st, slot, nbins, logn, rb, gamma, f0, f1, zs, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1u << logc);
    cfg.blockDim = dim3(kLscThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1u << logc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_lsc_fft, hist, (const BunchState *)st, slot, nbins, logn, logc, qm,
                              L * kClight / (double)N, (const double *)zs, (const double *)tw, V);
}

cudaError_t launch_wake_conv_t(const unsigned long long *dip, const double *wfun_t, int nbins, double qm, double *V,
                               cudaStream_t s) {
    k_wake_conv_t<<<dim3(conv_blocks(nbins), 2), kConvThreads, 0, s>>>(dip, wfun_t, nbins, qm, V);
    return cudaGetLastError();
}

cudaError_t launch_wake_conv(const uint32_t *hist, const double *wfun, int nbins, double qm, double *V,
                             cudaStream_t s) {
    k_wake_conv<<<conv_blocks(nbins), kConvThreads, 0, s>>>(hist, wfun, nbins, qm, V);
    return cudaGetLastError();
}

}  // namespace trk
