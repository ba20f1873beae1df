// Wake path (Sec. 2.2 histogram, Sec. 2.3 convolution; Table 1 WAKE, TRWAKE):
// l-window by min/max over alive particles, privatised shared-memory histogram
// with an exact bin index, causal convolution with the wake function, and (in
// the tracking kernel) the interpolated energy kick.  With a transverse
// strength the same pass sums x and y per bin (the dipole moments), in 64-bit
// fixed point so that the sums do not depend on the order of the atomics, and
// two more convolutions give the transverse voltages for the slope kicks.
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
