// trk_wake_static: the standalone longitudinal wake without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a wake
// step: code that runs while another component owns the allocator (a memory
// pool that must not grow, a plug-in hosted by an application that forbids
// cudaMalloc after start-up), or a process whose device memory is already
// committed to other buffers.  This entry point takes the particles and the
// outputs from the caller and keeps its working arrays (l-window keys,
// histogram, wake-function samples, voltages) in one file-scope device array
// of fixed size, which every GPU that loads the library holds until the
// process exits.
//
// The device address of that array is obtained once per device, with the
// device current, by cudaGetSymbolAddress on the first call made on that
// device, and cached for the life of the process; make that first call before
// any stream capture, and do not use the library across a cudaDeviceReset (the
// cached address would then point at freed memory).  All calls share the
// array and it keeps the last call's contents, so each call clears what must
// start at zero; calls whose work overlaps on the GPU (different streams, or
// different host threads on one stream without ordering) race on it.
#include <cmath>
#include <mutex>
#include <string>

#include "trk_bins.cuh"
#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kStaticMaxBins = 16384;
// Layout in doubles: [0, 32) l-window keys (two uint64 used), then the histogram
// (kStaticMaxBins uint32 = kStaticMaxBins/2 doubles), wake-function samples and
// voltages (kStaticMaxBins doubles each).  Total 320.25 KiB.
constexpr int kKeysOff = 0;
constexpr int kHistOff = 32;
constexpr int kWfunOff = kHistOff + kStaticMaxBins / 2;
constexpr int kVOff = kWfunOff + kStaticMaxBins;
constexpr int kScratchDoubles = kVOff + kStaticMaxBins;

static __device__ __align__(256) double g_wake_scratch[kScratchDoubles];

constexpr int kThreads = 256;
constexpr int kSmemBins = 8192;

__global__ void k_static_reset(double *scratch, int nbins) {
    uint64_t *keys = reinterpret_cast<uint64_t *>(scratch + kKeysOff);
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + kHistOff);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x) hist[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        keys[0] = ~0ull;
        keys[1] = 0ull;
    }
}

__global__ void k_static_minmax(const double *__restrict__ coords, int64_t pitch, int64_t n, double *scratch) {
    __shared__ unsigned long long mm[2];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch + kKeysOff);
    unsigned long long kmin = ~0ull, kmax = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
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
        atomicMin(&keys[0], mm[0]);
        atomicMax(&keys[1], mm[1]);
    }
}

__device__ __forceinline__ void window(const double *scratch, int nbins, double &lmin, double &dl, bool &any) {
    const uint64_t *keys = reinterpret_cast<const uint64_t *>(scratch + kKeysOff);
    const uint64_t kmin = keys[0], kmax = keys[1];
    any = kmin <= kmax;
    lmin = any ? dkey_inv(kmin) : 0.0;
    const double lmax = any ? dkey_inv(kmax) : 0.0;
    dl = (lmax - lmin) / nbins;
}

__global__ void __launch_bounds__(kThreads) k_static_hist(const double *__restrict__ coords, int64_t pitch, int64_t n,
                                                           int nbins, double w0, double sc, double *scratch) {
    __shared__ uint32_t sh[kSmemBins];
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + kHistOff);
    double *wfun = scratch + kWfunOff;
    double lmin, dl;
    bool any;
    window(scratch, nbins, lmin, dl, any);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nbins; m += gridDim.x * blockDim.x) {
        const double s = (double)m * dl;
        wfun[m] = w0 / sqrt(s > sc ? s : sc);
    }
    if (!any) return;
    const bool smem = nbins <= kSmemBins;
    if (smem) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0u;
        __syncthreads();
    }
    double rdl_s;
    long long bin_m;
    bin_consts(dl, nbins, rdl_s, bin_m);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin_of(coords[4 * pitch + i], lmin, dl, rdl_s, bin_m, nbins);
        if (smem)
            atomicAdd(sh + b, 1u);
        else
            atomicAdd(hist + b, 1u);
    }
    if (smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (sh[b]) atomicAdd(hist + b, sh[b]);
    }
}

__global__ void k_static_kick(double *__restrict__ coords, int64_t pitch, int64_t n, int nbins, double p0c,
                              const double *scratch) {
    const double *V = scratch + kVOff;
    double lmin, dl;
    bool any;
    window(scratch, nbins, lmin, dl, any);
    if (!any) return;
    const bool flat = !(dl > 0.0);
    const double idl = flat ? 0.0 : 1.0 / dl;
    const double ip0 = 1.0 / p0c;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (flat) {
            v = V[0];
        } else {
            const double u = fma(coords[4 * pitch + i] - lmin, idl, -0.5);
            const double k0 = floor(u);
            if (!(k0 >= 0.0))
                v = V[0];
            else if (k0 >= (double)(nbins - 1))
                v = V[nbins - 1];
            else {
                const int k = (int)k0;
                v = fma(u - k0, V[k + 1] - V[k], V[k]);
            }
        }
        coords[5 * pitch + i] = fma(v, ip0, coords[5 * pitch + i]);
    }
}

int grid_for(int64_t n, int cap) {
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

// Device address of the scratch array on the current device (set up once).
static cudaError_t static_scratch(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_wake_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace trk

using namespace trk;

extern "C" trk_status trk_wake_static(double *d_coords, int64_t pitch, int64_t n, int32_t nbins, double w0,
                                      double sc, double charge, double p0c_ev, uint32_t *d_hist, double *d_volt,
                                      void *stream) {
    if (nbins < 1 || nbins > kStaticMaxBins)
        return set_error(TRK_EINVAL, "trk_wake_static: nbins must be 1.." + std::to_string(kStaticMaxBins));
    if (n < 0 || pitch < n || (n > 0 && !d_coords)) return set_error(TRK_EINVAL, "trk_wake_static: bad particle array");
    if (!(p0c_ev > 0.0)) return set_error(TRK_EINVAL, "trk_wake_static: p0c_ev must be > 0");
    double *scratch = nullptr;
    cudaError_t e = static_scratch(&scratch);
    if (e != cudaSuccess)
        return set_error(TRK_ECUDA, std::string("trk_wake_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    if (n == 0) return TRK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_static_reset<<<grid_for(nbins, 64), kThreads, 0, s>>>(scratch, nbins);
    k_static_minmax<<<grid_for(n, 152 * 8), kThreads, 0, s>>>(d_coords, pitch, n, scratch);
    const int gh = grid_for(n, 152 * 4) > (nbins + kThreads - 1) / kThreads ? grid_for(n, 152 * 4)
                                                                            : (nbins + kThreads - 1) / kThreads;
    k_static_hist<<<gh, kThreads, 0, s>>>(d_coords, pitch, n, nbins, w0, sc, scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + kHistOff);
    e = launch_wake_conv(hist, scratch + kWfunOff, nbins, charge / (double)n, scratch + kVOff, s);
    if (e == cudaSuccess) {
        k_static_kick<<<grid_for(n, 152 * 8), kThreads, 0, s>>>(d_coords, pitch, n, nbins, p0c_ev, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_hist)
        e = cudaMemcpyAsync(d_hist, hist, nbins * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_volt)
        e = cudaMemcpyAsync(d_volt, scratch + kVOff, nbins * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(TRK_ECUDA, std::string("trk_wake_static: ") + cudaGetErrorString(e));
    return TRK_OK;
}
