// FP64 issue-rate probe: the measured denominator beside the derived FP64 peak
// of the tracking roofline (no counterpart in the paper).
//
// Every thread runs kChains independent FMA chains v = fma(v, a, b) (a, b
// kernel arguments, so nothing folds); the grid holds 4 blocks of 256 threads
// per SM.  Rates are thread-level operations per second.
#include <string>

#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(256) k_probe(double *__restrict__ out, int iters, double a, double b) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) v[c] = fma(v[c], a, b);
            if (OP == 1) v[c] = v[c] * a;
            if (OP == 2) v[c] = v[c] + b;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
cudaError_t time_probe(double *buf, int grid, int iters, cudaStream_t s, double *ops_per_s) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    k_probe<OP><<<grid, 256, 0, s>>>(buf, 16, 0.9999999, 1e-7);  // warm-up
    cudaEventRecord(e0, s);
    k_probe<OP><<<grid, 256, 0, s>>>(buf, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ops_per_s = e == cudaSuccess && ms > 0.0f ? (double)grid * 256 * iters * kChains / (ms * 1e-3) : 0.0;
    return e;
}

}  // namespace
}  // namespace trk

using namespace trk;

extern "C" trk_status trk_probe_fp64(double *out, void *stream) {
    if (!out) return set_error(TRK_EINVAL, "trk_probe_fp64: NULL output");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 4 * nsm;
    double *buf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)grid * 256 * sizeof(double));
    cudaStream_t s = (cudaStream_t)stream;
    const int iters = 4000;
    if (e == cudaSuccess) e = time_probe<0>(buf, grid, iters, s, &out[0]);
    if (e == cudaSuccess) e = time_probe<1>(buf, grid, iters, s, &out[1]);
    if (e == cudaSuccess) e = time_probe<2>(buf, grid, iters, s, &out[2]);
    cudaFree(buf);
    if (e != cudaSuccess) return set_error(TRK_ECUDA, std::string("trk_probe_fp64: ") + cudaGetErrorString(e));
    return TRK_OK;
}
