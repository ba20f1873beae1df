// Dynamic-aperture survival scans on top of the batched tracker: particles are
// placed at (x0, 0, y0, 0, 0, 0), tracked through every variant's lattice, and
// the turn of each loss is turned into a survival count.
#include "trk_internal.cuh"

namespace trk {
namespace {

// Particles i < n of one variant's slice from points first + i.
__global__ void k_da_init(double *__restrict__ coords, int64_t pitch, int32_t *__restrict__ ids,
                          const double *__restrict__ x0, const double *__restrict__ y0, int64_t first, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        coords[i] = x0[first + i];
        coords[pitch + i] = 0.0;
        coords[2 * pitch + i] = y0[first + i];
        coords[3 * pitch + i] = 0.0;
        coords[4 * pitch + i] = 0.0;
        coords[5 * pitch + i] = 0.0;
        ids[i] = (int32_t)(first + i);
    }
}

__global__ void k_da_survival(const int32_t *__restrict__ ids, const int32_t *__restrict__ lt, int64_t n,
                              int32_t n_turns, int32_t *__restrict__ survival) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = lt[i];
        survival[ids[i]] = t >= 0 ? t + 1 : n_turns + 1;
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_da_init(double *coords, int64_t pitch, int32_t *ids, const double *x0, const double *y0,
                           int64_t first, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_da_init<<<grid_for(n), 256, 0, s>>>(coords, pitch, ids, x0, y0, first, n);
    return cudaGetLastError();
}

cudaError_t launch_da_survival(const int32_t *ids, const int32_t *lt, int64_t n, int32_t n_turns, int32_t *survival,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_da_survival<<<grid_for(n), 256, 0, s>>>(ids, lt, n, n_turns, survival);
    return cudaGetLastError();
}

}  // namespace trk
