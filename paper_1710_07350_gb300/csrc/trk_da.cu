// Dynamic-aperture survival scans on top of the batched tracker: particles are
// placed at (x0, 0, y0, 0, 0, 0), tracked through every variant's lattice, and
// the turn of each loss is turned into a survival count.
//
// For few particles the scan is bound by one particle's chain of dependent
// FP64 operations over all turns, not by throughput.  k_da_lanes then gives a
// particle 8 lanes, lane r holding coordinate r: the six rows of a map are
// evaluated on six lanes at once (coordinates exchanged by warp shuffles),
// thin sextupoles and drifts update their lanes, and every lane takes the same
// aperture decision.  Each row sums its terms in the order, and with the
// operations, of the tracking kernel, so the survival turns are bit-identical.
#include "trk_device.cuh"
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

// Particle i of the point list takes threads 8 i .. 8 i + 7; its variant is the
// v with offsets[v] <= i < offsets[v + 1].  Lattices hold MAP, EDRIFT and
// THINSEXT elements only (checked on the host).
__global__ void __launch_bounds__(256) k_da_lanes(const LatticeView *__restrict__ views, int n_var,
                                                  const int64_t *__restrict__ offsets,
                                                  const double *__restrict__ x0, const double *__restrict__ y0,
                                                  int64_t n, int32_t n_turns, int32_t *__restrict__ survival) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    if (i >= n) return;   // whole 8-lane groups leave together
    const int r = threadIdx.x & 7;
    const int g0 = (threadIdx.x & 31) & ~7;
    const unsigned gm = 0xFFu << g0;
    int lo = 0, hi = n_var;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid;
    }
    const LatticeView L = views[lo];
    double c = r == 0 ? x0[i] : (r == 2 ? y0[i] : 0.0);
    int32_t surv = n_turns + 1;
    bool alive = true;
    for (int turn = 0; alive && turn < n_turns; ++turn) {
        for (int e = 0; e < L.n_elem; ++e) {
            const DevElem *E = L.elems + e;
            const int type = __ldg(&E->type);
            if (type == TRK_MAP) {
                const uint32_t flags = __ldg(&E->flags);
                const int4 rbv = __ldg(reinterpret_cast<const int4 *>(E->rb));
                const int16_t *rb = reinterpret_cast<const int16_t *>(&rbv);
                const double2 *t = reinterpret_cast<const double2 *>(L.terms + __ldg(&E->term0));
                int nmax = 0;
#pragma unroll
                for (int q = 0; q < 6; ++q) nmax = rb[q + 1] - rb[q] > nmax ? rb[q + 1] - rb[q] : nmax;
                const int kb = r < 6 ? rb[r] : 0, len = r < 6 ? rb[r + 1] - rb[r] : 0;
                double acc = (r < 6 && ((flags >> r) & 1u)) ? c : 0.0;
                for (int k = 0; k < nmax; ++k) {
                    const bool on = k < len;
                    const double2 tv = on ? __ldg(t + kb + k) : make_double2(0.0, 0.0);
                    const int code = (int)(unsigned)(__double_as_longlong(tv.y) & 0xffffffffll);
                    const int deg = code & 3, j = (code >> 2) & 7, jk = (code >> 5) & 7, jl = (code >> 8) & 7;
                    const double v1 = __shfl_sync(gm, c, g0 + j);
                    const double v2 = __shfl_sync(gm, c, g0 + jk);
                    const double v3 = __shfl_sync(gm, c, g0 + jl);
                    double m = 1.0;
                    if (deg >= 1) m = v1;
                    if (deg >= 2) m *= v2;
                    if (deg >= 3) m *= v3;
                    if (on) acc = fma(tv.x, m, acc);
                }
                if (r < 6) c = acc;
            } else if (type == TRK_THINSEXT) {
                const double x = __shfl_sync(gm, c, g0), y = __shfl_sync(gm, c, g0 + 2);
                const double k2 = __ldg(&E->p[0]), hk = __ldg(&E->p[1]);
                if (r == 1) c = fma(-hk, (x - y) * (x + y), c);
                if (r == 3) c = fma(k2, x * y, c);
            } else if (type == TRK_EDRIFT) {
                const double xp = __shfl_sync(gm, c, g0 + 1), yp = __shfl_sync(gm, c, g0 + 3);
                const double Ld = __ldg(&E->p[0]);
                if (r == 0) c = fma(Ld, xp, c);
                if (r == 2) c = fma(Ld, yp, c);
                if (r == 4) c = fma(Ld, edrift_g(fma(xp, xp, yp * yp)), c);
            }
            const double x = __shfl_sync(gm, c, g0), y = __shfl_sync(gm, c, g0 + 2);
            if (!inside(x, y, L)) {
                surv = turn + 1;
                alive = false;
                break;
            }
        }
    }
    if (r == 0) survival[i] = surv;
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

cudaError_t launch_da_lanes(const LatticeView *views, int n_var, const int64_t *offsets, const double *x0,
                            const double *y0, int64_t n, int32_t n_turns, int32_t *survival, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = 8 * n;
    k_da_lanes<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(views, n_var, offsets, x0, y0, n, n_turns, survival);
    return cudaGetLastError();
}

cudaError_t launch_da_survival(const int32_t *ids, const int32_t *lt, int64_t n, int32_t n_turns, int32_t *survival,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_da_survival<<<grid_for(n), 256, 0, s>>>(ids, lt, n, n_turns, survival);
    return cudaGetLastError();
}

}  // namespace trk
