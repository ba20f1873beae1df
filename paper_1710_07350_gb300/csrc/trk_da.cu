// Dynamic-aperture survival scans on top of the batched tracker: particles are
// placed at (x0, 0, y0, 0, 0, 0), tracked through every variant's lattice, and
// the turn of each loss is turned into a survival count.
//
// For few particles the scan is bound by one particle's chain of dependent
// FP64 operations over all turns, not by throughput.  k_da_lanes then gives a
// particle 8 lanes: the six rows of a map are evaluated on six lanes at once
// and exchanged by warp shuffles; everything else runs replicated on every
// lane.  Each row sums its terms in the order, and with the operations, of the
// tracking kernel, so the survival turns are bit-identical.
//
// Both scans (this kernel and the batched tracker under trk_da_survival)
// evaluate only the map rows in the lattice's survival rows: the rows on which
// an aperture test depends, directly or through other rows (for a ring of maps
// and thin sextupoles without RF, every row but the path length).  A skipped
// row is never read by an evaluated one, so every loss decision is the one
// full tracking takes.
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

// q[j] for a runtime j by selects, so that q stays in registers.
__device__ __forceinline__ double sel6(const double (&q)[6], int j) {
    double v = q[0];
    v = j == 1 ? q[1] : v;
    v = j == 2 ? q[2] : v;
    v = j == 3 ? q[3] : v;
    v = j == 4 ? q[4] : v;
    v = j == 5 ? q[5] : v;
    return v;
}

// Particle i of the point list takes threads LANES i .. LANES i + LANES - 1; its
// variant is the v with offsets[v] <= i < offsets[v + 1].  Every lane of the
// group holds all six coordinates; lane r < min(6, LANES) sums row r of a map,
// and as many independent shuffles hand the new coordinates to the group.  Thin
// sextupoles, drifts and the aperture test run on every lane with the same
// operations (no exchange).  LANES = 4 serves views whose survival rows are
// among x, x', y, y' (rows 4 and 5 are then read by no evaluated row and keep
// their values); it halves the replicated work, which binds passes of a few
// thousand points.  Lattices hold MAP, EDRIFT and THINSEXT elements only
// (checked on the host).
template <int LANES>
__global__ void __launch_bounds__(256) k_da_lanes(const LatticeView *__restrict__ views, int n_var,
                                                  const int64_t *__restrict__ offsets,
                                                  const double *__restrict__ x0, const double *__restrict__ y0,
                                                  int64_t n, int32_t n_turns, double zero,
                                                  int32_t *__restrict__ survival) {
    static_assert(LANES == 4 || LANES == 8, "lane groups of 4 or 8");
    constexpr int kRows = LANES < 6 ? LANES : 6;   // map rows evaluated by the group
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
    if (i >= n) return;   // whole lane groups leave together
    const int r = threadIdx.x & (LANES - 1);
    const int g0 = (threadIdx.x & 31) & ~(LANES - 1);
    const unsigned gm = ((1u << LANES) - 1u) << g0;
    int lo = 0, hi = n_var;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid;
    }
    const LatticeView L = views[lo];
    double q[6] = {x0[i], 0.0, y0[i], 0.0, 0.0, 0.0};
    int32_t surv = n_turns + 1;
    bool alive = true;
    for (int turn = 0; alive && turn < n_turns; ++turn) {
        for (int e = 0; e < L.n_elem; ++e) {
            const DevElem *E = L.elems + e;
            // the record's first 48 bytes (type, n, term0, flags; row offsets; p[0], p[1])
            // in three independent loads, whatever the element needs of them
            const int4 hd = __ldg(reinterpret_cast<const int4 *>(E));
            const int4 rbv = __ldg(reinterpret_cast<const int4 *>(E->rb));
            const double2 pp = __ldg(reinterpret_cast<const double2 *>(E->p));
            const int type = hd.x;
            if (type == TRK_MAP) {
                const uint32_t flags = (uint32_t)hd.w;
                const int16_t *rb = reinterpret_cast<const int16_t *>(&rbv);
                const double2 *t = reinterpret_cast<const double2 *>(L.terms + hd.z);
                const int rr = r < kRows ? r : 0;
                const int kb = rb[rr], len = (r < kRows && ((L.row_mask >> rr) & 1u)) ? rb[rr + 1] - rb[rr] : 0;
                double acc = (r < kRows && ((flags >> rr) & 1u)) ? sel6(q, rr) : 0.0;
                // +0 at run time: fma(a, b, z0) rounds as a * b, as the tracking
                // kernel's map (whose z0 = p * 0.0 may be -0: only the sign of an
                // exact zero can differ, and no loss decision depends on it)
                const double z0 = zero;
                for (int k = 0; k < len; ++k) {
                    const double2 tv = __ldg(t + kb + k);
                    const int code = (int)(unsigned)(__double_as_longlong(tv.y) & 0xffffffffll);
                    const int deg = code & 3, j = (code >> 2) & 7, jk = (code >> 5) & 7, jl = (code >> 8) & 7;
                    double m = 1.0;
                    if (deg >= 1) m = sel6(q, j);
                    if (deg >= 2) m = fma(m, sel6(q, jk), z0);
                    if (deg >= 3) m = fma(m, sel6(q, jl), z0);
                    acc = fma(tv.x, m, acc);
                }
#pragma unroll
                for (int c = 0; c < kRows; ++c) q[c] = __shfl_sync(gm, acc, g0 + c);
            } else if (type == TRK_THINSEXT) {
                const double k2 = pp.x, hk = pp.y;
                const double x = q[0], y = q[2], z0 = zero;   // as the tracking kernel (see the map)
                q[1] = fma(-hk, fma(x, x, -fma(y, y, z0)), q[1]);
                q[3] = fma(k2, fma(x, y, z0), q[3]);
            } else if (type == TRK_EDRIFT) {
                const double Ld = pp.x;
                const double xp = q[1], yp = q[3];
                const double g = edrift_g(fma(xp, xp, yp * yp));
                q[0] = fma(Ld, xp, q[0]);
                q[2] = fma(Ld, yp, q[2]);
                q[4] = fma(Ld, g, q[4]);
            }
            if (!inside(q[0], q[2], L)) {
                surv = turn + 1;
                alive = false;
                break;
            }
        }
    }
    if (r == 0) survival[i] = surv;
}

// particles per block of k_da_lanes: 8 up to kLaneSmall points, 16 above
constexpr int kLaneSmall = 4096;

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
                            const double *y0, int64_t n, int32_t n_turns, int lanes, int32_t *survival,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (lanes != 4 && lanes != 8) return cudaErrorInvalidValue;
    // small blocks spread few particles over many SMs: each SM's L1 then holds
    // the records of fewer variants' lattices (measured: a 34-point pass over 34
    // variants 45 ms at 32 particles per block, 23 ms at 8; above a few thousand
    // points 16 per block keep more warps per SM in flight)
    const int per = n <= kLaneSmall ? 8 : 16;
    const unsigned grid = (unsigned)((n + per - 1) / per);
    if (lanes == 4)
        k_da_lanes<4><<<grid, 4 * per, 0, s>>>(views, n_var, offsets, x0, y0, n, n_turns, 0.0, survival);
    else
        k_da_lanes<8><<<grid, 8 * per, 0, s>>>(views, n_var, offsets, x0, y0, n, n_turns, 0.0, survival);
    return cudaGetLastError();
}

cudaError_t launch_da_survival(const int32_t *ids, const int32_t *lt, int64_t n, int32_t n_turns, int32_t *survival,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_da_survival<<<grid_for(n), 256, 0, s>>>(ids, lt, n, n_turns, survival);
    return cudaGetLastError();
}

}  // namespace trk
