// Surrogate-triaged dynamic-aperture scan (no counterpart in the paper).
//
// For every lattice variant and every cell of an nx x ny grid of initial
// amplitudes: track a coarse sub-grid exactly, train the MLP surrogate on those
// survival labels (features x/w, y/w and the variant's 6 normalised
// parameters), predict the survival mask of every cell, mark a band of cells
// within Chebyshev distance r of a predicted-boundary cell (a cell whose 8
// neighbours hold both classes) plus caller-chosen audit cells, re-track those
// exactly in FP64, and merge.  The band is then re-derived from the merged mask
// and the cells it newly reaches are tracked, until every cell within the band
// radius of the merged boundary is exact (the band follows the true boundary
// wherever the prediction misplaced it); later passes also take every cell
// within expand_radius of a cell whose label the last merge flipped.  Sentinel
// cells on a regular sub-lattice are tracked with the coarse cells, before any
// prediction: with sentinel stride <= 2 band_radius + 1 every
// (2 band_radius + 1)^2 block holds an exact cell, which is what makes the
// one-cell boundary criterion hold by construction (an untracked wrong cell two
// or more cells from the exhaustive boundary would need a whole uniform 5 x 5
// block without an exact cell).  With use_mlp = 0 the prediction is the label
// of the nearest known (coarse or sentinel) cell instead: the same pipeline
// without the network.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "trk_internal.cuh"

namespace trk {
namespace {

// Cell centre -w + (i + 1/2)(2w/n), rounded operation by operation (no FMA
// contraction) so that it equals the same expression evaluated on the host.
__device__ __forceinline__ double cell_centre(int i, int n, double w) {
    return __dadd_rn(-w, __dmul_rn(__dadd_rn((double)i, 0.5), __ddiv_rn(__dmul_rn(2.0, w), (double)n)));
}

// Known cells of every variant: cells[j] (j < per_v) is the j-th known cell of
// a variant -- the coarse cells first (row by row), then the sentinel cells.
// Points i = v * per_v + j.
__global__ void k_known_points(const int2 *__restrict__ cells, int per_v, int n_var, int nx, int ny, double w,
                               double *__restrict__ x0, double *__restrict__ y0) {
    const int64_t n = (int64_t)n_var * per_v;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 c = cells[i % per_v];
        x0[i] = cell_centre(c.x, nx, w);
        y0[i] = cell_centre(c.y, ny, w);
    }
}

// Training features and labels of the coarse cells (the first n_c known cells
// of each variant); feature row v * n_c + j.
__global__ void k_coarse_features(const double *__restrict__ x0, const double *__restrict__ y0,
                                  const int32_t *__restrict__ surv, const float *__restrict__ params, int n_c,
                                  int per_v, int n_var, double w, int32_t n_turns, float *__restrict__ X,
                                  float *__restrict__ y) {
    const int64_t n = (int64_t)n_c * n_var;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(k / n_c);
        const int64_t i = (int64_t)v * per_v + k % n_c;
        X[k * 8 + 0] = (float)(x0[i] / w);
        X[k * 8 + 1] = (float)(y0[i] / w);
        for (int q = 0; q < 6; ++q) X[k * 8 + 2 + q] = params[v * 6 + q];
        y[k] = surv[i] == n_turns + 1 ? 1.0f : 0.0f;
    }
}

// Features of cells [c0, c0 + m) of the full grid (cell = (v * ny + iy) * nx + ix).
__global__ void k_grid_features(int64_t c0, int64_t m, int nx, int ny, double w, const float *__restrict__ params,
                                float *__restrict__ X) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + i;
        const int ix = (int)(c % nx);
        const int iy = (int)((c / nx) % ny);
        const int v = (int)(c / ((int64_t)nx * ny));
        X[i * 8 + 0] = (float)(cell_centre(ix, nx, w) / w);
        X[i * 8 + 1] = (float)(cell_centre(iy, ny, w) / w);
        for (int k = 0; k < 6; ++k) X[i * 8 + 2 + k] = params[v * 6 + k];
    }
}

// Features of the listed cells idx[0, m).
__global__ void k_list_features(const int64_t *__restrict__ idx, int64_t m, int nx, int ny, double w,
                                const float *__restrict__ params, float *__restrict__ X) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx[i];
        const int ix = (int)(c % nx);
        const int iy = (int)((c / nx) % ny);
        const int v = (int)(c / ((int64_t)nx * ny));
        X[i * 8 + 0] = (float)(cell_centre(ix, nx, w) / w);
        X[i * 8 + 1] = (float)(cell_centre(iy, ny, w) / w);
        for (int k = 0; k < 6; ++k) X[i * 8 + 2 + k] = params[v * 6 + k];
    }
}

// The cells with bit 0 of region set, in any order (each cell's prediction
// depends on its own features only, so the order does not reach the mask); one
// atomic per warp and step (the warp's set lanes take consecutive slots).
__global__ void k_region_list(const uint8_t *__restrict__ region, int64_t n, int64_t *__restrict__ idx,
                              unsigned long long *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of steps (the bound is rounded up to whole warps)
    const int64_t n_up = (n + 31) / 32 * 32;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_up; c += stride) {
        const bool set = c < n && (region[c] & 1);
        const unsigned m = __ballot_sync(0xffffffffu, set);
        if (!m) continue;
        unsigned long long base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (set) idx[base + __popc(m & ((1u << lane) - 1u))] = c;
    }
}

__global__ void k_list_threshold(const int64_t *__restrict__ idx, const float *__restrict__ logit, int64_t m,
                                 uint8_t *__restrict__ mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        mask[idx[i]] = logit[i] > 0.0f ? 1 : 0;
}

__global__ void k_threshold(const float *__restrict__ logit, int64_t m, uint8_t *__restrict__ mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        mask[i] = logit[i] > 0.0f ? 1 : 0;
}

// Prediction without the network: label of the nearest known cell -- the
// nearest coarse cell (per axis j = (i - off + stride/2) / stride, clamped), or
// the nearest sentinel cell (per-axis tables nsx, nsy of sentinel indices,
// sx_n sentinels per row) where its squared index distance is strictly smaller.
__global__ void k_nearest_known(const int32_t *__restrict__ surv, const int2 *__restrict__ cells, int nx, int ny,
                                int stride, int off, int cx, int cy, int per_v, const int *__restrict__ nsx,
                                const int *__restrict__ nsy, int sx_n, int n_var, int32_t n_turns,
                                uint8_t *__restrict__ mask) {
    const int64_t n = (int64_t)n_var * nx * ny;
    const int n_c = cx * cy;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)((c / nx) % ny), v = (int)(c / ((int64_t)nx * ny));
        int jx = (ix - off + stride / 2) / stride, jy = (iy - off + stride / 2) / stride;
        if (ix < off) jx = 0;
        if (iy < off) jy = 0;
        jx = jx < cx - 1 ? jx : cx - 1;
        jy = jy < cy - 1 ? jy : cy - 1;
        int j = jy * cx + jx;
        if (per_v > n_c) {
            const int2 pc = cells[j];
            const int k = n_c + nsy[iy] * sx_n + nsx[ix];
            const int2 ps = cells[k];
            const int dc = (pc.x - ix) * (pc.x - ix) + (pc.y - iy) * (pc.y - iy);
            const int ds = (ps.x - ix) * (ps.x - ix) + (ps.y - iy) * (ps.y - iy);
            if (ds < dc) j = k;
        }
        mask[c] = surv[(int64_t)v * per_v + j] == n_turns + 1 ? 1 : 0;
    }
}

// Known labels override the prediction; their survival is exact.
__global__ void k_apply_known(const int32_t *__restrict__ surv, const int2 *__restrict__ cells, int per_v, int nx,
                              int ny, int n_var, int32_t n_turns, uint8_t *__restrict__ mask,
                              uint8_t *__restrict__ known, int32_t *__restrict__ out_surv) {
    const int64_t n = (int64_t)n_var * per_v;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / per_v);
        const int2 cl = cells[i % per_v];
        const int64_t c = ((int64_t)v * ny + cl.y) * nx + cl.x;
        const int32_t sv = surv[i];
        mask[c] = sv == n_turns + 1 ? 1 : 0;
        known[c] = 1;
        out_surv[c] = sv;
    }
}

// Boundary cells: the 8-neighbourhood (within the grid) holds both classes.
__global__ void k_boundary(const uint8_t *__restrict__ mask, int nx, int ny, int n_var, uint8_t *__restrict__ bnd) {
    const int64_t n = (int64_t)n_var * nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)((c / nx) % ny);
        const int64_t base = c - (int64_t)iy * nx - ix;
        int ones = 0, cnt = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int jx = ix + dx, jy = iy + dy;
                if (jx < 0 || jy < 0 || jx >= nx || jy >= ny) continue;
                ones += mask[base + (int64_t)jy * nx + jx];
                ++cnt;
            }
        bnd[c] = (ones > 0 && ones < cnt) ? 1 : 0;
    }
}

// Horizontal then vertical pass of two box dilations at once: bit 0 of the
// result = a boundary cell within Chebyshev distance r, bit 1 = a flipped cell
// within distance R (both limited to the variant's grid).
__global__ void k_dilate_x(const uint8_t *__restrict__ bnd, const uint8_t *__restrict__ flip, int nx, int ny,
                           int n_var, int r, int R, uint8_t *__restrict__ out) {
    const int64_t n = (int64_t)n_var * nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx);
        const int64_t row = c - ix;
        uint8_t b = 0;
        for (int jx = ix - r < 0 ? 0 : ix - r, je = ix + r < nx ? ix + r : nx - 1; jx <= je && !b; ++jx)
            b = bnd[row + jx] ? 1 : 0;
        if (flip)
            for (int jx = ix - R < 0 ? 0 : ix - R, je = ix + R < nx ? ix + R : nx - 1; jx <= je; ++jx)
                if (flip[row + jx]) {
                    b |= 2;
                    break;
                }
        out[c] = b;
    }
}
__global__ void k_dilate_y(const uint8_t *__restrict__ in, int nx, int ny, int n_var, int r, int R,
                           uint8_t *__restrict__ near) {
    const int64_t n = (int64_t)n_var * nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)((c / nx) % ny);
        const int64_t base = c - (int64_t)iy * nx;
        const int m = r > R ? r : R;
        uint8_t b = 0;
        for (int jy = iy - m < 0 ? 0 : iy - m, je = iy + m < ny ? iy + m : ny - 1; jy <= je && b != 3; ++jy) {
            const int d = jy > iy ? jy - iy : iy - jy;
            const uint8_t v = in[base + (int64_t)jy * nx];
            if (d <= r) b |= v & 1;
            if (d <= R) b |= v & 2;
        }
        near[c] = b;
    }
}

// Cells to re-track: near (a boundary cell within the band radius or a flipped
// cell within the expansion radius) or audit cells, and not already known.
__global__ void k_band(const uint8_t *__restrict__ near, const uint8_t *__restrict__ audit,
                       const uint8_t *__restrict__ known, int64_t n, uint8_t *__restrict__ todo,
                       uint8_t *__restrict__ is_audit) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool nr = near[c] != 0;
        const bool au = audit && audit[c] && !nr;
        todo[c] = (!known[c] && (nr || au)) ? 1 : 0;
        is_audit[c] = (!known[c] && au) ? 1 : 0;
    }
}

// Per-variant counts of cells to track (block per variant).
__global__ void k_count(const uint8_t *__restrict__ todo, int64_t per, int64_t *__restrict__ counts) {
    __shared__ int64_t sh[256];
    int64_t s = 0;
    const uint8_t *t = todo + (int64_t)blockIdx.x * per;
    for (int64_t i = threadIdx.x; i < per; i += blockDim.x) s += t[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = sh[0];
}

// Stable per-variant compaction of the cells to track into point lists (one
// block per variant, chunks of blockDim cells scanned in order).
__global__ void k_gather_todo(const uint8_t *__restrict__ todo, int64_t per, int nx, int ny, double w,
                              const int64_t *__restrict__ offsets, double *__restrict__ x0, double *__restrict__ y0,
                              int64_t *__restrict__ cell) {
    __shared__ int wsum[32];
    __shared__ int64_t running;
    const int v = blockIdx.x;
    const uint8_t *t = todo + (int64_t)v * per;
    if (threadIdx.x == 0) running = offsets[v];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c0 = 0; c0 < per; c0 += blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        const bool on = c < per && t[c];
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int j = 0; j < nw; ++j) {
            if (j < wid) before += wsum[j];
            total += wsum[j];
        }
        if (on) {
            const int64_t dst = running + before + __popc(bal & ((1u << lane) - 1u));
            const int ix = (int)(c % nx), iy = (int)(c / nx);
            x0[dst] = cell_centre(ix, nx, w);
            y0[dst] = cell_centre(iy, ny, w);
            cell[dst] = (int64_t)v * per + c;
        }
        __syncthreads();
        if (threadIdx.x == 0) running += total;
        __syncthreads();
    }
}

__global__ void k_merge(const int64_t *__restrict__ cell, const int32_t *__restrict__ surv, int64_t n,
                        int32_t n_turns, const uint8_t *__restrict__ is_audit, uint8_t *__restrict__ mask,
                        uint8_t *__restrict__ known, uint8_t *__restrict__ flip, int32_t *__restrict__ out_surv,
                        unsigned long long *__restrict__ wrong) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cell[i];
        const uint8_t m = surv[i] == n_turns + 1 ? 1 : 0;
        if (is_audit[c] && m != mask[c]) atomicAdd(wrong, 1ull);
        flip[c] = m != mask[c] ? 1 : 0;
        mask[c] = m;
        known[c] = 1;
        out_surv[c] = surv[i];
    }
}

// Cells never tracked: survival from the prediction.
__global__ void k_fill_predicted(const uint8_t *__restrict__ mask, const uint8_t *__restrict__ known, int64_t n,
                                 int32_t n_turns, int32_t *__restrict__ out_surv) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        if (!known[c]) out_surv[c] = mask[c] ? n_turns + 1 : 0;
}

constexpr int64_t kLaneCells = 16384;
constexpr int64_t kOnePerThreadCells = 1 << 20;   // band passes up to this size: one particle per thread

// Sentinel positions on an axis of n cells: off, off + stride, ... up to
// n - 1 - off, plus n - 1 - off itself (off = stride / 2), inside [0, n).
void sentinel_positions(int n, int stride, std::vector<int> &pos) {
    const int off = stride / 2, last = n - 1 - off;
    pos.clear();
    for (int p = off; p <= last; p += stride) pos.push_back(p);
    if (last >= 0 && last < n && (pos.empty() || pos.back() != last)) pos.push_back(last);
}

// For every cell of the axis the index of the closest position (the lower on a tie).
void nearest_positions(const std::vector<int> &pos, std::vector<int> &out) {
    for (int i = 0; i < (int)out.size(); ++i) {
        int best = 0;
        for (int k = 1; k < (int)pos.size(); ++k)
            if (std::abs(pos[k] - i) < std::abs(pos[best] - i)) best = k;
        out[i] = best;
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename T>
struct DBuf {
    T *p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, (n ? n : 1) * sizeof(T)); }
    void reset() {
        cudaFree(p);
        p = nullptr;
    }
    ~DBuf() { cudaFree(p); }
};

}  // namespace
}  // namespace trk

using namespace trk;

#define TRI_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return set_error(TRK_ECUDA, std::string("trk_da_triage: ") + #call + ": " + \
                                                               cudaGetErrorString(e_));                 \
    } while (0)

extern "C" trk_status trk_da_triage(const trk_lattice *const *lats, int32_t n_var, const float *d_params,
                                    const uint8_t *d_audit, trk_mlp *net, const int32_t *d_perm,
                                    const trk_triage_opts *o, uint8_t *d_mask, int32_t *d_survival,
                                    trk_triage_stats *stats, void *stream) {
    if (!lats || n_var < 1 || !d_params || !o || !d_mask || !d_survival)
        return set_error(TRK_EINVAL, "trk_da_triage: NULL argument");
    if (o->nx < 2 || o->ny < 2 || !(o->half_width > 0.0) || o->n_turns < 1 || o->coarse_stride < 1 ||
        o->band_radius < 0 || o->sentinel_stride < 0 || o->expand_radius < 0 ||
        (o->use_mlp && (!net || o->epochs < 1 || o->batch < 1)))
        return set_error(TRK_EINVAL, "trk_da_triage: bad options");
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = o->nx, ny = o->ny, st = o->coarse_stride, off = st / 2;
    const int cx = (nx - off + st - 1) / st, cy = (ny - off + st - 1) / st;
    const double w = o->half_width;
    const int64_t per = (int64_t)nx * ny, n_all = per * n_var;
    const int n_c = cx * cy;
    trk_triage_stats S;
    std::memset(&S, 0, sizeof S);
    S.n_cells = n_all;
    S.n_coarse = (int64_t)n_c * n_var;
    double t0 = now_ms();

    // 1. exact survival of the known cells of every variant: the coarse cells
    // (row by row), then the sentinel cells (row by row), in one scan
    std::vector<int2> cells;
    for (int jy = 0; jy < cy; ++jy)
        for (int jx = 0; jx < cx; ++jx) cells.push_back(make_int2(off + jx * st, off + jy * st));
    std::vector<int> sxp, syp, nsx(nx, 0), nsy(ny, 0);
    if (o->sentinel_stride > 0) {
        sentinel_positions(nx, o->sentinel_stride, sxp);
        sentinel_positions(ny, o->sentinel_stride, syp);
        for (int b = 0; b < (int)syp.size(); ++b)
            for (int a = 0; a < (int)sxp.size(); ++a) cells.push_back(make_int2(sxp[a], syp[b]));
        nearest_positions(sxp, nsx);
        nearest_positions(syp, nsy);
    }
    const int per_v = (int)cells.size();
    const int64_t n_known = (int64_t)per_v * n_var;
    S.n_sentinel = (int64_t)(per_v - n_c) * n_var;
    DBuf<int2> dcells;
    DBuf<int> dnsx, dnsy;
    DBuf<double> kx0, ky0;
    DBuf<int32_t> ksurv;
    if (dcells.alloc(per_v) || dnsx.alloc(nx) || dnsy.alloc(ny) || kx0.alloc(n_known) || ky0.alloc(n_known) ||
        ksurv.alloc(n_known))
        return set_error(TRK_ENOMEM, "trk_da_triage: known-cell allocation failed");
    TRI_CUDA(cudaMemcpyAsync(dcells.p, cells.data(), per_v * sizeof(int2), cudaMemcpyHostToDevice, s));
    TRI_CUDA(cudaMemcpyAsync(dnsx.p, nsx.data(), nx * sizeof(int), cudaMemcpyHostToDevice, s));
    TRI_CUDA(cudaMemcpyAsync(dnsy.p, nsy.data(), ny * sizeof(int), cudaMemcpyHostToDevice, s));
    k_known_points<<<grid_for(n_known), 256, 0, s>>>(dcells.p, per_v, n_var, nx, ny, w, kx0.p, ky0.p);
    TRI_CUDA(cudaGetLastError());
    std::vector<int64_t> offs(n_var + 1);
    for (int v = 0; v <= n_var; ++v) offs[v] = (int64_t)v * per_v;
    trk_status r = trk_da_survival(lats, n_var, offs.data(), kx0.p, ky0.p, o->n_turns, nullptr, ksurv.p, stream);
    if (r != TRK_OK) return r;
    double t1 = now_ms();
    S.ms_coarse = t1 - t0;

    // 2. train the surrogate on the coarse labels
    DBuf<uint8_t> mask_known, todo, bnd, audit_c, flip, tmp;
    if (mask_known.alloc(n_all) || todo.alloc(n_all) || bnd.alloc(n_all) || audit_c.alloc(n_all) ||
        flip.alloc(n_all) || tmp.alloc(n_all))
        return set_error(TRK_ENOMEM, "trk_da_triage: mask allocation failed");
    TRI_CUDA(cudaMemsetAsync(mask_known.p, 0, n_all, s));
    TRI_CUDA(cudaMemsetAsync(flip.p, 0, n_all, s));
    if (o->use_mlp) {
        const int64_t n_train = S.n_coarse;
        DBuf<float> X, y;
        if (X.alloc(n_train * 8) || y.alloc(n_train)) return set_error(TRK_ENOMEM, "trk_da_triage: feature allocation failed");
        k_coarse_features<<<grid_for(n_train), 256, 0, s>>>(kx0.p, ky0.p, ksurv.p, d_params, n_c, per_v, n_var, w,
                                                            o->n_turns, X.p, y.p);
        TRI_CUDA(cudaGetLastError());
        r = trk_mlp_train(net, X.p, y.p, n_train, o->batch, o->epochs, d_perm, o->lr, nullptr, stream);
        if (r != TRK_OK) return r;
    }
    double t2 = now_ms();
    S.ms_train = t2 - t1;

    // 3. predicted mask of every cell
    if (o->use_mlp == 2) {
        // nearest known cell everywhere, then the network where the known cells
        // disagree: within distance 3 of a boundary cell of that prediction
        k_nearest_known<<<grid_for(n_all), 256, 0, s>>>(ksurv.p, dcells.p, nx, ny, st, off, cx, cy, per_v, dnsx.p,
                                                        dnsy.p, (int)sxp.size(), n_var, o->n_turns, d_mask);
        DBuf<uint8_t> rb, rt;
        DBuf<unsigned long long> rcount;
        if (rb.alloc(n_all) || rt.alloc(n_all) || rcount.alloc(1))
            return set_error(TRK_ENOMEM, "trk_da_triage: region allocation failed");
        k_boundary<<<grid_for(n_all), 256, 0, s>>>(d_mask, nx, ny, n_var, rb.p);
        k_dilate_x<<<grid_for(n_all), 256, 0, s>>>(rb.p, nullptr, nx, ny, n_var, 3, 0, rt.p);
        k_dilate_y<<<grid_for(n_all), 256, 0, s>>>(rt.p, nx, ny, n_var, 3, 0, rb.p);
        TRI_CUDA(cudaMemsetAsync(rcount.p, 0, sizeof(unsigned long long), s));
        DBuf<int64_t> ridx;
        if (ridx.alloc(n_all)) return set_error(TRK_ENOMEM, "trk_da_triage: region allocation failed");
        k_region_list<<<grid_for(n_all), 256, 0, s>>>(rb.p, n_all, ridx.p, rcount.p);
        TRI_CUDA(cudaGetLastError());
        unsigned long long nr = 0;
        TRI_CUDA(cudaMemcpyAsync(&nr, rcount.p, sizeof nr, cudaMemcpyDeviceToHost, s));
        TRI_CUDA(cudaStreamSynchronize(s));
        S.n_region = (int64_t)nr;
        const int64_t chunk = 1 << 20;
        DBuf<float> X, logit;
        if (X.alloc(chunk * 8) || logit.alloc(chunk)) return set_error(TRK_ENOMEM, "trk_da_triage: inference allocation failed");
        for (int64_t c0 = 0; c0 < (int64_t)nr; c0 += chunk) {
            const int64_t m = (int64_t)nr - c0 < chunk ? (int64_t)nr - c0 : chunk;
            k_list_features<<<grid_for(m), 256, 0, s>>>(ridx.p + c0, m, nx, ny, w, d_params, X.p);
            r = trk_mlp_forward(net, X.p, m, logit.p, stream);
            if (r != TRK_OK) return r;
            k_list_threshold<<<grid_for(m), 256, 0, s>>>(ridx.p + c0, logit.p, m, d_mask);
        }
    } else if (o->use_mlp) {
        S.n_region = n_all;
        const int64_t chunk = 1 << 20;
        DBuf<float> X, logit;
        if (X.alloc(chunk * 8) || logit.alloc(chunk)) return set_error(TRK_ENOMEM, "trk_da_triage: inference allocation failed");
        for (int64_t c0 = 0; c0 < n_all; c0 += chunk) {
            const int64_t m = n_all - c0 < chunk ? n_all - c0 : chunk;
            k_grid_features<<<grid_for(m), 256, 0, s>>>(c0, m, nx, ny, w, d_params, X.p);
            r = trk_mlp_forward(net, X.p, m, logit.p, stream);
            if (r != TRK_OK) return r;
            k_threshold<<<grid_for(m), 256, 0, s>>>(logit.p, m, d_mask + c0);
        }
    } else {
        k_nearest_known<<<grid_for(n_all), 256, 0, s>>>(ksurv.p, dcells.p, nx, ny, st, off, cx, cy, per_v, dnsx.p,
                                                        dnsy.p, (int)sxp.size(), n_var, o->n_turns, d_mask);
    }
    TRI_CUDA(cudaGetLastError());
    TRI_CUDA(cudaStreamSynchronize(s));
    double t3 = now_ms();
    S.ms_infer = t3 - t2;

    // 4./5. known labels; then, pass after pass, the band around the boundary of
    // the current mask (plus the audit cells in the first pass) is gathered into
    // point lists, re-tracked exactly in FP64 and merged, until a pass finds no
    // cell left to track.
    k_apply_known<<<grid_for(n_known), 256, 0, s>>>(ksurv.p, dcells.p, per_v, nx, ny, n_var, o->n_turns, d_mask,
                                                    mask_known.p, d_survival);
    TRI_CUDA(cudaGetLastError());
    DBuf<int64_t> dcounts, doffs;
    DBuf<unsigned long long> wrong;
    if (dcounts.alloc(n_var) || doffs.alloc(n_var + 1) || wrong.alloc(1))
        return set_error(TRK_ENOMEM, "trk_da_triage: count allocation failed");
    TRI_CUDA(cudaMemsetAsync(wrong.p, 0, sizeof(unsigned long long), s));
    const int max_passes = o->max_passes > 0 ? o->max_passes : 64;
    std::vector<int64_t> counts(n_var), toffs(n_var + 1, 0);
    DBuf<int64_t> tcell;
    DBuf<double> tx0, ty0;
    DBuf<int32_t> tsurv;
    int64_t cap = 0;
    double t_band = 0.0, t_track = 0.0;
    for (int pass = 0; pass < max_passes; ++pass) {
        const double p0 = now_ms();
        k_boundary<<<grid_for(n_all), 256, 0, s>>>(d_mask, nx, ny, n_var, bnd.p);
        const int R = pass == 0 ? 0 : o->expand_radius;
        k_dilate_x<<<grid_for(n_all), 256, 0, s>>>(bnd.p, R > 0 ? flip.p : nullptr, nx, ny, n_var, o->band_radius, R,
                                                   tmp.p);
        k_dilate_y<<<grid_for(n_all), 256, 0, s>>>(tmp.p, nx, ny, n_var, o->band_radius, R, bnd.p);
        k_band<<<grid_for(n_all), 256, 0, s>>>(bnd.p, pass == 0 ? d_audit : nullptr, mask_known.p, n_all, todo.p,
                                               audit_c.p);
        k_count<<<n_var, 256, 0, s>>>(todo.p, per, dcounts.p);
        TRI_CUDA(cudaGetLastError());
        TRI_CUDA(cudaMemcpyAsync(counts.data(), dcounts.p, n_var * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (pass == 0) {
            DBuf<int64_t> acount;
            if (acount.alloc(n_var)) return set_error(TRK_ENOMEM, "trk_da_triage: count allocation failed");
            k_count<<<n_var, 256, 0, s>>>(audit_c.p, per, acount.p);
            TRI_CUDA(cudaGetLastError());
            std::vector<int64_t> ac(n_var);
            TRI_CUDA(cudaMemcpyAsync(ac.data(), acount.p, n_var * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            TRI_CUDA(cudaStreamSynchronize(s));
            for (int v = 0; v < n_var; ++v) S.n_audit += ac[v];
        }
        TRI_CUDA(cudaStreamSynchronize(s));
        for (int v = 0; v < n_var; ++v) toffs[v + 1] = toffs[v] + counts[v];
        const int64_t n_todo = toffs[n_var];
        if (n_todo == 0) {
            t_band += now_ms() - p0;
            break;
        }
        S.n_tracked += n_todo;
        S.n_passes = pass + 1;
        S.pass_cells[pass < 15 ? pass : 15] += n_todo;
        if (n_todo > cap) {
            tcell.reset();
            tx0.reset();
            ty0.reset();
            tsurv.reset();
            if (tcell.alloc(n_todo) || tx0.alloc(n_todo) || ty0.alloc(n_todo) || tsurv.alloc(n_todo))
                return set_error(TRK_ENOMEM, "trk_da_triage: band allocation failed");
            cap = n_todo;
        }
        TRI_CUDA(cudaMemcpyAsync(doffs.p, toffs.data(), (n_var + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        k_gather_todo<<<n_var, 256, 0, s>>>(todo.p, per, nx, ny, w, doffs.p, tx0.p, ty0.p, tcell.p);
        TRI_CUDA(cudaGetLastError());
        const double p1 = now_ms();
        t_band += p1 - p0;
        // Few cells: the pass is bound by one particle's latency over all turns,
        // so the lane-parallel scan (4 or 8 lanes per particle) takes it where the
        // lattices allow; otherwise one particle per thread up to about a million
        // cells keeps one chain per thread and spreads the warps over the SMs
        // (measured: 484 k random cells 67 ms at one particle per thread, 103 ms at
        // two; equal near 1 M; two per thread ahead from 2 M).
        r = TRK_EUNSUPPORTED;
        if (n_todo <= kLaneCells)
            r = trk_da_survival_lanes(lats, n_var, toffs.data(), tx0.p, ty0.p, o->n_turns, tsurv.p, stream);
        if (r == TRK_EUNSUPPORTED) {
            trk_schedule sch = {128, n_todo <= kOnePerThreadCells ? 1 : 2, 1, 2};
            r = trk_da_survival(lats, n_var, toffs.data(), tx0.p, ty0.p, o->n_turns, &sch, tsurv.p, stream);
        }
        if (r != TRK_OK) return r;
        TRI_CUDA(cudaMemsetAsync(flip.p, 0, n_all, s));
        k_merge<<<grid_for(n_todo), 256, 0, s>>>(tcell.p, tsurv.p, n_todo, o->n_turns, audit_c.p, d_mask,
                                                 mask_known.p, flip.p, d_survival, wrong.p);
        TRI_CUDA(cudaGetLastError());
        TRI_CUDA(cudaStreamSynchronize(s));
        const double p2 = now_ms();
        t_track += p2 - p1;
        S.pass_ms[pass < 15 ? pass : 15] += p2 - p0;
    }
    k_fill_predicted<<<grid_for(n_all), 256, 0, s>>>(d_mask, mask_known.p, n_all, o->n_turns, d_survival);
    TRI_CUDA(cudaGetLastError());
    unsigned long long nw = 0;
    TRI_CUDA(cudaMemcpyAsync(&nw, wrong.p, sizeof nw, cudaMemcpyDeviceToHost, s));
    TRI_CUDA(cudaStreamSynchronize(s));
    S.ms_band = t_band;
    S.ms_retrack = t_track;
    S.n_band = S.n_tracked - S.n_audit;
    S.n_audit_wrong = (int64_t)nw;
    if (stats) *stats = S;
    return TRK_OK;
}
