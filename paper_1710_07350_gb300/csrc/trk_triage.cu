// Surrogate-triaged dynamic-aperture scan (no counterpart in the paper).
//
// For every lattice variant and every cell of an nx x ny grid of initial
// amplitudes: track a coarse sub-grid exactly, train the MLP surrogate on those
// survival labels (features x/w, y/w and the variant's 6 normalised
// parameters), predict the survival mask of every cell, mark a band of cells
// within Chebyshev distance r of a predicted-boundary cell (a cell whose 8
// neighbours hold both classes) plus caller-chosen audit cells, re-track those
// exactly in FP64, and merge.  With use_mlp = 0 the prediction is the label of
// the nearest coarse cell instead (the same pipeline without the network).
#include <chrono>
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

// Coarse cells (ix, iy) with ix % stride == off, iy % stride == off, per variant.
__global__ void k_coarse_points(int nx, int ny, int stride, int off, double w, int cx, int cy, int n_var,
                                double *__restrict__ x0, double *__restrict__ y0) {
    const int64_t n = (int64_t)n_var * cx * cy;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i % ((int64_t)cx * cy);
        const int jx = (int)(c % cx), jy = (int)(c / cx);
        x0[i] = cell_centre(off + jx * stride, nx, w);
        y0[i] = cell_centre(off + jy * stride, ny, w);
    }
}

// Training features and labels of the coarse cells.
__global__ void k_coarse_features(const double *__restrict__ x0, const double *__restrict__ y0,
                                  const int32_t *__restrict__ surv, const float *__restrict__ params, int cx, int cy,
                                  int n_var, double w, int32_t n_turns, float *__restrict__ X, float *__restrict__ y) {
    const int64_t per = (int64_t)cx * cy, n = per * n_var;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / per);
        X[i * 8 + 0] = (float)(x0[i] / w);
        X[i * 8 + 1] = (float)(y0[i] / w);
        for (int k = 0; k < 6; ++k) X[i * 8 + 2 + k] = params[v * 6 + k];
        y[i] = surv[i] == n_turns + 1 ? 1.0f : 0.0f;
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

__global__ void k_threshold(const float *__restrict__ logit, int64_t m, uint8_t *__restrict__ mask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        mask[i] = logit[i] > 0.0f ? 1 : 0;
}

// Prediction without the network: label of the coarse cell nearest to each cell.
__global__ void k_nearest_coarse(const int32_t *__restrict__ surv, int nx, int ny, int stride, int off, int cx, int cy,
                                 int n_var, int32_t n_turns, uint8_t *__restrict__ mask) {
    const int64_t n = (int64_t)n_var * nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)((c / nx) % ny), v = (int)(c / ((int64_t)nx * ny));
        int jx = (ix - off + stride / 2) / stride, jy = (iy - off + stride / 2) / stride;
        if (ix < off) jx = 0;
        if (iy < off) jy = 0;
        jx = jx < cx - 1 ? jx : cx - 1;
        jy = jy < cy - 1 ? jy : cy - 1;
        mask[c] = surv[((int64_t)v * cy + jy) * cx + jx] == n_turns + 1 ? 1 : 0;
    }
}

// Coarse truth overrides the prediction; survival of coarse cells is exact.
__global__ void k_apply_coarse(const int32_t *__restrict__ surv, int nx, int ny, int stride, int off, int cx, int cy,
                               int n_var, int32_t n_turns, uint8_t *__restrict__ mask, uint8_t *__restrict__ known,
                               int32_t *__restrict__ out_surv) {
    const int64_t n = (int64_t)n_var * cx * cy;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t per = (int64_t)cx * cy;
        const int v = (int)(i / per);
        const int jx = (int)((i % per) % cx), jy = (int)((i % per) / cx);
        const int64_t c = ((int64_t)v * ny + off + jy * stride) * nx + off + jx * stride;
        const int32_t s = surv[i];
        mask[c] = s == n_turns + 1 ? 1 : 0;
        known[c] = 1;
        out_surv[c] = s;
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

// Cells to re-track: within Chebyshev distance r of a boundary cell, or audit
// cells, and not already known exactly.
__global__ void k_band(const uint8_t *__restrict__ bnd, const uint8_t *__restrict__ audit,
                       const uint8_t *__restrict__ known, int nx, int ny, int n_var, int r,
                       uint8_t *__restrict__ todo, uint8_t *__restrict__ is_audit) {
    const int64_t n = (int64_t)n_var * nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(c % nx), iy = (int)((c / nx) % ny);
        const int64_t base = c - (int64_t)iy * nx - ix;
        bool near = false;
        for (int dy = -r; dy <= r && !near; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const int jx = ix + dx, jy = iy + dy;
                if (jx < 0 || jy < 0 || jx >= nx || jy >= ny) continue;
                if (bnd[base + (int64_t)jy * nx + jx]) {
                    near = true;
                    break;
                }
            }
        const bool au = audit && audit[c] && !near;
        todo[c] = (!known[c] && (near || au)) ? 1 : 0;
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
                        int32_t *__restrict__ out_surv, unsigned long long *__restrict__ wrong) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cell[i];
        const uint8_t m = surv[i] == n_turns + 1 ? 1 : 0;
        if (is_audit[c] && m != mask[c]) atomicAdd(wrong, 1ull);
        mask[c] = m;
        out_surv[c] = surv[i];
    }
}

// Cells neither tracked nor coarse: survival from the prediction.
__global__ void k_fill_predicted(const uint8_t *__restrict__ mask, const uint8_t *__restrict__ known,
                                 const uint8_t *__restrict__ todo, int64_t n, int32_t n_turns,
                                 int32_t *__restrict__ out_surv) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        if (!known[c] && !todo[c]) out_surv[c] = mask[c] ? n_turns + 1 : 0;
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
        o->band_radius < 0 || (o->use_mlp && (!net || o->epochs < 1 || o->batch < 1)))
        return set_error(TRK_EINVAL, "trk_da_triage: bad options");
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = o->nx, ny = o->ny, st = o->coarse_stride, off = st / 2;
    const int cx = (nx - off + st - 1) / st, cy = (ny - off + st - 1) / st;
    const double w = o->half_width;
    const int64_t per = (int64_t)nx * ny, n_all = per * n_var, n_coarse = (int64_t)cx * cy * n_var;
    trk_triage_stats S;
    std::memset(&S, 0, sizeof S);
    S.n_cells = n_all;
    S.n_coarse = n_coarse;
    double t0 = now_ms();

    // 1. exact survival of the coarse cells
    DBuf<double> cx0, cy0;
    DBuf<int32_t> csurv;
    if (cx0.alloc(n_coarse) || cy0.alloc(n_coarse) || csurv.alloc(n_coarse))
        return set_error(TRK_ENOMEM, "trk_da_triage: coarse allocation failed");
    k_coarse_points<<<grid_for(n_coarse), 256, 0, s>>>(nx, ny, st, off, w, cx, cy, n_var, cx0.p, cy0.p);
    TRI_CUDA(cudaGetLastError());
    std::vector<int64_t> offs(n_var + 1);
    for (int v = 0; v <= n_var; ++v) offs[v] = (int64_t)v * cx * cy;
    trk_status r = trk_da_survival(lats, n_var, offs.data(), cx0.p, cy0.p, o->n_turns, nullptr, csurv.p, stream);
    if (r != TRK_OK) return r;
    double t1 = now_ms();
    S.ms_coarse = t1 - t0;

    // 2. train the surrogate on the coarse labels
    DBuf<uint8_t> mask_known, todo, bnd, audit_c;
    if (mask_known.alloc(n_all) || todo.alloc(n_all) || bnd.alloc(n_all) || audit_c.alloc(n_all))
        return set_error(TRK_ENOMEM, "trk_da_triage: mask allocation failed");
    TRI_CUDA(cudaMemsetAsync(mask_known.p, 0, n_all, s));
    if (o->use_mlp) {
        DBuf<float> X, y;
        if (X.alloc(n_coarse * 8) || y.alloc(n_coarse)) return set_error(TRK_ENOMEM, "trk_da_triage: feature allocation failed");
        k_coarse_features<<<grid_for(n_coarse), 256, 0, s>>>(cx0.p, cy0.p, csurv.p, d_params, cx, cy, n_var, w,
                                                             o->n_turns, X.p, y.p);
        TRI_CUDA(cudaGetLastError());
        r = trk_mlp_train(net, X.p, y.p, n_coarse, o->batch, o->epochs, d_perm, o->lr, nullptr, stream);
        if (r != TRK_OK) return r;
    }
    double t2 = now_ms();
    S.ms_train = t2 - t1;

    // 3. predicted mask of every cell
    if (o->use_mlp) {
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
        k_nearest_coarse<<<grid_for(n_all), 256, 0, s>>>(csurv.p, nx, ny, st, off, cx, cy, n_var, o->n_turns, d_mask);
    }
    TRI_CUDA(cudaGetLastError());
    TRI_CUDA(cudaStreamSynchronize(s));
    double t3 = now_ms();
    S.ms_infer = t3 - t2;

    // 4. coarse truth, boundary band, audit cells; point lists to re-track
    k_apply_coarse<<<grid_for(n_coarse), 256, 0, s>>>(csurv.p, nx, ny, st, off, cx, cy, n_var, o->n_turns, d_mask,
                                                      mask_known.p, d_survival);
    k_boundary<<<grid_for(n_all), 256, 0, s>>>(d_mask, nx, ny, n_var, bnd.p);
    k_band<<<grid_for(n_all), 256, 0, s>>>(bnd.p, d_audit, mask_known.p, nx, ny, n_var, o->band_radius, todo.p,
                                           audit_c.p);
    DBuf<int64_t> dcounts;
    if (dcounts.alloc(n_var)) return set_error(TRK_ENOMEM, "trk_da_triage: count allocation failed");
    k_count<<<n_var, 256, 0, s>>>(todo.p, per, dcounts.p);
    TRI_CUDA(cudaGetLastError());
    std::vector<int64_t> counts(n_var);
    TRI_CUDA(cudaMemcpyAsync(counts.data(), dcounts.p, n_var * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRI_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> toffs(n_var + 1, 0);
    for (int v = 0; v < n_var; ++v) toffs[v + 1] = toffs[v] + counts[v];
    const int64_t n_todo = toffs[n_var];
    S.n_tracked = n_todo;
    DBuf<int64_t> doffs, tcell;
    DBuf<double> tx0, ty0;
    DBuf<int32_t> tsurv;
    if (doffs.alloc(n_var + 1) || tcell.alloc(n_todo) || tx0.alloc(n_todo) || ty0.alloc(n_todo) || tsurv.alloc(n_todo))
        return set_error(TRK_ENOMEM, "trk_da_triage: band allocation failed");
    TRI_CUDA(cudaMemcpyAsync(doffs.p, toffs.data(), (n_var + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_gather_todo<<<n_var, 256, 0, s>>>(todo.p, per, nx, ny, w, doffs.p, tx0.p, ty0.p, tcell.p);
    TRI_CUDA(cudaGetLastError());
    TRI_CUDA(cudaStreamSynchronize(s));
    double t4 = now_ms();
    S.ms_band = t4 - t3;

    // 5. exact FP64 re-track of the band and audit cells, merge
    DBuf<unsigned long long> wrong;
    if (wrong.alloc(1)) return set_error(TRK_ENOMEM, "trk_da_triage: counter allocation failed");
    TRI_CUDA(cudaMemsetAsync(wrong.p, 0, sizeof(unsigned long long), s));
    if (n_todo > 0) {
        r = trk_da_survival(lats, n_var, toffs.data(), tx0.p, ty0.p, o->n_turns, nullptr, tsurv.p, stream);
        if (r != TRK_OK) return r;
        k_merge<<<grid_for(n_todo), 256, 0, s>>>(tcell.p, tsurv.p, n_todo, o->n_turns, audit_c.p, d_mask, d_survival,
                                                 wrong.p);
    }
    k_fill_predicted<<<grid_for(n_all), 256, 0, s>>>(d_mask, mask_known.p, todo.p, n_all, o->n_turns, d_survival);
    TRI_CUDA(cudaGetLastError());
    unsigned long long nw = 0;
    TRI_CUDA(cudaMemcpyAsync(&nw, wrong.p, sizeof nw, cudaMemcpyDeviceToHost, s));
    // audit and band sizes
    DBuf<int64_t> acount;
    if (acount.alloc(n_var)) return set_error(TRK_ENOMEM, "trk_da_triage: count allocation failed");
    k_count<<<n_var, 256, 0, s>>>(audit_c.p, per, acount.p);
    std::vector<int64_t> ac(n_var);
    TRI_CUDA(cudaMemcpyAsync(ac.data(), acount.p, n_var * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRI_CUDA(cudaStreamSynchronize(s));
    double t5 = now_ms();
    S.ms_retrack = t5 - t4;
    for (int v = 0; v < n_var; ++v) S.n_audit += ac[v];
    S.n_band = n_todo - S.n_audit;
    S.n_audit_wrong = (int64_t)nw;
    if (stats) *stats = S;
    return TRK_OK;
}
