// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "trk.h"

namespace trk {

constexpr int kMaxBins = 65536;
constexpr int kMomentsN = 28;   // n, 6 means, 21 second moments

// Device element record (128 bytes, read warp-uniformly).
//   KQUAD/KSEXT  p[0] d1 = w1 h / 2     p[1] d2 = (w0 + w1) h / 2   p[2] dm = w1 h
//                p[3] a1 = K1 w1 h       p[4] a0 = K1 w0 h
//                p[5] hb1 = K2 w1 h / 2  p[6] hb0 = K2 w0 h / 2
//                p[7] d1 / 2, p[8] 3 d1 / 8, p[9] d2 / 2, p[10] 3 d2 / 8, p[11] 3 dm / 8
//                (drift series constants; dm = 2 d1 exactly, so dm / 2 = d1)
//                n = steps; flags bit0 = has K1, bit1 = has K2
//   EDRIFT       p[0] L, p[1] L / 2, p[2] 3 L / 8
//   THINSEXT     p[0] K2L, p[1] K2L / 2
//   RFCA         p[0] V, p[1] phi [rad], p[2] k_rf = 2 pi f / c, p[3] G = V cos(phi)
//   WAKE         p[0] W0, p[1] s_c, p[2] charge, p[3] W0T (transverse, 0 = none);
//                n = nbins; term0 = wake ordinal
//   SBEND        p[0] L, p[1] theta, p[2] rho, p[3] 1/rho, p[4] sin theta, p[5] cos theta
//   LSC          p[2] charge, p[4] K L; n = nbins; flags = smoothing passes;
//                term0 = wake ordinal (kicked like a wake); impedance mode:
//                p[5] r_b (> 0), p[6] rest energy mc^2 [eV], p[7] f0, p[8] f1, p[9] L
//   MAP          term0 = first term; rb[r]..rb[r+1] = terms of output row r;
//                flags bit r (r < 6) = row r starts from x_r (R_rr == 1 folded);
//                flags bit 6 = row 5 (delta) changes
struct alignas(16) DevElem {
    int32_t type;
    int32_t n;
    int32_t term0;
    uint32_t flags;
    int16_t rb[8];
    double p[12];
};
static_assert(sizeof(DevElem) == 128, "DevElem layout");

// One map term: coefficient and monomial code deg | j << 2 | k << 5 | l << 8.
struct alignas(16) DevTerm {
    double c;
    int32_t code;
    int32_t pad;
};

struct LatticeView {
    const DevElem *elems;
    const DevTerm *terms;
    int32_t n_elem;
    int32_t ap_type;
    // Map rows evaluated (bit r = row r): all six for tracking; in survival
    // scans only the rows the aperture test depends on (see survival_rows).
    uint32_t row_mask;
    int32_t pad_;
    double ap_a, ap_b;
    unsigned long long ap_a_key, ap_b_key;   // bit patterns of a, b (> 0) shifted left by one
    unsigned long long ap_ia_key, ap_ib_key; // the same of 0.7 a, 0.7 b: inner box of the ellipse
};

// The l window of the collective elements, two slots: order keys of the l
// min/max ([2s] min, [2s+1] max) and, for the j-th collective element (0 or 1)
// of the group on slot s, 1/dl of its histogram at [2s + j] (0 for an empty or
// zero-width window): the histogram pass writes it once so that the kick does
// not divide in every thread.  Two adjacent elements share the window but may
// have different bin counts, hence one value each.
struct WakeWindow {
    uint64_t key[4];
    double idl[4];
};

// Device-resident bunch state.
struct BunchState {
    int64_t n_alive;        // alive particles occupy [0, n_alive)
    int64_t n_alive_next;   // result of the pending compaction
    WakeWindow win;
    int32_t error;
    int32_t pad;
};

// Arguments of one fused tracking launch over elements [e0, e1).
struct TrackArgs {
    double *coords;
    int64_t pitch;
    int32_t *loss_turn;     // -1 = alive
    int32_t *loss_elem;
    BunchState *st;
    WakeWindow *win;          // l window of the collective elements: &st->win, or the first part's
                              // for a bunch held in several parts
    LatticeView lat;
    int32_t e0, e1;
    int32_t n_turns;        // > 1 only when [e0, e1) is the whole lattice
    int32_t turn_abs0;      // absolute turn number of the first turn
    int32_t local_turn0;    // row of the first turn in the partial-sum buffer
    int32_t kick_wake;      // element index of a wake to kick with first, or -1
    int32_t kick_wake2;     // a second collective element right after it (same window), or -1
    int32_t kick_slot;      // their key slot
    int32_t minmax_slot;    // key slot to fill with l min/max at the end, or -1
    int32_t do_moments;     // per-turn moments at the end of each turn
    int32_t n_tiles;        // stride of the partial-sum rows
    double p0c;             // reference momentum at element e0 [eV]
    double ip0c;            // 1 / p0c (computed on the host)
    // n_turns == 1: 1 / p0' after the first n_rf_ip RF cavities of [e0, e1), in
    // order, computed on the host from the same sums as the kernel's p0
    double rf_ip[4];
    int32_t n_rf_ip;
    int32_t pad_rf;
    double zero;            // 0.0 (a value the compiler cannot see: see track_tile)
    double *partials;       // [turn][tile][28]
    int32_t *tile_alive;    // alive count per tile at the end (may be null)
    const double *wake_V;   // voltages of the kicking wake
    const double *wake_Vx;  // its transverse voltages (x then y, 2 x nbins), or null
    int32_t wake_nbins;
    int32_t wake_nbins2;    // the same of the second kick
    const double *wake_V2;
    const double *wake_Vx2;
    int32_t tile;           // particles per tile (block * per_thread)
    double *mom_out;        // finalised moments of this launch's first turn (batched path)
};

// Arguments of the loss compaction of one bunch.
struct CompactArgs {
    double *coords;
    int64_t pitch;
    int32_t *ids, *lt, *le;
    double *cb;
    int32_t *ib, *ltb, *leb;
    const int32_t *tile_alive;
    int64_t *tile_off;
    BunchState *st;
    int32_t tile;
    int32_t n_tiles;
};

// Launchers (trk_track.cu / trk_wake.cu); all asynchronous on `s`.
cudaError_t launch_track(const TrackArgs &a, int block, int per_thread, int n_tiles, cudaStream_t s);
cudaError_t launch_moments_finalize(const double *partials, int n_tiles, int n_turns, const BunchState *st,
                                    int tile, double *out, cudaStream_t s);
cudaError_t launch_compact(const CompactArgs &c, int n_tiles, cudaStream_t s);
// One chunk of a batched call: fused tracking of every (variant, tile) item,
// moment finalisation and compaction of every variant.
cudaError_t launch_batch_chunk(const TrackArgs *args, const CompactArgs *cargs, const int2 *items, int n_items,
                               int n_var, int n_chunks, int chunk, int block, int per_thread, int tile,
                               int max_turns, bool moments, cudaStream_t s);
cudaError_t launch_init_bunch(BunchState *st, int32_t *lt, int32_t *le, int64_t n, cudaStream_t s);
// Transverse dipole sums are 64-bit fixed point, 2^-40 m per unit.
constexpr double kDipoleScale = 1099511627776.0;   // 2^40 per metre
// Zero the histogram (and the dipole sums if dip) and, with reset_keys, the l
// window of key slot `slot`.
cudaError_t launch_wake_reset(BunchState *st, int slot, uint32_t *hist, unsigned long long *dip, int nbins,
                              bool reset_keys, cudaStream_t s);
cudaError_t launch_wake_minmax(const double *coords, int64_t pitch, const int32_t *lt, BunchState *st,
                               int slot, int64_t n_max, cudaStream_t s);
cudaError_t launch_wake_hist(const double *coords, int64_t pitch, const int32_t *lt, const BunchState *st,
                             WakeWindow *win, int slot, int which, int nbins,
                             double w0, double sc, uint32_t *hist, double *wfun, double w0t, unsigned long long *dip,
                             double *wfun_t, int64_t n_max, cudaStream_t s);
cudaError_t launch_wake_conv(const uint32_t *hist, const double *wfun, int nbins, double qm, double *V,
                             cudaStream_t s);
// Transverse voltages V_c[k] = q_m sum_{j<=k} D_c[j] W_T((k - j) dl) for c = x, y
// (dip[c * nbins + j] fixed point, V[c * nbins + k]).
// Long-wavelength space-charge field on the bins of slot `slot`:
// V_k = KL d_k (see TRK_LSC); a, b scratch of nbins doubles.
cudaError_t launch_lsc_field(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double KL,
                             int passes, double *a, double *b, double *V, cudaStream_t s);
// Space-charge field of the round-beam impedance on the bins of slot `slot`
// (see TRK_LSC): the impedance and twiddle tables over the whole GPU, then the
// two transforms of the line density zero-padded to N = 2 nbins (nbins a power
// of two, <= kLscImpMaxBins) on one CTA or a cluster of 8 sharing their halves
// through distributed shared memory.  scratch: 3 nbins + 1 doubles.
constexpr int kLscImpMaxBins = 4096;
cudaError_t launch_lsc_imp(const uint32_t *hist, const BunchState *st, int slot, int nbins, double qm, double L,
                           double rb, double gamma, double f0, double f1, double *scratch, double *V,
                           cudaStream_t s);
cudaError_t launch_wake_conv_t(const unsigned long long *dip, const double *wfun_t, int nbins, double qm, double *V,
                               cudaStream_t s);

// Dynamic-aperture helpers (trk_da.cu).
// tcgen05 surrogate inference layers (trk_mlp_umma.cu); BF16 passed as uint16_t.
size_t umma_layer_smem(int K);
cudaError_t launch_umma_layer(const uint16_t *A_tiled, const uint16_t *W_tiled, const float *bias, int K,
                              int64_t n_tiles, uint16_t *out_tiled, int *d_err, cudaStream_t s);
cudaError_t launch_to_tiled(const uint16_t *src, int64_t rows, int K, int tile_rows, uint16_t *dst, cudaStream_t s);
cudaError_t launch_from_tiled(const uint16_t *src, int64_t rows, uint16_t *dst, cudaStream_t s);
// Programmatic dependent launch for the training step's chain of small
// kernels: a kernel launched by pdl_launch may be scheduled while the kernel
// before it in the stream finishes; it must call pdl_wait() before it reads or
// writes global memory that an earlier kernel of the stream uses, and it calls
// pdl_trigger() to let the next kernel be scheduled in turn.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... Exp, typename... Act>
cudaError_t pdl_launch(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Act &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Act &&>(args)...);
}
#endif
// Training products on tcgen05 (trk_mlp_umma.cu): one output tile per CTA.
cudaError_t launch_train_fwd(const uint16_t *H_tiled, int K, const uint16_t *W_tiled, const float *bias,
                             int64_t m_pad, float *Z, uint16_t *Hout_tiled, uint16_t *Hout_T, uint16_t *Hout_rm,
                             int *d_err, cudaStream_t s);
cudaError_t launch_train_dx(const uint16_t *dzb_tiled, const uint16_t *WT_tiled, const float *Zin, int64_t m_pad,
                            float *dz, uint16_t *dzb_out_tiled, uint16_t *dzb_out_T, int *d_err, cudaStream_t s);
int train_dw_splits(int64_t m_pad);
cudaError_t launch_train_dw(const uint16_t *dzb_T, const uint16_t *H_T, int n_in, int64_t m_pad, float *part,
                            int *d_err, cudaStream_t s);
// Training inputs in both layouts; with step != NULL the batch rows are
// gathered through perm at the device step counter (labels into yb).
cudaError_t launch_train_input(const float *X, int64_t M, int64_t m_pad, uint16_t *H0, uint16_t *H0T,
                               const int32_t *perm, int64_t n, int64_t batch, int64_t spe, const int64_t *step,
                               const float *y, float *yb, cudaStream_t s);
// Logits of the tiled last hidden layer and the head's backward step in one
// launch (dlogit, dz_4 FP32 and its BF16 copy tiled and transposed-tiled,
// the loss terms); rows [M, m_pad) get zeros.
cudaError_t launch_train_head(const uint16_t *H4_tiled, const uint16_t *w5, const float *b5, const float *y,
                              int64_t M, int64_t m_pad, const float *Z4, float *logit, float *dl, float *dz,
                              uint16_t *dzb, uint16_t *dzbT, float *loss_terms, cudaStream_t s);
// Adam on the FP32 master weights with the BF16 and tiled weight copies and
// the device step counter; with wpart, the hidden layers' weight gradients are
// summed from their batch-split partials (in split order) and stored to g.
cudaError_t launch_adam_step(float *p, float *m, float *v, float *g, uint16_t *pb, int64_t n, float lr,
                             const float *c12, int64_t *step, const float *loss, float *loss_hist, unsigned *ticket,
                             const size_t *w_off, const size_t *w_end, const size_t *wt_off, const size_t *wtT_off,
                             const int *in_pad, uint16_t *wt, uint16_t *wtT, const float *const *wpart, int splits,
                             cudaStream_t s);
cudaError_t launch_retile_weights(const uint16_t *pb, const size_t *w_off, const size_t *wt_off, const size_t *wtT_off,
                                  const int *in_pad, uint16_t *wt, uint16_t *wtT, cudaStream_t s);
cudaError_t launch_input_tiled(const float *X, int64_t M, int64_t m_pad, uint16_t *H0, cudaStream_t s);
cudaError_t launch_head_tiled(const uint16_t *H4, const uint16_t *w5, const float *b5, int64_t M, float *logit,
                              cudaStream_t s);
cudaError_t launch_da_init(double *coords, int64_t pitch, int32_t *ids, const double *x0, const double *y0,
                           int64_t first, int64_t n, cudaStream_t s);
// lanes: 8, or 4 when every view's row_mask lies within rows 0..3
cudaError_t launch_da_lanes(const LatticeView *views, int n_var, const int64_t *offsets, const double *x0,
                            const double *y0, int64_t n, int32_t n_turns, int lanes, int32_t *survival,
                            cudaStream_t s);
cudaError_t launch_da_survival(const int32_t *ids, const int32_t *lt, int64_t n, int32_t n_turns, int32_t *survival,
                               cudaStream_t s);

// Records the calling thread's error text (returned by trk_last_error) and
// passes the status through.
trk_status set_error(trk_status s, const char *msg);
inline trk_status set_error(trk_status s, const std::string &msg) { return set_error(s, msg.c_str()); }

// Order-preserving 64-bit key of a double (non-NaN) and its inverse.
__host__ __device__ inline uint64_t dkey(double v) {
#ifdef __CUDA_ARCH__
    uint64_t b = (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    __builtin_memcpy(&b, &v, 8);
#endif
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double dkey_inv(uint64_t k) {
    uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    __builtin_memcpy(&v, &b, 8);
    return v;
#endif
}

}  // namespace trk
