/*
 * trk.h -- C ABI of the GB300 (sm_103a) FP64 particle tracker.
 *
 * The library implements the data-parallel hot path of GPU-accelerated Elegant
 * (King et al., "GPU acceleration and performance of the particle-beam-dynamics
 * code Elegant", arXiv:1710.07350): the per-turn 6D tracking loop through
 * lumped elements (Sec. 1; Table 1), particle loss at apertures (Sec. 2.5),
 * per-turn beam moments by reduction (Sec. 2.4), and the longitudinal wakefield
 * path of histogram (Sec. 2.2), convolution (Sec. 2.3) and energy kick
 * (Table 1, WAKE / RFCW).
 *
 * Conventions shared by every call
 *   Coordinates  per particle (x [m], x' [rad], y [m], y' [rad], l [m], delta):
 *                slopes as in the paper's exactDrift listings (Sec. 2.1); l is
 *                the path-length DEVIATION from the reference particle; delta
 *                is the relative momentum deviation from the reference p0.
 *                Particles are ultra-relativistic (beta = 1).
 *   Layout       structure of arrays (Sec. 2, barrier 1): coordinate c of
 *                particle i is coords[c * pitch + i], FP64, device memory.
 *                pitch >= n; coords must be 16-byte aligned.
 *   Ownership    particle arrays and outputs passed as device pointers are
 *                owned by the CALLER (e.g. PyTorch tensors) and only borrowed.
 *                Lattices and all scratch are owned by the library and freed by
 *                trk_destroy_lattice / trk_bunch_free.
 *   Streams      device work is enqueued on the bunch's CUDA stream; calls that
 *                enqueue work return before it completes.  Calls that return
 *                host data (trk_moments, trk_lost, trk_n_alive, trk_bunch_p0c)
 *                synchronise that stream first.
 *   Errors       every call returns a trk_status; nothing aborts, exits or
 *                traps.  trk_last_error() gives the calling thread's text for
 *                the last non-OK status.  Device-side failures surface as
 *                TRK_ECUDA at the next call that synchronises.
 *   Ordering     after trk_track the alive particles occupy slots [0, n_alive)
 *                in their previous relative order (stable compaction); lost
 *                particles follow in order of loss.  Identify particles by id.
 */
#ifndef TRK_H
#define TRK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRK_OK = 0,
    TRK_EINVAL = 1,       /* invalid argument or descriptor */
    TRK_ENOMEM = 2,       /* device or host allocation failed */
    TRK_ECUDA = 3,        /* a CUDA runtime call failed */
    TRK_EKERNEL = 4,      /* a kernel reported an internal error */
    TRK_ETIMEOUT = 5,     /* a bounded device wait ran out */
    TRK_EUNSUPPORTED = 6  /* valid request the library does not implement */
} trk_status;

/* Element types (Table 1 of the paper). */
typedef enum {
    TRK_MAP = 1,       /* polynomial transport map of order 1..3 (R, T, U):
                          "transport matrices (up to third order)", Sec. 1;
                          track_particles M1/M2/M3 rows of Table 1.
                          x_i <- C_i + sum_j R_ij x_j + sum_{j<=k} T_i(jk) x_j x_k
                                     + sum_{j<=k<=l} U_i(jkl) x_j x_k x_l
                          evaluated from the input vector (simultaneous update) */
    TRK_EDRIFT = 2,    /* exact drift (Sec. 2.1 listings): x += L x', y += L y',
                          l += L (sqrt(1 + x'^2 + y'^2) - 1) */
    TRK_KQUAD = 3,     /* thick quadrupole by canonical kick-drift integration,
                          4th-order Yoshida, n_kicks steps (Table 1,
                          multipole_tracking2; Sec. 3) */
    TRK_KSEXT = 4,     /* thick sextupole, same integrator (k1 may be nonzero) */
    TRK_THINSEXT = 5,  /* thin sextupole: x' -= (k2l/2)(x^2 - y^2), y' += k2l x y */
    TRK_RFCA = 6,      /* thin RF cavity with exact phase dependence (Table 1,
                          simple_rf_cavity): dE = V cos(phi + 2 pi f l / c),
                          P' = P + dE, p0' = p0 + V cos(phi),
                          delta' = P'/p0' - 1, x' and y' scaled by P/P' */
    TRK_WAKE = 7,      /* longitudinal wake (Table 1 WAKE; Sec. 2.2-2.3): l-window
                          [min, max] over alive particles, nbins equal bins,
                          counts h_j, V_k = -q_m sum_{j<=k} h_j W((k-j) dl) with
                          W(s) = w0 / sqrt(max(s, s_c)), q_m = charge / n,
                          delta += V(l) / p0c, V linearly interpolated between
                          bin centres and clamped at the end bins.  With
                          wake_w0t != 0 also the transverse dipole wake (Table 1
                          TRWAKE, the transverse half of RFCW): per-bin sums
                          D_j of x (and y) over alive particles with finite
                          offsets, V_x,k = +q_m sum_{j<=k} D_j W_T((k-j) dl),
                          x' += V_x(l) / (p0c (1 + delta)) (y likewise), applied
                          before the energy kick; voltages from the particles
                          entering the element */
    TRK_LSC = 8,       /* longitudinal space charge (Table 1 LSCDRIFT), a thin
                          kick of effective length `length` on the bins of
                          TRK_WAKE, line density lambda_k = q_m h_k / dl.
                          lsc_rb == 0, the long-wavelength limit: n_kicks passes
                          of lambda_k <- (lambda_{k-1} + 2 lambda_k + lambda_{k+1}) / 4
                          (end bins repeated), d_k = central difference (one-sided
                          at the ends), delta += lsc_k length d(l) / p0c with d
                          interpolated as the wake voltage.
                          lsc_rb > 0, the impedance of a round, transversely
                          uniform beam of radius r_b:
                          Z(k) = i sgn(k) Z0 / (pi |k| r_b^2) (1 - xi K1(xi)),
                          xi = |k| r_b / gamma, gamma = sqrt(1 + (p0c/lsc_mc2)^2),
                          times a cosine taper from lsc_f0 to lsc_f1 (fractions
                          of the Nyquist frequency); lambda zero-padded to
                          2 nbins, transformed, multiplied by Z, transformed
                          back: V(l) = length c (Z lambda)(l), delta += V / p0c.
                          nbins a power of two, 1 .. 4096, in this mode */
    TRK_SBEND = 9      /* sector dipole, hard edge, no gradient (Table 1 CSBEND
                          without fringe fields or radiation): the exact orbit in a
                          uniform field, a circle of radius rho p_h
                          (rho = length/angle, p_h = sqrt((1+delta)^2 - py^2)) from
                          the entrance face to the exit face at `angle`; x is
                          measured outward; angle 0 is the exact drift */
} trk_elem_type;

typedef enum { TRK_APERTURE_NONE = 0, TRK_APERTURE_RECT = 1, TRK_APERTURE_ELLIPSE = 2 } trk_aperture;

/* One element.  Map coefficient arrays are HOST pointers read (copied) by
 * trk_create_lattice; unused fields are ignored. */
typedef struct {
    int32_t type;       /* trk_elem_type */
    int32_t order;      /* TRK_MAP: 1, 2 or 3 (U ignored below 3, T below 2) */
    int32_t n_kicks;    /* TRK_KQUAD / TRK_KSEXT: Yoshida-4 steps (>= 1);
                           TRK_LSC: smoothing passes (0 .. 1000) */
    int32_t nbins;      /* TRK_WAKE, TRK_LSC: histogram bins (1 .. 65536) */
    double length;      /* m (TRK_EDRIFT, TRK_KQUAD, TRK_KSEXT) */
    double k1;          /* m^-2 (TRK_KQUAD, TRK_KSEXT) */
    double k2;          /* m^-3 (TRK_KSEXT) */
    double k2l;         /* m^-2 (TRK_THINSEXT) */
    double volt;        /* V (TRK_RFCA) */
    double phase_deg;   /* degrees (TRK_RFCA) */
    double freq_hz;     /* Hz (TRK_RFCA) */
    double wake_w0;     /* V m^1/2 / C (TRK_WAKE) */
    double wake_sc;     /* m, saturation length s_c (TRK_WAKE) */
    double charge;      /* C, bunch charge (TRK_WAKE) */
    double wake_w0t;    /* V m^-1/2 / C: transverse dipole wake
                           W_T(s) = wake_w0t / sqrt(max(s, s_c)) (TRK_WAKE; 0 = none) */
    double lsc_k;       /* V m / C per m of length: space-charge factor g / (4 pi eps0 gamma^2)
                           (TRK_LSC; uses length, nbins, charge, n_kicks) */
    double angle;       /* rad, bending angle (TRK_SBEND; |angle| < pi) */
    double lsc_rb;      /* m, beam radius of the space-charge impedance (TRK_LSC;
                           0 = the long-wavelength limit with lsc_k) */
    double lsc_mc2;     /* eV, rest energy of the particle (TRK_LSC with lsc_rb > 0) */
    double lsc_f0;      /* filter: start of the cosine taper, fraction of Nyquist (TRK_LSC, lsc_rb > 0) */
    double lsc_f1;      /* filter: end of the taper (0 from here on), f0 < f1 <= 1; <= 0 = no filter */
    const double *C;    /* TRK_MAP: [6] or NULL (zero) */
    const double *R;    /* TRK_MAP: [6*6] row-major */
    const double *T;    /* TRK_MAP: [6*21], (j,k) j<=k lexicographic, or NULL */
    const double *U;    /* TRK_MAP: [6*56], (j,k,l) j<=k<=l lexicographic, or NULL */
} trk_element_desc;

typedef struct {
    int32_t aperture;   /* trk_aperture, checked at the exit of every element
                           (Table 1 limit_amplitudes / RCOL / ECOL): RECT keeps
                           |x| <= a and |y| <= b, ELLIPSE keeps
                           (x/a)^2 + (y/b)^2 <= 1; NaN is lost */
    int32_t moments;    /* 1: compute per-turn moments (Sec. 2.4), 0: skip */
    double a, b;        /* aperture half-widths [m] */
    double p0c_ev;      /* reference momentum at the lattice entrance [eV] */
} trk_lattice_opts;

typedef struct trk_lattice trk_lattice;   /* opaque, library-owned */
typedef struct trk_bunch trk_bunch;       /* opaque view over caller arrays */

/* Compile n element descriptors into a device-resident lattice.  Returns
 * TRK_EINVAL for an unknown type, a MAP without R, order outside 1..3,
 * n_kicks < 1, nbins outside 1..65536, or a non-positive aperture. */
trk_status trk_create_lattice(const trk_element_desc *elems, int32_t n,
                              const trk_lattice_opts *opts, trk_lattice **out);
trk_status trk_destroy_lattice(trk_lattice *lat);

/* Wrap caller-owned device arrays as a bunch of n alive particles.
 *   d_coords  [6 * pitch] FP64, SoA as above, pitch >= n
 *   d_id      [n] int32 particle ids (permuted with the coordinates)
 *   stream    cudaStream_t (NULL = legacy default stream)
 * Allocates library scratch (loss records, compaction buffers, partial sums)
 * of about 80 bytes per particle.  The arrays must outlive the bunch. */
trk_status trk_bunch_wrap(double *d_coords, int64_t pitch, int32_t *d_id, int64_t n,
                          void *stream, trk_bunch **out);
/* Frees the wrapper and the library scratch only (never the caller arrays). */
trk_status trk_bunch_free(trk_bunch *b);

/* Reference momentum carried by the bunch [eV]; set from the lattice at the
 * first trk_track unless set explicitly.  trk_bunch_p0c synchronises. */
trk_status trk_bunch_set_p0c(trk_bunch *b, double p0c_ev);
trk_status trk_bunch_p0c(trk_bunch *b, double *p0c_ev);

/* Absolute turn counter of the bunch (turns tracked so far; loss records carry
 * it).  Checkpoint and restart: copy the alive slots [0, n_alive) of the
 * coordinates and ids, trk_bunch_p0c and trk_bunch_turn to the host; later wrap
 * copies of them as a new bunch and set its p0c and turn: tracking continues
 * bit-identically (the loss records before the checkpoint stay with the old
 * bunch).  trk_bunch_set_turn takes 0 .. 2^31 - 1; neither call touches the
 * device. */
trk_status trk_bunch_set_turn(trk_bunch *b, int64_t turn);
trk_status trk_bunch_turn(const trk_bunch *b, int64_t *turn);

/* Launch schedule: threads per block (64..256, multiple of 32), particles per
 * thread (1, 2 or 4, advanced in lock-step), turns per fused launch between
 * compactions (>= 1).  Zero
 * fields keep the current value. */
typedef struct {
    int32_t block;
    int32_t per_thread;
    int32_t chunk_turns;
    int32_t growth;      /* batched calls: 0 = every chunk chunk_turns long; g >= 2 =
                            chunks grow by g from chunk_turns up to 128 turns (dense
                            warps while many particles are lost early) */
} trk_schedule;
trk_status trk_bunch_set_schedule(trk_bunch *b, const trk_schedule *s);

/* Track the alive particles n_turns turns through the lattice (Sec. 2-3):
 * every element in order, the aperture at every element exit, moments after
 * every turn, stable compaction of survivors after each chunk of turns.
 * Asynchronous on the bunch's stream.  Loss records carry the absolute turn
 * (counted over all trk_track calls of this bunch) and the element index. */
trk_status trk_track(trk_bunch *b, const trk_lattice *lat, int32_t n_turns);

/* Track one physical bunch held in n_parts parts (Sec. 4: the particle count
 * grows beyond one kernel's working set, 8M particles per GPU and 1e9 in all;
 * Sec. 2.2-2.3: a wake's histogram is taken over the whole bunch).  Each part
 * is a trk_bunch over its own caller arrays (ids distinct across parts if the
 * caller wants to tell particles apart); the parts are tracked, compacted and
 * get per-turn moments each on their own (moments of part k are those of its
 * alive particles), but every collective element (TRK_WAKE, TRK_LSC) acts on
 * the union of the parts' alive particles: one l window over all parts, one
 * histogram, the field computed once with q_m = charge / (sum of the parts' n),
 * and the kick applied to every part.  The coordinates equal, bit for bit,
 * those of trk_track on one bunch holding all the particles: the window is an
 * exact min/max and the histogram and dipole sums are integer sums, whatever
 * the split.  All parts must use the same stream and share the
 * reference momentum and the turn counter (TRK_EINVAL otherwise); the first
 * part holds the collective scratch.  n_parts = 1 is trk_track. */
trk_status trk_track_parts(trk_bunch *const *parts, int32_t n_parts, const trk_lattice *lat, int32_t n_turns);

/* Per-turn moments of the last trk_track call, host_out[t*28 + q]:
 *   q = 0      number of alive particles after turn t
 *   q = 1..6   means of the 6 coordinates
 *   q = 7..27  population central second moments <d_j d_k>, j <= k
 *              lexicographic (0,0) (0,1) .. (0,5) (1,1) .. (5,5)
 * (all zero when no particle is alive).  cap_turns bounds the rows written;
 * *n_turns receives the number of rows available.  Synchronises. */
trk_status trk_moments(trk_bunch *b, double *host_out, int32_t cap_turns, int32_t *n_turns);

/* Lost particles so far (slots [n_alive, n)): ids, absolute loss turn and
 * element index, host arrays of capacity cap.  Synchronises. */
trk_status trk_lost(trk_bunch *b, int32_t *ids, int32_t *turn, int32_t *elem,
                    int64_t cap, int64_t *n_lost);
trk_status trk_n_alive(trk_bunch *b, int64_t *n_alive);

/* Standalone longitudinal wake (one TRK_WAKE element) on the alive particles
 * of the bunch, at reference momentum p0c_ev; q_m = charge / n (n = particles
 * wrapped).  d_hist [nbins] uint32 counts and d_volt [nbins] FP64 voltages are
 * optional caller device outputs (NULL to skip).  Asynchronous. */
trk_status trk_wake(trk_bunch *b, int32_t nbins, double w0, double sc, double charge,
                    double p0c_ev, uint32_t *d_hist, double *d_volt);

/* Batched tracking (many lattice variants with uneven particle counts in one
 * launch per turn chunk; no counterpart in the paper, which tracks one beamline).
 * A batch pairs bunch v with lattice v; every bunch must use the same stream and
 * no lattice may contain TRK_WAKE (TRK_EUNSUPPORTED).  trk_batch_track runs
 * n_turns turns of every pair: per chunk one fused launch over all (variant,
 * tile) items, then moment finalisation and stable compaction of every variant;
 * all chunks of a call are one CUDA graph, captured on the first call with a
 * given n_turns and schedule and replayed afterwards.  Per-bunch results
 * (trk_moments, trk_lost, trk_n_alive) are as after trk_track.  The batch only
 * borrows the bunches and lattices; they must outlive it. */
typedef struct trk_batch trk_batch;
trk_status trk_batch_create(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                            trk_batch **out);
trk_status trk_batch_set_schedule(trk_batch *B, const trk_schedule *s);
trk_status trk_batch_get_schedule(const trk_batch *B, trk_schedule *s);
trk_status trk_batch_track(trk_batch *B, int32_t n_turns);
trk_status trk_batch_destroy(trk_batch *B);
/* Project-written autotuner for batched calls: times probe_turns turns of
 * every candidate schedule -- (block, particles per thread) in {(128,1),
 * (128,2), (64,2), (256,2), (128,4), (64,4)} x chunk plan {fixed chunks of
 * probe_turns, growing chunks 1, 2, 4, ...} -- on shadow copies of the alive
 * particles (the caller's bunches are not changed), and returns the fastest in
 * *out (and its probe time in *best_ms if not NULL).  Synchronises. */
trk_status trk_autotune(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                        int32_t probe_turns, trk_schedule *out, double *best_ms);
/* One-shot form: create, set the schedule (if sched != NULL), track, destroy. */
trk_status trk_track_batch(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                           int32_t n_turns, const trk_schedule *sched);

/* Dynamic-aperture survival (no counterpart in the paper).  Variant v's points
 * are [offsets[v], offsets[v+1]) of the device arrays d_x0, d_y0 [m]; a particle
 * starts at (x0, 0, y0, 0, 0, 0) and is tracked through lattice v for up to
 * n_turns turns (batched, as trk_batch_track; the lattices' apertures decide
 * losses; create them with moments = 0 to skip the moment sums).
 * d_survival[p] (int32, device) receives the 1-based turn in which particle p
 * was lost, or n_turns + 1 if it survived.  offsets is a HOST array of n_var+1
 * entries starting at 0.  sched = NULL uses block 128, 2 particles per thread,
 * chunks of 1, 2, 4, ... 128 turns, or, for at most 16384 points on lattices of
 * MAP, EDRIFT and THINSEXT elements, trk_da_survival_lanes.  Only loss turns
 * leave the call, so map rows on which no aperture test depends (directly or
 * through other rows; for a ring of maps and thin sextupoles, the path-length
 * row) are not evaluated: every loss decision is the one full tracking takes.
 * Allocates its particle arrays and synchronises the stream before returning. */
trk_status trk_da_survival(const trk_lattice *const *lats, int32_t n_var, const int64_t *offsets,
                           const double *d_x0, const double *d_y0, int32_t n_turns, const trk_schedule *sched,
                           int32_t *d_survival, void *stream);

/* The same survival turns (bit-identical) for few points: each particle gets 8
 * GPU lanes (4 when no lattice's survival rows go beyond x, x', y, y'), lane r
 * evaluating map row r, so the rows of a map are evaluated in parallel and one
 * particle's chain of dependent operations per turn is shorter; one launch
 * covers all n_turns turns, lost particles stop at once.
 * Lattices may hold MAP, EDRIFT and THINSEXT elements only (TRK_EUNSUPPORTED
 * otherwise); at most 2^28 points.  Arguments as trk_da_survival.
 * Synchronises the stream before returning. */
trk_status trk_da_survival_lanes(const trk_lattice *const *lats, int32_t n_var, const int64_t *offsets,
                                 const double *d_x0, const double *d_y0, int32_t n_turns, int32_t *d_survival,
                                 void *stream);

/* MLP surrogate for dynamic-aperture triage (no counterpart in the paper).
 * Fixed architecture 8 -> 4 x [Linear 256 + GELU(erf)] -> Linear 256 -> 1 logit.
 * FP32 master weights and biases with BF16 copies; BF16 activations into the
 * tensor-core products (tcgen05, FP32 accumulation in tensor memory); BCE loss
 * on the logit; Adam (Kingma & Ba).  Rounding points: h0 = bf16(x),
 * z = h W^T + b (FP32), h = bf16(gelu(z)); dz = dh * gelu'(z) (FP32) rounded to
 * BF16 for dW = dz^T h and dh = dz W; db = sum dz (FP32).  Inference
 * (trk_mlp_forward) runs its hidden layers as persistent 128 x 256 tiles;
 * training (trk_mlp_grad, trk_mlp_train) runs every product -- forward, input
 * gradient, weight gradient split over the batch and summed in split order --
 * as 128 x 32 (forward, input gradient) and 128 x 64 (weight gradient) tiles;
 * the rounding points are the same.
 *   W[l], b[l]   HOST FP32 arrays, W[l] row-major [out][in]: l = 0: 256 x 8,
 *                l = 1..3: 256 x 256, l = 4: 1 x 256; b[l] [out]
 *   d_X          device FP32 [M][8] inputs; d_y device FP32 [M] labels (0/1)
 * trk_mlp_forward writes logits (device FP32 [M]); trk_mlp_grad computes the
 * gradients of the mean loss of M rows (kept inside; d_loss device FP32 [1]
 * or NULL); trk_mlp_adam applies one Adam step with them; trk_mlp_train runs
 * epochs over n rows in batches (d_perm: device int32 [epochs][n] row order
 * per epoch, or NULL for the stored order; d_loss_hist: device FP32, one
 * entry per step, or NULL).  trk_mlp_get copies weights, biases and the last
 * gradients to host arrays of the layout above (NULL entries skipped) and
 * synchronises.  All calls are asynchronous on `stream` except trk_mlp_get,
 * trk_mlp_train and trk_mlp_forward, which synchronise at the end
 * (trk_mlp_forward returns TRK_ETIMEOUT if a tensor-core layer gave up a
 * bounded wait). */
typedef struct trk_mlp trk_mlp;
trk_status trk_mlp_create(const float *const *W, const float *const *b, trk_mlp **out);
trk_status trk_mlp_destroy(trk_mlp *net);
trk_status trk_mlp_forward(trk_mlp *net, const float *d_X, int64_t M, float *d_logits, void *stream);
/* trk_mlp_forward that also copies each hidden layer's BF16 output (the
 * activations the next product reads) to d_hidden, device uint16 [4][M][256]
 * row-major (layer l, row m at (l * M + m) * 256); d_hidden NULL is plain
 * trk_mlp_forward.  For inspecting the network and for checking its rounding
 * layer by layer. */
trk_status trk_mlp_forward_hidden(trk_mlp *net, const float *d_X, int64_t M, float *d_logits, uint16_t *d_hidden,
                                  void *stream);
trk_status trk_mlp_grad(trk_mlp *net, const float *d_X, const float *d_y, int32_t M, float *d_loss, void *stream);
trk_status trk_mlp_adam(trk_mlp *net, float lr, float beta1, float beta2, float eps, void *stream);
trk_status trk_mlp_train(trk_mlp *net, const float *d_X, const float *d_y, int64_t n, int32_t batch,
                         int32_t epochs, const int32_t *d_perm, float lr, float *d_loss_hist, void *stream);
trk_status trk_mlp_get(trk_mlp *net, float *const *W, float *const *b, float *const *gW, float *const *gb);

/* Surrogate-triaged dynamic-aperture scan (no counterpart in the paper).  For
 * every variant v and cell (ix, iy) of an nx x ny grid (cell centres
 * -w + (i + 1/2) 2w/n, w = half_width):
 *   1. the coarse cells (every coarse_stride-th cell from stride/2) and the
 *      sentinel cells (sentinel_stride below) are tracked exactly in one scan
 *      (trk_da_survival);
 *   2. use_mlp = 1: the network is trained on the coarse cells (features x/w, y/w and the
 *      variant's 6 normalised parameters d_params[v][6]; label = survives all
 *      n_turns) with trk_mlp_train(epochs, batch, lr, d_perm) and predicts every
 *      cell (logit > 0 = survives); use_mlp = 0: every cell takes the label of
 *      its nearest known cell (the nearest coarse cell, or the nearest sentinel
 *      cell where that is strictly closer); use_mlp = 2: the network, trained
 *      as for 1, predicts only the cells within Chebyshev distance 3 of a
 *      boundary cell of the nearest-known prediction (where the known cells
 *      disagree), the nearest known cell the rest; the known labels override
 *      every form;
 *   3. cells within Chebyshev distance band_radius of a predicted-boundary cell
 *      (8-neighbourhood holding both classes), and the caller's audit cells
 *      (d_audit[v][iy][ix] != 0, optional), are re-tracked exactly in FP64 and
 *      merged; the boundary of the merged mask is taken again and the band
 *      cells not yet tracked are tracked, pass after pass (max_passes at most),
 *      until a pass finds none, so every cell within band_radius of the final
 *      boundary is exact (sentinel_stride, expand_radius below);
 *   4. d_mask (uint8 [n_var][ny][nx], 1 = survives) and d_survival (int32,
 *      1-based loss turn or n_turns + 1 where tracked; n_turns + 1 or 0 from the
 *      prediction elsewhere) receive the merged result; stats (host) counts
 *      cells, passes and audit disagreements (audit cells whose exact label
 *      differs from the prediction) and times each phase.
 * Allocates its working arrays and synchronises `stream`. */
typedef struct {
    int32_t nx, ny;
    double half_width;
    int32_t n_turns;
    int32_t coarse_stride;
    int32_t band_radius;
    int32_t use_mlp;
    int32_t epochs, batch;
    float lr;
    int32_t max_passes;       /* band passes at most (0: 64) */
    int32_t sentinel_stride;  /* > 0: also track, with the coarse cells, the cells of
                               * a sub-lattice with this stride on both axes (from
                               * stride/2, plus the cell stride/2 from the far edge);
                               * <= 2 band_radius + 1 makes the one-cell boundary
                               * criterion hold by construction; 0: none */
    int32_t expand_radius;    /* passes after the first also track the cells within
                               * this Chebyshev distance of a cell whose label the
                               * previous merge flipped (0: none) */
} trk_triage_opts;
typedef struct {
    int64_t n_cells, n_coarse, n_band, n_audit, n_tracked, n_audit_wrong;
    double ms_coarse, ms_train, ms_infer, ms_band, ms_retrack;
    int64_t n_passes;     /* band passes that tracked at least one cell */
    int64_t pass_cells[16];  /* cells tracked in pass k (passes past 15 add to [15]) */
    double pass_ms[16];      /* wall time of pass k: band, gather, track, merge */
    int64_t n_sentinel;      /* sentinel cells tracked with the coarse cells */
    int64_t n_region;        /* cells the network predicted (use_mlp 1: every cell; 2: the region) */
} trk_triage_stats;
trk_status trk_da_triage(const trk_lattice *const *lats, int32_t n_var, const float *d_params,
                         const uint8_t *d_audit, trk_mlp *net, const int32_t *d_perm, const trk_triage_opts *opts,
                         uint8_t *d_mask, int32_t *d_survival, trk_triage_stats *stats, void *stream);

/* Launch statistics of a bunch.  With timing enabled the library records CUDA
 * events on the bunch's stream around every fused tracking launch; the summed
 * device time of those launches is track_kernel_ms.  trk_bunch_stats
 * synchronises; reset != 0 zeroes the counters afterwards. */
typedef struct {
    double track_kernel_ms;   /* device time of the fused tracking launches [ms] */
    int64_t track_launches;   /* fused tracking launches */
    int64_t launches;         /* all kernel launches issued for this bunch */
} trk_stats;
trk_status trk_bunch_enable_timing(trk_bunch *b, int32_t on);
trk_status trk_bunch_stats(trk_bunch *b, trk_stats *out, int32_t reset);

/* The standalone wake of trk_wake for callers that cannot allocate device
 * memory.  The paper has no counterpart: it is an addition for code that runs
 * where allocation is not allowed (inside a fixed memory pool, a host
 * application that forbids cudaMalloc after start-up, or a device already
 * full).  The caller passes the particles and the outputs; nothing is
 * allocated.  The working arrays live in one file-scope device array of fixed
 * size (nbins <= 16384, 320.25 KiB) that every GPU loading the library holds
 * until the process exits.
 * Unlike trk_wake, which works on a bunch's alive particles, this call has no
 * id or alive array: EVERY one of the n particles counts as alive (in the l
 * window, the histogram and the kick), so a caller with lost particles passes
 * only the alive ones (compacted to the front).
 *   d_coords   [6 * pitch] FP64 SoA coordinates (caller-owned, device);
 *              delta (coordinate 5) receives the kick in place
 *   pitch, n   row pitch and particle count (0 <= n <= pitch)
 *   nbins      histogram bins over [min l, max l], 1..16384
 *   w0, sc     wake amplitude [V m^(1/2) / C] and cutoff distance [m]:
 *              W(s) = w0 / sqrt(max(s, sc)), as for trk_wake
 *   charge     total bunch charge [C]; divided by n inside as the charge per
 *              macro-particle q_m
 *   p0c_ev     reference momentum [eV] for the kick delta += V(l) / p0c
 *   d_hist     [nbins] uint32 counts, d_volt [nbins] FP64 voltages: optional
 *              caller device outputs (NULL to skip)
 *   stream     cudaStream_t (NULL = legacy default stream)
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it for the life
 * of the process; make that first call before any stream capture, and do not
 * use the library across a cudaDeviceReset (the cached address would then
 * point at memory that no longer exists).  Every call shares the array and
 * leaves its contents to the next; each call clears what must start at zero,
 * and calls whose work overlaps on the GPU race on it.  Returns TRK_EINVAL
 * for nbins outside 1..16384, n < 0, pitch < n or p0c_ev <= 0. */
trk_status trk_wake_static(double *d_coords, int64_t pitch, int64_t n, int32_t nbins, double w0, double sc,
                           double charge, double p0c_ev, uint32_t *d_hist, double *d_volt, void *stream);

/* Measured FP64 issue rates of the current device (no counterpart in the
 * paper; the measured denominator beside the derived FP64 peak of a roofline).
 * out[0], out[1], out[2] (host) receive thread-level DFMA, DMUL and DADD
 * operations per second of a kernel with 4 blocks of 256 threads per SM, each
 * thread running 8 independent dependent chains.  Allocates a small scratch
 * array, launches on `stream` and synchronises it. */
trk_status trk_probe_fp64(double *out, void *stream);

/* Text for the calling thread's last non-OK status ("" if none). */
const char *trk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TRK_H */
