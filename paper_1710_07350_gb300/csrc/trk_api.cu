// C ABI: lattice compilation, bunch scratch, and the launch schedule of
// trk_track (fused launches per turn chunk, wake steps, moment finalisation,
// loss compaction).  See include/trk.h for the contract of every call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "trk_internal.cuh"

using namespace trk;

namespace {

thread_local std::string g_err;

trk_status fail(trk_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define TRK_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(TRK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr double kClight = 299792458.0;

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// Monomial code of (j[,k[,l]]) for a map term.
int32_t mono_code(int deg, int j, int k, int l) { return deg | (j << 2) | (k << 5) | (l << 8); }

}  // namespace

struct trk_lattice {
    std::vector<DevElem> elems;
    std::vector<DevTerm> terms;
    DevElem *d_elems = nullptr;
    DevTerm *d_terms = nullptr;
    LatticeView view{};
    int moments = 1;
    double p0c = 0.0;
    std::vector<int> wakes;  // element indices of TRK_WAKE and TRK_LSC
    // collective groups: one collective element, or two adjacent ones (second >= 0),
    // which share one l window and kick together in the next segment's prologue
    std::vector<std::pair<int, int>> groups;
    int max_bins = 0;
    bool transverse = false; // a wake with a transverse part
    uint32_t survival_rows = 0x3Fu;  // map rows a survival scan needs (survival_rows())
    uint32_t survival_zero = 0u;     // coordinates that stay exactly zero in a survival scan (survival_zeros())
    // survival view: the elements with map rows limited to survival_rows and
    // without the terms that have a factor in survival_zero (its own copies when
    // that removes anything, else the tracking arrays)
    std::vector<DevElem> selems;
    std::vector<DevTerm> sterms;
    DevElem *d_selems = nullptr;
    DevTerm *d_sterms = nullptr;
    LatticeView sview{};
};

struct trk_bunch {
    double *coords = nullptr;
    int64_t pitch = 0;
    int32_t *ids = nullptr;
    int64_t n = 0;
    cudaStream_t stream = nullptr;
    int32_t *lt = nullptr, *le = nullptr;
    double *cb = nullptr;
    int32_t *ib = nullptr, *ltb = nullptr, *leb = nullptr;
    BunchState *st = nullptr;
    int block = 128, per_thread = 1, chunk = 100;
    int32_t *tile_alive = nullptr;
    int64_t *tile_off = nullptr;
    int64_t tiles_cap = 0;
    double *partials = nullptr;
    size_t partials_rows = 0;
    double *moments = nullptr;
    int moments_cap = 0, moments_turns = 0;
    uint32_t *hist = nullptr;
    double *wfun = nullptr, *V = nullptr;
    unsigned long long *dip = nullptr;            // transverse dipole sums [2][bins], fixed point
    double *wfun_t = nullptr, *Vt = nullptr;      // transverse wake samples, voltages [2][bins]
    double *V2 = nullptr, *Vt2 = nullptr;         // voltages of the second element of a group
    double *lsc = nullptr;                        // space-charge scratch [4 bins]
    int wake_cap = 0;
    int64_t turn = 0;
    double p0c = 0.0;
    bool p0c_set = false;
    // statistics
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;  // recorded pairs
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
    int64_t track_launches = 0, launches = 0;
    double track_ms = 0.0;
};

// Fused tracking launch with optional event timing and launch counting.
static cudaError_t track_launch(trk_bunch *b, const TrackArgs &a, int n_tiles) {
    // a launch that kicks with a collective element or fills its window reads
    // the window keys; never send it without them
    if ((a.kick_wake >= 0 || a.minmax_slot >= 0) && !a.win) return cudaErrorInvalidValue;
    std::pair<cudaEvent_t, cudaEvent_t> pr{nullptr, nullptr};
    if (b->timing) {
        if (!b->ev_free.empty()) {
            pr = b->ev_free.back();
            b->ev_free.pop_back();
        } else {
            cudaError_t e = cudaEventCreate(&pr.first);
            if (e == cudaSuccess) e = cudaEventCreate(&pr.second);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventRecord(pr.first, b->stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_track(a, b->block, b->per_thread, n_tiles, b->stream);
    if (e != cudaSuccess) return e;
    ++b->track_launches;
    ++b->launches;
    if (b->timing) {
        e = cudaEventRecord(pr.second, b->stream);
        if (e != cudaSuccess) return e;
        b->ev.push_back(pr);
    }
    return cudaSuccess;
}

// ------------------------------------------------------------- lattice ----

static trk_status compile_map(const trk_element_desc &d, int idx, DevElem &E, std::vector<DevTerm> &terms) {
    if (!d.R) return fail(TRK_EINVAL, "element " + std::to_string(idx) + ": TRK_MAP needs R");
    if (d.order < 1 || d.order > 3) return fail(TRK_EINVAL, "element " + std::to_string(idx) + ": order must be 1..3");
    if (d.order >= 2 && !d.T) return fail(TRK_EINVAL, "element " + std::to_string(idx) + ": order >= 2 needs T");
    if (d.order >= 3 && !d.U) return fail(TRK_EINVAL, "element " + std::to_string(idx) + ": order 3 needs U");
    E.term0 = (int32_t)terms.size();
    E.n = d.order;
    E.flags = 0;
    int pos = 0;
    bool delta_changes = false;
    for (int r = 0; r < 6; ++r) {
        E.rb[r] = (int16_t)pos;
        auto add = [&](double c, int32_t code) {
            if (c == 0.0) return;
            DevTerm t;
            t.c = c;
            t.code = code;
            t.pad = 0;
            terms.push_back(t);
            ++pos;
        };
        if (d.R[6 * r + r] == 1.0) E.flags |= 1u << r;
        if (d.C) add(d.C[r], mono_code(0, 0, 0, 0));
        for (int j = 0; j < 6; ++j) {
            if (j == r && d.R[6 * r + r] == 1.0) continue;
            add(d.R[6 * r + j], mono_code(1, j, 0, 0));
        }
        if (d.order >= 2) {
            int q = 0;
            for (int j = 0; j < 6; ++j)
                for (int k = j; k < 6; ++k, ++q) add(d.T[21 * r + q], mono_code(2, j, k, 0));
        }
        if (d.order >= 3) {
            int q = 0;
            for (int j = 0; j < 6; ++j)
                for (int k = j; k < 6; ++k)
                    for (int l = k; l < 6; ++l, ++q) add(d.U[56 * r + q], mono_code(3, j, k, l));
        }
        if (r == 5 && (pos > E.rb[5] || !(E.flags & 32u))) delta_changes = true;
        if (pos > 32000) return fail(TRK_EINVAL, "element " + std::to_string(idx) + ": too many map terms");
    }
    E.rb[6] = (int16_t)pos;
    E.rb[7] = (int16_t)pos;
    if (delta_changes) E.flags |= 64u;
    return TRK_OK;
}

// Coordinates a survival scan needs: the aperture reads x and y; a map row
// that is needed reads the coordinates of its terms (and its own, when its
// diagonal coefficient is 1), leaving out the terms with a factor in `zero`
// (survival_zeros: exactly zero, and dropped from the scan's terms); a thin
// sextupole reads x and y; an exact drift
// moves x, y by the slopes and l by a function of both.  The set is grown over
// the whole lattice until it stops changing (the lattice repeats every turn).
// Rows outside it never influence an aperture test, so a survival scan may
// skip them and still take bit-identical decisions.  Any other element type
// keeps every row.
static uint32_t survival_rows(const trk_lattice &L, uint32_t zero) {
    uint32_t need = 0x5u;   // x (0) and y (2)
    for (int it = 0; it < 8; ++it) {
        const uint32_t before = need;
        for (const DevElem &E : L.elems) {
            if (E.type == TRK_MAP) {
                for (int r = 0; r < 6; ++r) {
                    if (!((need >> r) & 1u)) continue;
                    for (int k = E.rb[r]; k < E.rb[r + 1]; ++k) {
                        const int code = L.terms[E.term0 + k].code;
                        const int deg = code & 3;
                        uint32_t f = 0;   // the term's factors
                        if (deg >= 1) f |= 1u << ((code >> 2) & 7);
                        if (deg >= 2) f |= 1u << ((code >> 5) & 7);
                        if (deg >= 3) f |= 1u << ((code >> 8) & 7);
                        if (!(f & zero)) need |= f;   // a term with a factor that stays zero is dropped
                    }
                }
            } else if (E.type == TRK_THINSEXT) {
                need |= 0x5u;
            } else if (E.type == TRK_EDRIFT) {
                if (need & 0x15u) need |= 0xAu;   // x, y or l needs the slopes
            } else {
                return 0x3Fu;
            }
        }
        if (need == before) break;
    }
    return need & 0x3Fu;
}

// Coordinates that stay exactly zero in a survival scan, which starts every
// particle at (x0, 0, y0, 0, 0, 0): the set starts as {x', y', l, delta} and a
// coordinate leaves it when an element can make it nonzero from coordinates
// outside the set -- a map row with a term none of whose factors is in the set
// (a constant term included), a thin sextupole (x', y' from x, y), an exact
// drift (l from the slopes).  Repeated over the lattice until it stops
// changing, this is the set that holds at every element of every turn.  A term
// with a factor in it is exactly zero and adds nothing (at most the sign of a
// zero sum changes, which no loss decision reads).  Any other element type:
// nothing is known to stay zero.
static uint32_t survival_zeros(const trk_lattice &L) {
    uint32_t zero = 0x3Au;   // x' (1), y' (3), l (4), delta (5)
    for (int it = 0; it < 8; ++it) {
        const uint32_t before = zero;
        for (const DevElem &E : L.elems) {
            if (E.type == TRK_MAP) {
                for (int r = 0; r < 6; ++r) {
                    if (!((zero >> r) & 1u)) continue;
                    for (int k = E.rb[r]; k < E.rb[r + 1]; ++k) {
                        const int code = L.terms[E.term0 + k].code;
                        const int deg = code & 3;
                        bool has_zero = false;
                        if (deg >= 1) has_zero |= (zero >> ((code >> 2) & 7)) & 1u;
                        if (deg >= 2) has_zero |= (zero >> ((code >> 5) & 7)) & 1u;
                        if (deg >= 3) has_zero |= (zero >> ((code >> 8) & 7)) & 1u;
                        if (!has_zero) {
                            zero &= ~(1u << r);
                            break;
                        }
                    }
                }
            } else if (E.type == TRK_THINSEXT) {
                if ((zero & 0x5u) != 0x5u) zero &= ~0xAu;   // x or y nonzero: x', y' may become nonzero
            } else if (E.type == TRK_EDRIFT) {
                if ((zero & 0xAu) != 0xAu) zero &= ~0x10u;  // a slope nonzero: l may become nonzero
            } else {
                return 0u;
            }
        }
        if (zero == before) break;
    }
    return zero;
}

// The survival view's element and term arrays (host): map rows outside
// `rows` get no terms, and terms with a factor in `zero` are left out.
static bool build_survival_terms(const trk_lattice &L, uint32_t rows, uint32_t zero, std::vector<DevElem> &elems,
                                 std::vector<DevTerm> &terms) {
    elems = L.elems;
    terms.clear();
    bool changed = false;
    for (size_t i = 0; i < elems.size(); ++i) {
        DevElem &E = elems[i];
        if (E.type != TRK_MAP) continue;
        const DevElem &O = L.elems[i];
        E.term0 = (int32_t)terms.size();
        int cnt = 0;
        for (int r = 0; r < 6; ++r) {
            E.rb[r] = (int16_t)cnt;
            if (!((rows >> r) & 1u)) {
                changed |= O.rb[r + 1] > O.rb[r];
                continue;
            }
            for (int k = O.rb[r]; k < O.rb[r + 1]; ++k) {
                const DevTerm &t = L.terms[O.term0 + k];
                const int deg = t.code & 3;
                bool has_zero = false;
                if (deg >= 1) has_zero |= (zero >> ((t.code >> 2) & 7)) & 1u;
                if (deg >= 2) has_zero |= (zero >> ((t.code >> 5) & 7)) & 1u;
                if (deg >= 3) has_zero |= (zero >> ((t.code >> 8) & 7)) & 1u;
                if (has_zero) {
                    changed = true;
                    continue;
                }
                terms.push_back(t);
                ++cnt;
            }
        }
        E.rb[6] = (int16_t)cnt;
        E.rb[7] = (int16_t)cnt;
    }
    return changed;
}

extern "C" trk_status trk_create_lattice(const trk_element_desc *elems, int32_t n, const trk_lattice_opts *opts,
                                         trk_lattice **out) {
    if (!out) return fail(TRK_EINVAL, "trk_create_lattice: out is NULL");
    *out = nullptr;
    if (!opts) return fail(TRK_EINVAL, "trk_create_lattice: opts is NULL");
    if (n < 0 || (n > 0 && !elems)) return fail(TRK_EINVAL, "trk_create_lattice: bad element array");
    if (!(opts->p0c_ev > 0.0)) return fail(TRK_EINVAL, "trk_create_lattice: p0c_ev must be > 0");
    if (opts->aperture != TRK_APERTURE_NONE && opts->aperture != TRK_APERTURE_RECT &&
        opts->aperture != TRK_APERTURE_ELLIPSE)
        return fail(TRK_EINVAL, "trk_create_lattice: unknown aperture type");
    if (opts->aperture != TRK_APERTURE_NONE && !(opts->a > 0.0 && opts->b > 0.0))
        return fail(TRK_EINVAL, "trk_create_lattice: aperture half-widths must be > 0");
    auto *L = new trk_lattice();
    L->moments = opts->moments ? 1 : 0;
    L->p0c = opts->p0c_ev;
    const double w1 = 1.0 / (2.0 - std::cbrt(2.0));
    const double w0 = 1.0 - 2.0 * w1;
    for (int i = 0; i < n; ++i) {
        const trk_element_desc &d = elems[i];
        DevElem E;
        std::memset(&E, 0, sizeof E);
        E.type = d.type;
        trk_status s = TRK_OK;
        switch (d.type) {
        case TRK_MAP: s = compile_map(d, i, E, L->terms); break;
        case TRK_EDRIFT:
            if (!std::isfinite(d.length)) s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": bad length");
            E.p[0] = d.length;
            E.p[1] = 0.5 * d.length;
            E.p[2] = 0.375 * d.length;
            break;
        case TRK_KQUAD:
        case TRK_KSEXT: {
            if (d.n_kicks < 1) {
                s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": n_kicks must be >= 1");
                break;
            }
            const double k2 = d.type == TRK_KSEXT ? d.k2 : 0.0;
            const double h = d.length / d.n_kicks;
            E.n = d.n_kicks;
            E.p[0] = 0.5 * w1 * h;
            E.p[1] = 0.5 * (w0 + w1) * h;
            E.p[2] = w1 * h;
            E.p[3] = d.k1 * (w1 * h);
            E.p[4] = d.k1 * (w0 * h);
            E.p[5] = (0.5 * k2) * (w1 * h);
            E.p[6] = (0.5 * k2) * (w0 * h);
            E.p[7] = 0.5 * E.p[0];
            E.p[8] = 0.375 * E.p[0];
            E.p[9] = 0.5 * E.p[1];
            E.p[10] = 0.375 * E.p[1];
            E.p[11] = 0.375 * E.p[2];
            E.flags = (d.k1 != 0.0 ? 1u : 0u) | (k2 != 0.0 ? 2u : 0u);
            break;
        }
        case TRK_THINSEXT:
            E.p[0] = d.k2l;
            E.p[1] = 0.5 * d.k2l;
            break;
        case TRK_RFCA: {
            const double phi = d.phase_deg * kPi / 180.0;
            E.p[0] = d.volt;
            E.p[1] = phi;
            E.p[2] = 2.0 * kPi * d.freq_hz / kClight;
            E.p[3] = d.volt * std::cos(phi);
            E.p[4] = std::cos(phi);
            E.p[5] = std::sin(phi);
            break;
        }
        case TRK_SBEND:
            if (!(d.length > 0.0) || !std::isfinite(d.length) || !(std::fabs(d.angle) < 3.14159265358979)) {
                s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": bad sector bend");
                break;
            }
            if (d.angle == 0.0) {   // the exact drift
                E.type = TRK_EDRIFT;
                E.p[0] = d.length;
                E.p[1] = 0.5 * d.length;
                E.p[2] = 0.375 * d.length;
                break;
            }
            E.p[0] = d.length;
            E.p[1] = d.angle;
            E.p[2] = d.length / d.angle;     // rho
            E.p[3] = d.angle / d.length;     // 1 / rho
            E.p[4] = std::sin(d.angle);
            E.p[5] = std::cos(d.angle);
            break;
        case TRK_LSC:
            if (d.nbins < 1 || d.nbins > kMaxBins || d.n_kicks < 0 || d.n_kicks > 1000 ||
                !std::isfinite(d.lsc_k) || !std::isfinite(d.length) || !std::isfinite(d.charge)) {
                s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": bad space-charge parameters");
                break;
            }
            E.n = d.nbins;
            E.flags = (uint32_t)d.n_kicks;
            E.term0 = (int32_t)L->wakes.size();
            if (d.lsc_rb != 0.0) {   // the impedance of a round beam
                const bool pow2 = (d.nbins & (d.nbins - 1)) == 0;
                const bool filt = !(d.lsc_f1 > 0.0) || (d.lsc_f0 >= 0.0 && d.lsc_f0 < d.lsc_f1 && d.lsc_f1 <= 1.0);
                if (!(d.lsc_rb > 0.0) || !std::isfinite(d.lsc_rb) || !(d.lsc_mc2 > 0.0) ||
                    !std::isfinite(d.lsc_mc2) || !pow2 || d.nbins > kLscImpMaxBins || !filt ||
                    !std::isfinite(d.lsc_f0) || !std::isfinite(d.lsc_f1)) {
                    s = fail(TRK_EINVAL, "element " + std::to_string(i) +
                                             ": bad space-charge impedance (r_b > 0, rest energy > 0, nbins a "
                                             "power of two up to 4096, 0 <= f0 < f1 <= 1 or f1 <= 0)");
                    break;
                }
                E.p[5] = d.lsc_rb;
                E.p[6] = d.lsc_mc2;
                E.p[7] = d.lsc_f0;
                E.p[8] = d.lsc_f1;
                E.p[9] = d.length;
            }
            E.p[2] = d.charge;
            E.p[4] = d.lsc_k * d.length;
            L->wakes.push_back(i);
            if (d.nbins > L->max_bins) L->max_bins = d.nbins;
            break;
        case TRK_WAKE:
            if (d.nbins < 1 || d.nbins > kMaxBins) {
                s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": nbins must be 1..65536");
                break;
            }
            E.n = d.nbins;
            E.term0 = (int32_t)L->wakes.size();
            if (!std::isfinite(d.wake_w0) || !std::isfinite(d.wake_w0t) || !(d.wake_sc > 0.0)) {
                s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": bad wake parameters");
                break;
            }
            E.p[0] = d.wake_w0;
            E.p[1] = d.wake_sc;
            E.p[2] = d.charge;
            E.p[3] = d.wake_w0t;
            if (d.wake_w0t != 0.0) L->transverse = true;
            L->wakes.push_back(i);
            if (d.nbins > L->max_bins) L->max_bins = d.nbins;
            break;
        default: s = fail(TRK_EINVAL, "element " + std::to_string(i) + ": unknown type " + std::to_string(d.type));
        }
        if (s != TRK_OK) {
            delete L;
            return s;
        }
        L->elems.push_back(E);
    }
    for (int w : L->wakes) {
        if (!L->groups.empty() && L->groups.back().second < 0 && L->groups.back().first + 1 == w)
            L->groups.back().second = w;
        else
            L->groups.push_back({w, -1});
    }
    cudaError_t e1 = dalloc(&L->d_elems, L->elems.size());
    cudaError_t e2 = dalloc(&L->d_terms, L->terms.size());
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFree(L->d_elems);
        cudaFree(L->d_terms);
        delete L;
        return fail(TRK_ENOMEM, "trk_create_lattice: device allocation failed");
    }
    cudaError_t e3 = cudaMemcpy(L->d_elems, L->elems.data(), L->elems.size() * sizeof(DevElem), cudaMemcpyHostToDevice);
    cudaError_t e4 = L->terms.empty() ? cudaSuccess
                                      : cudaMemcpy(L->d_terms, L->terms.data(), L->terms.size() * sizeof(DevTerm),
                                                   cudaMemcpyHostToDevice);
    if (e3 != cudaSuccess || e4 != cudaSuccess) {
        cudaFree(L->d_elems);
        cudaFree(L->d_terms);
        delete L;
        return fail(TRK_ECUDA, "trk_create_lattice: copy to device failed");
    }
    LatticeView &v = L->view;
    v.elems = L->d_elems;
    v.terms = L->d_terms;
    v.n_elem = n;
    v.ap_type = opts->aperture;
    v.row_mask = 0x3Fu;
    L->survival_zero = survival_zeros(*L);
    L->survival_rows = survival_rows(*L, L->survival_zero);
    v.ap_a = opts->a;
    v.ap_b = opts->b;
    // |x| <= a as integers: bit patterns of the positive bounds shifted left by one
    const auto key = [](double v) {
        uint64_t u;
        std::memcpy(&u, &v, 8);
        return (unsigned long long)(u << 1);
    };
    v.ap_a_key = key(opts->a);
    v.ap_b_key = key(opts->b);
    v.ap_ia_key = key(0.7 * opts->a);
    v.ap_ib_key = key(0.7 * opts->b);
    L->sview = v;
    L->sview.row_mask = L->survival_rows;
    if (build_survival_terms(*L, L->survival_rows, L->survival_zero, L->selems, L->sterms)) {
        cudaError_t e5 = dalloc(&L->d_selems, L->selems.size());
        if (e5 == cudaSuccess) e5 = dalloc(&L->d_sterms, L->sterms.size() ? L->sterms.size() : 1);
        if (e5 == cudaSuccess)
            e5 = cudaMemcpy(L->d_selems, L->selems.data(), L->selems.size() * sizeof(DevElem), cudaMemcpyHostToDevice);
        if (e5 == cudaSuccess && !L->sterms.empty())
            e5 = cudaMemcpy(L->d_sterms, L->sterms.data(), L->sterms.size() * sizeof(DevTerm), cudaMemcpyHostToDevice);
        if (e5 != cudaSuccess) {
            cudaFree(L->d_elems);
            cudaFree(L->d_terms);
            cudaFree(L->d_selems);
            cudaFree(L->d_sterms);
            delete L;
            return fail(TRK_ENOMEM, "trk_create_lattice: survival view allocation failed");
        }
        L->sview.elems = L->d_selems;
        L->sview.terms = L->d_sterms;
    }
    *out = L;
    return TRK_OK;
}

extern "C" trk_status trk_destroy_lattice(trk_lattice *L) {
    if (!L) return TRK_OK;
    cudaFree(L->d_elems);
    cudaFree(L->d_terms);
    cudaFree(L->d_selems);
    cudaFree(L->d_sterms);
    delete L;
    return TRK_OK;
}

// --------------------------------------------------------------- bunch ----

static void free_bunch_scratch(trk_bunch *b) {
    for (auto &pr : b->ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto &pr : b->ev_free) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    b->ev.clear();
    b->ev_free.clear();
    cudaFree(b->lt);
    cudaFree(b->le);
    cudaFree(b->cb);
    cudaFree(b->ib);
    cudaFree(b->ltb);
    cudaFree(b->leb);
    cudaFree(b->st);
    cudaFree(b->tile_alive);
    cudaFree(b->tile_off);
    cudaFree(b->partials);
    cudaFree(b->moments);
    cudaFree(b->hist);
    cudaFree(b->wfun);
    cudaFree(b->V);
    cudaFree(b->dip);
    cudaFree(b->wfun_t);
    cudaFree(b->Vt);
    cudaFree(b->V2);
    cudaFree(b->Vt2);
    cudaFree(b->lsc);
}

extern "C" trk_status trk_bunch_wrap(double *d_coords, int64_t pitch, int32_t *d_id, int64_t n, void *stream,
                                     trk_bunch **out) {
    if (!out) return fail(TRK_EINVAL, "trk_bunch_wrap: out is NULL");
    *out = nullptr;
    if (n < 0 || n > 0x7fffffffll) return fail(TRK_EINVAL, "trk_bunch_wrap: n must be 0 .. 2^31-1");
    if (pitch < n) return fail(TRK_EINVAL, "trk_bunch_wrap: pitch < n");
    if (n > 0 && (!d_coords || !d_id)) return fail(TRK_EINVAL, "trk_bunch_wrap: NULL array");
    if (((uintptr_t)d_coords & 15u) != 0) return fail(TRK_EINVAL, "trk_bunch_wrap: coords not 16-byte aligned");
    auto *b = new trk_bunch();
    b->coords = d_coords;
    b->pitch = pitch;
    b->ids = d_id;
    b->n = n;
    b->stream = (cudaStream_t)stream;
    const int64_t tiles = (n + 63) / 64 + 1;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&b->lt, n);
    if (e == cudaSuccess) e = dalloc(&b->le, n);
    if (e == cudaSuccess) e = dalloc(&b->cb, 6 * (size_t)pitch);
    if (e == cudaSuccess) e = dalloc(&b->ib, n);
    if (e == cudaSuccess) e = dalloc(&b->ltb, n);
    if (e == cudaSuccess) e = dalloc(&b->leb, n);
    if (e == cudaSuccess) e = dalloc(&b->st, 1);
    if (e == cudaSuccess) e = dalloc(&b->tile_alive, tiles);
    if (e == cudaSuccess) e = dalloc(&b->tile_off, tiles);
    if (e != cudaSuccess) {
        free_bunch_scratch(b);
        delete b;
        return fail(TRK_ENOMEM, std::string("trk_bunch_wrap: device allocation failed: ") + cudaGetErrorString(e));
    }
    b->tiles_cap = tiles;
    e = launch_init_bunch(b->st, b->lt, b->le, n, b->stream);
    if (e != cudaSuccess) {
        free_bunch_scratch(b);
        delete b;
        return fail(TRK_ECUDA, std::string("trk_bunch_wrap: init failed: ") + cudaGetErrorString(e));
    }
    *out = b;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_free(trk_bunch *b) {
    if (!b) return TRK_OK;
    cudaStreamSynchronize(b->stream);
    free_bunch_scratch(b);
    delete b;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_set_p0c(trk_bunch *b, double p0c) {
    if (!b || !(p0c > 0.0)) return fail(TRK_EINVAL, "trk_bunch_set_p0c: bad argument");
    b->p0c = p0c;
    b->p0c_set = true;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_p0c(trk_bunch *b, double *p0c) {
    if (!b || !p0c) return fail(TRK_EINVAL, "trk_bunch_p0c: bad argument");
    TRK_CUDA(cudaStreamSynchronize(b->stream));
    *p0c = b->p0c_set ? b->p0c : 0.0;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_set_turn(trk_bunch *b, int64_t turn) {
    if (!b || turn < 0 || turn > 0x7fffffffll) return fail(TRK_EINVAL, "trk_bunch_set_turn: bad argument");
    b->turn = turn;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_turn(const trk_bunch *b, int64_t *turn) {
    if (!b || !turn) return fail(TRK_EINVAL, "trk_bunch_turn: bad argument");
    *turn = b->turn;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_set_schedule(trk_bunch *b, const trk_schedule *s) {
    if (!b || !s) return fail(TRK_EINVAL, "trk_bunch_set_schedule: NULL argument");
    if (s->block && (s->block < 64 || s->block > 256 || s->block % 32))
        return fail(TRK_EINVAL, "trk_bunch_set_schedule: block must be 64..256, a multiple of 32");
    if (s->per_thread && s->per_thread != 1 && s->per_thread != 2 && s->per_thread != 4)
        return fail(TRK_EINVAL, "trk_bunch_set_schedule: per_thread must be 1, 2 or 4");
    if (s->chunk_turns < 0) return fail(TRK_EINVAL, "trk_bunch_set_schedule: chunk_turns must be >= 0");
    if (s->block) b->block = s->block;
    if (s->per_thread) b->per_thread = s->per_thread;
    if (s->chunk_turns) b->chunk = s->chunk_turns;
    return TRK_OK;
}

// ------------------------------------------------------------ tracking ----

static trk_status ensure_moments(trk_bunch *b, int n_turns, int n_tiles, int chunk) {
    if (n_turns > b->moments_cap) {
        cudaFree(b->moments);
        b->moments = nullptr;
        b->moments_cap = 0;
        if (dalloc(&b->moments, (size_t)n_turns * kMomentsN) != cudaSuccess)
            return fail(TRK_ENOMEM, "trk_track: moments allocation failed");
        b->moments_cap = n_turns;
    }
    const size_t rows = (size_t)chunk * n_tiles;
    if (rows > b->partials_rows) {
        cudaFree(b->partials);
        b->partials = nullptr;
        b->partials_rows = 0;
        if (dalloc(&b->partials, rows * kMomentsN) != cudaSuccess)
            return fail(TRK_ENOMEM, "trk_track: partial-sum allocation failed");
        b->partials_rows = rows;
    }
    return TRK_OK;
}

static trk_status ensure_wake(trk_bunch *b, int nbins, bool transverse) {
    if (nbins <= b->wake_cap && (!transverse || b->dip)) return TRK_OK;
    const int cap = nbins > b->wake_cap ? nbins : b->wake_cap;
    cudaFree(b->hist);
    cudaFree(b->wfun);
    cudaFree(b->V);
    cudaFree(b->dip);
    cudaFree(b->wfun_t);
    cudaFree(b->Vt);
    cudaFree(b->V2);
    cudaFree(b->Vt2);
    cudaFree(b->lsc);
    b->hist = nullptr;
    b->wfun = b->V = b->wfun_t = b->Vt = b->lsc = b->V2 = b->Vt2 = nullptr;
    b->dip = nullptr;
    b->wake_cap = 0;
    if (dalloc(&b->hist, cap) != cudaSuccess || dalloc(&b->wfun, cap) != cudaSuccess ||
        dalloc(&b->V, cap) != cudaSuccess || dalloc(&b->V2, cap) != cudaSuccess ||
        dalloc(&b->lsc, 4 * (size_t)cap) != cudaSuccess)
        return fail(TRK_ENOMEM, "wake scratch allocation failed");
    if (transverse && (dalloc(&b->dip, 2 * (size_t)cap) != cudaSuccess || dalloc(&b->wfun_t, cap) != cudaSuccess ||
                       dalloc(&b->Vt, 2 * (size_t)cap) != cudaSuccess ||
                       dalloc(&b->Vt2, 2 * (size_t)cap) != cudaSuccess))
        return fail(TRK_ENOMEM, "transverse wake scratch allocation failed");
    b->wake_cap = cap;
    return TRK_OK;
}

// p0 after elements [e0, e1) starting from p0 (same additions as the kernel).
static double advance_p0(const trk_lattice *L, int e0, int e1, double p0) {
    for (int e = e0; e < e1; ++e)
        if (L->elems[e].type == TRK_RFCA) p0 = p0 + L->elems[e].p[3];
    return p0;
}

static CompactArgs compact_args(trk_bunch *b, int tile, int n_tiles) {
    CompactArgs c;
    c.coords = b->coords;
    c.pitch = b->pitch;
    c.ids = b->ids;
    c.lt = b->lt;
    c.le = b->le;
    c.cb = b->cb;
    c.ib = b->ib;
    c.ltb = b->ltb;
    c.leb = b->leb;
    c.tile_alive = b->tile_alive;
    c.tile_off = b->tile_off;
    c.st = b->st;
    c.tile = tile;
    c.n_tiles = n_tiles;
    return c;
}

static TrackArgs base_args(trk_bunch *b, const trk_lattice *L, int n_tiles) {
    TrackArgs a;
    std::memset(&a, 0, sizeof a);
    a.coords = b->coords;
    a.pitch = b->pitch;
    a.loss_turn = b->lt;
    a.loss_elem = b->le;
    a.st = b->st;
    a.win = &b->st->win;
    a.lat = L->view;
    a.n_tiles = n_tiles;
    a.partials = b->partials;
    a.tile_alive = b->tile_alive;
    a.kick_wake = -1;
    a.kick_wake2 = -1;
    a.minmax_slot = -1;
    a.wake_V = b->V;
    a.wake_V2 = b->V2;
    a.tile = b->block * b->per_thread;
    return a;
}

// Tracks one physical bunch held in np parts (np = 1: an ordinary bunch).  The
// parts share the reference momentum and the turn counter; each part is
// tracked, compacted and gets its moments on its own, while every collective
// element (wake, space charge) sees the union of the parts' alive particles:
// the l window is reduced over all parts into the first part's keys, every
// part adds its particles to the first part's histogram, the field is computed
// once with q_m = Q / (sum of the parts' n), and every part takes its kick from
// those voltages in its next segment's prologue.
static trk_status track_parts(trk_bunch *const *P, int np, const trk_lattice *L, int32_t n_turns,
                              const char *who) {
    trk_bunch *lead = P[0];
    const std::string w(who);
    for (int k = 0; k < np; ++k) {
        trk_bunch *b = P[k];
        if (b->turn + n_turns > 0x7fffffffll) return fail(TRK_EINVAL, w + ": turn counter overflow");
        if (!b->p0c_set) {
            b->p0c = L->p0c;
            b->p0c_set = true;
        }
        b->moments_turns = 0;
    }
    for (int k = 1; k < np; ++k)
        if (P[k]->p0c != lead->p0c || P[k]->turn != lead->turn)
            return fail(TRK_EINVAL, w + ": the parts of a bunch must share the reference momentum and the turn");
    int64_t n_total = 0;
    for (int k = 0; k < np; ++k) n_total += P[k]->n;
    if (n_turns == 0 || n_total == 0) {
        for (int k = 0; k < np; ++k) P[k]->turn += n_turns;
        return TRK_OK;
    }
    const bool wakes = !L->wakes.empty();
    const int ne = L->view.n_elem;
    if (!wakes) {
        // no collective element: the parts are independent bunches
        for (int k = 0; k < np; ++k) {
            trk_bunch *b = P[k];
            if (b->n == 0) {
                b->turn += n_turns;
                continue;
            }
            const int tile = b->block * b->per_thread;
            const int n_tiles = (int)((b->n + tile - 1) / tile);
            const int chunk = b->chunk < n_turns ? b->chunk : n_turns;
            if (L->moments) {
                trk_status s = ensure_moments(b, n_turns, n_tiles, chunk);
                if (s != TRK_OK) return s;
            }
            for (int t0 = 0; t0 < n_turns; t0 += chunk) {
                const int nt = chunk < n_turns - t0 ? chunk : n_turns - t0;
                TrackArgs a = base_args(b, L, n_tiles);
                a.e0 = 0;
                a.e1 = ne;
                a.n_turns = nt;
                a.turn_abs0 = (int32_t)(b->turn + t0);
                a.local_turn0 = 0;
                a.do_moments = L->moments;
                a.p0c = b->p0c;
                a.ip0c = 1.0 / a.p0c;
                TRK_CUDA(track_launch(b, a, n_tiles));
                for (int t = 0; t < nt; ++t) b->p0c = advance_p0(L, 0, ne, b->p0c);
                if (L->moments) {
                    TRK_CUDA(launch_moments_finalize(b->partials, n_tiles, nt, b->st, tile,
                                                     b->moments + (size_t)t0 * kMomentsN, b->stream));
                    ++b->launches;
                }
                TRK_CUDA(launch_compact(compact_args(b, tile, n_tiles), n_tiles, b->stream));
                b->launches += 4;
            }
            b->turn += n_turns;
            b->moments_turns = L->moments ? n_turns : 0;
        }
        return TRK_OK;
    }
    const int chunk = lead->chunk < n_turns ? lead->chunk : n_turns;
    std::vector<int> tiles(np), n_tiles(np);
    for (int k = 0; k < np; ++k) {
        trk_bunch *b = P[k];
        tiles[k] = b->block * b->per_thread;
        n_tiles[k] = (int)((b->n + tiles[k] - 1) / tiles[k]);
        if (L->moments && b->n > 0) {
            trk_status s = ensure_moments(b, n_turns, n_tiles[k], chunk);
            if (s != TRK_OK) return s;
        }
    }
    {
        trk_status s = ensure_wake(lead, L->max_bins, L->transverse);
        if (s != TRK_OK) return s;
    }
    const double qm_base = 1.0 / (double)n_total;
    WakeWindow *win = &lead->st->win;
    const int ng = (int)L->groups.size();
    const auto transverse = [&](int e) {
        return e >= 0 && L->elems[e].type == TRK_WAKE && L->elems[e].p[3] != 0.0;
    };
    // histogram (over every part) and field of collective element e on the
    // window of `slot`, voltages into V (and the transverse ones into Vt)
    const auto collective = [&](int e, int slot, int which, double p0, double *V, double *Vt) -> trk_status {
        const DevElem &W = L->elems[e];
        const bool lsc = W.type == TRK_LSC;
        const bool tr = transverse(e);
        for (int k = 0; k < np; ++k) {
            trk_bunch *b = P[k];
            if (b->n == 0) continue;
            TRK_CUDA(launch_wake_hist(b->coords, b->pitch, b->lt, b->st, win, slot, which, W.n, lsc ? 0.0 : W.p[0],
                                      lsc ? 1.0 : W.p[1], lead->hist, lead->wfun, lsc ? 0.0 : W.p[3],
                                      tr ? lead->dip : nullptr, lead->wfun_t, b->n, lead->stream));
            ++b->launches;
        }
        if (lsc && W.p[5] > 0.0) {
            const double r = p0 / W.p[6];
            TRK_CUDA(launch_lsc_imp(lead->hist, lead->st, slot, W.n, W.p[2] / (double)n_total, W.p[9], W.p[5],
                                    std::sqrt(1.0 + r * r), W.p[7], W.p[8], lead->lsc, V, lead->stream));
            lead->launches += 2;
        } else {
            if (lsc)
                TRK_CUDA(launch_lsc_field(lead->hist, lead->st, slot, W.n, W.p[2] / (double)n_total, W.p[4], (int)W.flags,
                                          lead->wfun, lead->lsc, V, lead->stream));
            else
                TRK_CUDA(launch_wake_conv(lead->hist, lead->wfun, W.n, W.p[2] * qm_base, V, lead->stream));
            ++lead->launches;
        }
        if (tr) {
            TRK_CUDA(launch_wake_conv_t(lead->dip, lead->wfun_t, W.n, W.p[2] * qm_base, Vt, lead->stream));
            ++lead->launches;
        }
        return TRK_OK;
    };
    double p0c = lead->p0c;
    for (int t0 = 0; t0 < n_turns; t0 += chunk) {
        const int nt = chunk < n_turns - t0 ? chunk : n_turns - t0;
        for (int t = 0; t < nt; ++t) {
            int e_start = 0, prev = -1, prev2 = -1, prev_slot = 0;
            double p0 = p0c;
            for (int s = 0; s <= ng; ++s) {
                const int e_first = s < ng ? L->groups[s].first : ne;
                const int e_second = s < ng ? L->groups[s].second : -1;
                const int slot = s & 1;
                if (s < ng) {
                    TRK_CUDA(launch_wake_reset(lead->st, slot, lead->hist, transverse(e_first) ? lead->dip : nullptr,
                                               L->elems[e_first].n, true, lead->stream));
                    ++lead->launches;
                }
                for (int k = 0; k < np; ++k) {
                    trk_bunch *b = P[k];
                    if (b->n == 0) continue;
                    TrackArgs g = base_args(b, L, n_tiles[k]);
                    g.win = win;
                    g.wake_V = lead->V;
                    g.wake_V2 = lead->V2;
                    g.e0 = e_start;
                    g.e1 = e_first;
                    g.n_turns = 1;
                    g.turn_abs0 = (int32_t)(b->turn + t0 + t);
                    g.local_turn0 = t;
                    g.kick_wake = prev;
                    g.kick_wake2 = prev2;
                    g.kick_slot = prev_slot;
                    g.wake_nbins = prev >= 0 ? L->elems[prev].n : 0;
                    g.wake_Vx = transverse(prev) ? lead->Vt : nullptr;
                    g.wake_nbins2 = prev2 >= 0 ? L->elems[prev2].n : 0;
                    g.wake_Vx2 = transverse(prev2) ? lead->Vt2 : nullptr;
                    g.minmax_slot = s < ng ? slot : -1;
                    g.do_moments = L->moments && s == ng;
                    g.p0c = p0;
                    g.ip0c = 1.0 / p0;
                    {   // 1 / p0' after the segment's first RF cavities, as the kernel's p0 runs
                        double pr = p0;
                        g.n_rf_ip = 0;
                        for (int e = e_start; e < e_first && g.n_rf_ip < 4; ++e)
                            if (L->elems[e].type == TRK_RFCA) {
                                pr = pr + L->elems[e].p[3];
                                g.rf_ip[g.n_rf_ip++] = 1.0 / pr;
                            }
                    }
                    TRK_CUDA(track_launch(b, g, n_tiles[k]));
                }
                p0 = advance_p0(L, e_start, e_first, p0);
                if (s < ng) {
                    trk_status st = collective(e_first, slot, 0, p0, lead->V, lead->Vt);
                    if (st != TRK_OK) return st;
                    if (e_second >= 0) {   // same particles, same l: the window of `slot` stands
                        TRK_CUDA(launch_wake_reset(lead->st, slot, lead->hist,
                                                   transverse(e_second) ? lead->dip : nullptr,
                                                   L->elems[e_second].n, false, lead->stream));
                        ++lead->launches;
                        st = collective(e_second, slot, 1, p0, lead->V2, lead->Vt2);
                        if (st != TRK_OK) return st;
                    }
                }
                prev = s < ng ? e_first : -1;
                prev2 = e_second;
                prev_slot = slot;
                e_start = (e_second >= 0 ? e_second : e_first) + 1;
            }
            p0c = p0;
        }
        for (int k = 0; k < np; ++k) {
            trk_bunch *b = P[k];
            if (b->n == 0) continue;
            if (L->moments) {
                TRK_CUDA(launch_moments_finalize(b->partials, n_tiles[k], nt, b->st, tiles[k],
                                                 b->moments + (size_t)t0 * kMomentsN, b->stream));
                ++b->launches;
            }
            TRK_CUDA(launch_compact(compact_args(b, tiles[k], n_tiles[k]), n_tiles[k], b->stream));
            b->launches += 4;
        }
    }
    for (int k = 0; k < np; ++k) {
        P[k]->p0c = p0c;
        P[k]->turn += n_turns;
        P[k]->moments_turns = L->moments && P[k]->n > 0 ? n_turns : 0;
    }
    return TRK_OK;
}

extern "C" trk_status trk_track(trk_bunch *b, const trk_lattice *L, int32_t n_turns) {
    if (!b || !L) return fail(TRK_EINVAL, "trk_track: NULL bunch or lattice");
    if (n_turns < 0) return fail(TRK_EINVAL, "trk_track: n_turns < 0");
    return track_parts(&b, 1, L, n_turns, "trk_track");
}

extern "C" trk_status trk_track_parts(trk_bunch *const *parts, int32_t n_parts, const trk_lattice *L,
                                      int32_t n_turns) {
    if (!parts || n_parts < 1 || !L) return fail(TRK_EINVAL, "trk_track_parts: need n_parts >= 1 bunches and a lattice");
    if (n_turns < 0) return fail(TRK_EINVAL, "trk_track_parts: n_turns < 0");
    for (int k = 0; k < n_parts; ++k) {
        if (!parts[k]) return fail(TRK_EINVAL, "trk_track_parts: NULL part");
        if (parts[k]->stream != parts[0]->stream)
            return fail(TRK_EINVAL, "trk_track_parts: all parts must use the same stream");
        for (int j = 0; j < k; ++j)
            if (parts[j] == parts[k]) return fail(TRK_EINVAL, "trk_track_parts: a part appears twice");
    }
    return track_parts(parts, n_parts, L, n_turns, "trk_track_parts");
}

extern "C" trk_status trk_moments(trk_bunch *b, double *host_out, int32_t cap_turns, int32_t *n_turns) {
    if (!b) return fail(TRK_EINVAL, "trk_moments: NULL bunch");
    TRK_CUDA(cudaStreamSynchronize(b->stream));
    if (n_turns) *n_turns = b->moments_turns;
    const int rows = cap_turns < b->moments_turns ? cap_turns : b->moments_turns;
    if (rows > 0) {
        if (!host_out) return fail(TRK_EINVAL, "trk_moments: NULL output");
        TRK_CUDA(cudaMemcpy(host_out, b->moments, (size_t)rows * kMomentsN * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return TRK_OK;
}

extern "C" trk_status trk_n_alive(trk_bunch *b, int64_t *n_alive) {
    if (!b || !n_alive) return fail(TRK_EINVAL, "trk_n_alive: NULL argument");
    TRK_CUDA(cudaStreamSynchronize(b->stream));
    BunchState st;
    TRK_CUDA(cudaMemcpy(&st, b->st, sizeof st, cudaMemcpyDeviceToHost));
    *n_alive = st.n_alive;
    return TRK_OK;
}

extern "C" trk_status trk_lost(trk_bunch *b, int32_t *ids, int32_t *turn, int32_t *elem, int64_t cap,
                               int64_t *n_lost) {
    if (!b || !n_lost) return fail(TRK_EINVAL, "trk_lost: NULL argument");
    int64_t na = 0;
    trk_status s = trk_n_alive(b, &na);
    if (s != TRK_OK) return s;
    *n_lost = b->n - na;
    const int64_t m = cap < *n_lost ? cap : *n_lost;
    if (m > 0) {
        if (!ids || !turn || !elem) return fail(TRK_EINVAL, "trk_lost: NULL output");
        TRK_CUDA(cudaMemcpy(ids, b->ids + na, m * sizeof(int32_t), cudaMemcpyDeviceToHost));
        TRK_CUDA(cudaMemcpy(turn, b->lt + na, m * sizeof(int32_t), cudaMemcpyDeviceToHost));
        TRK_CUDA(cudaMemcpy(elem, b->le + na, m * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    return TRK_OK;
}

extern "C" trk_status trk_wake(trk_bunch *b, int32_t nbins, double w0, double sc, double charge, double p0c_ev,
                               uint32_t *d_hist, double *d_volt) {
    if (!b) return fail(TRK_EINVAL, "trk_wake: NULL bunch");
    if (nbins < 1 || nbins > kMaxBins) return fail(TRK_EINVAL, "trk_wake: nbins must be 1..65536");
    if (!(p0c_ev > 0.0)) return fail(TRK_EINVAL, "trk_wake: p0c_ev must be > 0");
    if (b->n == 0) return TRK_OK;
    trk_status s = ensure_wake(b, nbins, false);
    if (s != TRK_OK) return s;
    TRK_CUDA(launch_wake_reset(b->st, 0, b->hist, nullptr, nbins, true, b->stream));
    TRK_CUDA(launch_wake_minmax(b->coords, b->pitch, b->lt, b->st, 0, b->n, b->stream));
    TRK_CUDA(launch_wake_hist(b->coords, b->pitch, b->lt, b->st, &b->st->win,
                              0, 0, nbins, w0, sc, b->hist, b->wfun, 0.0, nullptr,
                              nullptr, b->n, b->stream));
    TRK_CUDA(launch_wake_conv(b->hist, b->wfun, nbins, charge / (double)b->n, b->V, b->stream));
    const int tile = b->block * b->per_thread;
    const int n_tiles = (int)((b->n + tile - 1) / tile);
    TrackArgs a;
    std::memset(&a, 0, sizeof a);
    a.coords = b->coords;
    a.pitch = b->pitch;
    a.loss_turn = b->lt;
    a.loss_elem = b->le;
    a.st = b->st;
    a.win = &b->st->win;   // the window the kick reads
    a.lat.ap_type = TRK_APERTURE_NONE;
    a.e0 = a.e1 = 0;
    a.n_turns = 1;
    a.turn_abs0 = (int32_t)b->turn;
    a.kick_wake = 0;
    a.kick_wake2 = -1;
    a.kick_slot = 0;
    a.minmax_slot = -1;
    a.p0c = p0c_ev;
    a.ip0c = 1.0 / p0c_ev;
    a.wake_V = b->V;
    a.wake_nbins = nbins;
    TRK_CUDA(track_launch(b, a, n_tiles));
    b->launches += 4;
    if (d_hist)
        TRK_CUDA(cudaMemcpyAsync(d_hist, b->hist, nbins * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->stream));
    if (d_volt)
        TRK_CUDA(cudaMemcpyAsync(d_volt, b->V, nbins * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    return TRK_OK;
}


// --------------------------------------------------------------- batch ----

struct trk_batch {
    std::vector<trk_bunch *> b;
    std::vector<const trk_lattice *> L;
    int n_var = 0;
    cudaStream_t stream = nullptr;   // the first bunch's stream: work is launched there
    cudaStream_t capture = nullptr;  // private stream used only to capture the graph
    int block = 128, per_thread = 2, chunk = 100, growth = 0;
    bool moments = false;
    bool survival_only = false;   // internal (survival scans): map rows limited to survival_rows
    // device tables
    TrackArgs *d_args = nullptr;
    size_t args_cap = 0;
    CompactArgs *d_cargs = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0;
    std::vector<TrackArgs> h_args;
    // cached graph of one call of `planned_turns` turns
    cudaGraphExec_t exec = nullptr;
    int planned_turns = -1;
    std::vector<int> chunks;
};

static std::vector<int> chunk_plan(int n_turns, int first, int growth) {
    std::vector<int> c;
    int len = first < 1 ? 1 : first;
    for (int t = 0; t < n_turns;) {
        const int k = len < n_turns - t ? len : n_turns - t;
        c.push_back(k);
        t += k;
        if (growth >= 2 && len < 128) len = len * growth > 128 ? 128 : len * growth;
    }
    return c;
}

static void batch_free_graph(trk_batch *B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    B->planned_turns = -1;
}

extern "C" trk_status trk_batch_create(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                                       trk_batch **out) {
    if (!out) return fail(TRK_EINVAL, "trk_batch_create: out is NULL");
    *out = nullptr;
    if (n_var < 1 || !bunches || !lats) return fail(TRK_EINVAL, "trk_batch_create: need n_var >= 1 bunches and lattices");
    for (int v = 0; v < n_var; ++v) {
        if (!bunches[v] || !lats[v]) return fail(TRK_EINVAL, "trk_batch_create: NULL bunch or lattice");
        if (!lats[v]->wakes.empty())
            return fail(TRK_EUNSUPPORTED, "trk_batch_create: lattices with TRK_WAKE are tracked with trk_track");
        if (bunches[v]->stream != bunches[0]->stream)
            return fail(TRK_EINVAL, "trk_batch_create: all bunches must use the same stream");
        if (lats[v]->moments != lats[0]->moments)
            return fail(TRK_EINVAL, "trk_batch_create: all lattices must agree on moments");
    }
    auto *B = new trk_batch();
    B->b.assign(bunches, bunches + n_var);
    B->L.assign(lats, lats + n_var);
    B->n_var = n_var;
    B->stream = bunches[0]->stream;
    B->moments = lats[0]->moments != 0;
    if (cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking) != cudaSuccess) {
        delete B;
        return fail(TRK_ECUDA, "trk_batch_create: stream creation failed");
    }
    *out = B;
    return TRK_OK;
}

extern "C" trk_status trk_batch_destroy(trk_batch *B) {
    if (!B) return TRK_OK;
    cudaStreamSynchronize(B->stream);
    batch_free_graph(B);
    cudaFree(B->d_args);
    cudaFree(B->d_cargs);
    cudaFree(B->d_items);
    if (B->capture) cudaStreamDestroy(B->capture);
    delete B;
    return TRK_OK;
}

extern "C" trk_status trk_batch_set_schedule(trk_batch *B, const trk_schedule *s) {
    if (!B || !s) return fail(TRK_EINVAL, "trk_batch_set_schedule: NULL argument");
    if (s->block && (s->block < 64 || s->block > 256 || s->block % 32))
        return fail(TRK_EINVAL, "trk_batch_set_schedule: block must be 64..256, a multiple of 32");
    if (s->per_thread && s->per_thread != 1 && s->per_thread != 2 && s->per_thread != 4)
        return fail(TRK_EINVAL, "trk_batch_set_schedule: per_thread must be 1, 2 or 4");
    if (s->chunk_turns < 0 || s->growth < 0 || s->growth == 1)
        return fail(TRK_EINVAL, "trk_batch_set_schedule: chunk_turns >= 0, growth 0 or >= 2");
    if (s->block) B->block = s->block;
    if (s->per_thread) B->per_thread = s->per_thread;
    if (s->chunk_turns) B->chunk = s->chunk_turns;
    B->growth = s->growth;
    batch_free_graph(B);
    B->n_items = 0;  // re-tile
    return TRK_OK;
}

extern "C" trk_status trk_batch_get_schedule(const trk_batch *B, trk_schedule *s) {
    if (!B || !s) return fail(TRK_EINVAL, "trk_batch_get_schedule: NULL argument");
    s->block = B->block;
    s->per_thread = B->per_thread;
    s->chunk_turns = B->chunk;
    s->growth = B->growth;
    return TRK_OK;
}

extern "C" trk_status trk_batch_track(trk_batch *B, int32_t n_turns) {
    if (!B) return fail(TRK_EINVAL, "trk_batch_track: NULL batch");
    if (n_turns < 0) return fail(TRK_EINVAL, "trk_batch_track: n_turns < 0");
    const int nv = B->n_var;
    const int tile = B->block * B->per_thread;
    for (int v = 0; v < nv; ++v) {
        trk_bunch *b = B->b[v];
        if (b->turn + n_turns > 0x7fffffffll) return fail(TRK_EINVAL, "trk_batch_track: turn counter overflow");
        if (!b->p0c_set) {
            b->p0c = B->L[v]->p0c;
            b->p0c_set = true;
        }
        b->moments_turns = 0;
        b->block = B->block;
        b->per_thread = B->per_thread;
    }
    if (n_turns == 0) return TRK_OK;
    const std::vector<int> chunks = chunk_plan(n_turns, B->chunk, B->growth);
    const int nc = (int)chunks.size();
    int max_chunk = 0;
    for (int c : chunks) max_chunk = c > max_chunk ? c : max_chunk;
    // per-variant scratch and the (variant, tile) item table
    std::vector<int2> items;
    std::vector<CompactArgs> cargs(nv);
    for (int v = 0; v < nv; ++v) {
        trk_bunch *b = B->b[v];
        const int nt = (int)((b->n + tile - 1) / tile);
        if (B->moments) {
            trk_status s = ensure_moments(b, n_turns, nt, max_chunk);
            if (s != TRK_OK) return s;
        }
        for (int t = 0; t < nt; ++t) items.push_back(make_int2(v, t));
        cargs[v] = compact_args(b, tile, nt);
    }
    const bool retile = B->n_items != (int)items.size() || !B->d_items;
    if (retile) {
        batch_free_graph(B);
        cudaFree(B->d_items);
        cudaFree(B->d_cargs);
        B->d_items = nullptr;
        B->d_cargs = nullptr;
        if (dalloc(&B->d_items, items.size()) != cudaSuccess || dalloc(&B->d_cargs, nv) != cudaSuccess)
            return fail(TRK_ENOMEM, "trk_batch_track: table allocation failed");
        TRK_CUDA(cudaMemcpy(B->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
        B->n_items = (int)items.size();
    }
    TRK_CUDA(cudaMemcpyAsync(B->d_cargs, cargs.data(), nv * sizeof(CompactArgs), cudaMemcpyHostToDevice, B->stream));
    // per (variant, chunk) launch arguments, with the reference momentum and the
    // absolute turn at the start of each chunk
    const size_t na = (size_t)nv * nc;
    if (na > B->args_cap) {
        batch_free_graph(B);
        cudaFree(B->d_args);
        B->d_args = nullptr;
        B->args_cap = 0;
        if (dalloc(&B->d_args, na) != cudaSuccess) return fail(TRK_ENOMEM, "trk_batch_track: argument table allocation failed");
        B->args_cap = na;
    }
    B->h_args.resize(na);
    for (int v = 0; v < nv; ++v) {
        trk_bunch *b = B->b[v];
        const trk_lattice *L = B->L[v];
        const int nt = cargs[v].n_tiles;
        const int ne = L->view.n_elem;
        int t0 = 0;
        for (int c = 0; c < nc; ++c) {
            TrackArgs a = base_args(b, L, nt);
            if (B->survival_only) a.lat = L->sview;
            a.e0 = 0;
            a.e1 = ne;
            a.n_turns = chunks[c];
            a.turn_abs0 = (int32_t)(b->turn + t0);
            a.local_turn0 = 0;
            a.do_moments = L->moments;
            a.p0c = b->p0c;
            a.ip0c = 1.0 / a.p0c;
            a.mom_out = b->moments ? b->moments + (size_t)t0 * kMomentsN : nullptr;
            B->h_args[(size_t)v * nc + c] = a;
            for (int t = 0; t < chunks[c]; ++t) b->p0c = advance_p0(L, 0, ne, b->p0c);
            t0 += chunks[c];
        }
    }
    TRK_CUDA(cudaMemcpyAsync(B->d_args, B->h_args.data(), na * sizeof(TrackArgs), cudaMemcpyHostToDevice, B->stream));
    // one CUDA graph holds every chunk of the call; it only reads the tables
    // above, so it is captured once per (n_turns, schedule, tiling) and replayed
    if (!B->exec || B->planned_turns != n_turns || B->chunks != chunks) {
        batch_free_graph(B);
        cudaGraph_t g = nullptr;
        TRK_CUDA(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int c = 0; c < nc && e == cudaSuccess; ++c)
            e = launch_batch_chunk(B->d_args, B->d_cargs, B->d_items, B->n_items, nv, nc, c, B->block,
                                   B->per_thread, tile, chunks[c], B->moments, B->capture);
        cudaError_t e2 = cudaStreamEndCapture(B->capture, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(TRK_ECUDA, std::string("trk_batch_track: graph capture failed: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&B->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            B->exec = nullptr;
            return fail(TRK_ECUDA, std::string("trk_batch_track: graph instantiation failed: ") + cudaGetErrorString(e));
        }
        B->planned_turns = n_turns;
        B->chunks = chunks;
    }
    TRK_CUDA(cudaGraphLaunch(B->exec, B->stream));
    for (int v = 0; v < nv; ++v) {
        trk_bunch *b = B->b[v];
        b->turn += n_turns;
        b->moments_turns = B->moments ? n_turns : 0;
        b->track_launches += nc;
        b->launches += (int64_t)nc * (B->moments ? 6 : 5);
    }
    return TRK_OK;
}

extern "C" trk_status trk_track_batch(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                                      int32_t n_turns, const trk_schedule *sched) {
    trk_batch *B = nullptr;
    trk_status s = trk_batch_create(bunches, lats, n_var, &B);
    if (s != TRK_OK) return s;
    if (sched) s = trk_batch_set_schedule(B, sched);
    if (s == TRK_OK) s = trk_batch_track(B, n_turns);
    trk_batch_destroy(B);
    return s;
}


// ----------------------------------------------------- dynamic aperture ----

// Below this many points a scan is bound by one particle's latency: 8 lanes per
// particle (k_da_lanes) then finish sooner than the batched tracker.
constexpr int64_t kLanePoints = 16384;

static bool lane_capable(const trk_lattice *L) {
    for (const DevElem &E : L->elems)
        if (E.type != TRK_MAP && E.type != TRK_EDRIFT && E.type != TRK_THINSEXT) return false;
    return true;
}

extern "C" trk_status trk_da_survival_lanes(const trk_lattice *const *lats, int32_t n_var, const int64_t *offsets,
                                            const double *d_x0, const double *d_y0, int32_t n_turns,
                                            int32_t *d_survival, void *stream) {
    if (n_var < 1 || !lats || !offsets) return fail(TRK_EINVAL, "trk_da_survival_lanes: need n_var >= 1, lattices, offsets");
    if (n_turns < 1) return fail(TRK_EINVAL, "trk_da_survival_lanes: n_turns must be >= 1");
    if (offsets[0] != 0) return fail(TRK_EINVAL, "trk_da_survival_lanes: offsets[0] must be 0");
    for (int v = 0; v < n_var; ++v) {
        if (!lats[v]) return fail(TRK_EINVAL, "trk_da_survival_lanes: NULL lattice");
        if (offsets[v + 1] < offsets[v]) return fail(TRK_EINVAL, "trk_da_survival_lanes: offsets must be non-decreasing");
        if (!lane_capable(lats[v]))
            return fail(TRK_EUNSUPPORTED, "trk_da_survival_lanes: lattices may hold MAP, EDRIFT and THINSEXT only");
    }
    const int64_t total = offsets[n_var];
    if (total == 0) return TRK_OK;
    if (total > ((int64_t)1 << 28)) return fail(TRK_EINVAL, "trk_da_survival_lanes: more than 2^28 points");
    if (!d_x0 || !d_y0 || !d_survival) return fail(TRK_EINVAL, "trk_da_survival_lanes: NULL point or output array");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<LatticeView> hv(n_var);
    int lanes = 4;   // 4 lanes per particle when no view evaluates rows 4 or 5
    for (int v = 0; v < n_var; ++v) {
        hv[v] = lats[v]->sview;
        if (hv[v].row_mask & ~0xFu) lanes = 8;
    }
    LatticeView *dv = nullptr;
    int64_t *doff = nullptr;
    cudaError_t e = cudaMalloc(&dv, n_var * sizeof(LatticeView));
    if (e == cudaSuccess) e = cudaMalloc(&doff, (n_var + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, hv.data(), n_var * sizeof(LatticeView), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, offsets, (n_var + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_da_lanes(dv, n_var, doff, d_x0, d_y0, total, n_turns, lanes, d_survival, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dv);
    cudaFree(doff);
    if (e != cudaSuccess) return fail(TRK_ECUDA, std::string("trk_da_survival_lanes: ") + cudaGetErrorString(e));
    return TRK_OK;
}

extern "C" trk_status trk_da_survival(const trk_lattice *const *lats, int32_t n_var, const int64_t *offsets,
                                      const double *d_x0, const double *d_y0, int32_t n_turns,
                                      const trk_schedule *sched, int32_t *d_survival, void *stream) {
    if (n_var < 1 || !lats || !offsets) return fail(TRK_EINVAL, "trk_da_survival: need n_var >= 1, lattices, offsets");
    if (n_turns < 1) return fail(TRK_EINVAL, "trk_da_survival: n_turns must be >= 1");
    if (offsets[0] != 0) return fail(TRK_EINVAL, "trk_da_survival: offsets[0] must be 0");
    for (int v = 0; v < n_var; ++v)
        if (offsets[v + 1] < offsets[v] || offsets[v + 1] - offsets[v] > 0x7fffffffll)
            return fail(TRK_EINVAL, "trk_da_survival: offsets must be non-decreasing, < 2^31 points per variant");
    const int64_t total = offsets[n_var];
    if (total == 0) return TRK_OK;
    if (!d_x0 || !d_y0 || !d_survival) return fail(TRK_EINVAL, "trk_da_survival: NULL point or output array");
    if (!sched && total <= kLanePoints) {
        bool ok = true;
        for (int v = 0; v < n_var && ok; ++v) ok = lats[v] && lane_capable(lats[v]);
        if (ok) return trk_da_survival_lanes(lats, n_var, offsets, d_x0, d_y0, n_turns, d_survival, stream);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // each variant's slice starts on a 32-byte boundary of the particle arrays
    std::vector<int64_t> slot(n_var + 1, 0);
    for (int v = 0; v < n_var; ++v) slot[v + 1] = slot[v] + (offsets[v + 1] - offsets[v] + 3) / 4 * 4;
    const int64_t pitch = slot[n_var] > 0 ? slot[n_var] : 1;
    double *coords = nullptr;
    int32_t *ids = nullptr;
    if (dalloc(&coords, 6 * (size_t)pitch) != cudaSuccess || dalloc(&ids, pitch) != cudaSuccess) {
        cudaFree(coords);
        return fail(TRK_ENOMEM, "trk_da_survival: particle allocation failed");
    }
    std::vector<trk_bunch *> bunches;
    std::vector<const trk_lattice *> L;
    trk_batch *B = nullptr;
    trk_status st = TRK_OK;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < n_var && e == cudaSuccess; ++v)
        e = launch_da_init(coords + slot[v], pitch, ids + slot[v], d_x0, d_y0, offsets[v], offsets[v + 1] - offsets[v], s);
    if (e != cudaSuccess) st = fail(TRK_ECUDA, std::string("trk_da_survival: ") + cudaGetErrorString(e));
    for (int v = 0; v < n_var && st == TRK_OK; ++v) {
        const int64_t n = offsets[v + 1] - offsets[v];
        if (n == 0) continue;
        trk_bunch *b = nullptr;
        st = trk_bunch_wrap(coords + slot[v], pitch, ids + slot[v], n, stream, &b);
        if (st == TRK_OK) {
            bunches.push_back(b);
            L.push_back(lats[v]);
        }
    }
    if (st == TRK_OK && !bunches.empty()) st = trk_batch_create(bunches.data(), L.data(), (int32_t)bunches.size(), &B);
    if (st == TRK_OK && B) B->survival_only = true;   // only the loss turns leave this call
    if (st == TRK_OK && B) {
        trk_schedule def = {128, 2, 1, 2};  // short chunks first: most lost particles leave early
        st = trk_batch_set_schedule(B, sched ? sched : &def);
    }
    if (st == TRK_OK && B) st = trk_batch_track(B, n_turns);
    for (size_t k = 0; k < bunches.size() && st == TRK_OK; ++k) {
        trk_bunch *b = bunches[k];
        e = launch_da_survival(b->ids, b->lt, b->n, n_turns, d_survival, s);
        if (e != cudaSuccess) st = fail(TRK_ECUDA, std::string("trk_da_survival: ") + cudaGetErrorString(e));
    }
    cudaStreamSynchronize(s);
    if (B) trk_batch_destroy(B);
    for (trk_bunch *b : bunches) trk_bunch_free(b);
    cudaFree(coords);
    cudaFree(ids);
    return st;
}


// ------------------------------------------------------------- autotune ----

extern "C" trk_status trk_autotune(trk_bunch *const *bunches, const trk_lattice *const *lats, int32_t n_var,
                                   int32_t probe_turns, trk_schedule *out, double *best_ms) {
    if (!bunches || !lats || n_var < 1 || !out || probe_turns < 1)
        return fail(TRK_EINVAL, "trk_autotune: bad argument");
    cudaStream_t s = bunches[0]->stream;
    // shadow copies of the alive particles, so the caller's bunches are untouched
    std::vector<double *> sc(n_var, nullptr);
    std::vector<int32_t *> si(n_var, nullptr);
    std::vector<trk_bunch *> sb(n_var, nullptr);
    trk_status st = TRK_OK;
    auto cleanup = [&]() {
        for (int v = 0; v < n_var; ++v) {
            if (sb[v]) trk_bunch_free(sb[v]);
            cudaFree(sc[v]);
            cudaFree(si[v]);
        }
    };
    for (int v = 0; v < n_var && st == TRK_OK; ++v) {
        trk_bunch *b = bunches[v];
        int64_t na = 0;
        st = trk_n_alive(b, &na);
        if (st != TRK_OK) break;
        const int64_t n = na > 0 ? na : 1;
        if (dalloc(&sc[v], 6 * (size_t)n) != cudaSuccess || dalloc(&si[v], n) != cudaSuccess) {
            st = fail(TRK_ENOMEM, "trk_autotune: shadow allocation failed");
            break;
        }
        if (na > 0) {
            cudaError_t e = cudaMemcpy2DAsync(sc[v], n * sizeof(double), b->coords, b->pitch * sizeof(double),
                                              na * sizeof(double), 6, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(si[v], b->ids, na * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) {
                st = fail(TRK_ECUDA, std::string("trk_autotune: copy failed: ") + cudaGetErrorString(e));
                break;
            }
        }
        st = trk_bunch_wrap(sc[v], n, si[v], na, s, &sb[v]);
        if (st == TRK_OK) {
            sb[v]->p0c = b->p0c_set ? b->p0c : lats[v]->p0c;
            sb[v]->p0c_set = true;
        }
    }
    if (st != TRK_OK) {
        cleanup();
        return st;
    }
    // candidate schedules: launch shape x chunk plan
    const int shapes[][2] = {{128, 1}, {128, 2}, {64, 2}, {256, 2}, {128, 4}, {64, 4}};
    const int plans[][2] = {{probe_turns, 0}, {1, 2}};
    double best = 1e300;
    trk_schedule best_s = {128, 2, probe_turns, 0};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (auto &sh : shapes) {
        for (auto &pl : plans) {
            trk_batch *B = nullptr;
            st = trk_batch_create(sb.data(), lats, n_var, &B);
            if (st != TRK_OK) break;
            trk_schedule cand = {sh[0], sh[1], pl[0], pl[1]};
            st = trk_batch_set_schedule(B, &cand);
            // the shadows advance with every probe; each probe starts from their
            // current state, which only shifts the turn counter
            if (st == TRK_OK) st = trk_batch_track(B, probe_turns);  // warm-up and graph capture
            if (st == TRK_OK) {
                cudaEventRecord(e0, s);
                st = trk_batch_track(B, probe_turns);
                cudaEventRecord(e1, s);
            }
            trk_batch_destroy(B);
            if (st != TRK_OK) break;
            float ms = 0.0f;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_s = cand;
            }
        }
        if (st != TRK_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    if (st != TRK_OK) return st;
    *out = best_s;
    if (best_ms) *best_ms = best;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_enable_timing(trk_bunch *b, int32_t on) {
    if (!b) return fail(TRK_EINVAL, "trk_bunch_enable_timing: NULL bunch");
    b->timing = on != 0;
    return TRK_OK;
}

extern "C" trk_status trk_bunch_stats(trk_bunch *b, trk_stats *out, int32_t reset) {
    if (!b || !out) return fail(TRK_EINVAL, "trk_bunch_stats: NULL argument");
    TRK_CUDA(cudaStreamSynchronize(b->stream));
    for (auto &pr : b->ev) {
        float ms = 0.0f;
        TRK_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        b->track_ms += ms;
        b->ev_free.push_back(pr);
    }
    b->ev.clear();
    out->track_kernel_ms = b->track_ms;
    out->track_launches = b->track_launches;
    out->launches = b->launches;
    if (reset) {
        b->track_ms = 0.0;
        b->track_launches = 0;
        b->launches = 0;
    }
    return TRK_OK;
}

trk_status trk::set_error(trk_status s, const char *msg) { return fail(s, msg); }

extern "C" const char *trk_last_error(void) { return g_err.c_str(); }
