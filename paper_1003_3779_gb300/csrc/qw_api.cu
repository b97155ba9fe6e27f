// qw_api.cu -- the C ABI of include/qw.h for single walks: handles, state and
// coin set-up, the step loop, marginals, plans and the autotuner.
//
// A walk is the one-step operator U = S (I (x) C) of Sec. 2.1 applied to the
// Z^1 / Z^2 walker states of Sec. 2.2-3 (cycle and torus, periodic, or the
// finite segment / line of Sec. 3 with broken links).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "qw_handle.h"

using namespace qw;

// ------------------------------------------------------------------ helpers
namespace qw {

qw_status set_error(qw_walk *w, qw_status st, const std::string &msg) {
    if (w) w->err = msg;
    return st;
}

qw_status cuda_error(qw_walk *w, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    (void)cudaGetLastError();  // clear a non-sticky error so the handle stays usable
    return set_error(w, e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA, m);
}

bool fault_injected(const char *what) {
    const char *f = std::getenv("QW_FAULT");
    return f && std::strstr(f, what);
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (fault_injected("alloc")) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

static int slot_bytes_of(int prec) {
    switch (prec) {
        case QW_F64: return 16;
        case QW_F32: return 8;
        case QW_F32_BF16STORE: return 4;
        case QW_F32_COMP: return 8;
    }
    return 0;
}

static size_t real_bytes(int prec) {  // bytes of one compute-precision real
    return prec == QW_F64 ? 8 : (prec == QW_F32_COMP ? 8 : 4);
}

static cudaError_t step1d(int prec, const Step1DArgs &a, const void *cp, int adj, cudaStream_t s) {
    switch (prec) {
        case QW_F64: return launch_step1d_f64(a, cp, adj, s);
        case QW_F32: return launch_step1d_f32(a, cp, adj, s);
        case QW_F32_BF16STORE: return launch_step1d_bf16(a, cp, adj, s);
        case QW_F32_COMP: return launch_step1d_comp(a, cp, adj, s);
    }
    return cudaErrorInvalidValue;
}
static cudaError_t step2d(int prec, const Step2DArgs &a, const void *cp, int adj, cudaStream_t s) {
    switch (prec) {
        case QW_F64: return launch_step2d_f64(a, cp, adj, s);
        case QW_F32: return launch_step2d_f32(a, cp, adj, s);
        case QW_F32_BF16STORE: return launch_step2d_bf16(a, cp, adj, s);
        case QW_F32_COMP: return launch_step2d_comp(a, cp, adj, s);
    }
    return cudaErrorInvalidValue;
}
static cudaError_t stepwin(int prec, const StepGenericArgs &a, const void *cp, const double *gains, int nsteps,
                           cudaStream_t s) {
    switch (prec) {
        case QW_F64: return launch_window1d_f64(a, cp, gains, nsteps, s);
        case QW_F32: return launch_window1d_f32(a, cp, gains, nsteps, s);
        case QW_F32_BF16STORE: return launch_window1d_bf16(a, cp, gains, nsteps, s);
        case QW_F32_COMP: return launch_window1d_comp(a, cp, gains, nsteps, s);
    }
    return cudaErrorInvalidValue;
}
static int64_t window_capacity(int prec) {
    switch (prec) {
        case QW_F64: return window1d_capacity_f64();
        case QW_F32: return window1d_capacity_f32();
        case QW_F32_BF16STORE: return window1d_capacity_bf16();
        case QW_F32_COMP: return window1d_capacity_comp();
    }
    return 0;
}

static cudaError_t stepgen(int prec, const StepGenericArgs &a, const void *cp, cudaStream_t s) {
    switch (prec) {
        case QW_F64: return launch_generic_f64(a, cp, s);
        case QW_F32: return launch_generic_f32(a, cp, s);
        case QW_F32_BF16STORE: return launch_generic_bf16(a, cp, s);
        case QW_F32_COMP: return launch_generic_comp(a, cp, s);
    }
    return cudaErrorInvalidValue;
}
static int tile1d(int prec, int tile, int kind, int adj) {
    switch (prec) {
        case QW_F64: return tile1d_f64(tile, kind, adj);
        case QW_F32: return tile1d_f32(tile, kind, adj);
        case QW_F32_BF16STORE: return tile1d_bf16(tile, kind, adj);
        case QW_F32_COMP: return tile1d_comp(tile, kind, adj);
    }
    return 0;
}
// Sweep plans: `tile` is the sites per lane (0 or an uncompiled value: the
// launcher's default for this cycle length).
static bool sweep_ok(const qw_walk *w, int K, int tile) {
    if (w->ndim != 1 || w->bc != QW_BC_PERIODIC || links_on(w)) return false;
    switch (w->prec) {
        case QW_F64: return sweep_ok_f64(w->nx, K, w->kind, tile);
        case QW_F32: return sweep_ok_f32(w->nx, K, w->kind, tile);
        case QW_F32_BF16STORE: return sweep_ok_bf16(w->nx, K, w->kind, tile);
    }
    return false;
}
static int sweep_tile(const qw_walk *w, int tile) {
    switch (w->prec) {
        case QW_F64: return sweep_tile_f64(w->nx, tile);
        case QW_F32: return sweep_tile_f32(w->nx, tile);
        case QW_F32_BF16STORE: return sweep_tile_bf16(w->nx, tile);
    }
    return 0;
}

// tiles compiled for the forward 1D kernel, per precision
static void tiles_of(int prec, int &a, int &b) {
    if (prec == QW_F64 || prec == QW_F32_COMP) { a = 4; b = 8; }
    else { a = 8; b = 16; }
}

// Warps the 2D streaming kernel can keep busy at depth KT: 64-column strips
// with KT columns of halo per side, row chunks of at least 8 KT rows.
static int64_t tb_warps(const qw_walk *w, int KT) {
    const int64_t W = 64 - 2 * KT;
    return ((w->nx + W - 1) / W) * ((w->ny + 8 * KT - 1) / (8 * KT));
}

static void default_plan(const qw_walk *w, int &k, int &tile, int &variant) {
    variant = 0;
    if (w->ndim == 2) {
        // the streaming kernel where the lattice gives it two waves of warps
        // (8 per SM), else the fused single step
        tile = 0;
        k = 1;
        if (w->bc != QW_BC_PERIODIC || links_on(w)) return;
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        }
        const int64_t enough = (int64_t)sms * 8 * 2;
        for (int KT : {8, 4})
            if (step2d_tb_ok(w->prec, w->kind, KT, w->shift) && tb_warps(w, KT) >= enough) { k = KT; break; }
        return;
    }
    switch (w->prec) {
        case QW_F64: tile = 8; k = 8; break;
        case QW_F32_COMP: tile = 4; k = 8; break;
        default: tile = 16; k = 32; break;
    }
    if (sweep_ok(w, w->prec == QW_F64 ? 8 : 64, 0)) {
        variant = 1;
        k = w->prec == QW_F64 ? 8 : 64;
        tile = sweep_tile(w, 0);
    }
}

static void effective_plan(const qw_walk *w, int &k, int &tile, int &variant) {
    default_plan(w, k, tile, variant);
    if (w->plan_k > 0) {
        k = w->plan_k;
        tile = w->plan_tile ? w->plan_tile : tile;
        variant = w->plan_variant >= 0 ? w->plan_variant : 0;
    }
}
static void effective_plan(const qw_walk *w, int &k, int &tile) {
    int v;
    effective_plan(w, k, tile, v);
}

// Global coin: store, classify, and convert to the compute precision.
//
// The specialised kernels (Grover, H (x) H, the Hadamard class lambda * M)
// apply their own matrix, not the caller's.  In float compute a coin within
// 1e-15 (absolute) or 1e-14 (relative) of one of them rounds to the same
// float matrix, so the substitution changes nothing.  The double and
// double-float forms carry the caller's entries to 53 / ~48 bits: there a coin
// is specialised only when every entry lies within one double ulp of the
// specialised matrix (|h - 1/2| <= 2^-53; for lambda * M the four magnitudes
// within 2^-52 relative of their mean).  Such a substitution moves each entry
// by no more than one rounding, as the arithmetic of a step does anyway; a
// coin that differs by more runs as given.  (kron(H, H) of the rounded 1/sqrt2,
// whose entries are 1/2 - 2^-53, and SU(2) at theta = pi/4, whose cos and sin
// differ by one ulp, stay specialised.)
static void apply_global_coin(qw_walk *w, const double *h) {
    const int d = w->d, n = d * d;
    std::memcpy(w->coin_host, h, sizeof(double) * 2 * n);
    const bool wide = w->prec == QW_F64 || w->prec == QW_F32_COMP;
    const double tol_abs = wide ? 0x1p-53 : 1e-15, tol_rel = wide ? 0x1p-52 : 1e-14;
    bool real = true;
    for (int i = 0; i < n; ++i) real = real && h[2 * i + 1] == 0.0;
    int kind = real ? CK_REAL : CK_COMPLEX;
    if (d == 4 && real) {
        bool grover = true, hh = true;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                const double g = (r == c) ? -0.5 : 0.5;
                const int sgn = ((r & c & 1) ^ ((r >> 1) & (c >> 1) & 1)) ? -1 : 1;  // H(x)H, c = 2j+k
                grover = grover && std::fabs(h[2 * (4 * r + c)] - g) <= tol_abs;
                hh = hh && std::fabs(h[2 * (4 * r + c)] - 0.5 * sgn) <= tol_abs;
            }
        if (grover) kind = CK_GROVER;
        else if (hh) kind = CK_HH;
    }
    w->kind = kind;
    std::memset(w->coinp, 0, sizeof(w->coinp));
    double fro = 0.0;   // |C_f|_F^2 of the coin as the kernels see it
    if (w->prec == QW_F64) {
        auto *cp = reinterpret_cast<CoinP<double> *>(w->coinp);
        for (int i = 0; i < n; ++i) { cp->re[i] = h[2 * i]; cp->im[i] = h[2 * i + 1]; }
        for (int i = 0; i < n; ++i) fro += cp->re[i] * cp->re[i] + cp->im[i] * cp->im[i];
    } else if (w->prec == QW_F32_COMP) {
        auto *cp = reinterpret_cast<CoinP<ff> *>(w->coinp);
        for (int i = 0; i < n; ++i) {
            const float rh = (float)h[2 * i], ih = (float)h[2 * i + 1];
            cp->re[i] = {rh, (float)(h[2 * i] - (double)rh)};
            cp->im[i] = {ih, (float)(h[2 * i + 1] - (double)ih)};
        }
        fro = (double)d;    // hi + lo carries ~48 bits: no drift to compensate
    } else {
        auto *cp = reinterpret_cast<CoinP<float> *>(w->coinp);
        for (int i = 0; i < n; ++i) { cp->re[i] = (float)h[2 * i]; cp->im[i] = (float)h[2 * i + 1]; }
        for (int i = 0; i < n; ++i) fro += (double)cp->re[i] * cp->re[i] + (double)cp->im[i] * cp->im[i];
    }
    // For a unitary coin rounded to C_f, C_f^dagger C_f = alpha^2 I (exactly for
    // rotation / Hadamard-type coins, to first order otherwise): every step scales
    // the norm by alpha.  The kernels divide it back out.  A coin that is not
    // close to unitary (|alpha - 1| > 1e-5, e.g. a deliberately lossy one) is
    // applied as given.  The double form applies the caller's double entries
    // themselves (no rounding by the library), so it compensates nothing: a
    // coin a few ulps from unitary is the caller's coin, not a rounding drift.
    if (w->prec == QW_F64) fro = (double)d;
    const double alpha = std::sqrt(fro / d);
    w->coin_alpha = std::fabs(alpha - 1.0) <= 1e-5 ? alpha : 1.0;
    w->gain_fb = 1.0;
    w->drift_pending = 1.0;

    // Hadamard class on the cycle with the moving shift: C = lambda * M, M in
    // {+-1}^{2x2}, M = diag(a, c) H diag(1, s) (needs m11 = -m10 m01 m00).
    if (d == 2 && real && w->shift == QW_SHIFT_MOVING) {
        double mag[4], lam = 0.0;
        for (int i = 0; i < 4; ++i) { mag[i] = std::fabs(h[2 * i]); lam += mag[i] / 4; }
        bool eq = lam > 0.0;
        for (int i = 0; i < 4; ++i) eq = eq && std::fabs(mag[i] - lam) <= tol_rel * lam;
        if (eq) {
            const int m00 = h[0] > 0 ? 1 : -1, m01 = h[2] > 0 ? 1 : -1;
            const int m10 = h[4] > 0 ? 1 : -1, m11 = h[6] > 0 ? 1 : -1;
            if (m11 == -m10 * m01 * m00) {
                w->sign_lambda = lam;
                w->sign_a = m00;
                w->sign_s = m01 * m00;
                w->sign_c = m10;
                w->sign_sigma = w->sign_a * w->sign_s * w->sign_c;
                w->kind = w->sign_sigma > 0 ? CK_SIGN_P : CK_SIGN_M;
            }
        }
    }
}

static bool rounds_to_float(const qw_walk *w) {
    return w->prec == QW_F32 || w->prec == QW_F32_BF16STORE;
}

// The factor that actually reaches the kernel for an ideal positive factor
// `ideal`, with error feedback: the rounding residue of earlier launches is
// folded into this one, so the product of applied factors tracks the product
// of ideal ones to one rounding instead of one rounding per launch.
static double feedback_gain(qw_walk *w, double ideal, bool update = true) {
    if (ideal == 1.0 && w->gain_fb == 1.0) return 1.0;
    const double want = ideal / w->gain_fb;
    const double applied = rounds_to_float(w) ? (double)(float)want : want;
    if (update) w->gain_fb *= applied / ideal;
    return applied;
}

// Norm-drift compensation of a rounded coin.  Each launch of K steps scales
// the norm by alpha^K; the ideal correction alpha^-K is accumulated here and
// applied in the last launch of a qw_step call (or as soon as it exceeds
// 2^-16).  Applying factors within a few ulps of 1 at every launch would itself
// be biased: round-to-nearest of x * (1 - 2^-24) is always x - ulp(x).
static double take_drift(qw_walk *w, int steps, bool last) {
    if (w->kind == CK_PERSITE || w->kind == CK_PHASE || w->coin_alpha == 1.0) return 1.0;
    w->drift_pending *= std::pow(w->coin_alpha, -(double)steps);
    if (!last && std::fabs(w->drift_pending - 1.0) < 1.0 / 65536) return 1.0;
    const double applied = rounds_to_float(w) ? (double)(float)w->drift_pending : w->drift_pending;
    w->drift_pending /= applied;
    return applied;
}

// Per-step factor for the 2D and generic kernels: drift_gain(w, 1, last).
static double drift_gain(qw_walk *w, int steps, bool last = true) { return take_drift(w, steps, last); }

// Pre / post per-plane factors of one 1D launch of K steps.
static void launch_gains_1d(qw_walk *w, int K, int adj, Step1DArgs &a, bool update = true, bool last = true) {
    if (w->kind == CK_SIGN_P || w->kind == CK_SIGN_M) {
        // the sweep kernel rescales by 2^-SIGN_RESCALE_LOG2 every SIGN_RESCALE_STEPS steps
        const int m = a.variant == 1 ? K / SIGN_RESCALE_STEPS : 0;
        const double mag = feedback_gain(w, std::ldexp(std::pow(w->sign_lambda, (double)K), SIGN_RESCALE_LOG2 * m),
                                         update);
        const double ak1 = ((K - 1) % 2 == 0 || w->sign_a > 0) ? 1.0 : -1.0;   // a^{K-1}
        if (!adj) {
            a.pre0 = 1.0; a.pre1 = (double)(w->sign_sigma * w->sign_s);
            a.post0 = mag * ak1 * w->sign_a; a.post1 = mag * ak1 * w->sign_c;
        } else {
            a.pre0 = (double)w->sign_a; a.pre1 = (double)(w->sign_sigma * w->sign_c);
            a.post0 = mag * ak1; a.post1 = mag * ak1 * w->sign_s;
        }
        return;
    }
    const double g = update ? take_drift(w, K, last) : 1.0;
    a.pre0 = a.pre1 = 1.0;
    a.post0 = a.post1 = g;
}

static qw_status ensure_staging(qw_walk *w, size_t bytes) {
    if (w->staging_bytes >= bytes) return QW_OK;
    if (w->staging) { cudaStreamSynchronize(w->stream); cudaFree(w->staging); w->staging = nullptr; w->staging_bytes = 0; }
    cudaError_t e = dev_alloc(&w->staging, bytes);
    if (e != cudaSuccess) return cuda_error(w, e, "staging allocation");
    w->staging_bytes = bytes;
    return QW_OK;
}

static constexpr size_t STAGE_CHUNK = size_t(32) << 20;  // bytes per host conversion chunk

// ---------------------------------------------------------------- light-cone clipping
// A walker started on a few sites (the line computations of Sec. 3 start at
// one site, MP, and step only the window that its light cone has reached) is
// zero outside a box that widens by one site per step on each side.  The box
// of the state set by qw_set_state is searched on the GPU (launch_support);
// the steps then run on the box widened by their depth, and the box grows
// with them until it covers the lattice.  Both state buffers are zero outside
// the box (the other buffer is cleared once, before the first clipped step),
// and each output is computed by the same arithmetic as in a full launch, so
// the results equal those of the full launches bit for bit.

// Is the walk's stream being captured into a CUDA graph?  Then nothing may
// wait for its work: the search is skipped and the steps run in full.
static bool capturing(const qw_walk *w) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(w->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// Queue the search for the support box of the current state (qw_set_state).
static qw_status queue_support(qw_walk *w) {
    w->next_clear = false;
    if (!w->clip_on || capturing(w)) {
        (void)cudaGetLastError();
        w->sup_mode = 0;
        return QW_OK;
    }
    cudaError_t e = launch_support(w->prec == QW_F64 ? P_F64 : w->prec == QW_F32 ? P_F32
                                   : w->prec == QW_F32_BF16STORE ? P_BF16 : P_COMP,
                                   cur_view(w), w->nx, w->ny, w->sup_dev, w->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->sup_host, w->sup_dev, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaEventRecord(w->sup_ev, w->stream);
    if (e != cudaSuccess) { w->sup_mode = 0; return cuda_error(w, e, "support search"); }
    w->sup_mode = 1;
    return QW_OK;
}

// Take the searched box (waits for the search only, not for later work).
static qw_status resolve_support(qw_walk *w) {
    if (w->sup_mode != 1) return QW_OK;
    w->sup_mode = 0;
    if (capturing(w)) { (void)cudaGetLastError(); return QW_OK; }   // step in full
    cudaError_t e = cudaEventSynchronize(w->sup_ev);
    if (e != cudaSuccess) return cuda_error(w, e, "support search");
    const unsigned long long *b = w->sup_host;
    if (b[0] > b[1] || b[2] > b[3]) return QW_OK;   // a zero state: stepped in full
    w->bx0 = (int64_t)b[0]; w->bw = (int64_t)(b[1] - b[0]) + 1;
    w->by0 = (int64_t)b[2]; w->bh = (int64_t)(b[3] - b[2]) + 1;
    if (w->bw >= w->nx) { w->bx0 = 0; w->bw = w->nx; }
    if (w->bh >= w->ny) { w->by0 = 0; w->bh = w->ny; }
    w->sup_mode = (w->bw < w->nx || w->bh < w->ny) ? 2 : 0;
    return QW_OK;
}

// The box after K more steps: one site more on each side per step, modulo the
// lattice on the periodic one, cut at its ends on the segment and the line.
static void grow_axis(int64_t &b0, int64_t &bw, int64_t n, int K, bool periodic) {
    if (bw >= n) return;
    if (periodic) {
        bw += 2 * (int64_t)K;
        b0 = ((b0 - K) % n + n) % n;
    } else {
        const int64_t lo = std::max<int64_t>(0, b0 - K), hi = std::min<int64_t>(n, b0 + bw + K);
        b0 = lo;
        bw = hi - lo;
    }
    if (bw >= n) { b0 = 0; bw = n; }
}
static void grow_support(qw_walk *w, int K) {
    if (w->sup_mode != 2) return;
    const bool per = w->bc == QW_BC_PERIODIC;
    grow_axis(w->bx0, w->bw, w->nx, K, per);
    grow_axis(w->by0, w->bh, w->ny, K, per);
    if (w->bw >= w->nx && w->bh >= w->ny) w->sup_mode = 0;
}

// Before a clipped step: the other buffer must be zero outside the box.
static qw_status clear_next(qw_walk *w) {
    if (w->next_clear) return QW_OK;
    cudaError_t e = cudaMemsetAsync(w->buf[w->cur ^ 1], 0, w->state_bytes, w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "clear");
    w->next_clear = true;
    return QW_OK;
}

qw_status run_steps(qw_walk *w, int64_t T, int adj) {
    if (T < 0) return set_error(w, QW_EINVAL, "T must be >= 0");
    if (T == 0) return QW_OK;
    const void *cp = w->coinp;
    bool generic = w->bc != QW_BC_PERIODIC || links_on(w);
    if (!generic && w->ndim == 2) {
        if (w->kind == CK_PERSITE) generic = true;
        if (w->kind == CK_PHASE && !(w->prec == QW_F32 || w->prec == QW_F64)) generic = true;
    }
    cudaError_t e = cudaSuccess;
    {
        qw_status st = resolve_support(w);
        if (st != QW_OK) return st;
        if (w->sup_mode == 2 && (st = clear_next(w)) != QW_OK) return st;
    }
    if (generic) {
        StepGenericArgs a{};
        a.ndim = w->ndim; a.nx = w->nx; a.ny = w->ny; a.shift = w->shift; a.bc = w->bc;
        a.kind = w->kind; a.coins = w->coins_dev; a.phi = w->phi_dev;
        a.links = w->has_links ? w->links_dev : nullptr; a.adjoint = adj;
        a.rthr = w->link_thr;
        a.rk0 = (uint32_t)w->link_seed; a.rk1 = (uint32_t)(w->link_seed >> 32);
        if (w->kind == CK_SIGN_P || w->kind == CK_SIGN_M) a.kind = CK_COMPLEX;   // generic reads the matrix
        // a clipped forward walk on the segment or the line: as many steps as keep
        // the box (after them) within one CTA's window go into one launch
        const bool win_ok = w->ndim == 1 && !adj && w->bc != QW_BC_PERIODIC &&
                            (w->shift == QW_SHIFT_MOVING || w->shift == QW_SHIFT_FLIPFLOP) && w->nx < (int64_t(1) << 30);
        const int64_t win_cap = win_ok ? window_capacity(w->prec) : 0;
        for (int64_t t = 0; t < T; ++t) {
            if (win_ok && w->sup_mode == 2) {
                int ns = (int)std::min<int64_t>(T - t, WINDOW_MAX_STEPS);
                auto width = [&](int k) {
                    return std::min<int64_t>(w->nx, w->bx0 + w->bw + k) - std::max<int64_t>(0, w->bx0 - k);
                };
                while (ns > 0 && width(ns) > win_cap) --ns;
                if (ns > 0) {
                    double gains[WINDOW_MAX_STEPS];
                    for (int i = 0; i < ns; ++i) gains[i] = drift_gain(w, 1, t + i + 1 == T);
                    a.rstep = (uint32_t)w->link_step;   // the first step's; step i draws rstep + i
                    if (w->link_thr) w->link_step += ns;
                    a.gain = 1.0;
                    a.in = cur_view(w); a.out = next_view(w);
                    a.bx0 = w->bx0; a.bw = w->bw; a.by0 = 0; a.bh = 1;
                    if ((e = stepwin(w->prec, a, cp, gains, ns, w->stream)) != cudaSuccess)
                        return cuda_error(w, e, "window step launch");
                    grow_support(w, ns);
                    w->cur ^= 1;
                    t += ns - 1;
                    continue;
                }
            }
            // random links: a forward step draws the mask of its index, then counts
            // up; the adjoint counts down first, so it undoes the last forward step
            if (w->link_thr && adj) --w->link_step;
            a.rstep = (uint32_t)w->link_step;
            if (w->link_thr && !adj) ++w->link_step;
            a.gain = drift_gain(w, 1, t + 1 == T);
            a.in = cur_view(w); a.out = next_view(w);
            // the tiled forward kernels run only the tiles around the support box
            // (the others, and the per-site kernel, step the whole lattice)
            if (w->sup_mode == 2) { a.bx0 = w->bx0; a.bw = w->bw; a.by0 = w->by0; a.bh = w->bh; }
            else { a.bx0 = a.by0 = a.bh = 0; a.bw = 0; }
            if ((e = stepgen(w->prec, a, cp, w->stream)) != cudaSuccess) return cuda_error(w, e, "generic step launch");
            grow_support(w, 1);
            w->cur ^= 1;
        }
        return QW_OK;
    }
    if (w->ndim == 1) {
        int K, tile, variant;
        effective_plan(w, K, tile, variant);
        const int teff = tile1d(w->prec, tile, w->kind, adj);
        if (variant != 1) K = std::min(K, 8 * teff);
        Step1DArgs a{};
        a.n = w->nx; a.shift = w->shift; a.kind = w->kind; a.coins = w->coins_dev;
        for (int64_t rem = T; rem > 0;) {
            a.K = (int)std::min<int64_t>(K, rem);
            const bool clip = w->sup_mode == 2;
            // the last, shorter launch of a sweep plan falls back to the tile kernel
            // if needed; a clipped launch always runs the tiles
            a.variant = (!clip && variant == 1 && sweep_ok(w, a.K, tile)) ? 1 : 0;
            a.tile = a.variant == 1 ? tile : teff;
            if (a.variant == 0) a.K = std::min(a.K, 8 * teff);
            launch_gains_1d(w, a.K, adj, a, true, rem - a.K == 0);
            a.in = cur_view(w); a.out = next_view(w);
            a.obeg = a.oend = 0;
            const int64_t n = w->nx, len = w->bw + 2 * (int64_t)a.K;
            if (!clip || len >= n) {
                e = step1d(w->prec, a, cp, adj, w->stream);
            } else {
                // the outputs: the support widened by K, as one or two ranges inside [0, n)
                const int64_t b0 = ((w->bx0 - a.K) % n + n) % n;
                a.obeg = b0; a.oend = std::min(n, b0 + len);
                e = step1d(w->prec, a, cp, adj, w->stream);
                if (e == cudaSuccess && b0 + len > n) {
                    a.obeg = 0; a.oend = b0 + len - n;
                    e = step1d(w->prec, a, cp, adj, w->stream);
                }
            }
            if (e != cudaSuccess) return cuda_error(w, e, "1D step launch");
            grow_support(w, a.K);
            w->cur ^= 1;
            rem -= a.K;
        }
        return QW_OK;
    }
    Step2DArgs a{};
    a.nx = w->nx; a.ny = w->ny; a.shift = w->shift; a.kind = w->kind; a.coins = w->coins_dev;
    a.phi = w->phi_dev; a.K = 1;
    // the support box of the launch's input (bw = 0: the whole torus)
    auto set_box = [&](Step2DArgs &b) {
        if (w->sup_mode == 2) { b.bx0 = w->bx0; b.bw = w->bw; b.by0 = w->by0; b.bh = w->bh; }
        else { b.bx0 = b.by0 = b.bh = 0; b.bw = 0; }
    };
    int K2, t2;
    effective_plan(w, K2, t2);
    if (!adj && K2 > 1 && step2d_tb_ok(w->prec, w->kind, K2, w->shift)) {
        // whole blocks of K2 steps in the streaming kernel, the rest one step at a time
        Step2DArgs b = a;
        b.K = K2;
        while (T >= K2) {
            b.gain = drift_gain(w, K2, T - K2 == 0);   // applied once, to the launch's output
            b.in = cur_view(w); b.out = next_view(w);
            set_box(b);
            if ((e = launch_step2d_tb(b, cp, w->stream)) != cudaSuccess) return cuda_error(w, e, "2D blocked step launch");
            grow_support(w, K2);
            w->cur ^= 1;
            T -= K2;
        }
    }
    for (int64_t t = 0; t < T; ++t) {
        a.gain = drift_gain(w, 1, t + 1 == T);
        a.in = cur_view(w); a.out = next_view(w);
        set_box(a);
        if ((e = step2d(w->prec, a, cp, adj, w->stream)) != cudaSuccess) return cuda_error(w, e, "2D step launch");
        grow_support(w, 1);
        w->cur ^= 1;
    }
    return QW_OK;
}

}  // namespace qw

// ------------------------------------------------------------------ ABI
extern "C" {

const char *qw_version(void) { return "qw 0.1 sm_103a"; }

const char *qw_status_string(qw_status s) {
    switch (s) {
        case QW_OK: return "ok";
        case QW_EINVAL: return "invalid argument";
        case QW_ENOMEM: return "out of memory";
        case QW_ECUDA: return "CUDA error";
        case QW_ESTATE: return "invalid state for this call";
        case QW_ETIMEOUT: return "device wait timed out";
        case QW_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *qw_last_error(const qw_walk *w) { return w ? w->err.c_str() : "null handle"; }

qw_status qw_destroy(qw_walk *w) {
    if (!w) return QW_OK;
    cudaStreamSynchronize(w->stream);
    cudaFree(w->buf[0]);
    cudaFree(w->buf[1]);
    cudaFree(w->coins_dev);
    cudaFree(w->phi_dev);
    cudaFree(w->links_dev);
    cudaFree(w->partials);
    cudaFree(w->norm_dev);
    cudaFree(w->p_dev);
    cudaFree(w->staging);
    cudaFree(w->grad_scratch);
    cudaFree(w->buf3);
    cudaFree(w->pipe_p[0]);
    cudaFree(w->pipe_p[1]);
    cudaFree(w->pipe_norm);
    if (w->s_in) cudaStreamDestroy(w->s_in);
    if (w->s_out) cudaStreamDestroy(w->s_out);
    if (w->host_scalar) cudaFreeHost(w->host_scalar);
    cudaFree(w->sup_dev);
    if (w->sup_host) cudaFreeHost(w->sup_host);
    if (w->sup_ev) cudaEventDestroy(w->sup_ev);
    delete w;
    return QW_OK;
}

qw_status qw_create(int ndim, const int64_t *dims, int coin_dim, qw_boundary bc, qw_shift shift,
                    qw_precision prec, void *cuda_stream, qw_walk **out) {
    if (!out) return QW_EINVAL;
    *out = nullptr;
    if ((ndim != 1 && ndim != 2) || !dims || coin_dim != 2 * ndim) return QW_EINVAL;
    if (dims[0] < 1 || (ndim == 2 && dims[1] < 1)) return QW_EINVAL;
    if ((int)bc < 0 || (int)bc > 2 || (int)shift < 0 || (int)shift > 2 || (int)prec < 0 || (int)prec > 3)
        return QW_EINVAL;
    if (shift == QW_SHIFT_DIAGONAL && (ndim != 2 || bc != QW_BC_PERIODIC)) return QW_EINVAL;
    const int64_t nx = dims[0], ny = ndim == 2 ? dims[1] : 1;
    if (nx > (int64_t(1) << 40) || ny > (int64_t(1) << 40) || nx * ny > (int64_t(1) << 40)) return QW_EINVAL;

    qw_walk *w = new (std::nothrow) qw_walk();
    if (!w) return QW_ENOMEM;
    w->ndim = ndim; w->d = coin_dim; w->nx = nx; w->ny = ny; w->ns = nx * ny;
    w->bc = bc; w->shift = shift; w->prec = prec;
    w->stream = static_cast<cudaStream_t>(cuda_stream);
    w->pitch = (w->ns + 63) / 64 * 64;
    w->nslots = w->d * (prec == QW_F32_COMP ? 2 : 1);
    w->slot_bytes = slot_bytes_of(prec);
    w->state_bytes = (size_t)w->nslots * w->pitch * w->slot_bytes;

    cudaError_t e = cudaGetDevice(&w->device);
    if (e == cudaSuccess) e = dev_alloc(&w->buf[0], w->state_bytes);
    if (e == cudaSuccess) e = dev_alloc(&w->buf[1], w->state_bytes);
    if (e == cudaSuccess) e = dev_alloc((void **)&w->partials, sizeof(double) * marginal_blocks());
    if (e == cudaSuccess) e = dev_alloc((void **)&w->norm_dev, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&w->host_scalar, sizeof(double) * 4);
    if (e == cudaSuccess) e = dev_alloc((void **)&w->sup_dev, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&w->sup_host, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->sup_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->buf[0], 0, w->state_bytes, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->buf[1], 0, w->state_bytes, w->stream);
    if (e != cudaSuccess) {
        qw_status st = e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA;
        (void)cudaGetLastError();
        qw_destroy(w);
        return st;
    }
    double ident[32] = {0};
    for (int i = 0; i < coin_dim; ++i) ident[2 * (i * coin_dim + i)] = 1.0;
    apply_global_coin(w, ident);
    *out = w;
    return QW_OK;
}

int64_t qw_nsites(const qw_walk *w) { return w ? w->ns : -1; }

qw_status qw_synchronize(qw_walk *w) {
    if (!w) return QW_EINVAL;
    cudaError_t e = cudaStreamSynchronize(w->stream);
    return e == cudaSuccess ? QW_OK : cuda_error(w, e, "synchronize");
}

qw_status qw_set_coin(qw_walk *w, const double *coin, int per_site, int on_device) {
    if (!w) return QW_EINVAL;
    if (!coin) return set_error(w, QW_EINVAL, "coin is NULL");
    const int d = w->d;
    cudaError_t e;
    if (!per_site) {
        double h[32];
        if (on_device) {
            e = cudaMemcpyAsync(h, coin, sizeof(double) * 2 * d * d, cudaMemcpyDeviceToHost, w->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
            if (e != cudaSuccess) return cuda_error(w, e, "coin copy");
        } else {
            std::memcpy(h, coin, sizeof(double) * 2 * d * d);
        }
        apply_global_coin(w, h);
        return QW_OK;
    }
    const int64_t count = w->ns * d * d;   // complex entries
    const size_t want = (size_t)count * 2 * real_bytes(w->prec);
    if (w->coins_bytes != want) {
        cudaStreamSynchronize(w->stream);
        cudaFree(w->coins_dev);
        w->coins_dev = nullptr; w->coins_bytes = 0;
        if ((e = dev_alloc(&w->coins_dev, want)) != cudaSuccess) return cuda_error(w, e, "per-site coin allocation");
        w->coins_bytes = want;
    }
    if (on_device) {
        if ((e = launch_convert_coins(w->prec, coin, w->coins_dev, count, w->stream)) != cudaSuccess)
            return cuda_error(w, e, "coin conversion");
    } else {
        qw_status st = ensure_staging(w, STAGE_CHUNK);
        if (st != QW_OK) return st;
        const int64_t per = (int64_t)(STAGE_CHUNK / 16);
        for (int64_t off = 0; off < count; off += per) {
            const int64_t n = std::min(per, count - off);
            e = cudaMemcpyAsync(w->staging, coin + 2 * off, (size_t)n * 16, cudaMemcpyHostToDevice, w->stream);
            if (e == cudaSuccess)
                e = launch_convert_coins(w->prec, (const double *)w->staging,
                                         (char *)w->coins_dev + (size_t)off * 2 * real_bytes(w->prec), n, w->stream);
            if (e != cudaSuccess) return cuda_error(w, e, "coin upload");
        }
    }
    w->kind = CK_PERSITE;
    return QW_OK;
}

qw_status qw_set_coin_phases(qw_walk *w, const double *base, const float *phi, int on_device) {
    if (!w) return QW_EINVAL;
    if (!base || !phi) return set_error(w, QW_EINVAL, "base and phi are required");
    const int d = w->d;
    const size_t pbytes = sizeof(float) * (size_t)w->ns * d;
    cudaError_t e;
    if (!w->phi_dev) {
        if ((e = dev_alloc((void **)&w->phi_dev, pbytes)) != cudaSuccess) return cuda_error(w, e, "phase allocation");
    }
    e = cudaMemcpyAsync(w->phi_dev, phi, pbytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "phase copy");
    apply_global_coin(w, base);   // the kernels read the base coin from here
    if (w->ndim == 2) {
        w->kind = CK_PHASE;
        return QW_OK;
    }
    // 1D: expand to per-site matrices once
    const size_t want = (size_t)w->ns * d * d * 2 * real_bytes(w->prec);
    if (w->coins_bytes != want) {
        cudaStreamSynchronize(w->stream);
        cudaFree(w->coins_dev);
        w->coins_dev = nullptr; w->coins_bytes = 0;
        if ((e = dev_alloc(&w->coins_dev, want)) != cudaSuccess) return cuda_error(w, e, "per-site coin allocation");
        w->coins_bytes = want;
    }
    qw_status st = ensure_staging(w, 256);
    if (st != QW_OK) return st;
    e = cudaMemcpyAsync(w->staging, base, sizeof(double) * 2 * d * d, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = launch_phase_coins(w->prec, (const double *)w->staging, w->phi_dev, w->coins_dev, w->ns, d, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);  // base lives on the caller's stack
    if (e != cudaSuccess) return cuda_error(w, e, "phase coin expansion");
    w->kind = CK_PERSITE;
    return QW_OK;
}

qw_status qw_set_links(qw_walk *w, const uint8_t *closed, int on_device) {
    if (!w) return QW_EINVAL;
    if (!closed) { w->has_links = false; return QW_OK; }
    if (w->shift == QW_SHIFT_DIAGONAL) return set_error(w, QW_EUNSUPPORTED, "broken links are defined on the axis lattice");
    const size_t bytes = (size_t)w->ndim * w->ns;
    cudaError_t e;
    if (!w->links_dev && (e = dev_alloc((void **)&w->links_dev, bytes)) != cudaSuccess)
        return cuda_error(w, e, "link mask allocation");
    e = cudaMemcpyAsync(w->links_dev, closed, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "link mask copy");
    if (!on_device && (e = cudaStreamSynchronize(w->stream)) != cudaSuccess) return cuda_error(w, e, "link mask copy");
    w->has_links = true;
    return QW_OK;
}

qw_status qw_set_link_noise(qw_walk *w, double p, uint64_t seed, int64_t step) {
    if (!w) return QW_EINVAL;
    if (!(p >= 0.0 && p <= 1.0)) return set_error(w, QW_EINVAL, "p must be in [0, 1]");
    if (p > 0.0 && w->shift == QW_SHIFT_DIAGONAL)
        return set_error(w, QW_EUNSUPPORTED, "broken links are defined on the axis lattice");
    const double scaled = p * 4294967296.0;
    w->link_thr = scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
    w->link_seed = seed;
    w->link_step = step;
    return QW_OK;
}

qw_status qw_get_link_step(const qw_walk *w, int64_t *step) {
    if (!w || !step) return QW_EINVAL;
    *step = w->link_step;
    return QW_OK;
}

static bool direct_layout(const qw_walk *w, qw_cdtype dt) {
    return (w->prec == QW_F32 && dt == QW_C64) || (w->prec == QW_F64 && dt == QW_C128);
}

qw_status qw_set_state(qw_walk *w, const void *amp, qw_cdtype dtype, int on_device) {
    if (!w) return QW_EINVAL;
    if (!amp || (dtype != QW_C128 && dtype != QW_C64)) return set_error(w, QW_EINVAL, "bad state buffer or dtype");
    const size_t eb = dtype == QW_C128 ? 16 : 8;
    const size_t plane = (size_t)w->ns * eb;
    cudaError_t e = cudaSuccess;
    const View dst = cur_view(w);
    w->gain_fb = 1.0;
    w->drift_pending = 1.0;
    w->sup_mode = 0;
    if (direct_layout(w, dtype)) {
        e = cudaMemcpy2DAsync(w->buf[w->cur], (size_t)w->pitch * w->slot_bytes, amp, plane, plane, w->d,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, w->stream);
        if (e != cudaSuccess) return cuda_error(w, e, "state copy");
        return queue_support(w);
    }
    if (w->prec == QW_F32_COMP) {  // clear the lo slots first (a complex64 input has none)
        e = cudaMemsetAsync((char *)w->buf[w->cur] + (size_t)w->d * w->pitch * w->slot_bytes, 0,
                            (size_t)w->d * w->pitch * w->slot_bytes, w->stream);
        if (e != cudaSuccess) return cuda_error(w, e, "state clear");
    }
    for (int c = 0; c < w->d; ++c) {
        const char *src = static_cast<const char *>(amp) + c * plane;
        if (on_device) {
            if ((e = launch_import(w->prec, dst, w->ns, src, dtype == QW_C64, 0, w->ns, c, w->stream)) != cudaSuccess)
                return cuda_error(w, e, "state import");
            continue;
        }
        qw_status st = ensure_staging(w, STAGE_CHUNK);
        if (st != QW_OK) return st;
        const int64_t per = (int64_t)(STAGE_CHUNK / eb);
        for (int64_t off = 0; off < w->ns; off += per) {
            const int64_t n = std::min(per, w->ns - off);
            e = cudaMemcpyAsync(w->staging, src + off * eb, (size_t)n * eb, cudaMemcpyHostToDevice, w->stream);
            if (e == cudaSuccess) e = launch_import(w->prec, dst, w->ns, w->staging, dtype == QW_C64, off, n, c, w->stream);
            if (e != cudaSuccess) return cuda_error(w, e, "state upload");
        }
    }
    return queue_support(w);
}

qw_status qw_get_state(qw_walk *w, void *amp_out, qw_cdtype dtype, int on_device) {
    if (!w) return QW_EINVAL;
    if (!amp_out || (dtype != QW_C128 && dtype != QW_C64)) return set_error(w, QW_EINVAL, "bad state buffer or dtype");
    const size_t eb = dtype == QW_C128 ? 16 : 8;
    const size_t plane = (size_t)w->ns * eb;
    cudaError_t e = cudaSuccess;
    const View src = cur_view(w);
    if (direct_layout(w, dtype)) {
        e = cudaMemcpy2DAsync(amp_out, plane, w->buf[w->cur], (size_t)w->pitch * w->slot_bytes, plane, w->d,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(w->stream);
        return e == cudaSuccess ? QW_OK : cuda_error(w, e, "state copy");
    }
    for (int c = 0; c < w->d; ++c) {
        char *dst = static_cast<char *>(amp_out) + c * plane;
        if (on_device) {
            if ((e = launch_export(w->prec, src, w->ns, dst, dtype == QW_C64, 0, w->ns, c, w->stream)) != cudaSuccess)
                return cuda_error(w, e, "state export");
            continue;
        }
        qw_status st = ensure_staging(w, STAGE_CHUNK);
        if (st != QW_OK) return st;
        const int64_t per = (int64_t)(STAGE_CHUNK / eb);
        for (int64_t off = 0; off < w->ns; off += per) {
            const int64_t n = std::min(per, w->ns - off);
            e = launch_export(w->prec, src, w->ns, w->staging, dtype == QW_C64, off, n, c, w->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst + off * eb, w->staging, (size_t)n * eb, cudaMemcpyDeviceToHost, w->stream);
            if (e != cudaSuccess) return cuda_error(w, e, "state download");
        }
    }
    if (!on_device && (e = cudaStreamSynchronize(w->stream)) != cudaSuccess) return cuda_error(w, e, "state download");
    return QW_OK;
}

qw_status qw_step(qw_walk *w, int64_t T) {
    if (!w) return QW_EINVAL;
    NvtxRange nvtx("qw_step");
    return run_steps(w, T, 0);
}

qw_status qw_step_adjoint(qw_walk *w, int64_t T) {
    if (!w) return QW_EINVAL;
    NvtxRange nvtx("qw_step_adjoint");
    return run_steps(w, T, 1);
}

qw_status qw_probabilities(qw_walk *w, void *P_out, qw_rdtype pdtype, int on_device, double *norm_out) {
    if (!w) return QW_EINVAL;
    NvtxRange nvtx("qw_probabilities");
    if (pdtype != QW_R64 && pdtype != QW_R32) return set_error(w, QW_EINVAL, "bad probability dtype");
    const size_t pb = (size_t)w->ns * (pdtype == QW_R32 ? 4 : 8);
    void *pdst = nullptr;
    cudaError_t e;
    if (P_out) {
        if (on_device) {
            pdst = P_out;
        } else {
            if (w->p_bytes < pb) {
                cudaStreamSynchronize(w->stream);
                cudaFree(w->p_dev);
                w->p_dev = nullptr; w->p_bytes = 0;
                if ((e = dev_alloc(&w->p_dev, pb)) != cudaSuccess) return cuda_error(w, e, "probability buffer");
                w->p_bytes = pb;
            }
            pdst = w->p_dev;
        }
    }
    e = launch_marginals(w->prec, cur_view(w), w->ns, pdst, pdtype == QW_R32, w->partials, marginal_blocks(),
                         w->norm_dev, w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "marginal launch");
    if (P_out && !on_device) {
        if ((e = cudaMemcpyAsync(P_out, w->p_dev, pb, cudaMemcpyDeviceToHost, w->stream)) != cudaSuccess)
            return cuda_error(w, e, "probability download");
    }
    if (norm_out) {
        if ((e = cudaMemcpyAsync(w->host_scalar, w->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, w->stream)) != cudaSuccess)
            return cuda_error(w, e, "norm download");
    }
    if (norm_out || (P_out && !on_device)) {
        if ((e = cudaStreamSynchronize(w->stream)) != cudaSuccess) return cuda_error(w, e, "marginals");
        if (norm_out) *norm_out = *w->host_scalar;
    }
    return QW_OK;
}

qw_status qw_run_host_batch(qw_walk *w, int count, const void *amp_in, int64_t in_stride, qw_cdtype dtype, int64_t T,
                            void *P_out, int64_t p_stride, qw_rdtype pdtype, double *norms_out) {
    if (!w) return QW_EINVAL;
    NvtxRange nvtx("qw_run_host_batch");
    if (count < 0 || T < 0 || in_stride < 0 || p_stride < 0 || (count && (!amp_in || !P_out)) ||
        (pdtype != QW_R64 && pdtype != QW_R32))
        return set_error(w, QW_EINVAL, "bad count, T, strides, buffers or probability dtype");
    if (!direct_layout(w, dtype))
        return set_error(w, QW_EUNSUPPORTED, "pipelined runs take complex64 states for FP32 and complex128 for FP64");
    if (count == 0) return QW_OK;
    w->sup_mode = 0;   // arbitrary host states: every run steps the whole lattice
    const size_t plane = (size_t)w->ns * (dtype == QW_C128 ? 16 : 8);
    const size_t pb = (size_t)w->ns * (pdtype == QW_R32 ? 4 : 8);
    cudaError_t e = cudaSuccess;
    if (!w->buf3 && (e = dev_alloc(&w->buf3, w->state_bytes)) != cudaSuccess) return cuda_error(w, e, "third state buffer");
    if (w->pipe_p_bytes < pb) {
        cudaStreamSynchronize(w->stream);
        cudaFree(w->pipe_p[0]); cudaFree(w->pipe_p[1]);
        w->pipe_p[0] = w->pipe_p[1] = nullptr; w->pipe_p_bytes = 0;
        if ((e = dev_alloc(&w->pipe_p[0], pb)) == cudaSuccess) e = dev_alloc(&w->pipe_p[1], pb);
        if (e != cudaSuccess) return cuda_error(w, e, "pipelined probability buffers");
        w->pipe_p_bytes = pb;
    }
    if (w->pipe_norm_cap < count) {
        cudaStreamSynchronize(w->stream);
        cudaFree(w->pipe_norm);
        w->pipe_norm = nullptr; w->pipe_norm_cap = 0;
        if ((e = dev_alloc((void **)&w->pipe_norm, sizeof(double) * (size_t)count)) != cudaSuccess)
            return cuda_error(w, e, "pipelined norms");
        w->pipe_norm_cap = count;
    }
    if (!w->s_in && (e = cudaStreamCreateWithFlags(&w->s_in, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_error(w, e, "copy stream");
    if (!w->s_out && (e = cudaStreamCreateWithFlags(&w->s_out, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_error(w, e, "copy stream");
    // events: state i arrived; run i's buffers and P slot free again (compute done);
    // P slot of run i copied out
    std::vector<cudaEvent_t> ev_in(count), ev_done(count), ev_out(count);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming);
    }
    auto destroy_events = [&]() {
        for (int i = 0; i < count; ++i) {
            if (ev_in[i]) cudaEventDestroy(ev_in[i]);
            if (ev_done[i]) cudaEventDestroy(ev_done[i]);
            if (ev_out[i]) cudaEventDestroy(ev_out[i]);
        }
    };
    if (e != cudaSuccess) { destroy_events(); return cuda_error(w, e, "pipeline events"); }

    // Three buffers rotate: run i reads its state from X_i and ping-pongs with
    // Y_i; run i+1's state is copied into the third, Z_i, which run i-1 may
    // still be using until its event, while run i computes.
    void *bufs[3] = {w->buf[w->cur], w->buf[w->cur ^ 1], w->buf3};
    auto copy_in = [&](int i, void *dst) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        if (i >= 2) r = cudaStreamWaitEvent(w->s_in, ev_done[i - 2], 0);   // dst was run i-2's buffer
        if (r == cudaSuccess)
            r = cudaMemcpy2DAsync(dst, (size_t)w->pitch * w->slot_bytes, static_cast<const char *>(amp_in) + i * in_stride,
                                  plane, plane, w->d, cudaMemcpyHostToDevice, w->s_in);
        if (r == cudaSuccess) r = cudaEventRecord(ev_in[i], w->s_in);
        return r;
    };
    // wait for work the caller queued on the walk's stream before touching its buffers
    cudaEvent_t start_ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming)) == cudaSuccess &&
        (e = cudaEventRecord(start_ev, w->stream)) == cudaSuccess &&
        (e = cudaStreamWaitEvent(w->s_in, start_ev, 0)) == cudaSuccess)
        e = copy_in(0, bufs[0]);
    int x = 0;   // index in bufs of run i's input
    qw_status st = QW_OK;
    for (int i = 0; i < count && e == cudaSuccess && st == QW_OK; ++i) {
        const int y = (x + 1) % 3, z = (x + 2) % 3;
        if (i + 1 < count && (e = copy_in(i + 1, bufs[z])) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(w->stream, ev_in[i], 0)) != cudaSuccess) break;
        if (i >= 2 && (e = cudaStreamWaitEvent(w->stream, ev_out[i - 2], 0)) != cudaSuccess) break;   // P slot free
        // the walk's two buffers for this run: the arrived state and a free one
        w->cur = 0;
        w->buf[0] = bufs[x];
        w->buf[1] = bufs[y];
        w->gain_fb = 1.0;
        w->drift_pending = 1.0;
        if ((st = run_steps(w, T, 0)) != QW_OK) break;
        void *pslot = w->pipe_p[i & 1];
        e = launch_marginals(w->prec, cur_view(w), w->ns, pslot, pdtype == QW_R32, w->partials, marginal_blocks(),
                             w->pipe_norm + i, w->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev_done[i], w->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(w->s_out, ev_done[i], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char *>(P_out) + i * p_stride, pslot, pb, cudaMemcpyDeviceToHost, w->s_out);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[i], w->s_out);
        // the run's result is in w->buf[w->cur]; the next run's input is in bufs[z]
        const int res = w->buf[w->cur] == bufs[x] ? x : y;
        // rotate so that the next run reads bufs[z] and ping-pongs with the
        // buffer not holding this run's result (its P is computed already, in
        // stream order, before the next run's first kernel)
        const int other = res == x ? y : x;
        void *const nz = bufs[z], *const no = bufs[other], *const nr = bufs[res];
        bufs[0] = nz; bufs[1] = no; bufs[2] = nr;
        x = 0;
    }
    // leave the walk holding the last run's result as its state
    cudaError_t e2 = cudaStreamSynchronize(w->s_in);
    cudaError_t e3 = cudaStreamSynchronize(w->s_out);
    cudaError_t e4 = cudaStreamSynchronize(w->stream);
    // after the loop bufs[2] holds the last result; the other two are free
    w->buf[0] = bufs[2];
    w->buf[1] = bufs[1];
    w->buf3 = bufs[0];
    w->cur = 0;
    if (start_ev) cudaEventDestroy(start_ev);
    destroy_events();
    if (st != QW_OK) return st;
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
    // the norms of all runs in one copy once everything is done (norms_out may
    // be pageable: a copy per run would hold the host until that run ended)
    if (e == cudaSuccess && norms_out) {
        e = cudaMemcpyAsync(norms_out, w->pipe_norm, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    }
    if (e != cudaSuccess) return cuda_error(w, e, "pipelined runs");
    return QW_OK;
}

qw_status qw_set_plan(qw_walk *w, int depth_k, int tile) {
    if (!w) return QW_EINVAL;
    if (depth_k == 0) { w->plan_k = 0; w->plan_tile = 0; w->plan_user = false; return QW_OK; }
    if (depth_k < 0 || tile < 0) return set_error(w, QW_EINVAL, "negative plan");
    if (w->ndim == 2) {
        if (depth_k != 1 && depth_k != 4 && depth_k != 8)
            return set_error(w, QW_EINVAL, "2D plans take k = 1, 4 or 8");
        w->plan_k = depth_k; w->plan_tile = 0; w->plan_user = true;
        return QW_OK;
    }
    int dk, dt, dv;
    default_plan(w, dk, dt, dv);
    const int teff = tile1d(w->prec, tile ? tile : dt, CK_REAL, 0);
    if (tile && teff != tile) return set_error(w, QW_EINVAL, "tile not compiled for this precision");
    if (depth_k > 8 * teff) return set_error(w, QW_EINVAL, "k exceeds 8 * tile");
    w->plan_k = depth_k; w->plan_tile = teff; w->plan_variant = 0; w->plan_user = true;
    return QW_OK;
}

qw_status qw_set_plan_ex(qw_walk *w, int depth_k, int tile, int variant) {
    if (!w) return QW_EINVAL;
    if (variant != 1) {
        qw_status st = qw_set_plan(w, depth_k, tile);
        if (st == QW_OK && depth_k == 0) w->plan_variant = -1;
        return st;
    }
    if (w->ndim != 1 || depth_k < 1 || !sweep_ok(w, std::max(depth_k, 2), tile))
        return set_error(w, QW_EINVAL, "the sweep kernel needs the periodic 1D walk, N at least its "
                                       "chunk (32 x tile sites), a global coin, FP32/BF16/FP64 and "
                                       "1 <= k < chunk / 2");
    w->plan_k = depth_k; w->plan_tile = sweep_tile(w, tile); w->plan_variant = 1;
    w->plan_user = true;
    return QW_OK;
}

qw_status qw_get_plan_ex(const qw_walk *w, int *depth_k, int *tile, int *variant) {
    if (!w || !depth_k || !tile || !variant) return QW_EINVAL;
    int k, t, v;
    effective_plan(w, k, t, v);
    if (w->ndim == 1) t = v == 1 ? sweep_tile(w, t) : tile1d(w->prec, t, w->kind, 0);
    *depth_k = k; *tile = t; *variant = v;
    return QW_OK;
}

qw_status qw_set_clipping(qw_walk *w, int on) {
    if (!w) return QW_EINVAL;
    w->clip_on = on != 0;
    if (!w->clip_on) w->sup_mode = 0;
    return QW_OK;
}

qw_status qw_describe(const qw_walk *w, char *buf, size_t len) {
    if (!w || !buf || !len) return QW_EINVAL;
    static const char *kinds[] = {"real", "complex", "grover", "hadamard2", "per_site", "phase",
                                  "hadamard_class", "hadamard_class"};
    int k, t, var;
    effective_plan(w, k, t, var);
    if (w->ndim == 1) t = var == 1 ? sweep_tile(w, t) : tile1d(w->prec, t, w->kind, 0);
    const bool generic = w->bc != QW_BC_PERIODIC || links_on(w) ||
                         (w->ndim == 2 && (w->kind == CK_PERSITE ||
                                           (w->kind == CK_PHASE && !(w->prec == QW_F32 || w->prec == QW_F64))));
    // a clipped walk on the segment or the line whose box (one step on) fits the
    // window CTA runs its steps in the window kernel
    const bool window = generic && w->ndim == 1 && w->bc != QW_BC_PERIODIC && w->sup_mode == 2 &&
                        (w->shift == QW_SHIFT_MOVING || w->shift == QW_SHIFT_FLIPFLOP) && w->nx < (int64_t(1) << 30) &&
                        std::min<int64_t>(w->nx, w->bx0 + w->bw + 1) - std::max<int64_t>(0, w->bx0 - 1) <=
                            window_capacity(w->prec);
    char sup[96];
    if (w->sup_mode == 2)
        std::snprintf(sup, sizeof sup, "[%lld, %lld, %lld, %lld]", (long long)w->bx0, (long long)w->bw,
                      (long long)w->by0, (long long)w->bh);
    else
        std::snprintf(sup, sizeof sup, "\"%s\"", w->sup_mode == 1 ? "pending" : "full");
    std::snprintf(buf, len,
                  "{\"ndim\": %d, \"sites\": %lld, \"coin_dim\": %d, \"precision\": %d, \"coin_kind\": \"%s\", "
                  "\"k\": %d, \"tile\": %d, \"path\": \"%s\", \"state_bytes\": %zu, \"clipping\": %d, "
                  "\"support\": %s}",
                  w->ndim, (long long)w->ns, w->d, w->prec, kinds[w->kind], k, t,
                  window ? "k_step1d_window" : generic ? "generic"
                          : (w->ndim == 1 ? (var == 1 && w->sup_mode != 2 ? "k_step1d_sweep" : "k_step1d")
                                          : (k > 1 && step2d_tb_ok(w->prec, w->kind, k, w->shift) ? "k_step2d_tb" : "k_step2d")),
                  w->state_bytes, (int)w->clip_on, sup);
    return QW_OK;
}

qw_status qw_get_plan(const qw_walk *w, int *depth_k, int *tile) {
    if (!w || !depth_k || !tile) return QW_EINVAL;
    int k, t;
    effective_plan(w, k, t);
    if (w->ndim == 1) t = tile1d(w->prec, t, w->kind, 0);
    *depth_k = k;
    *tile = t;
    return QW_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;  // key -> (tile, k)
bool g_tune_loaded = false;

std::string tune_key(const qw_walk *w) {
    char b[128];
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= w->ns) ++lg;
    std::snprintf(b, sizeof b, "%dd_p%d_k%d_s%d_n2^%d", w->ndim, w->prec, w->kind, w->shift, lg);
    return b;
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("QW_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[128];
    int tile, k;
    // format: one entry per line:  "key": [tile, k],
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        if (std::sscanf(line, " \"%127[^\"]\": [%d, %d]", key, &tile, &k) == 3) g_tune[key] = {tile, k};
    }
    std::fclose(f);
}

void tune_save() {
    const char *path = std::getenv("QW_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : g_tune)
        std::fprintf(f, "  \"%s\": [%d, %d]%s\n", kv.first.c_str(), kv.second.first, kv.second.second,
                     ++i < g_tune.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
}

}  // namespace

extern "C" qw_status qw_autotune(qw_walk *w, char *report, size_t report_len) {
    if (!w) return QW_EINVAL;
    auto put = [&](const char *s) {
        if (report && report_len) { std::strncpy(report, s, report_len - 1); report[report_len - 1] = 0; }
    };
    if (w->bc != QW_BC_PERIODIC || links_on(w)) {
        put("{\"tuned\": false, \"reason\": \"the generic boundary / broken-link kernel has no plan space\"}");
        return QW_OK;
    }
    if (w->ndim == 2) {
        // k = 1 (fused step) against the streaming kernel at k = 4 and 8
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        Step2DArgs a{};
        a.nx = w->nx; a.ny = w->ny; a.shift = w->shift; a.kind = w->kind; a.coins = w->coins_dev;
        a.phi = w->phi_dev; a.gain = 1.0;
        a.in = cur_view(w); a.out = next_view(w);
        float best = 1e30f;
        int best_k = 1;
        cudaError_t err = cudaSuccess;
        for (int k : {1, 4, 8}) {
            if (k > 1 && !step2d_tb_ok(w->prec, w->kind, k, w->shift)) continue;
            a.K = k;
            auto launch = [&]() { return k == 1 ? step2d(w->prec, a, w->coinp, 0, w->stream) : launch_step2d_tb(a, w->coinp, w->stream); };
            if ((err = launch()) != cudaSuccess) break;
            cudaEventRecord(e0, w->stream);
            for (int r = 0; r < 3; ++r) launch();
            cudaEventRecord(e1, w->stream);
            if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / (3 * k) < best) { best = ms / (3 * k); best_k = k; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err != cudaSuccess) return cuda_error(w, err, "autotune");
        w->plan_k = best_k; w->plan_tile = 0; w->plan_user = true;
        char b2[256];
        std::snprintf(b2, sizeof b2, "{\"tuned\": true, \"ndim\": 2, \"k\": %d, \"ms_per_step\": %.6g}", best_k, best);
        put(b2);
        return QW_OK;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    const std::string key = tune_key(w);
    auto it = g_tune.find(key);
    char buf[512];
    if (it != g_tune.end()) {
        w->plan_tile = std::abs(it->second.first);   // a negative tile records the sweep kernel
        w->plan_variant = it->second.first < 0 ? 1 : 0;
        w->plan_k = it->second.second;
        std::snprintf(buf, sizeof buf, "{\"tuned\": true, \"cached\": true, \"key\": \"%s\", \"tile\": %d, \"k\": %d}",
                      key.c_str(), w->plan_tile, w->plan_k);
        put(buf);
        return QW_OK;
    }
    int ta, tb;
    tiles_of(w->prec, ta, tb);
    const int tiles[2] = {ta, tb};
    const int ks[] = {1, 2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64, 96, 128};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_t = ta, best_k = 1;
    Step1DArgs a{};
    a.n = w->nx; a.shift = w->shift; a.kind = w->kind; a.coins = w->coins_dev;
    a.in = cur_view(w); a.out = next_view(w);   // reads the state, writes only the scratch buffer
    cudaError_t err = cudaSuccess;
    for (int ti = 0; ti < 2; ++ti) {
        const int teff = tile1d(w->prec, tiles[ti], w->kind, 0);
        if (ti == 1 && teff == tile1d(w->prec, tiles[0], w->kind, 0)) break;  // kind has one tile only
        for (int k : ks) {
            if (k > 8 * teff) break;
            a.tile = teff; a.K = k;
            launch_gains_1d(w, k, 0, a, false);
            err = step1d(w->prec, a, w->coinp, 0, w->stream);   // warm-up
            if (err != cudaSuccess) break;
            cudaEventRecord(e0, w->stream);
            const int reps = 3;
            for (int r = 0; r < reps; ++r) step1d(w->prec, a, w->coinp, 0, w->stream);
            cudaEventRecord(e1, w->stream);
            if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const float per_step = ms / (reps * k);
            if (per_step < best) { best = per_step; best_t = teff; best_k = k; }
        }
        if (err != cudaSuccess) break;
    }
    int best_v = 0;
    if (err == cudaSuccess) {
        // both sweep tiles (even k: an odd k adds a register copy per chunk)
        const int sks[] = {8, 16, 24, 32, 48, 64, 96, 128, 160, 192, 224, 254, 288, 320, 384, 448, 510};
        int last_r = 0;
        for (int st : {8, 16, 32}) {
            const int r = sweep_tile(w, st);
            if (r != st || r == last_r) continue;   // not compiled for this precision
            last_r = r;
            for (int k : sks) {
                if (!sweep_ok(w, k, r)) continue;
                a.K = k; a.variant = 1; a.tile = r;
                launch_gains_1d(w, k, 0, a, false);
                err = step1d(w->prec, a, w->coinp, 0, w->stream);
                if (err != cudaSuccess) break;
                cudaEventRecord(e0, w->stream);
                const int reps = 3;
                for (int rep = 0; rep < reps; ++rep) step1d(w->prec, a, w->coinp, 0, w->stream);
                cudaEventRecord(e1, w->stream);
                if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                const float per_step = ms / (reps * k);
                if (per_step < best) { best = per_step; best_k = k; best_v = 1; best_t = r; }
            }
            if (err != cudaSuccess) break;
        }
        a.variant = 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_error(w, err, "autotune");
    w->plan_tile = best_t;
    w->plan_k = best_k;
    w->plan_variant = best_v;
    g_tune[key] = {best_v ? -best_t : best_t, best_k};
    tune_save();
    std::snprintf(buf, sizeof buf,
                  "{\"tuned\": true, \"cached\": false, \"key\": \"%s\", \"tile\": %d, \"k\": %d, "
                  "\"variant\": \"%s\", \"ms_per_step\": %.6g}",
                  key.c_str(), best_t, best_k, best_v ? "sweep" : "tiles", best);
    put(buf);
    return QW_OK;
}

// ------------------------------------------------------------------ bounded wait self test
__global__ void k_bounded_wait(volatile int *flag, long long spins, int *status) {
    long long i = 0;
    while (i < spins && *flag == 0) {
        __nanosleep(100);
        ++i;
    }
    *status = (*flag == 0) ? 1 : 0;
}

extern "C" qw_status qw_debug_bounded_wait(int64_t spins, void *cuda_stream) {
    if (spins < 0) return QW_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int *mem = nullptr;
    cudaError_t e = dev_alloc((void **)&mem, 2 * sizeof(int));
    if (e != cudaSuccess) { (void)cudaGetLastError(); return e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA; }
    int host[2] = {0, 0};
    e = cudaMemsetAsync(mem, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) {
        k_bounded_wait<<<1, 1, 0, s>>>(mem, (long long)spins, mem + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, mem, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mem);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return QW_ECUDA; }
    return host[1] ? QW_ETIMEOUT : QW_OK;
}
