// qw_handle.h -- the walk handle behind the opaque qw_walk of the C ABI, and the
// host helpers every ABI source file shares.
#pragma once
#include <string>

#include "qw_internal.cuh"

struct qw_walk {
    // lattice (Sec. 2.2): 1D cycle of nx sites or 2D torus nx * ny, coin dim d
    int ndim = 1, d = 2;
    int64_t nx = 1, ny = 1, ns = 1;
    int bc = QW_BC_PERIODIC, shift = QW_SHIFT_MOVING, prec = QW_F32;
    cudaStream_t stream = nullptr;
    int device = 0;

    // state: two buffers (current / next) of nslots padded planes
    int64_t pitch = 0;
    int nslots = 0, slot_bytes = 0;
    size_t state_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;

    // coin
    int kind = qw::CK_REAL;
    double coin_host[32] = {0};            // global / base coin, row-major complex
    double coin_alpha = 1.0;               // sqrt(tr(C_f^dagger C_f) / d) of the rounded coin
    // Hadamard-class coin lambda * diag(a, c) H diag(1, s) (1D moving shift)
    double sign_lambda = 1.0;
    int sign_a = 1, sign_c = 1, sign_s = 1, sign_sigma = 1;
    // error feedback of the rounded per-launch gains: product of applied / ideal
    double gain_fb = 1.0;
    // norm-drift factor of the rounded coin not yet applied to the state
    double drift_pending = 1.0;
    alignas(16) unsigned char coinp[512];  // CoinP<real> in compute precision
    void *coins_dev = nullptr;             // per-site matrices (compute precision)
    size_t coins_bytes = 0;
    float *phi_dev = nullptr;              // per-site phases, nsites * d
    uint8_t *links_dev = nullptr;          // closed-link flags, ndim * nsites
    bool has_links = false;
    // links broken at random at every step (qw_set_link_noise): Philox threshold
    // (0: off), key, and the index of the next forward step
    uint32_t link_thr = 0;
    uint64_t link_seed = 0;
    int64_t link_step = 0;

    // reductions
    double *partials = nullptr;
    double *norm_dev = nullptr;
    double *host_scalar = nullptr;  // pinned
    void *p_dev = nullptr;          // device probabilities for host readout
    size_t p_bytes = 0;

    // staging for host conversions
    void *staging = nullptr;
    size_t staging_bytes = 0;
    // pipelined host runs (qw_run_host_batch): a third state buffer, two
    // probability / norm slots and the copy streams
    void *buf3 = nullptr;
    void *pipe_p[2] = {nullptr, nullptr};
    size_t pipe_p_bytes = 0;
    double *pipe_norm = nullptr;   // one norm per run of qw_run_host_batch
    int64_t pipe_norm_cap = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;

    // Light-cone clipping (the growing computation window of a localised walk,
    // Sec. 3): the bounding box of the state's support, columns [bx0, bx0 + bw)
    // and rows [by0, by0 + bh) modulo the lattice.  sup_mode 0: the whole
    // lattice is stepped; 1: qw_set_state has queued the box search, whose
    // result arrives in sup_host (event sup_ev); 2: the box is known and the
    // steps run on it, widening it by one site per step and side.  next_clear:
    // the other state buffer is zero outside the box.
    bool clip_on = true;
    int sup_mode = 0;
    int64_t bx0 = 0, bw = 0, by0 = 0, bh = 0;
    bool next_clear = false;
    unsigned long long *sup_dev = nullptr;    // 4 values (device)
    unsigned long long *sup_host = nullptr;   // 4 values (pinned)
    cudaEvent_t sup_ev = nullptr;

    // execution plan
    int plan_k = 0, plan_tile = 0;
    int plan_variant = -1;   // 1D kernel: -1 automatic, 0 independent warp tiles, 1 time-skewed sweep
    bool plan_user = false;

    // adjoint / gradient scratch
    void *grad_scratch = nullptr;
    size_t grad_scratch_bytes = 0;

    std::string err;
};

// NVTX ranges around the public calls that launch work, for timelines in a
// profiler; header-only, and nothing happens when no tool is attached
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#else
struct NvtxRange {
    explicit NvtxRange(const char *) {}
};
#endif

namespace qw {

qw_status set_error(qw_walk *w, qw_status st, const std::string &msg);
qw_status cuda_error(qw_walk *w, cudaError_t e, const char *where);
bool fault_injected(const char *what);
cudaError_t dev_alloc(void **p, size_t bytes);

inline View view_of(const qw_walk *w, int which) {
    return View{w->buf[which], w->pitch, w->d};
}
inline View cur_view(const qw_walk *w) { return view_of(w, w->cur); }
// any closed links, fixed or broken at random: the generic kernel then runs
inline bool links_on(const qw_walk *w) { return w->has_links || w->link_thr != 0; }
inline View next_view(const qw_walk *w) { return view_of(w, w->cur ^ 1); }

// Runs T steps of U (adj = 0) or U^dagger (adj = 1) from buffer `src` into
// the other buffer and flips w->cur; used by qw_step and the adjoint.
qw_status run_steps(qw_walk *w, int64_t T, int adj);

// Launch helpers implemented in the per-precision translation units.
cudaError_t launch_step1d_f32(const Step1DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step1d_f64(const Step1DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step1d_bf16(const Step1DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step1d_comp(const Step1DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step2d_f32(const Step2DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step2d_f64(const Step2DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step2d_bf16(const Step2DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_step2d_comp(const Step2DArgs &, const void *, int, cudaStream_t);
cudaError_t launch_generic_f32(const StepGenericArgs &, const void *, cudaStream_t);
cudaError_t launch_generic_f64(const StepGenericArgs &, const void *, cudaStream_t);
cudaError_t launch_generic_bf16(const StepGenericArgs &, const void *, cudaStream_t);
cudaError_t launch_generic_comp(const StepGenericArgs &, const void *, cudaStream_t);
// steps per launch of the 1D window kernel (k_window1d.cuh, WIN_MAX_STEPS there)
constexpr int WINDOW_MAX_STEPS = 256;
cudaError_t launch_window1d_f32(const StepGenericArgs &, const void *, const double *, int, cudaStream_t);
cudaError_t launch_window1d_f64(const StepGenericArgs &, const void *, const double *, int, cudaStream_t);
cudaError_t launch_window1d_bf16(const StepGenericArgs &, const void *, const double *, int, cudaStream_t);
cudaError_t launch_window1d_comp(const StepGenericArgs &, const void *, const double *, int, cudaStream_t);
int64_t window1d_capacity_f32();
int64_t window1d_capacity_f64();
int64_t window1d_capacity_bf16();
int64_t window1d_capacity_comp();
bool sweep_ok_f32(int64_t, int, int, int);
bool sweep_ok_f64(int64_t, int, int, int);
bool sweep_ok_bf16(int64_t, int, int, int);
int sweep_tile_f32(int64_t, int);
int sweep_tile_f64(int64_t, int);
int sweep_tile_bf16(int64_t, int);
int tile1d_f32(int, int, int);
int tile1d_f64(int, int, int);
int tile1d_bf16(int, int, int);
int tile1d_comp(int, int, int);

// streaming temporal blocking on the torus (step2d_tb.cu)
bool step2d_tb_ok(int prec, int kind, int K, int shift);
cudaError_t launch_step2d_tb(const Step2DArgs &a, const void *coinp, cudaStream_t s);

// per-site coin conversion kernels (qw_coins.cu)
cudaError_t launch_convert_coins(int prec, const double *src, void *dst, int64_t count, cudaStream_t s);
cudaError_t launch_phase_coins(int prec, const double *base, const float *phi, void *dst, int64_t ns,
                               int d, cudaStream_t s);

}  // namespace qw
