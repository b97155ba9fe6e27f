// qw_internal.cuh -- types shared by the kernels and the C ABI layer of libqw.
//
// Arithmetic of one walk step U = S (I (x) C) (Sawerwain & Gielerak, Sec. 2.1):
// every kernel applies the coin at the source site and moves the result along
// the shift.  Real types: float, double, and the double-float pair `ff` used by
// the compensated precision form.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "qw.h"

namespace qw {

// ------------------------------------------------------------------ precision
enum Prec { P_F64 = 0, P_F32 = 1, P_BF16 = 2, P_COMP = 3 };

// ------------------------------------------------------------------ double-float
// An unevaluated sum hi + lo of two floats, |lo| <= ulp(hi)/2.  The error-free
// transformations are Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based
// TwoProduct; addition and multiplication follow the double-word algorithms of
// Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44(2), 2017 (AccurateDWPlusDW and
// DWTimesDW with FMA).  Compiled without contraction changes: every operation
// below is written with explicit __fadd_rn / __fmul_rn / __fmaf_rn.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff operator+(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    ff t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    ff v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ ff operator-(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff operator*(ff x, ff y) {
    float ch = __fmul_rn(x.hi, y.hi);
    float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(cl1, cl2);
    return fast_two_sum(ch, cl3);
}
__device__ __forceinline__ ff ff_from(float a) { return {a, 0.f}; }

// ------------------------------------------------------------------ complex
template <class R>
struct Cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
// a * b for complex a, b
template <class R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// acc + a * b
template <class R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc) {
    return {acc.re + a.re * b.re - a.im * b.im, acc.im + a.re * b.im + a.im * b.re};
}
// real r times complex b, plus acc
template <class R>
__device__ __forceinline__ Cx<R> rfma(R r, Cx<R> b, Cx<R> acc) {
    return {acc.re + r * b.re, acc.im + r * b.im};
}
template <class R>
__device__ __forceinline__ Cx<R> rmul(R r, Cx<R> b) { return {r * b.re, r * b.im}; }
template <class R>
__device__ __forceinline__ Cx<R> conjmul(Cx<R> a, Cx<R> b) {  // conj(a) * b
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// float / double specialisations with explicit FMAs (contraction is allowed on
// the GPU path; the FMA form is the cheapest)
template <>
__device__ __forceinline__ Cx<float> cfma(Cx<float> a, Cx<float> b, Cx<float> acc) {
    float re = __fmaf_rn(a.re, b.re, acc.re);
    re = __fmaf_rn(-a.im, b.im, re);
    float im = __fmaf_rn(a.re, b.im, acc.im);
    im = __fmaf_rn(a.im, b.re, im);
    return {re, im};
}
template <>
__device__ __forceinline__ Cx<float> rfma(float r, Cx<float> b, Cx<float> acc) {
    return {__fmaf_rn(r, b.re, acc.re), __fmaf_rn(r, b.im, acc.im)};
}
template <>
__device__ __forceinline__ Cx<double> cfma(Cx<double> a, Cx<double> b, Cx<double> acc) {
    double re = __fma_rn(a.re, b.re, acc.re);
    re = __fma_rn(-a.im, b.im, re);
    double im = __fma_rn(a.re, b.im, acc.im);
    im = __fma_rn(a.im, b.re, im);
    return {re, im};
}
template <>
__device__ __forceinline__ Cx<double> rfma(double r, Cx<double> b, Cx<double> acc) {
    return {__fma_rn(r, b.re, acc.re), __fma_rn(r, b.im, acc.im)};
}

template <class R> __device__ __forceinline__ R rzero();
template <> __device__ __forceinline__ float rzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double rzero<double>() { return 0.0; }
template <> __device__ __forceinline__ ff rzero<ff>() { return {0.f, 0.f}; }
template <class R> __device__ __forceinline__ Cx<R> czero() { return {rzero<R>(), rzero<R>()}; }

// warp shuffles of compute values
__device__ __forceinline__ float shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ ff shfl_up(ff v, int d) { return {shfl_up(v.hi, d), shfl_up(v.lo, d)}; }
__device__ __forceinline__ ff shfl_down(ff v, int d) { return {shfl_down(v.hi, d), shfl_down(v.lo, d)}; }
__device__ __forceinline__ float shfl_idx(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double shfl_idx(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
template <class R> __device__ __forceinline__ Cx<R> shfl_idx(Cx<R> v, int l) { return {shfl_idx(v.re, l), shfl_idx(v.im, l)}; }
template <class R> __device__ __forceinline__ Cx<R> shfl_up(Cx<R> v, int d) { return {shfl_up(v.re, d), shfl_up(v.im, d)}; }
template <class R> __device__ __forceinline__ Cx<R> shfl_down(Cx<R> v, int d) { return {shfl_down(v.re, d), shfl_down(v.im, d)}; }

// |a|^2 accumulated in double
__device__ __forceinline__ double norm2d(Cx<float> a) { return (double)a.re * a.re + (double)a.im * a.im; }
__device__ __forceinline__ double norm2d(Cx<double> a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double norm2d(Cx<ff> a) {
    double re = (double)a.re.hi + (double)a.re.lo, im = (double)a.im.hi + (double)a.im.lo;
    return re * re + im * im;
}

// ------------------------------------------------------------------ storage
// State loads are plain (coherent) global loads, never the read-only path:
// the batched kernel reads back, in the same launch, what its block wrote.
// A state buffer is `nslots` plane slots of `pitch` sites each; slot c holds
// coin c (QW_F32_COMP: slot c the hi parts, slot d+c the lo parts).  pitch is a
// multiple of 64 sites and the buffer is 256-byte aligned, so every slot is
// 16-byte aligned and a 16-byte vector covers VEC whole sites.
struct View {
    void *p;
    int64_t pitch;   // sites per slot
    int d;           // coin dimension
};

template <int P> struct St;

template <> struct St<P_F32> {
    using real = float;
    static constexpr int VEC = 2;
    static constexpr int SLOT_BYTES = 8;  // bytes per site per slot
    static constexpr int SLOTS_PER_COIN = 1;
    __device__ static Cx<float> ld(View v, int c, int64_t i) {
        float2 a = reinterpret_cast<const float2 *>(v.p)[c * v.pitch + i];
        return {a.x, a.y};
    }
    __device__ static void st(View v, int c, int64_t i, Cx<float> a) {
        reinterpret_cast<float2 *>(v.p)[c * v.pitch + i] = make_float2(a.re, a.im);
    }
    __device__ static void ldv(View v, int c, int64_t i, Cx<float> *o) {
        float4 a = *reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(v.p) + c * v.pitch + i);
        o[0] = {a.x, a.y};
        o[1] = {a.z, a.w};
    }
    __device__ static void stv(View v, int c, int64_t i, const Cx<float> *a) {
        *reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(v.p) + c * v.pitch + i) =
            make_float4(a[0].re, a[0].im, a[1].re, a[1].im);
    }
    __device__ static void unpack(uint4 u, Cx<float> *o) {
        o[0] = {__uint_as_float(u.x), __uint_as_float(u.y)};
        o[1] = {__uint_as_float(u.z), __uint_as_float(u.w)};
    }
};

template <> struct St<P_F64> {
    using real = double;
    static constexpr int VEC = 1;
    static constexpr int SLOT_BYTES = 16;
    static constexpr int SLOTS_PER_COIN = 1;
    __device__ static Cx<double> ld(View v, int c, int64_t i) {
        double2 a = reinterpret_cast<const double2 *>(v.p)[c * v.pitch + i];
        return {a.x, a.y};
    }
    __device__ static void st(View v, int c, int64_t i, Cx<double> a) {
        reinterpret_cast<double2 *>(v.p)[c * v.pitch + i] = make_double2(a.re, a.im);
    }
    __device__ static void ldv(View v, int c, int64_t i, Cx<double> *o) { o[0] = ld(v, c, i); }
    __device__ static void stv(View v, int c, int64_t i, const Cx<double> *a) { st(v, c, i, a[0]); }
    __device__ static void unpack(uint4 u, Cx<double> *o) {
        o[0] = {__hiloint2double(u.y, u.x), __hiloint2double(u.w, u.z)};
    }
};

template <> struct St<P_BF16> {
    using real = float;
    static constexpr int VEC = 4;
    static constexpr int SLOT_BYTES = 4;
    static constexpr int SLOTS_PER_COIN = 1;
    __device__ static Cx<float> ld(View v, int c, int64_t i) {
        __nv_bfloat162 a = reinterpret_cast<const __nv_bfloat162 *>(v.p)[c * v.pitch + i];
        float2 f = __bfloat1622float2(a);
        return {f.x, f.y};
    }
    __device__ static void st(View v, int c, int64_t i, Cx<float> a) {
        reinterpret_cast<__nv_bfloat162 *>(v.p)[c * v.pitch + i] = __floats2bfloat162_rn(a.re, a.im);
    }
    __device__ static void ldv(View v, int c, int64_t i, Cx<float> *o) {
        uint4 u = *reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat162 *>(v.p) + c * v.pitch + i);
        const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(b[k]);
            o[k] = {f.x, f.y};
        }
    }
    __device__ static void stv(View v, int c, int64_t i, const Cx<float> *a) {
        uint4 u;
        __nv_bfloat162 *b = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = __floats2bfloat162_rn(a[k].re, a[k].im);
        *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat162 *>(v.p) + c * v.pitch + i) = u;
    }
    __device__ static void unpack(uint4 u, Cx<float> *o) {
        const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(b[k]);
            o[k] = {f.x, f.y};
        }
    }
};

template <> struct St<P_COMP> {
    using real = ff;
    static constexpr int VEC = 2;
    static constexpr int SLOT_BYTES = 8;
    static constexpr int SLOTS_PER_COIN = 2;
    __device__ static Cx<ff> ld(View v, int c, int64_t i) {
        const float2 *p = reinterpret_cast<const float2 *>(v.p);
        float2 h = p[c * v.pitch + i], l = p[(v.d + c) * v.pitch + i];
        return {{h.x, l.x}, {h.y, l.y}};
    }
    __device__ static void st(View v, int c, int64_t i, Cx<ff> a) {
        float2 *p = reinterpret_cast<float2 *>(v.p);
        p[c * v.pitch + i] = make_float2(a.re.hi, a.im.hi);
        p[(v.d + c) * v.pitch + i] = make_float2(a.re.lo, a.im.lo);
    }
    __device__ static void ldv(View v, int c, int64_t i, Cx<ff> *o) {
        const float2 *p = reinterpret_cast<const float2 *>(v.p);
        float4 h = *reinterpret_cast<const float4 *>(p + c * v.pitch + i);
        float4 l = *reinterpret_cast<const float4 *>(p + (v.d + c) * v.pitch + i);
        o[0] = {{h.x, l.x}, {h.y, l.y}};
        o[1] = {{h.z, l.z}, {h.w, l.w}};
    }
    __device__ static void stv(View v, int c, int64_t i, const Cx<ff> *a) {
        float2 *p = reinterpret_cast<float2 *>(v.p);
        *reinterpret_cast<float4 *>(p + c * v.pitch + i) = make_float4(a[0].re.hi, a[0].im.hi, a[1].re.hi, a[1].im.hi);
        *reinterpret_cast<float4 *>(p + (v.d + c) * v.pitch + i) = make_float4(a[0].re.lo, a[0].im.lo, a[1].re.lo, a[1].im.lo);
    }
};

// ------------------------------------------------------------------ coins
// Coin kinds the kernels specialise on.
enum CoinKind {
    CK_REAL = 0,      // one global matrix with zero imaginary parts
    CK_COMPLEX = 1,   // one global complex matrix
    CK_GROVER = 2,    // (2/d) J - I: phi_c = (2/d) sum psi - psi_c
    CK_HH = 3,        // H (x) H (2D only)
    CK_PERSITE = 4,   // one matrix per site, read from device memory
    CK_PHASE = 5,     // base . diag(e^{i phi_{v,k}}), phases read from device memory
    // 1D moving shift, coin lambda * M with M a +-1 matrix (Hadamard class):
    // M = diag(a, c) H diag(1, s), H = [[1, 1], [1, -1]].  diag(a, c) commutes
    // with the moving shift, so K steps are
    //   (S M)^K = lambda^K a^{K-1} diag(a, c) [S H_sigma]^K diag(1, sigma s),
    // H_sigma = H diag(1, sigma), sigma = a s c: only additions per step, the
    // signs and lambda^K are applied once per launch (pre / post gains).
    CK_SIGN_P = 6,    // sigma = +1: p0 = a0 + a1, p1 = a0 - a1
    CK_SIGN_M = 7     // sigma = -1: p0 = a0 - a1, p1 = a0 + a1
};

// The Hadamard-class kernels add without the factor lambda = 1/sqrt(2) per
// step, so amplitudes grow by sqrt(2) per step; float overflows after about
// 250 steps.  The sweep kernel, which runs up to 511 steps per launch,
// multiplies the state by 2^-SIGN_RESCALE_LOG2 (exact) after every
// SIGN_RESCALE_STEPS steps, and the host folds 2^(SIGN_RESCALE_LOG2 * m), m the
// number of rescales in the launch, into the launch's lambda^K.
constexpr int SIGN_RESCALE_STEPS = 64;
constexpr int SIGN_RESCALE_LOG2 = 32;

// One global d x d coin in compute precision, passed by value (kernel
// parameter space, read through the constant cache).
template <class R>
struct CoinP {
    R re[16];
    R im[16];
};

// double -> compute real, on the host (kernel arguments)
template <class R> inline R real_from_double(double x) { return (R)x; }
template <> inline ff real_from_double<ff>(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
template <class R> __device__ __forceinline__ bool is_one(R g) { return g == (R)1; }
template <> __device__ __forceinline__ bool is_one<ff>(ff g) { return g.hi == 1.f && g.lo == 0.f; }

// ------------------------------------------------------------------ errors
struct Err {
    qw_status st;
    const char *what;
};

// ------------------------------------------------------------------ launchers
// Each launcher enqueues work on `s` and returns the launch status.
struct Step1DArgs {
    View in, out;
    int64_t n;         // sites
    int K;             // steps in this launch
    int tile;          // sites per lane (R)
    int shift;         // 0 moving, 1 flip-flop
    int kind;          // CoinKind
    const void *coins; // CK_PERSITE: nsites x 4 complex in compute precision
    double pre0, pre1;   // per-plane factors applied after the load
    double post0, post1; // per-plane factors applied before the store
    int variant;         // 0 independent warp tiles (halo recomputed), 1 time-skewed sweep
    int chunks;          // sweep: chunks per warp segment (0 = default)
    // output range [obeg, oend) inside [0, n) when oend > obeg (the light-cone
    // window of a localised state: warp tiles only); else the whole cycle
    int64_t obeg, oend;
};
cudaError_t launch_step1d(int prec, const Step1DArgs &a, const void *coinp, cudaStream_t s);
cudaError_t launch_step1d_adjoint(int prec, const Step1DArgs &a, const void *coinp, cudaStream_t s);

struct Step2DArgs {
    View in, out;
    int64_t nx, ny;
    int shift;
    int kind;
    const void *coins;   // CK_PERSITE: nsites x 16 complex (compute precision)
    const float *phi;    // CK_PHASE: nsites x 4
    int K;               // temporal depth (1 = plain fused step)
    double gain;         // factor applied to every step's coin output
    // Support of the input state (the light-cone window of a localised
    // state): columns [bx0, bx0 + bw) and rows [by0, by0 + bh), both modulo
    // the torus; the state is zero outside.  bw = 0: the whole torus.
    int64_t bx0, bw, by0, bh;
};
cudaError_t launch_step2d(int prec, const Step2DArgs &a, const void *coinp, cudaStream_t s);
cudaError_t launch_step2d_adjoint(int prec, const Step2DArgs &a, const void *coinp, cudaStream_t s);

// generic (any boundary / links) single step, slow path
struct StepGenericArgs {
    View in, out;
    int ndim;
    int64_t nx, ny;
    int shift, bc;
    int kind;
    const void *coins;
    const float *phi;
    const uint8_t *links;
    int adjoint;
    double gain;         // factor applied to every step's output
    // links broken at random: closed when Philox word 0 < rthr (0: off), key
    // (rk0, rk1), step index rstep
    uint32_t rthr, rk0, rk1, rstep;
    // support box of the input state as in Step2DArgs (modulo the lattice on
    // the periodic one, inside it otherwise); bw = 0: the whole lattice
    int64_t bx0, bw, by0, bh;
};
cudaError_t launch_step_generic(int prec, const StepGenericArgs &a, const void *coinp, cudaStream_t s);

// marginals + norm
cudaError_t launch_marginals(int prec, View v, int64_t nsites, void *P, int p_f32,
                             double *partials, int nblocks, double *norm_dev, cudaStream_t s);
int marginal_blocks();

// conversions between caller layout (dense planes, complex128/complex64) and storage
cudaError_t launch_import(int prec, View dst, int64_t nsites, const void *src, int src_c64,
                          int64_t first_site, int64_t count, int plane, cudaStream_t s);
cudaError_t launch_export(int prec, View src, int64_t nsites, void *dst, int dst_c64,
                          int64_t first_site, int64_t count, int plane, cudaStream_t s);
cudaError_t launch_zero_state(View v, int nslots, int slot_bytes, cudaStream_t s);
// bounding box of the nonzero amplitudes: box[0..1] columns, box[2..3] rows
cudaError_t launch_support(int prec, View v, int64_t nx, int64_t ny, unsigned long long *box, cudaStream_t s);

}  // namespace qw
