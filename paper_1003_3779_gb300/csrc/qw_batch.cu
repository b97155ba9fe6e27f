// qw_batch.cu -- many independent walks on cycles in one persistent launch.
//
// Each walk is the 1D walk of Sec. 2.2 (cycle Z_N, coin dim 2, U = S (I (x) C)
// of Sec. 2.1) with its own N, T and 2x2 coin, started localised at x0.  The
// walks are sorted by light-cone work, largest first, and popped from global
// counters by persistent CTAs or warps, which zero the walk's two state
// buffers, place the initial amplitude and advance the walk k steps per round.
// The walk's state ping-pongs between two global buffers; a walk of at most
// 65536 sites is 1 MiB per buffer in FP32 (0.5 MiB in bfloat16), so it mostly
// stays in L2 while it is worked on.  Two kernels:
//
// - k_batch (variant 0): one CTA per walk; its four warps share the register
//   tiles (tb_tile, with a halo of k sites per side) of a round and meet at a
//   __syncthreads between rounds.
// - k_batch_sweep (variant 1): the time-skewed sweep of the single cycle over
//   the chunks that cover the walk's light cone, with no halo.  The largest
//   walks run on a CTA's four warps as segments; the rest on single warps.
//
// Light cone (Sec. 3, the "line" computation window): after t steps from a
// single site x0 the state is zero outside [x0 - t, x0 + t].  Variant 0 skips
// the tiles whose outputs all lie outside the cone of the current round (their
// buffer region is still the zero written at the start); variant 1 sweeps only
// the window from the cone's left end.  (Shorter rounds while the cone is
// narrow clip it more tightly but cost more per-round traffic and
// synchronisation than they save on this workload: measured 28 ms against
// 17 ms for 4096 walks in variant 0, so a single k is used; Ks stays
// available.)
//
// At the end of its walk the group writes P(x) = |psi0|^2 + |psi1|^2 (float)
// and the walk's norm (double, fixed order) to the batch outputs.  There are
// no waits other than __syncthreads / __syncwarp: nothing spins.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "qw_handle.h"
#include "k_step1d.cuh"

namespace qw {

struct WalkDesc {
    int64_t n, T, x0;
    int64_t base;    // first site slot of the walk in each state buffer (plane 0; plane 1 at +pitch)
    int64_t pitch;   // sites per plane, a multiple of 64
    int64_t poff;    // first index of the walk in the concatenated probabilities
    float c[8];      // coin, row-major complex (re, im)
    float clo[8];    // QW_F32_COMP: the low parts, coin = c + clo to ~48 bits (else 0)
    // norm-drift compensation of the float-rounded coin (alpha = sqrt(|C_f|_F^2 / 2)):
    // the last round applies alpha^-T (g_last), the others g_main = 1; computed on
    // the host, so the kernel does no double arithmetic per round
    float g_main, g_last;
    double alpha;
};

struct BatchArgs {
    const WalkDesc *walks;
    const int *order;
    int nwalks;
    void *buf0, *buf1;
    float *P;
    double *norms;
    int *counter;    // [0]: next walk (variant 0; variant 1: next big walk), [1]: next small walk
    int *final_buf;
    int nbig;        // variant 1: walks order[0, nbig) run on a whole CTA, the rest on single warps
    int K;           // steps per round once the light cone covers the cycle
    int Ks;          // steps per round while it does not (finer cone clipping)
    float cs[4];     // coin state at x0: (re, im) of coin 0 and coin 1
    float cs_lo[4];  // QW_F32_COMP: their low parts
};

constexpr int BATCH_THREADS = 128;
constexpr int BATCH_R = 16;
// Sites per lane of the warp tiles: the double-float form holds four floats per
// amplitude, so its tiles are half as long to stay in registers.
constexpr int BATCH_R_COMP = 8;
template <int P> constexpr int batch_r() { return P == P_COMP ? BATCH_R_COMP : BATCH_R; }

// A compute real from the hi / lo floats the host split a double into.
template <class R> __device__ __forceinline__ R real_hl(float hi, float lo);
template <> __device__ __forceinline__ float real_hl<float>(float hi, float) { return hi; }
template <> __device__ __forceinline__ ff real_hl<ff>(float hi, float lo) { return {hi, lo}; }

// P(x) as the batch reports it (float) and its double contribution to the norm.
// Float forms: the sum of squares in float, as the single walks' marginals;
// the double-float form: in double from hi + lo, rounded once.
template <int P>
__device__ __forceinline__ float site_prob(View v, int64_t x, double &pd) {
    using S = St<P>;
    if constexpr (P == P_COMP) {
        pd = norm2d(S::ld(v, 0, x)) + norm2d(S::ld(v, 1, x));
        return (float)pd;
    } else {
        const Cx<float> u = S::ld(v, 0, x), w = S::ld(v, 1, x);
        const float p = __fmaf_rn(u.re, u.re, __fmaf_rn(u.im, u.im, __fmaf_rn(w.re, w.re, w.im * w.im)));
        pd = (double)p;
        return p;
    }
}

// Does the tile output range [a, b) meet the circular interval [x0 - r, x0 + r] (mod n)?
__device__ __forceinline__ bool meets_cone(int64_t a, int64_t b, int64_t x0, int64_t r, int64_t n) {
    int64_t lo = x0 - r, hi = x0 + r + 1;   // half-open, 2r + 1 < n
    if (lo < 0) return (a < hi) || (b > lo + n);
    if (hi > n) return (b > lo) || (a < hi - n);
    return a < hi && b > lo;
}

// ---------------------------------------------------------------- window sweep
// The time-skewed sweep of k_step1d_sweep, over a window of one walk's cycle:
// frame chunks j of B = 32R sites start at site L + jB (mod n); after K levels
// chunk j holds sites L + jB - K + [0, B), which it writes out.  The walk only
// depends on its left in the frame, so a chunk needs from the chunk before it
// the two values per level that lane 31 hands over through the edge buffer.
// Chunks [j0, j1) of one segment are swept in order by one warp.  The first
// chunk's left edge is either zero (warm = false: the state is zero left of
// the window, outside the light cone) or comes from a warm-up chunk j0 - 1
// recomputed from a zero edge (its error front moves two sites per level, so
// K < B/2 - 1 leaves its right edge exact).  Chunks that are not a contiguous,
// 16-byte aligned run of the cycle (across site n-1 -> 0, or after it when n is
// odd) are fetched site by site.
__device__ __forceinline__ void cp_async_bytes8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_bytes4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int P, int CK>
__device__ __forceinline__ void window_segment(View in, View out, int64_t n, int K, int64_t L, int j0, int j1,
                                            bool warm, CoinP<float> cp, float post, unsigned char *wbase,
                                            int lane) {
    using S = St<P>;
    using C = Cx<float>;
    constexpr int R = BATCH_R;
    using SW = Sweep<P, R>;
    constexpr int B = SW::B, CPL = SW::CPL, VEC = S::VEC, UPV = 16 / S::SLOT_BYTES;
    uint4 *cbuf = reinterpret_cast<uint4 *>(wbase);
    C *edge = reinterpret_cast<C *>(wbase + SW::chunk_bytes);
    const int jfirst = warm ? j0 - 1 : j0;
    {   // the first chunk reads its left edge from parity (jfirst & 1) ^ 1
        C *e0 = edge + (size_t)((jfirst & 1) ^ 1) * K * 2;
        for (int i = lane; i < 2 * K; i += 32) e0[i] = C{0.f, 0.f};
    }
    __syncwarp();
    auto site = [&](int64_t x) { const int64_t r = x % n; return r < 0 ? r + n : r; };
    auto prefetch = [&](int j) {
        const int64_t start = site(L + (int64_t)j * B);
        if (start + B <= n && start % VEC == 0) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const char *g = static_cast<const char *>(in.p) + (c * in.pitch + start) * S::SLOT_BYTES;
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int u = i * 32 + lane;
                    cp_async16(cbuf + c * 32 * CPL + swz<CPL>(u / CPL, u % CPL), g + (size_t)u * 16);
                }
            }
        } else {
            // this lane's own R sites, one slot at a time, wrapping around the cycle
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int64_t g = site(start + (int64_t)lane * R + i);
                    unsigned char *dst = reinterpret_cast<unsigned char *>(cbuf + c * 32 * CPL + swz<CPL>(lane, i / UPV)) +
                                         (i % UPV) * S::SLOT_BYTES;
                    const char *src = static_cast<const char *>(in.p) + (c * in.pitch + g) * S::SLOT_BYTES;
                    if constexpr (S::SLOT_BYTES == 8) cp_async_bytes8(dst, src);
                    else cp_async_bytes4(dst, src);
                }
            }
        }
        cp_async_commit();
    };

    C a0[R], a1[R];
    prefetch(jfirst);
    const int from = (lane + 31) & 31;
    for (int j = jfirst; j < j1; ++j) {
        cp_async_wait_all();
        __syncwarp();
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            S::unpack(cbuf[swz<CPL>(lane, u)], &a0[u * VEC]);
            S::unpack(cbuf[32 * CPL + swz<CPL>(lane, u)], &a1[u * VEC]);
        }
        __syncwarp();
        if (j + 1 < j1) prefetch(j + 1);
        const int par = j & 1;
        const unsigned si = (unsigned)__cvta_generic_to_shared(edge + (size_t)(par ^ 1) * K * 2);
        const unsigned so = (unsigned)__cvta_generic_to_shared(edge + (size_t)par * K * 2);
        // one level of the moving walk in the sliding frame (see k_step1d_sweep)
        auto level = [&](int t, const C (&s0)[R], const C (&s1)[R], C (&d0)[R], C (&d1)[R]) {
            C top2, top1;
#pragma unroll
            for (int i = R - 1; i >= 0; --i) {
                C n0, n1;
                coin2<CK>(cp, (const C *)nullptr, s0[i], s1[i], n0, n1);
                d0[i] = n0;
                if (i + 2 < R) d1[i + 2] = n1;
                else if (i == R - 1) top1 = n1;
                else top2 = n1;
                if (i == R - 2) edge_swap31(lane, so + t * 2 * (unsigned)sizeof(C), si + t * 2 * (unsigned)sizeof(C), top2, top1);
            }
            d1[0] = shfl_idx(top2, from);
            d1[1] = shfl_idx(top1, from);
        };
        C b0[R], b1[R];
        int t = 0;
#pragma unroll 1
        for (; t + 1 < K; t += 2) {
            level(t, a0, a1, b0, b1);
            level(t + 1, b0, b1, a0, a1);
        }
        if (t < K) {
            level(t, a0, a1, b0, b1);
#pragma unroll
            for (int i = 0; i < R; ++i) { a0[i] = b0[i]; a1[i] = b1[i]; }
        }
        if (j >= j0) {
            if (post != 1.f) {
#pragma unroll
                for (int i = 0; i < R; ++i) { a0[i] = rmul(post, a0[i]); a1[i] = rmul(post, a1[i]); }
            }
            const int64_t g0 = site(L + (int64_t)j * B - K + (int64_t)lane * R);
            if (g0 + R <= n && g0 % VEC == 0) {
#pragma unroll
                for (int i = 0; i < R; i += VEC) { S::stv(out, 0, g0 + i, &a0[i]); S::stv(out, 1, g0 + i, &a1[i]); }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int64_t g = site(g0 + i);
                    S::st(out, 0, g, a0[i]);
                    S::st(out, 1, g, a1[i]);
                }
            }
        }
    }
}

// Variant 0: one CTA per walk, warp register tiles with a halo of k sites
// (tb_tile), tiles outside the light cone skipped.
template <int P, int CK>
__global__ void __launch_bounds__(BATCH_THREADS)
k_batch(BatchArgs a) {
    using S = St<P>;
    using real = typename S::real;
    constexpr int R = batch_r<P>();
    constexpr int VEC = S::VEC;
    __shared__ int s_q;
    __shared__ double s_red[BATCH_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_q = atomicAdd(a.counter, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= a.nwalks) return;
        const int w = a.order[q];
        const WalkDesc d = a.walks[w];
        View in{static_cast<char *>(a.buf0) + d.base * S::SLOT_BYTES, d.pitch, 2};
        View out{static_cast<char *>(a.buf1) + d.base * S::SLOT_BYTES, d.pitch, 2};

        // zero both buffers of this walk (all plane slots), then place the start
        {
            const int64_t nvec = 2 * S::SLOTS_PER_COIN * d.pitch * S::SLOT_BYTES / 16;
            uint4 z = make_uint4(0, 0, 0, 0);
            for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) {
                reinterpret_cast<uint4 *>(in.p)[i] = z;
                reinterpret_cast<uint4 *>(out.p)[i] = z;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S::st(in, 0, d.x0, Cx<real>{real_hl<real>(a.cs[0], a.cs_lo[0]), real_hl<real>(a.cs[1], a.cs_lo[1])});
            S::st(in, 1, d.x0, Cx<real>{real_hl<real>(a.cs[2], a.cs_lo[2]), real_hl<real>(a.cs[3], a.cs_lo[3])});
        }
        __syncthreads();

        CoinP<real> cp;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            cp.re[e] = real_hl<real>(d.c[2 * e], d.clo[2 * e]);
            cp.im[e] = real_hl<real>(d.c[2 * e + 1], d.clo[2 * e + 1]);
        }
        const real one = real_hl<real>(1.f, 0.f);
        int cur = 0;
        for (int64_t t0 = 0; t0 < d.T;) {
            // while the cone is narrower than the cycle, short rounds clip it more tightly
            const int kr = (2 * t0 + 1 < d.n) ? min(a.Ks, a.K) : a.K;
            const int k = (int)min((int64_t)kr, d.T - t0);
            const int64_t W = (32LL * R - 2LL * k - (VEC - 1)) / VEC * VEC;
            const int64_t ntiles = (d.n + W - 1) / W;
            const int64_t r = t0 + k;
            const bool all = 2 * r + 1 >= d.n;
            const real g = real_hl<real>((t0 + k >= d.T) ? d.g_last : d.g_main, 0.f);
            for (int64_t tile = wid; tile < ntiles; tile += nw) {
                const int64_t o0 = tile * W, o1 = min(o0 + W, d.n);
                if (!all && !meets_cone(o0, o1, d.x0, r, d.n)) continue;
                tb_tile<P, R, CK, 0, 0>(in, out, d.n, k, o0, (int)(o1 - o0), lane, cp, nullptr, one, one, g, g);
            }
            __syncthreads();
            View t = in; in = out; out = t;
            cur ^= 1;
            t0 += k;
        }

        // marginals and norm of the final state: P(x) is float output, the
        // running norm in double
        double acc = 0.0;
        for (int64_t x = threadIdx.x; x < d.n; x += blockDim.x) {
            double pd;
            a.P[d.poff + x] = site_prob<P>(in, x, pd);
            acc += pd;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) s_red[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < nw; ++i) tot += s_red[i];
            a.norms[w] = tot;
            a.final_buf[w] = cur;
        }
    }
}


// Variant 1: the window sweep.  A walk is advanced in passes of k steps; a
// pass sweeps the chunks that cover the light cone (frame from the cone's left
// end, whose left is zero), or the whole cycle with a warm-up chunk once the
// cone, widened by the margins, reaches round it.  The largest walks
// (order[0, nbig)) are each shared by the four warps of a CTA, which split the
// chunks of a pass into segments (each after the first with a warm-up chunk)
// and meet at a barrier between passes; every other walk is swept by a single
// warp alone, with no warm-up chunks and no barrier.  Results are the same
// bits either way.
template <int P, int CK>
__device__ __forceinline__ void run_walk_sweep(const BatchArgs &a, int w, bool cta, int g, int gs, int wid, int nw,
                                               double *s_red, unsigned char *wbase) {
    using S = St<P>;
    constexpr int R = BATCH_R, B = 32 * R, VEC = S::VEC;
    const int lane = threadIdx.x & 31;
    auto sync = [cta] { if (cta) __syncthreads(); else __syncwarp(); };
    const WalkDesc d = a.walks[w];
    View in{static_cast<char *>(a.buf0) + d.base * S::SLOT_BYTES, d.pitch, 2};
    View out{static_cast<char *>(a.buf1) + d.base * S::SLOT_BYTES, d.pitch, 2};
    {
        const int64_t nvec = 2 * d.pitch * S::SLOT_BYTES / 16;
        uint4 z = make_uint4(0, 0, 0, 0);
        for (int64_t i = g; i < nvec; i += gs) {
            reinterpret_cast<uint4 *>(in.p)[i] = z;
            reinterpret_cast<uint4 *>(out.p)[i] = z;
        }
    }
    sync();
    if (g == 0) {
        S::st(in, 0, d.x0, Cx<float>{a.cs[0], a.cs[1]});
        S::st(in, 1, d.x0, Cx<float>{a.cs[2], a.cs[3]});
    }
    sync();
    CoinP<float> cp;
#pragma unroll
    for (int e = 0; e < 4; ++e) { cp.re[e] = d.c[2 * e]; cp.im[e] = d.c[2 * e + 1]; }
    int cur = 0;
    for (int64_t t0 = 0; t0 < d.T;) {
        const int k = (int)min((int64_t)a.K, d.T - t0);
        // window: from the cone's left end at t0 (rounded down to the vector
        // width) far enough that the outputs, shifted left by k, cover the
        // cone's right end at t0 + k
        int64_t L = d.x0 - t0;
        L -= ((L % VEC) + VEC) % VEC;
        const int64_t span = d.x0 + t0 + 2 * k + 1 - L;
        const bool win = span + 2 * k + B <= d.n;   // the zero run left of L is outside the cone, not its far side
        int nch;
        if (win) {
            nch = (int)((span + B - 1) / B);
        } else {
            L = 0;
            nch = (int)((d.n + B - 1) / B);
        }
        // on a CTA, one segment per warp (down to one chunk each): the CTA walks
        // are the critical path, so the extra warm-up chunks buy a shorter pass
        const int nseg = max(1, min(nw, nch));
        const float gl = (t0 + k >= d.T) ? d.g_last : d.g_main;
        if (wid < nseg) {
            const int j0 = (int)((int64_t)nch * wid / nseg), j1 = (int)((int64_t)nch * (wid + 1) / nseg);
            window_segment<P, CK>(in, out, d.n, k, L, j0, j1, !win || wid > 0, cp, gl, wbase, lane);
        }
        sync();
        View tv = in; in = out; out = tv;
        cur ^= 1;
        t0 += k;
    }
    double acc = 0.0;
    for (int64_t x = g; x < d.n; x += gs) {
        double pd;
        a.P[d.poff + x] = site_prob<P>(in, x, pd);
        acc += pd;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (cta) {
        if (lane == 0) s_red[wid] = acc;
        __syncthreads();
        if (g == 0) {
            double tot = 0.0;
            for (int i = 0; i < nw; ++i) tot += s_red[i];
            a.norms[w] = tot;
            a.final_buf[w] = cur;
        }
        __syncthreads();
    } else if (lane == 0) {
        a.norms[w] = acc;
        a.final_buf[w] = cur;
    }
}

template <int P, int CK>
__global__ void __launch_bounds__(BATCH_THREADS)
k_batch_sweep(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_q;
    __shared__ double s_red[BATCH_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned char *wbase = bsm + (size_t)wid * Sweep<P, BATCH_R>::warp_bytes(a.K);
    bool cta = true;   // uniform over the CTA until it leaves the big walks
    for (;;) {
        int q;
        if (cta) {
            __syncthreads();
            if (threadIdx.x == 0) s_q = atomicAdd(&a.counter[0], 1);
            __syncthreads();
            q = s_q;
            if (q >= a.nbig) { cta = false; continue; }
        } else {
            q = 0;
            if (lane == 0) q = atomicAdd(&a.counter[1], 1);
            q = a.nbig + __shfl_sync(0xffffffffu, q, 0);
            if (q >= a.nwalks) return;
        }
        // one call site: one inlined copy of the walk code for both modes
        run_walk_sweep<P, CK>(a, a.order[q], cta, cta ? (int)threadIdx.x : lane, cta ? (int)blockDim.x : 32,
                              cta ? wid : 0, cta ? nw : 1, s_red, wbase);
    }
}

}  // namespace qw

using namespace qw;

struct qw_batch {
    int nwalks = 0;
    int prec = QW_F32;
    int kind = CK_REAL;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t cap = nullptr;         // private stream the graph is captured on
    std::vector<WalkDesc> walks;
    std::vector<int> order;
    int64_t total_sites = 0, total_slots = 0;
    size_t buf_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    WalkDesc *walks_dev = nullptr;
    int *order_dev = nullptr;
    float *P_dev = nullptr;
    double *norms_dev = nullptr;
    int *counter = nullptr;             // two queue counters (see BatchArgs)
    int *final_dev = nullptr;
    std::vector<double> work;           // light-cone site-steps of each walk
    int nbig = 0;                       // variant 1: the nbig walks with the most work run on a CTA
    int K = 96;
    int variant = 1;                    // 0: warp tiles with halos, 1: light-cone window sweep
    int grid = 0, grid1 = 0;            // persistent grid of each variant (one wave)
    float cs[4] = {0, 0, 0, 0};
    float cs_lo[4] = {0, 0, 0, 0};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ran = false;
    std::string err;
};

static qw_status batch_fail(qw_batch *b, qw_status st, const std::string &m) {
    if (b) b->err = m;
    return st;
}

static qw_status batch_cuda(qw_batch *b, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    (void)cudaGetLastError();
    return batch_fail(b, e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA, m);
}

static int batch_slot_bytes(int prec) { return prec == QW_F32_BF16STORE ? 4 : 8; }
static int batch_slots(int prec) { return prec == QW_F32_COMP ? 4 : 2; }    // plane slots per walk
static int batch_tile(int prec) { return prec == QW_F32_COMP ? BATCH_R_COMP : BATCH_R; }
static int batch_kmax(int prec) { return 8 * batch_tile(prec); }
static int batch_prec_code(int prec) {
    return prec == QW_F32_BF16STORE ? P_BF16 : (prec == QW_F32_COMP ? P_COMP : P_F32);
}

// The window sweep's shared memory: a chunk buffer and the k-level edge
// buffer per warp.
static size_t batch_smem(int prec, int variant, int K) {
    if (variant != 1) return 0;
    const size_t w = prec == QW_F32_BF16STORE ? Sweep<P_BF16, BATCH_R>::warp_bytes(K) : Sweep<P_F32, BATCH_R>::warp_bytes(K);
    return w * (BATCH_THREADS / 32);
}

template <int P, int CK>
static cudaError_t launch_batch_kernel(qw_batch *b, const BatchArgs &a, cudaStream_t s) {
    if (b->variant == 1) {
        const size_t smem = batch_smem(b->prec, 1, b->K);
        cudaError_t e = cudaFuncSetAttribute(k_batch_sweep<P, CK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_batch_sweep<P, CK><<<b->grid1, BATCH_THREADS, smem, s>>>(a);
    } else {
        k_batch<P, CK><<<b->grid, BATCH_THREADS, 0, s>>>(a);
    }
    return cudaSuccess;
}

static cudaError_t batch_launch(qw_batch *b, cudaStream_t s) {
    BatchArgs a{};
    a.walks = b->walks_dev; a.order = b->order_dev; a.nwalks = b->nwalks;
    a.buf0 = b->buf[0]; a.buf1 = b->buf[1]; a.P = b->P_dev; a.norms = b->norms_dev;
    a.counter = b->counter; a.final_buf = b->final_dev; a.K = b->K; a.Ks = b->K;
    std::memcpy(a.cs, b->cs, sizeof a.cs);
    std::memcpy(a.cs_lo, b->cs_lo, sizeof a.cs_lo);
    a.nbig = b->nbig;
    cudaError_t e = cudaMemsetAsync(b->counter, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (b->prec == QW_F32_COMP) {   // warp tiles only (no double-float sweep)
        if (b->kind == CK_REAL) k_batch<P_COMP, CK_REAL><<<b->grid, BATCH_THREADS, 0, s>>>(a);
        else k_batch<P_COMP, CK_COMPLEX><<<b->grid, BATCH_THREADS, 0, s>>>(a);
    } else if (b->prec == QW_F32_BF16STORE) {
        if (b->kind == CK_REAL) e = launch_batch_kernel<P_BF16, CK_REAL>(b, a, s);
        else e = launch_batch_kernel<P_BF16, CK_COMPLEX>(b, a, s);
    } else {
        if (b->kind == CK_REAL) e = launch_batch_kernel<P_F32, CK_REAL>(b, a, s);
        else e = launch_batch_kernel<P_F32, CK_COMPLEX>(b, a, s);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Per-walk drift factors (see WalkDesc): the whole correction alpha^-T is
// applied once, in the walk's last round.  Factors within a few ulps of 1,
// applied every round, would be biased by round-to-nearest.
static void set_gains(qw_batch *b, int K) {
    (void)K;
    for (auto &d : b->walks) {
        d.g_main = 1.f;
        d.g_last = (d.T <= 0 || d.alpha == 1.0) ? 1.f : (float)std::pow(d.alpha, -(double)d.T);
    }
}

static void drop_graph(qw_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

extern "C" {

qw_status qw_batch_destroy(qw_batch *b) {
    if (!b) return QW_OK;
    cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamSynchronize(b->cap);
    drop_graph(b);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->walks_dev);
    cudaFree(b->order_dev);
    cudaFree(b->P_dev);
    cudaFree(b->norms_dev);
    cudaFree(b->counter);
    cudaFree(b->final_dev);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return QW_OK;
}

const char *qw_batch_last_error(const qw_batch *b) { return b ? b->err.c_str() : "null handle"; }

qw_status qw_batch_create(int nwalks, const int64_t *N, const int64_t *T, const double *coins,
                          const int64_t *x0, const double *coin_state, qw_precision prec,
                          void *cuda_stream, qw_batch **out) {
    if (!out) return QW_EINVAL;
    *out = nullptr;
    if (nwalks < 1 || !N || !T || !coins || !x0 || !coin_state) return QW_EINVAL;
    if (prec != QW_F32 && prec != QW_F32_BF16STORE && prec != QW_F32_COMP) return QW_EUNSUPPORTED;
    for (int i = 0; i < nwalks; ++i)
        if (N[i] < 1 || N[i] > (int64_t(1) << 31) || T[i] < 0 || x0[i] < 0 || x0[i] >= N[i]) return QW_EINVAL;

    qw_batch *b = new (std::nothrow) qw_batch();
    if (!b) return QW_ENOMEM;
    b->nwalks = nwalks;
    b->prec = prec;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < 4; ++i) {
        b->cs[i] = (float)coin_state[i];
        if (prec == QW_F32_COMP) b->cs_lo[i] = (float)(coin_state[i] - (double)b->cs[i]);
    }
    b->walks.resize(nwalks);
    bool real = true;
    int64_t base = 0, poff = 0;
    for (int i = 0; i < nwalks; ++i) {
        WalkDesc &d = b->walks[i];
        d.n = N[i]; d.T = T[i]; d.x0 = x0[i];
        d.pitch = (N[i] + 63) / 64 * 64;
        d.base = base;
        d.poff = poff;
        base += batch_slots(prec) * d.pitch;
        poff += N[i];
        double fro = 0.0;
        for (int e = 0; e < 8; ++e) {
            d.c[e] = (float)coins[8 * i + e];
            d.clo[e] = prec == QW_F32_COMP ? (float)(coins[8 * i + e] - (double)d.c[e]) : 0.f;
            fro += (double)d.c[e] * d.c[e];
            if (e % 2 == 1 && coins[8 * i + e] != 0.0) real = false;
        }
        const double alpha = std::sqrt(fro / 2.0);
        // hi + lo carries the coin to ~48 bits: no norm drift to compensate
        d.alpha = (prec != QW_F32_COMP && std::fabs(alpha - 1.0) <= 1e-5) ? alpha : 1.0;
    }
    b->kind = real ? CK_REAL : CK_COMPLEX;
    b->total_slots = base;
    b->total_sites = poff;
    b->order.resize(nwalks);
    std::iota(b->order.begin(), b->order.end(), 0);
    // longest first by light-cone work, sum_{t<T} min(N, 2t+1) site-steps (the
    // tiles a walk actually computes), not by N*T
    b->work.resize(nwalks);
    for (int i = 0; i < nwalks; ++i) {
        const double n = (double)N[i], t = (double)T[i];
        const double tc = std::min(t, std::ceil((n - 1) / 2));   // steps before the cone covers the cycle
        b->work[i] = tc * tc + (t - tc) * n;
    }
    std::stable_sort(b->order.begin(), b->order.end(), [&](int p, int q) { return b->work[p] > b->work[q]; });
    b->buf_bytes = (size_t)base * batch_slot_bytes(prec);

    cudaError_t e = cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, prec == QW_F32_BF16STORE ? (const void *)k_batch<P_BF16, CK_REAL>
                     : prec == QW_F32_COMP    ? (const void *)k_batch<P_COMP, CK_REAL>
                                              : (const void *)k_batch<P_F32, CK_REAL>,
            BATCH_THREADS, 0);
    int per_sm1 = 0;
    if (e == cudaSuccess && prec != QW_F32_COMP) {
        // the window sweep at the largest k it is planned with (the occupancy of smaller k is no lower)
        const size_t smem = batch_smem(prec, 1, 8 * BATCH_R);
        const void *f1 = prec == QW_F32_BF16STORE ? (const void *)k_batch_sweep<P_BF16, CK_REAL> : (const void *)k_batch_sweep<P_F32, CK_REAL>;
        e = cudaFuncSetAttribute(f1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, f1, BATCH_THREADS, smem);
    }
    if (e == cudaSuccess) e = dev_alloc(&b->buf[0], b->buf_bytes);
    if (e == cudaSuccess) e = dev_alloc(&b->buf[1], b->buf_bytes);
    if (e == cudaSuccess) e = dev_alloc((void **)&b->walks_dev, sizeof(WalkDesc) * nwalks);
    if (e == cudaSuccess) e = dev_alloc((void **)&b->order_dev, sizeof(int) * nwalks);
    if (e == cudaSuccess) e = dev_alloc((void **)&b->P_dev, sizeof(float) * (size_t)b->total_sites);
    if (e == cudaSuccess) e = dev_alloc((void **)&b->norms_dev, sizeof(double) * nwalks);
    if (e == cudaSuccess) e = dev_alloc((void **)&b->counter, 2 * sizeof(int));
    if (e == cudaSuccess) e = dev_alloc((void **)&b->final_dev, sizeof(int) * nwalks);
    set_gains(b, b->K);
    if (e == cudaSuccess) e = cudaMemcpy(b->walks_dev, b->walks.data(), sizeof(WalkDesc) * nwalks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->order_dev, b->order.data(), sizeof(int) * nwalks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        qw_status st = e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA;
        (void)cudaGetLastError();
        qw_batch_destroy(b);
        return st;
    }
    b->grid = std::max(1, std::min(nwalks, sms * std::max(1, per_sm)));
    b->grid1 = std::max(1, std::min(nwalks, sms * std::max(1, per_sm1)));
    b->nbig = nwalks / 16;   // the largest sixteenth on CTAs (the autotuner refines it)
    if (prec == QW_F32_COMP) { b->variant = 0; b->K = 32; }
    *out = b;
    return QW_OK;
}

qw_status qw_batch_step(qw_batch *b) {
    if (!b) return QW_EINVAL;
    NvtxRange nvtx("qw_batch_step");
    cudaError_t e;
    if (!b->exec) {
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return batch_cuda(b, e, "graph capture begin");
        cudaError_t le = batch_launch(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (le != cudaSuccess) { drop_graph(b); return batch_cuda(b, le, "batch launch (capture)"); }
        if (e != cudaSuccess) { drop_graph(b); return batch_cuda(b, e, "graph capture end"); }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) { drop_graph(b); return batch_cuda(b, e, "graph instantiate"); }
    }
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "graph launch");
    b->ran = true;
    return QW_OK;
}

qw_status qw_batch_set_plan(qw_batch *b, int depth_k) {
    if (!b) return QW_EINVAL;
    if (depth_k < 1 || depth_k > batch_kmax(b->prec))
        return batch_fail(b, QW_EINVAL, "k must be in [1, " + std::to_string(batch_kmax(b->prec)) + "]");
    if (depth_k != b->K) {
        cudaStreamSynchronize(b->stream);
        drop_graph(b);   // the captured launch carries k
        b->K = depth_k;
        set_gains(b, depth_k);
        cudaError_t e = cudaMemcpy(b->walks_dev, b->walks.data(), sizeof(WalkDesc) * b->nwalks, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return batch_cuda(b, e, "batch plan");
    }
    return QW_OK;
}

qw_status qw_batch_get_plan(const qw_batch *b, int *depth_k, int *tile) {
    if (!b || !depth_k || !tile) return QW_EINVAL;
    *depth_k = b->K;
    *tile = batch_tile(b->prec);
    return QW_OK;
}

qw_status qw_batch_set_plan_ex(qw_batch *b, int depth_k, int variant) {
    if (!b) return QW_EINVAL;
    if (variant != 0 && variant != 1) return batch_fail(b, QW_EINVAL, "variant must be 0 (tiles) or 1 (window sweep)");
    if (variant == 1 && b->prec == QW_F32_COMP)
        return batch_fail(b, QW_EUNSUPPORTED, "the double-float batch runs the warp tiles (variant 0) only");
    qw_status st = qw_batch_set_plan(b, depth_k);
    if (st != QW_OK) return st;
    if (variant != b->variant) {
        cudaStreamSynchronize(b->stream);
        drop_graph(b);   // the captured launch is one kernel variant
        b->variant = variant;
    }
    return QW_OK;
}

qw_status qw_batch_set_cta_walks(qw_batch *b, int n) {
    if (!b) return QW_EINVAL;
    if (n < 0) return batch_fail(b, QW_EINVAL, "the number of CTA walks must be >= 0");
    n = std::min(n, b->nwalks);
    if (n != b->nbig) {
        cudaStreamSynchronize(b->stream);
        drop_graph(b);   // the captured launch carries the split
        b->nbig = n;
    }
    return QW_OK;
}

int qw_batch_cta_walks(const qw_batch *b) { return b ? b->nbig : -1; }

qw_status qw_batch_get_plan_ex(const qw_batch *b, int *depth_k, int *tile, int *variant) {
    if (!b || !depth_k || !tile || !variant) return QW_EINVAL;
    *depth_k = b->K;
    *tile = batch_tile(b->prec);
    *variant = b->variant;
    return QW_OK;
}

qw_status qw_batch_autotune(qw_batch *b, char *report, size_t report_len) {
    if (!b) return QW_EINVAL;
    const int ks[] = {8, 16, 24, 32, 48, 64, 96, 128};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_k = b->K, best_v = b->variant;
    int best_n = b->nbig;
    cudaError_t e = cudaSuccess;
    // time the current plan (after a capturing warm-up run)
    auto time_plan = [&](float &ms) -> bool {
        if (qw_batch_step(b) != QW_OK) { e = cudaErrorUnknown; return false; }
        cudaEventRecord(e0, b->stream);
        qw_batch_step(b);
        cudaEventRecord(e1, b->stream);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return false;
        cudaEventElapsedTime(&ms, e0, e1);
        return true;
    };
    // variant 0 over k
    for (int k : ks) {
        if (k > batch_kmax(b->prec)) break;
        float ms = 0.f;
        if (qw_batch_set_plan_ex(b, k, 0) != QW_OK) { e = cudaErrorUnknown; break; }
        if (!time_plan(ms)) break;
        if (ms < best) { best = ms; best_k = k; best_v = 0; }
    }
    // variant 1: how many of the largest walks run on CTAs (the rest on single
    // warps), at k = 96, then k at that split
    int n1 = b->nbig;
    float best1 = 1e30f;
    if (e == cudaSuccess && b->prec != QW_F32_COMP && qw_batch_set_plan_ex(b, std::min(96, 8 * BATCH_R), 1) == QW_OK) {
        for (int n : {0, 16, 32, 64, 128, 256, 512, 1024, b->nwalks}) {
            if (n > b->nwalks) continue;
            qw_batch_set_cta_walks(b, n);
            float ms = 0.f;
            if (!time_plan(ms)) break;
            if (ms < best1) { best1 = ms; n1 = n; }
        }
        qw_batch_set_cta_walks(b, n1);
    }
    for (int k : ks) {
        if (e != cudaSuccess || b->prec == QW_F32_COMP || k > 8 * BATCH_R) break;
        float ms = 0.f;
        if (qw_batch_set_plan_ex(b, k, 1) != QW_OK) { e = cudaErrorUnknown; break; }
        if (!time_plan(ms)) break;
        if (ms < best) { best = ms; best_k = k; best_v = 1; best_n = n1; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    qw_batch_set_cta_walks(b, best_n);
    if (e != cudaSuccess) return e == cudaErrorUnknown ? QW_ECUDA : batch_cuda(b, e, "batch autotune");
    qw_batch_set_plan_ex(b, best_k, best_v);
    if (report && report_len) {
        std::snprintf(report, report_len,
                      "{\"tuned\": true, \"k\": %d, \"tile\": %d, \"variant\": \"%s\", \"cta_walks\": %d, "
                      "\"ms\": %.6g}", best_k, batch_tile(b->prec), best_v ? "window_sweep" : "tiles", best_v ? b->nbig : b->nwalks, best);
    }
    return QW_OK;
}

qw_status qw_batch_probabilities(qw_batch *b, float *P_concat, int on_device, double *norms) {
    if (!b) return QW_EINVAL;
    if (!b->ran) return batch_fail(b, QW_ESTATE, "qw_batch_step has not run");
    cudaError_t e = cudaSuccess;
    if (P_concat)
        e = cudaMemcpyAsync(P_concat, b->P_dev, sizeof(float) * (size_t)b->total_sites,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && norms)
        e = cudaMemcpyAsync(norms, b->norms_dev, sizeof(double) * b->nwalks, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? QW_OK : batch_cuda(b, e, "batch probabilities");
}

qw_status qw_batch_get_state(qw_batch *b, int walk, void *amp_out, qw_cdtype dtype) {
    if (!b) return QW_EINVAL;
    if (walk < 0 || walk >= b->nwalks || !amp_out || (dtype != QW_C128 && dtype != QW_C64))
        return batch_fail(b, QW_EINVAL, "bad walk index, buffer or dtype");
    if (!b->ran) return batch_fail(b, QW_ESTATE, "qw_batch_step has not run");
    const WalkDesc &d = b->walks[walk];
    int which = 0;
    cudaError_t e = cudaMemcpyAsync(&which, b->final_dev + walk, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "batch state");
    View v{static_cast<char *>(b->buf[which]) + d.base * batch_slot_bytes(b->prec), d.pitch, 2};
    const size_t eb = dtype == QW_C128 ? 16 : 8;
    void *tmp = nullptr;
    e = dev_alloc(&tmp, 2 * (size_t)d.n * eb);
    if (e != cudaSuccess) return batch_cuda(b, e, "batch state staging");
    const int prec = batch_prec_code(b->prec);
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = launch_export(prec, v, d.n, static_cast<char *>(tmp) + c * d.n * eb, dtype == QW_C64, 0, d.n, c, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(amp_out, tmp, 2 * (size_t)d.n * eb, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    return e == cudaSuccess ? QW_OK : batch_cuda(b, e, "batch state");
}

}  // extern "C"
