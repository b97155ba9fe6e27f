// k_step1d.cuh -- fused coin + shift on the cycle Z_N with temporal blocking.
//
// One step is U = S (I (x) C) (Sec. 2.1) on the 1D walk of Sec. 2.2: coin 0 moves
// x -> x-1, coin 1 moves x -> x+1 (moving shift) or the same moves with the
// coin flipped (flip-flop).  The paper's kernel (Sec. 3, figure "one iteration
// segment") does one step per launch, one thread per site, reading both coin
// planes from global memory.  Here each warp owns a tile of 32*R consecutive
// sites held in registers (R per lane), applies K steps back to back, moving
// the one value per plane that crosses a lane boundary with a warp shuffle,
// and writes only the 32R - 2K central sites: the light cone of a site after
// K steps is +-K sites, so those outputs never saw the tile edge.  Tiles of
// neighbouring warps overlap by 2K sites (recomputed redundantly), which is
// what lets warps run with no synchronisation at all.  HBM traffic per step
// is (2 planes read + 2 written) / K per site.
//
// The same kernel, with ADJ=1, applies U^dagger = (I (x) C^dagger) S^dagger.
//
// Per-plane factors: `pre` after the load, `post` before the store.  They carry
// the signs and the scale lambda^K of the Hadamard-class coin (CK_SIGN_*), and
// for other global coins the compensation of the one systematic error of a
// rounded coin: with C_f the coin rounded to the compute precision,
// C_f^dagger C_f = alpha^2 I (exactly for rotation / Hadamard-type coins, to
// first order otherwise), so K steps scale the norm by alpha^K and the host
// passes post = alpha^-K.  Without it 1/sqrt2 rounded to float shrinks the norm
// by 3.6e-8 per step (1.5e-4 after 4096 steps).
#pragma once
#include "qw_internal.cuh"

namespace qw {

__device__ __forceinline__ int64_t wrap_index(int64_t g, int64_t n) {
    int64_t r = g % n;
    return r < 0 ? r + n : r;
}

// Load R consecutive sites starting at global site s (periodic wrap), one plane.
template <int P, int R>
__device__ __forceinline__ void load_run(View v, int c, int64_t s, int64_t n,
                                         Cx<typename St<P>::real> (&o)[R]) {
    using S = St<P>;
    if (s >= 0 && s + R <= n && (s % S::VEC) == 0) {
#pragma unroll
        for (int j = 0; j < R; j += S::VEC) S::ldv(v, c, s + j, &o[j]);
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) o[j] = S::ld(v, c, wrap_index(s + j, n));
    }
}

// Store the lane's R sites (global s .. s+R-1, tile positions j0 .. j0+R-1),
// keeping only tile positions in [lo, hi).
template <int P, int R>
__device__ __forceinline__ void store_run(View v, int c, int64_t s, int j0, int lo, int hi,
                                          const Cx<typename St<P>::real> (&a)[R]) {
    using S = St<P>;
    if (j0 >= lo && j0 + R <= hi && (s % S::VEC) == 0) {
#pragma unroll
        for (int j = 0; j < R; j += S::VEC) S::stv(v, c, s + j, &a[j]);
    } else if (j0 + R > lo && j0 < hi) {   // a lane straddling an end of the output range
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (j0 + j >= lo && j0 + j < hi) S::st(v, c, s + j, a[j]);
    }                                      // lanes holding only halo sites store nothing
}

// phi = C psi for one site, d = 2.
template <int CK, class R>
__device__ __forceinline__ void coin2(const CoinP<R> &cp, const Cx<R> *m, Cx<R> a0, Cx<R> a1,
                                      Cx<R> &p0, Cx<R> &p1) {
    if (CK == CK_REAL) {
        p0 = rfma(cp.re[1], a1, rmul(cp.re[0], a0));
        p1 = rfma(cp.re[3], a1, rmul(cp.re[2], a0));
    } else if (CK == CK_COMPLEX) {
        Cx<R> c00{cp.re[0], cp.im[0]}, c01{cp.re[1], cp.im[1]};
        Cx<R> c10{cp.re[2], cp.im[2]}, c11{cp.re[3], cp.im[3]};
        p0 = cfma(c01, a1, cmul(c00, a0));
        p1 = cfma(c11, a1, cmul(c10, a0));
    } else if (CK == CK_SIGN_P) {
        p0 = cadd(a0, a1);
        p1 = csub(a0, a1);
    } else if (CK == CK_SIGN_M) {
        p0 = csub(a0, a1);
        p1 = cadd(a0, a1);
    } else {  // CK_PERSITE: m points at this site's 4 entries
        p0 = cfma(m[1], a1, cmul(m[0], a0));
        p1 = cfma(m[3], a1, cmul(m[2], a0));
    }
}

// psi = C^dagger b for one site, d = 2.
template <int CK, class R>
__device__ __forceinline__ void coin2_adj(const CoinP<R> &cp, const Cx<R> *m, Cx<R> b0, Cx<R> b1,
                                          Cx<R> &a0, Cx<R> &a1) {
    if (CK == CK_REAL) {
        a0 = rfma(cp.re[2], b1, rmul(cp.re[0], b0));
        a1 = rfma(cp.re[3], b1, rmul(cp.re[1], b0));
    } else if (CK == CK_COMPLEX) {
        Cx<R> c00{cp.re[0], cp.im[0]}, c01{cp.re[1], cp.im[1]};
        Cx<R> c10{cp.re[2], cp.im[2]}, c11{cp.re[3], cp.im[3]};
        a0 = cadd(conjmul(c00, b0), conjmul(c10, b1));
        a1 = cadd(conjmul(c01, b0), conjmul(c11, b1));
    } else if (CK == CK_SIGN_P || CK == CK_SIGN_M) {
        // (U^dagger)^K = lambda^K a^{K-1} diag(1, s) [H_sigma S^dagger]^K diag(a, sigma c):
        // the same addition pattern, applied after the pull
        coin2<CK>(cp, m, b0, b1, a0, a1);
    } else {
        a0 = cadd(conjmul(m[0], b0), conjmul(m[2], b1));
        a1 = cadd(conjmul(m[1], b0), conjmul(m[3], b1));
    }
}

// Tile origin of a warp whose first output site is out0: out0 - K rounded down
// to the vector width, so that every lane's run starts on a 16-byte boundary
// whatever K is.  W (outputs per warp) is a multiple of VEC with
// 32R >= W + 2K + VEC - 1, so the tile still covers the light cone.
template <int VEC>
__device__ __forceinline__ int64_t tile_origin(int64_t out0, int K) {
    const int64_t t = out0 - K;
    return t >= 0 ? t - t % VEC : -((-t + VEC - 1) / VEC) * VEC;
}

// One warp tile: K steps on the 32R sites around the wthis outputs
// [out0, out0 + wthis), a range inside [0, n).  Called by the cycle kernel
// below and by the batched kernel (one walk per CTA).
template <int P, int R, int CK, int FF, int ADJ>
__device__ __forceinline__ void tb_tile(View in, View out, int64_t n, int K, int64_t out0, int wthis, int lane,
                                        const CoinP<typename St<P>::real> &cp,
                                        const Cx<typename St<P>::real> *__restrict__ coins,
                                        typename St<P>::real pre0, typename St<P>::real pre1,
                                        typename St<P>::real post0, typename St<P>::real post1) {
    using real = typename St<P>::real;
    using C = Cx<real>;
    const int j0 = lane * R;
    const int64_t ts = tile_origin<St<P>::VEC>(out0, K);
    const int lo = (int)(out0 - ts);   // first output's tile position, in [K, K + VEC)
    const int64_t s = ts + j0;

    C a0[R], a1[R];
    load_run<P, R>(in, 0, s, n, a0);
    load_run<P, R>(in, 1, s, n, a1);
    if (!is_one(pre0)) {
#pragma unroll
        for (int i = 0; i < R; ++i) a0[i] = rmul(pre0, a0[i]);
    }
    if (!is_one(pre1)) {
#pragma unroll
        for (int i = 0; i < R; ++i) a1[i] = rmul(pre1, a1[i]);
    }

    // per-site coins stay with their site while the amplitudes move through
    constexpr int NM = (CK == CK_PERSITE) ? 4 * R : 1;
    C m[NM];
    if (CK == CK_PERSITE) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            int64_t g = wrap_index(s + i, n);
#pragma unroll
            for (int e = 0; e < 4; ++e) m[4 * i + e] = coins[4 * g + e];
        }
    }

    // unrolled by two so the register shift of one step is a renaming into the
    // other step's registers instead of moves at the loop back edge
#pragma unroll 2
    for (int t = 0; t < K; ++t) {
        if (!ADJ) {
            C p0[R], p1[R];
#pragma unroll
            for (int i = 0; i < R; ++i) coin2<CK>(cp, &m[(CK == CK_PERSITE) ? 4 * i : 0], a0[i], a1[i], p0[i], p1[i]);
            // coin 0 arrives from the right neighbour site, coin 1 from the left
            C from_right = shfl_down(p0[0], 1);
            C from_left = shfl_up(p1[R - 1], 1);
            if (!FF) {
#pragma unroll
                for (int i = 0; i < R - 1; ++i) a0[i] = p0[i + 1];
                a0[R - 1] = from_right;
#pragma unroll
                for (int i = R - 1; i > 0; --i) a1[i] = p1[i - 1];
                a1[0] = from_left;
            } else {
#pragma unroll
                for (int i = 0; i < R - 1; ++i) a1[i] = p0[i + 1];
                a1[R - 1] = from_right;
#pragma unroll
                for (int i = R - 1; i > 0; --i) a0[i] = p1[i - 1];
                a0[0] = from_left;
            }
        } else {
            // S^dagger: moving  b0(x) = psi0(x-1), b1(x) = psi1(x+1);
            //           flip-flop b0(x) = psi1(x-1), b1(x) = psi0(x+1)
            C lsrc[R], rsrc[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                lsrc[i] = FF ? a1[i] : a0[i];
                rsrc[i] = FF ? a0[i] : a1[i];
            }
            C from_left = shfl_up(lsrc[R - 1], 1);
            C from_right = shfl_down(rsrc[0], 1);
            C b0[R], b1[R];
#pragma unroll
            for (int i = R - 1; i > 0; --i) b0[i] = lsrc[i - 1];
            b0[0] = from_left;
#pragma unroll
            for (int i = 0; i < R - 1; ++i) b1[i] = rsrc[i + 1];
            b1[R - 1] = from_right;
#pragma unroll
            for (int i = 0; i < R; ++i) coin2_adj<CK>(cp, &m[(CK == CK_PERSITE) ? 4 * i : 0], b0[i], b1[i], a0[i], a1[i]);
        }
    }
    if (!is_one(post0)) {
#pragma unroll
        for (int i = 0; i < R; ++i) a0[i] = rmul(post0, a0[i]);
    }
    if (!is_one(post1)) {
#pragma unroll
        for (int i = 0; i < R; ++i) a1[i] = rmul(post1, a1[i]);
    }
    store_run<P, R>(out, 0, s, j0, lo, lo + wthis, a0);
    store_run<P, R>(out, 1, s, j0, lo, lo + wthis, a1);
}

// W output sites per warp (see tile_origin) over the output range [obeg, oend)
// inside [0, n) (the whole cycle, or the light-cone window of a localised
// state); nwarps = ceil((oend - obeg) / W).
template <int P, int R, int CK, int FF, int ADJ>
__global__ void __launch_bounds__(128)
k_step1d(View in, View out, int64_t n, int K, int64_t W, int64_t obeg, int64_t oend, int64_t nwarps,
         CoinP<typename St<P>::real> cp, const Cx<typename St<P>::real> *__restrict__ coins,
         typename St<P>::real pre0, typename St<P>::real pre1,
         typename St<P>::real post0, typename St<P>::real post1) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nwarps) return;  // uniform per warp
    const int64_t out0 = obeg + warp * W;
    tb_tile<P, R, CK, FF, ADJ>(in, out, n, K, out0, (int)min(W, oend - out0), lane, cp, coins, pre0, pre1, post0,
                               post1);
}

// ---------------------------------------------------------------- k = 1
// One step per launch, streaming: each lane owns one 16-byte vector per plane
// (VEC sites), so every warp load / store is one fully coalesced 512-byte
// access.  The value that enters a lane from its neighbour comes by shuffle;
// at the warp edges lane 0 and lane 31 evaluate the one site outside the
// warp's range themselves (periodic), so nothing is recomputed elsewhere.
template <int P, int CK, int FF, int ADJ>
__device__ void step1d_site(View in, View out, int64_t n, int64_t x, const CoinP<typename St<P>::real> &cp,
                            const Cx<typename St<P>::real> *coins, typename St<P>::real pre0,
                            typename St<P>::real pre1, typename St<P>::real post0,
                            typename St<P>::real post1) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    const int64_t xm = x == 0 ? n - 1 : x - 1, xp = x + 1 == n ? 0 : x + 1;
    C r0, r1;
    if (!ADJ) {
        // coin at x+1 (its coin-0 output moves to x) and at x-1 (coin 1 moves to x)
        C u0 = rmul(pre0, S::ld(in, 0, xp)), u1 = rmul(pre1, S::ld(in, 1, xp)), p0, p1;
        coin2<CK>(cp, coins + 4 * xp, u0, u1, p0, p1);
        C v0 = rmul(pre0, S::ld(in, 0, xm)), v1 = rmul(pre1, S::ld(in, 1, xm)), q0, q1;
        coin2<CK>(cp, coins + 4 * xm, v0, v1, q0, q1);
        r0 = FF ? q1 : p0;
        r1 = FF ? p0 : q1;
    } else {
        C b0, b1;
        if (!FF) { b0 = rmul(pre0, S::ld(in, 0, xm)); b1 = rmul(pre1, S::ld(in, 1, xp)); }
        else { b0 = rmul(pre1, S::ld(in, 1, xm)); b1 = rmul(pre0, S::ld(in, 0, xp)); }
        coin2_adj<CK>(cp, coins + 4 * x, b0, b1, r0, r1);
    }
    S::st(out, 0, x, rmul(post0, r0));
    S::st(out, 1, x, rmul(post1, r1));
}

template <int P, int CK, int FF, int ADJ>
__global__ void __launch_bounds__(256)
k_step1d_k1(View in, View out, int64_t n, int64_t nwarps, CoinP<typename St<P>::real> cp,
            const Cx<typename St<P>::real> *__restrict__ coins, typename St<P>::real pre0,
            typename St<P>::real pre1, typename St<P>::real post0, typename St<P>::real post1) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    constexpr int R = S::VEC;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nwarps) return;  // uniform per warp
    const int64_t x0 = warp * (32 * R);
    const int64_t xs = x0 + lane * R;
    if (x0 + 32 * R > n) {       // ragged tail (uniform per warp): per-site pull
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (xs + i < n) step1d_site<P, CK, FF, ADJ>(in, out, n, xs + i, cp, coins, pre0, pre1, post0, post1);
        return;
    }
    C a0[R], a1[R];
    S::ldv(in, 0, xs, a0);
    S::ldv(in, 1, xs, a1);
#pragma unroll
    for (int i = 0; i < R; ++i) { a0[i] = rmul(pre0, a0[i]); a1[i] = rmul(pre1, a1[i]); }
    const int64_t xl = x0 == 0 ? n - 1 : x0 - 1;        // site left of the warp
    const int64_t xr = (x0 + 32 * R == n) ? 0 : x0 + 32 * R;  // site right of the warp
    C r0[R], r1[R];
    if (!ADJ) {
        C p0[R], p1[R];
#pragma unroll
        for (int i = 0; i < R; ++i) coin2<CK>(cp, coins + 4 * (xs + i), a0[i], a1[i], p0[i], p1[i]);
        C halo = czero<real>();
        if (lane == 0 || lane == 31) {
            const int64_t xh = lane == 0 ? xl : xr;
            C h0 = rmul(pre0, S::ld(in, 0, xh)), h1 = rmul(pre1, S::ld(in, 1, xh)), q0, q1;
            coin2<CK>(cp, coins + 4 * xh, h0, h1, q0, q1);
            halo = lane == 0 ? q1 : q0;
        }
        C from_right = shfl_down(p0[0], 1);
        C from_left = shfl_up(p1[R - 1], 1);
        if (lane == 31) from_right = halo;
        if (lane == 0) from_left = halo;
        // coin 0 arrives from x+1, coin 1 from x-1; flip-flop swaps the planes
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const C in0 = (i == R - 1) ? from_right : p0[i + 1];
            const C in1 = (i == 0) ? from_left : p1[i - 1];
            r0[i] = FF ? in1 : in0;
            r1[i] = FF ? in0 : in1;
        }
    } else {
        // S^dagger: moving b0(x) = psi0(x-1), b1(x) = psi1(x+1); flip-flop b0(x) = psi1(x-1), b1(x) = psi0(x+1)
        C lsrc[R], rsrc[R];
#pragma unroll
        for (int i = 0; i < R; ++i) { lsrc[i] = FF ? a1[i] : a0[i]; rsrc[i] = FF ? a0[i] : a1[i]; }
        C halo = czero<real>();
        if (lane == 0) halo = FF ? rmul(pre1, S::ld(in, 1, xl)) : rmul(pre0, S::ld(in, 0, xl));
        if (lane == 31) halo = FF ? rmul(pre0, S::ld(in, 0, xr)) : rmul(pre1, S::ld(in, 1, xr));
        C from_left = shfl_up(lsrc[R - 1], 1);
        C from_right = shfl_down(rsrc[0], 1);
        if (lane == 0) from_left = halo;
        if (lane == 31) from_right = halo;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const C b0 = (i == 0) ? from_left : lsrc[i - 1];
            const C b1 = (i == R - 1) ? from_right : rsrc[i + 1];
            coin2_adj<CK>(cp, coins + 4 * (xs + i), b0, b1, r0[i], r1[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) { r0[i] = rmul(post0, r0[i]); r1[i] = rmul(post1, r1[i]); }
    S::stv(out, 0, xs, r0);
    S::stv(out, 1, xs, r1);
}

// ---------------------------------------------------------------- time-skewed sweep
// The same k steps per HBM round trip as tb_tile, without recomputing a halo.
// A warp walks a segment of the cycle chunk by chunk (32R sites per chunk).
// The frame slides one site to the left per step: after t steps a chunk that
// was loaded at [x, x + 32R) holds [x - t, x + 32R - t).  In that frame the
// walk depends on the left only: one plane keeps its index, the other takes
// the value two sites to its left (moving shift: coin 0 arrives from x+1, coin
// 1 from x-1).  The two values a chunk needs from the chunk before it, at each
// of the k time levels, are handed over through a small per-warp edge array in
// shared memory.  Only the first chunk of a segment is recomputed (a warm-up
// chunk whose own left edge starts as zeros; its error front moves two sites
// per step, so k < 16R keeps the handed-over values exact).  The next chunk is
// prefetched with cp.async into a swizzled shared buffer while the current one
// computes; each lane then reads its own run conflict-free.  Any n >= 32R: the
// last chunk may reach past site n - 1 and wrap.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// One site's slot (4, 8 or 16 bytes), both addresses aligned to its size.
template <int BYTES>
__device__ __forceinline__ void cp_async_slot(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Lane 31 stores (v2, v1) at eout and loads (v2, v1) from ein; the other lanes
// keep their values.  Predicated shared accesses: no branch, no select.
// Float pairs are one 16-byte access each way (both addresses 16-byte aligned).
__device__ __forceinline__ void edge_swap31(int lane, unsigned eout, unsigned ein, Cx<float> &v2, Cx<float> &v1) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %4, 31;\n\t"
                 "@p st.shared.v4.f32 [%5], {%0, %1, %2, %3};\n\t"
                 "@p ld.shared.v4.f32 {%0, %1, %2, %3}, [%6];\n\t}"
                 : "+f"(v2.re), "+f"(v2.im), "+f"(v1.re), "+f"(v1.im)
                 : "r"(lane), "r"(eout), "r"(ein)
                 : "memory");
}
__device__ __forceinline__ void edge_swap31(int lane, unsigned eout, unsigned ein, Cx<double> &v2, Cx<double> &v1) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %4, 31;\n\t"
                 "@p st.shared.v2.f64 [%5], {%0, %1};\n\t"
                 "@p st.shared.v2.f64 [%5+16], {%2, %3};\n\t"
                 "@p ld.shared.v2.f64 {%0, %1}, [%6];\n\t"
                 "@p ld.shared.v2.f64 {%2, %3}, [%6+16];\n\t}"
                 : "+d"(v2.re), "+d"(v2.im), "+d"(v1.re), "+d"(v1.im)
                 : "r"(lane), "r"(eout), "r"(ein)
                 : "memory");
}

// Position of a lane's c-th 16-byte unit in the chunk buffer: the XOR keeps the
// eight lanes that share a shared-memory wavefront on distinct bank groups.
template <int CPL>
__device__ __forceinline__ int swz(int lane, int c) {
    if constexpr (CPL >= 8) {
        return lane * CPL + (c ^ (lane & 7));
    } else {
        constexpr int G = 8 / CPL;
        return lane * CPL + (c ^ ((lane / G) & (CPL - 1)));
    }
}

template <int P, int R>
struct Sweep {
    static constexpr int B = 32 * R;                              // sites per chunk
    static constexpr int CPL = R * St<P>::SLOT_BYTES / 16;        // 16-byte units per lane and plane
    static constexpr size_t chunk_bytes = 2 * 32 * CPL * 16;
    __host__ __device__ static size_t edge_bytes(int K) { return 2 * (size_t)K * 2 * sizeof(Cx<typename St<P>::real>); }
    __host__ __device__ static size_t warp_bytes(int K) { return chunk_bytes + edge_bytes(K); }
};

template <int P, int R, int CK, int FF, int ADJ>
__global__ void __launch_bounds__(128)
k_step1d_sweep(View in, View out, int64_t n, int K, int nch, int64_t nseg, CoinP<typename St<P>::real> cp,
               typename St<P>::real pre0, typename St<P>::real pre1,
               typename St<P>::real post0, typename St<P>::real post1) {
    using S = St<P>;
    using real = typename S::real;
    using C = Cx<real>;
    using SW = Sweep<P, R>;
    constexpr int B = SW::B, CPL = SW::CPL, VEC = S::VEC;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (seg >= nseg) return;   // uniform per warp
    unsigned char *wbase = smem + wib * SW::warp_bytes(K);
    uint4 *cbuf = reinterpret_cast<uint4 *>(wbase);
    C *edge = reinterpret_cast<C *>(wbase + SW::chunk_bytes);
    const int64_t s0 = seg * (int64_t)nch * B;
    // the last chunk of the cycle may run past site n - 1: it wraps to the first
    // sites, which it recomputes (with their true left context) to the same bits
    const int nchs = (int)min((int64_t)nch, (n - s0 + B - 1) / B);

    auto prefetch = [&](int j) {
        int64_t start = s0 + (int64_t)j * B;
        if (start < 0) start += n;
        if (start + B <= n && start % VEC == 0) {   // a contiguous, 16-byte aligned run
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const char *g = static_cast<const char *>(in.p) + (c * in.pitch + start) * S::SLOT_BYTES;
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int u = i * 32 + lane;
                    cp_async16(cbuf + c * 32 * CPL + swz<CPL>(u / CPL, u % CPL), g + (size_t)u * 16);
                }
            }
        } else {   // across site n - 1 (or after it, unaligned): this lane's own sites one by one
            // (rolled loops: the rare path must not cost the main loop registers)
            constexpr int UPV = 16 / S::SLOT_BYTES;
#pragma unroll 1
            for (int c = 0; c < 2; ++c) {
#pragma unroll 1
                for (int i = 0; i < R; ++i) {
                    const int64_t g = (start + (int64_t)lane * R + i) % n;
                    void *dst = reinterpret_cast<unsigned char *>(cbuf + c * 32 * CPL + swz<CPL>(lane, i / UPV)) +
                                (i % UPV) * S::SLOT_BYTES;
                    cp_async_slot<S::SLOT_BYTES>(dst, static_cast<const char *>(in.p) + (c * in.pitch + g) * S::SLOT_BYTES);
                }
            }
        }
        cp_async_commit();
    };

    // the warm-up chunk (j = -1) reads its left edge from the parity-0 edge
    // buffer: zero it once, so the level loop needs no special case.  After
    // this, lane 31 alone writes and reads the edge entries.
    for (int i = lane; i < 2 * K; i += 32) edge[i] = czero<real>();
    __syncwarp();

    C a0[R], a1[R];
    prefetch(-1);
    for (int j = -1; j < nchs; ++j) {
        cp_async_wait_all();
        __syncwarp();
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            S::unpack(cbuf[swz<CPL>(lane, u)], &a0[u * VEC]);
            S::unpack(cbuf[32 * CPL + swz<CPL>(lane, u)], &a1[u * VEC]);
        }
        __syncwarp();
        if (j + 1 < nchs) prefetch(j + 1);
        if (!is_one(pre0)) {
#pragma unroll
            for (int i = 0; i < R; ++i) a0[i] = rmul(pre0, a0[i]);
        }
        if (!is_one(pre1)) {
#pragma unroll
            for (int i = 0; i < R; ++i) a1[i] = rmul(pre1, a1[i]);
        }
        const int par = j & 1;
        const int from = (lane + 31) & 31;   // the lane below, lane 31 for lane 0
        // shared addresses of the edge entries handed over by the previous chunk
        // (ein) and to the next one (eout)
        const unsigned si = (unsigned)__cvta_generic_to_shared(edge + (size_t)(par ^ 1) * K * 2);
        const unsigned so = (unsigned)__cvta_generic_to_shared(edge + (size_t)par * K * 2);
        // One level of the sliding frame, from (s0, s1) into fresh arrays (d0, d1).
        // Two levels per loop iteration ping-pong between a and b, so results
        // always go to registers that hold nothing live (no moves at all).
        // The two values that leave a lane at its top go to the lane above by a
        // rotating shuffle; lane 31's pair instead goes to the next chunk through
        // eout, and lane 31 sends on, in its place, the pair the previous chunk
        // left in ein (zeros for the warm-up chunk), which the rotation delivers
        // to lane 0.  Predicated shared accesses of lane 31, no selects.
        auto level = [&](int t, const C (&s0)[R], const C (&s1)[R], C (&d0)[R], C (&d1)[R]) {
            if (!ADJ) {
                C top2, top1;   // coin-1 results of the two highest sites: they leave the lane
#pragma unroll
                for (int i = R - 1; i >= 0; --i) {
                    C n0, n1;
                    coin2<CK>(cp, (const C *)nullptr, s0[i], s1[i], n0, n1);
                    // moving: coin 0 keeps its frame index, coin 1 moves two up;
                    // flip-flop: the same values land in the other plane
                    if (!FF) d0[i] = n0; else d1[i] = n0;
                    if (i + 2 < R) { if (!FF) d1[i + 2] = n1; else d0[i + 2] = n1; }
                    else if (i == R - 1) top1 = n1;
                    else top2 = n1;
                    if (i == R - 2)   // both leave-values ready: lane 31 swaps in ein's
                        edge_swap31(lane, so + t * 2 * (unsigned)sizeof(C), si + t * 2 * (unsigned)sizeof(C), top2, top1);
                }
                const C lm2 = shfl_idx(top2, from), lm1 = shfl_idx(top1, from);
                if (!FF) { d1[0] = lm2; d1[1] = lm1; } else { d0[0] = lm2; d0[1] = lm1; }
            } else {
                // S^dagger in the sliding frame: moving b1 = a1 (same index), b0 = a0 two down;
                // flip-flop b1 = a0, b0 = a1 two down.  Then C^dagger at the site.
                C e2 = FF ? s1[R - 2] : s0[R - 2], e1 = FF ? s1[R - 1] : s0[R - 1];
                edge_swap31(lane, so + t * 2 * (unsigned)sizeof(C), si + t * 2 * (unsigned)sizeof(C), e2, e1);
                const C lm2 = shfl_idx(e2, from), lm1 = shfl_idx(e1, from);
#pragma unroll
                for (int i = R - 1; i >= 0; --i) {
                    const C b0 = i >= 2 ? (FF ? s1[i - 2] : s0[i - 2]) : (i == 0 ? lm2 : lm1);
                    const C b1 = FF ? s0[i] : s1[i];
                    coin2_adj<CK>(cp, (const C *)nullptr, b0, b1, d0[i], d1[i]);
                }
            }
        };
        C b0[R], b1[R];
        // blocks of levels; the Hadamard class rescales after each full block of
        // SIGN_RESCALE_STEPS (its unnormalised additions grow by sqrt(2) per step)
        constexpr bool SIGN = CK == CK_SIGN_P || CK == CK_SIGN_M;
        const int blk = SIGN ? SIGN_RESCALE_STEPS : K;
        int t = 0;
#pragma unroll 1
        for (int tb = 0; tb + 1 < K; tb += blk) {
            const int te = min(tb + blk, K);
#pragma unroll 1
            for (t = tb; t + 1 < te; t += 2) {
                level(t, a0, a1, b0, b1);
                level(t + 1, b0, b1, a0, a1);
            }
            if (SIGN && t == tb + SIGN_RESCALE_STEPS) {   // 2^-SIGN_RESCALE_LOG2, exact
                const real sc = (real)(1.0 / (double)(1ull << SIGN_RESCALE_LOG2));
#pragma unroll
                for (int i = 0; i < R; ++i) { a0[i] = rmul(sc, a0[i]); a1[i] = rmul(sc, a1[i]); }
            }
        }
        if (t < K) {
            level(t, a0, a1, b0, b1);
#pragma unroll
            for (int i = 0; i < R; ++i) { a0[i] = b0[i]; a1[i] = b1[i]; }
        }
        if (j >= 0) {
            if (!is_one(post0)) {
#pragma unroll
                for (int i = 0; i < R; ++i) a0[i] = rmul(post0, a0[i]);
            }
            if (!is_one(post1)) {
#pragma unroll
                for (int i = 0; i < R; ++i) a1[i] = rmul(post1, a1[i]);
            }
            const int64_t g0 = s0 + (int64_t)j * B - K + lane * R;
            if (g0 >= 0 && g0 + R <= n && (g0 % VEC) == 0) {
#pragma unroll
                for (int i = 0; i < R; i += VEC) { S::stv(out, 0, g0 + i, &a0[i]); S::stv(out, 1, g0 + i, &a1[i]); }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int64_t g = wrap_index(g0 + i, n);
                    S::st(out, 0, g, a0[i]);
                    S::st(out, 1, g, a1[i]);
                }
            }
        }
    }
}

}  // namespace qw
