// k_step2d_tb.cuh -- temporal blocking on the torus: KT walk steps per HBM
// round trip, by streaming rows through a pipeline of KT time levels.
//
// The step is the 2D walk of Sec. 2.2 / Sec. 3 (U = S (C (x) I)): with
// phi = C psi at every site, the moving shift gives
//     psi'(x, y, 0) = phi(x-1, y, 0)   psi'(x, y, 1) = phi(x+1, y, 1)
//     psi'(x, y, 2) = phi(x, y-1, 2)   psi'(x, y, 3) = phi(x, y+1, 3)
// (flip-flop: the same values land in planes 1, 0, 3, 2).  Level s of the
// pipeline produces row r of psi_s once level s-1 has produced row r+1, so
// level s runs one row behind level s-1.  Each level keeps, per column, the
// coin outputs of planes 0..2 of its input's previous row and plane 2 of the
// row before: four complex numbers of delay line per level and column, all in
// registers.  A warp owns a strip of 32R columns (R per lane) and a chunk of H
// rows; planes 0 and 1 cross lane boundaries with one shuffle each, so the
// valid columns shrink by one per level on both sides (KT columns of halo per
// side, recomputed by the neighbouring strip) and the chunk needs KT rows of
// warm-up below and above.  HBM traffic: one read and one write of the 4
// planes per KT steps, plus the halo.
#pragma once
#include "qw_internal.cuh"
#include "k_step2d.cuh"
#include "k_step1d.cuh"   // wrap_index

namespace qw {

// Site-free coin for the streaming kernel (global coins only).  H (x) H is
// applied without its factor 1/2 (the butterflies only, exact in binary
// scaling): the kernel multiplies the output by 2^-KT once, exactly.
template <int CK, class R>
__device__ __forceinline__ void coin4g(const CoinP<R> &cp, const Cx<R> (&a)[4], Cx<R> (&p)[4]) {
    if constexpr (CK == CK_HH) {
        const Cx<R> u0 = cadd(a[0], a[1]), u1 = csub(a[0], a[1]);
        const Cx<R> u2 = cadd(a[2], a[3]), u3 = csub(a[2], a[3]);
        p[0] = cadd(u0, u2);
        p[1] = cadd(u1, u3);
        p[2] = csub(u0, u2);
        p[3] = csub(u1, u3);
    } else {
        SiteCoin<R> sc;
        coin4<CK, R>(cp, (const Cx<R> *)nullptr, sc, a, p);
    }
}

// Rows of psi_0 in flight per warp: each row is cp.async-copied into a ring
// of shared-memory slots TB_RING - 1 rows before it is needed, so the global
// latency hides behind that many rows of compute (one row, about the time of
// the KT levels, is not enough).  Each lane copies and reads back only its own
// 16 bytes per plane.
constexpr int TB_RING = 4;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Dynamic shared memory of one 128-thread block.
inline size_t step2d_tb_smem() { return (size_t)(128 / 32) * TB_RING * 4 * 32 * 16; }

template <int P, int KT, int CK, int FF>
__global__ void __launch_bounds__(128)
k_step2d_tb(View in, View out, int64_t nx, int64_t ny, int64_t W, int64_t nstrips, int64_t H, int64_t nchunks,
            CoinP<typename St<P>::real> cp, typename St<P>::real gain) {
    using S = St<P>;
    using real = typename S::real;
    using C = Cx<real>;
    constexpr int R = 2;   // sites per lane (one 16-byte vector per plane in FP32)
    static_assert(P == P_F32 && R * S::SLOT_BYTES == 16, "one 16-byte ring slot per lane and plane");
    extern __shared__ __align__(16) unsigned char tsm[];
    uint4 *ring = reinterpret_cast<uint4 *>(tsm) + (size_t)(threadIdx.x >> 5) * TB_RING * 4 * 32;   // [slot][plane][lane]
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= nstrips * nchunks) return;   // uniform per warp
    const int64_t strip = gw % nstrips, chunk = gw / nstrips;
    const int64_t xo = strip * W;                       // first output column
    const int wthis = (int)min(W, nx - xo);
    const int64_t y0 = chunk * H;
    const int64_t hthis = min(H, ny - y0);
    const int j0 = lane * R;                            // tile column of the lane's first site
    const int64_t xs = xo - KT + j0;                    // its global column (may wrap)
    const bool vec = (xs >= 0) && (xs + R <= nx) && (xs % S::VEC == 0) && (R % S::VEC == 0);
    int64_t cx[R];
#pragma unroll
    for (int i = 0; i < R; ++i) cx[i] = wrap_index(xs + i, nx);

    C A[KT][R][3];   // level s input's previous row: coin outputs of planes 0, 1, 2
    C B[KT][R];      // plane 2 from the row before that
#pragma unroll
    for (int s = 0; s < KT; ++s)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            B[s][i] = czero<real>();
#pragma unroll
            for (int c = 0; c < 3; ++c) A[s][i][c] = czero<real>();
        }
    if constexpr (CK == CK_HH) gain = gain * (real)(1.0 / (double)(1u << KT));   // the factors 1/2 of H (x) H
    const bool gain_one = is_one(gain);

    // rows stay within one period of the torus (H <= ny, KT < ny is not needed:
    // q is at most one period outside [0, ny)), so a conditional add wraps them
    auto wrap_row = [&](int64_t q) { return q < 0 ? q + ny * ((-q + ny - 1) / ny) : (q >= ny ? q % ny : q); };
    const int64_t qbeg = y0 - KT, qend = y0 + hthis + KT;
    // copy row q of psi_0 (this lane's R sites of each plane) into its ring slot;
    // one commit group per row, empty past the end, so the waits count rows
    auto issue_row = [&](int64_t q) {
        if (q < qend) {
            const int64_t row = wrap_row(q) * nx;
            uint4 *dst = ring + (int)((q - qbeg) % TB_RING) * 4 * 32 + lane;
            const char *base = static_cast<const char *>(in.p);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (vec) {
                    cp_async16(dst + c * 32, base + (c * in.pitch + row + xs) * S::SLOT_BYTES);
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        cp_async8(reinterpret_cast<unsigned char *>(dst + c * 32) + i * S::SLOT_BYTES,
                                  base + (c * in.pitch + row + cx[i]) * S::SLOT_BYTES);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int r = 0; r < TB_RING - 1; ++r) issue_row(qbeg + r);
    for (int64_t q = qbeg; q < qend; ++q) {
        // psi_0 of row q with the coin applied: the newest input of level 1
        C N[R][4];
        {
            issue_row(q + TB_RING - 1);
            cp_async_wait_pending<TB_RING - 1>();   // row q has landed
            C a[4][R];
            const uint4 *src = ring + (int)((q - qbeg) % TB_RING) * 4 * 32 + lane;
#pragma unroll
            for (int c = 0; c < 4; ++c) S::unpack(src[c * 32], &a[c][0]);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                C ai[4] = {a[0][i], a[1][i], a[2][i], a[3][i]}, pi[4];
                coin4g<CK, real>(cp, ai, pi);
#pragma unroll
                for (int c = 0; c < 4; ++c) N[i][c] = pi[c];
            }
        }
        // levels 1..KT: level s produces psi_s of row q - s
        C psi[R][4];
#pragma unroll
        for (int s = 0; s < KT; ++s) {
            // x-moving planes of the previous row (A), from the neighbouring columns
            C fl = shfl_up(A[s][R - 1][0], 1);      // coin 0 arrives from x-1
            C fr = shfl_down(A[s][0][1], 1);        // coin 1 arrives from x+1
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const C m0 = i == 0 ? fl : A[s][i - 1][0];
                const C m1 = i == R - 1 ? fr : A[s][i + 1][1];
                const C m2 = B[s][i];               // coin 2 arrives from the row below
                const C m3 = N[i][3];               // coin 3 arrives from the row above
                psi[i][FF ? 1 : 0] = m0;
                psi[i][FF ? 0 : 1] = m1;
                psi[i][FF ? 3 : 2] = m2;
                psi[i][FF ? 2 : 3] = m3;
            }
            // rotate this level's delay line (after every column has read it)
#pragma unroll
            for (int i = 0; i < R; ++i) {
                B[s][i] = A[s][i][2];
                A[s][i][0] = N[i][0];
                A[s][i][1] = N[i][1];
                A[s][i][2] = N[i][2];
            }
            if (s + 1 < KT) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    C pi[4];
                    coin4g<CK, real>(cp, psi[i], pi);
#pragma unroll
                    for (int c = 0; c < 4; ++c) N[i][c] = pi[c];
                }
            }
        }
        // psi_KT of row q - KT: store the columns whose light cone stayed inside the strip
        const int64_t r = q - KT;
        if (r >= y0) {
            if (!gain_one) {   // the launch's drift correction, once per KT steps
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) psi[i][c] = rmul(gain, psi[i][c]);
            }
            const int64_t orow = wrap_row(r) * nx;
            if (j0 >= KT && j0 + R <= KT + wthis && vec) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    C v[R];
#pragma unroll
                    for (int i = 0; i < R; ++i) v[i] = psi[i][c];
#pragma unroll
                    for (int i = 0; i < R; i += S::VEC) S::stv(out, c, orow + xs + i, &v[i]);
                }
            } else if (j0 + R > KT && j0 < KT + wthis) {
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (j0 + i >= KT && j0 + i < KT + wthis)
#pragma unroll
                        for (int c = 0; c < 4; ++c) S::st(out, c, orow + cx[i], psi[i][c]);
            }
        }
    }
}

}  // namespace qw
