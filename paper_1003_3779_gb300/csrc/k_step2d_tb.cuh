// k_step2d_tb.cuh -- temporal blocking on the torus: KT walk steps per HBM
// round trip, by streaming rows through a pipeline of KT time levels.
//
// The step is the 2D walk of Sec. 2.2 / Sec. 3 (U = S (C (x) I)): with
// phi = C psi at every site, the moving shift gives
//     psi'(x, y, 0) = phi(x-1, y, 0)   psi'(x, y, 1) = phi(x+1, y, 1)
//     psi'(x, y, 2) = phi(x, y-1, 2)   psi'(x, y, 3) = phi(x, y+1, 3)
// (flip-flop: the same values land in planes 1, 0, 3, 2), and the diagonal
// lattice (Fig. 1(c)), coin c = 2j + k displaced by ((-1)^j, (-1)^k),
//     psi'(x, y, 0) = phi(x-1, y-1, 0)   psi'(x, y, 1) = phi(x-1, y+1, 1)
//     psi'(x, y, 2) = phi(x+1, y-1, 2)   psi'(x, y, 3) = phi(x+1, y+1, 3).
//
// Level s of the pipeline produces row r of psi_s once level s-1 has produced
// row r+1, so level s runs one row behind level s-1.  Its input is the coin
// output phi of psi_{s-1}: row r+1 arrives now, row r arrived one row ago and
// row r-1 two rows ago.  What a level keeps between rows, per column:
// - axis lattice: planes 0 and 1 of row r (one row of delay) in registers,
//   in two register sets that alternate with the row parity -- the row loop
//   is unrolled by two, so the coin output of row r+1 is written straight
//   into the set that is free, with no copies -- and plane 2 of rows r and
//   r-1 (two rows of delay) in a per-warp shared-memory ring of two slots;
// - diagonal lattice: planes 0 and 2 of rows r and r-1, stored already
//   moved in x, plane 0 in registers (two slots per level, selected by the
//   row parity, which the unrolled row loop makes a literal) and plane 2 in
//   the ring; planes 1 and 3 come from the newest row.
// A slot is read (row r-1) and rewritten (row r+1) by the same lane in the
// same level, so the ring needs no synchronisation.
//
// A warp owns a strip of 32R columns (R = 2 per lane) and a chunk of H rows;
// planes that move in x cross lane boundaries with one shuffle each, so the
// valid columns shrink by one per level on both sides (KT columns of halo per
// side, recomputed by the neighbouring strip) and the chunk needs KT rows of
// warm-up below and above.  Rows of psi_0 arrive through a cp.async ring in
// shared memory, TB_RING - 1 rows ahead.  HBM traffic: one read and one write
// of the 4 planes per KT steps, plus the halo.
#pragma once
#include "qw_internal.cuh"
#include "k_step2d.cuh"
#include "k_step1d.cuh"   // wrap_index, cp_async16, cp_async_commit

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
// latency hides behind that many rows of compute.  Each lane copies and reads
// back only its own 16 bytes per plane.
constexpr int TB_RING = 4;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Planes that pass through the shared-memory delay ring: plane 2 on both
// lattices (the diagonal lattice keeps plane 0's two-row delay in registers).
template <int SH> constexpr int tb_delay_planes() { return 1; }

// 16-byte units of shared memory per warp: the input ring ([slot][plane][lane])
// and the delay ring ([level][slot][delayed plane][lane]).
template <int KT, int SH> constexpr int tb_warp_units() { return TB_RING * 4 * 32 + KT * 2 * tb_delay_planes<SH>() * 32; }

// Dynamic shared memory of one 128-thread block.
template <int KT, int SH> constexpr size_t step2d_tb_smem() { return (size_t)(128 / 32) * tb_warp_units<KT, SH>() * 16; }

__device__ __forceinline__ uint4 pack2(const Cx<float> (&v)[2]) {
    return make_uint4(__float_as_uint(v[0].re), __float_as_uint(v[0].im), __float_as_uint(v[1].re),
                      __float_as_uint(v[1].im));
}

// The outputs are the box of columns [ox0, ox0 + ow) and rows [oy0, oy0 + oh)
// (modulo the torus): the whole torus, or the light-cone window of a localised
// state after the launch's KT steps.
template <int P, int KT, int CK, int SH>
__global__ void __launch_bounds__(128)
k_step2d_tb(View in, View out, int64_t nx, int64_t ny, int64_t ox0, int64_t ow, int64_t oy0, int64_t oh, int64_t W,
            int64_t nstrips, int64_t H, int64_t nchunks, CoinP<typename St<P>::real> cp,
            typename St<P>::real gain) {
    using S = St<P>;
    using real = typename S::real;
    using C = Cx<real>;
    constexpr int R = 2;   // sites per lane (one 16-byte vector per plane in FP32)
    static_assert(P == P_F32 && R * S::SLOT_BYTES == 16, "one 16-byte ring slot per lane and plane");
    constexpr bool DIAG = SH == QW_SHIFT_DIAGONAL, FF = SH == QW_SHIFT_FLIPFLOP;
    constexpr int NDP = tb_delay_planes<SH>();
    extern __shared__ __align__(16) unsigned char tsm[];
    const int lane = threadIdx.x & 31;
    uint4 *ring = reinterpret_cast<uint4 *>(tsm) + (size_t)(threadIdx.x >> 5) * tb_warp_units<KT, SH>();
    uint4 *dly = ring + TB_RING * 4 * 32 + lane;   // this lane's delay slots: [level][slot][plane] x 32
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= nstrips * nchunks) return;   // uniform per warp
    const int64_t strip = gw % nstrips, chunk = gw / nstrips;
    const int64_t xo = ox0 + strip * W;                 // first output column (wrapped below)
    const int wthis = (int)min(W, ow - strip * W);
    const int64_t y0 = oy0 + chunk * H;                 // first output row (wrapped below)
    const int64_t hthis = min(H, oh - chunk * H);
    const int j0 = lane * R;                            // tile column of the lane's first site
    const int64_t xs = xo - KT + j0;                    // its global column (may wrap)
    const bool vec = (xs >= 0) && (xs + R <= nx) && (xs % S::VEC == 0) && (R % S::VEC == 0);
    int64_t cx[R];
#pragma unroll
    for (int i = 0; i < R; ++i) cx[i] = wrap_index(xs + i, nx);

    // The delay ring starts at zero.  (Its first values only feed rows of the
    // warm-up band, which are never stored; zeros keep them finite.)
#pragma unroll
    for (int u = 0; u < KT * 2 * NDP; ++u) dly[u * 32] = make_uint4(0, 0, 0, 0);
    // axis lattice: planes 0 and 1 of the previous row per level, two sets
    // alternating with the row parity (the diagonal lattice keeps none)
    constexpr int NA = DIAG ? 1 : KT;
    C Aa[NA][2][R], Ab[NA][2][R];
#pragma unroll
    for (int s = 0; s < NA; ++s)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int i = 0; i < R; ++i) { Aa[s][c][i] = czero<real>(); Ab[s][c][i] = czero<real>(); }
    // diagonal lattice: plane 0 of the rows two and one before the newest, per
    // level, already moved in x ([level][slot parity], as the ring's slots)
    constexpr int ND = DIAG ? KT : 1;
    C D0[ND][2][R];
#pragma unroll
    for (int s = 0; s < ND; ++s)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int i = 0; i < R; ++i) D0[s][q][i] = czero<real>();
    if constexpr (CK == CK_HH) gain = gain * (real)(1.0 / (double)(1u << KT));   // the factors 1/2 of H (x) H
    const bool gain_one = is_one(gain);

    // rows stay within one period of the torus (q is at most one period
    // outside [0, ny)), so a conditional add wraps them
    auto wrap_row = [&](int64_t q) { return q < 0 ? q + ny * ((-q + ny - 1) / ny) : (q >= ny ? q % ny : q); };
    const int64_t qbeg = y0 - KT;
    const int nrows = (int)(hthis + 2 * KT);        // rows qbeg .. qend - 1 pass through the pipeline
    const int64_t nn = nx * ny;
    const int64_t pitch_b = in.pitch * S::SLOT_BYTES;
    const char *inx = static_cast<const char *>(in.p) + xs * S::SLOT_BYTES;   // this lane's columns (vec)
    const char *inb = static_cast<const char *>(in.p);
    // Running element offsets (row * nx) of the next row to copy in and the
    // next row to store, and the count of rows copied in: no per-row division.
    int64_t ld_off = wrap_row(qbeg) * nx, st_off = wrap_row(y0) * nx;
    int ld_cnt = 0;
    // copy the next row of psi_0 (this lane's R sites of each plane) into its
    // ring slot; one commit group per row, empty past the end, so the waits
    // count rows
    auto issue_next = [&]() {
        if (ld_cnt < nrows) {
            uint4 *dst = ring + (ld_cnt & (TB_RING - 1)) * 4 * 32 + lane;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (vec) {
                    cp_async16(dst + c * 32, inx + c * pitch_b + ld_off * S::SLOT_BYTES);
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        cp_async8(reinterpret_cast<unsigned char *>(dst + c * 32) + i * S::SLOT_BYTES,
                                  inb + c * pitch_b + (ld_off + cx[i]) * S::SLOT_BYTES);
                }
            }
            ld_off += nx;
            if (ld_off >= nn) ld_off -= nn;
        }
        ++ld_cnt;
        cp_async_commit();
    };
    // a value of the neighbouring column: from x-1 (left) or from x+1 (right)
    auto from_left = [&](const C (&v)[R], C (&o)[R]) {
        const C l = shfl_up(v[R - 1], 1);
#pragma unroll
        for (int i = R - 1; i > 0; --i) o[i] = v[i - 1];
        o[0] = l;
    };
    auto from_right = [&](const C (&v)[R], C (&o)[R]) {
        const C r = shfl_down(v[0], 1);
#pragma unroll
        for (int i = 0; i < R - 1; ++i) o[i] = v[i + 1];
        o[R - 1] = r;
    };

    // One input row (the rc-th, row qbeg + rc): levels 1..KT, level s
    // producing row qbeg + rc - s of psi_s.  PAR = rc & 1 is a literal at each
    // (inlined) call: it selects the register set read (Ar: the level's input
    // row before the newest) and written (Aw: the newest), and the delay-ring
    // slot.
    auto row = [&](const int PAR, int rc, C (&Ar)[NA][2][R], C (&Aw)[NA][2][R]) {
        issue_next();
        cp_async_wait_pending<TB_RING - 1>();   // row rc has landed
        C N[4][R];                              // coin output of the level's newest input row
        {
            C a[4][R];
            const uint4 *src = ring + (rc & (TB_RING - 1)) * 4 * 32 + lane;
#pragma unroll
            for (int c = 0; c < 4; ++c) S::unpack(src[c * 32], &a[c][0]);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                C ai[4] = {a[0][i], a[1][i], a[2][i], a[3][i]}, pi[4];
                coin4g<CK, real>(cp, ai, pi);
#pragma unroll
                for (int c = 0; c < 4; ++c) N[c][i] = pi[c];
            }
        }
        // ring slot of level s for this row: the newest row and the one two
        // rows before it share a parity; read the old value, write the new.
        // The old values of the next level are loaded one level ahead.
        auto slot_of = [&](int s) { return dly + ((s * 2 + ((PAR + s) & 1)) * NDP) * 32; };
        uint4 dv[NDP];
#pragma unroll
        for (int p = 0; p < NDP; ++p) dv[p] = slot_of(0)[p * 32];
        C psi[4][R];
#pragma unroll
        for (int s = 0; s < KT; ++s) {
            uint4 dn[NDP];
            if (s + 1 < KT) {
#pragma unroll
                for (int p = 0; p < NDP; ++p) dn[p] = slot_of(s + 1)[p * 32];
            }
            uint4 *d = slot_of(s);
            if constexpr (!DIAG) {
                C old2[R];
                S::unpack(dv[0], old2);
                d[0] = pack2(N[2]);
                C m0[R], m1[R];
                from_left(Ar[s][0], m0);      // coin 0 arrives from x-1
                from_right(Ar[s][1], m1);     // coin 1 arrives from x+1
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    psi[FF ? 1 : 0][i] = m0[i];
                    psi[FF ? 0 : 1][i] = m1[i];
                    psi[FF ? 3 : 2][i] = old2[i];   // coin 2 from the row below
                    psi[FF ? 2 : 3][i] = N[3][i];   // coin 3 from the row above
                    Aw[s][0][i] = N[0][i];
                    Aw[s][1][i] = N[1][i];
                }
            } else {
                // planes 0 and 2 are delayed already moved in x, two rows
                // before they are used, so their shuffles stay off this level's
                // dependency chain: plane 0 in registers, plane 2 in the ring
                const int q = (PAR + s) & 1;
                C s0[R], s2[R];
                from_left(N[0], s0);           // to (x+1, y+1) two rows on
                from_right(N[2], s2);          // to (x-1, y+1) two rows on
#pragma unroll
                for (int i = 0; i < R; ++i) psi[0][i] = D0[DIAG ? s : 0][q][i];   // from (x-1, y-1)
                S::unpack(dv[0], psi[2]);      // from (x+1, y-1)
#pragma unroll
                for (int i = 0; i < R; ++i) D0[DIAG ? s : 0][q][i] = s0[i];
                d[0] = pack2(s2);
                from_left(N[1], psi[1]);       // from (x-1, y+1)
                from_right(N[3], psi[3]);      // from (x+1, y+1)
            }
            if (s + 1 < KT) {
#pragma unroll
                for (int p = 0; p < NDP; ++p) dv[p] = dn[p];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    C ai[4] = {psi[0][i], psi[1][i], psi[2][i], psi[3][i]}, pi[4];
                    coin4g<CK, real>(cp, ai, pi);
#pragma unroll
                    for (int c = 0; c < 4; ++c) N[c][i] = pi[c];
                }
            }
        }
        // psi_KT of row qbeg + rc - KT: store the columns whose light cone
        // stayed inside the strip, once the row is at or past y0
        if (rc >= 2 * KT) {
            if (!gain_one) {   // the launch's drift correction, once per KT steps
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int i = 0; i < R; ++i) psi[c][i] = rmul(gain, psi[c][i]);
            }
            if (j0 >= KT && j0 + R <= KT + wthis && vec) {
#pragma unroll
                for (int c = 0; c < 4; ++c) S::stv(out, c, st_off + xs, psi[c]);
            } else if (j0 + R > KT && j0 < KT + wthis) {
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (j0 + i >= KT && j0 + i < KT + wthis)
#pragma unroll
                        for (int c = 0; c < 4; ++c) S::st(out, c, st_off + cx[i], psi[c][i]);
            }
            st_off += nx;
            if (st_off >= nn) st_off -= nn;
        }
    };

#pragma unroll
    for (int r = 0; r < TB_RING - 1; ++r) issue_next();
    int rc = 0;
#pragma unroll 1
    for (; rc + 1 < nrows; rc += 2) {
        row(0, rc, Aa, Ab);
        row(1, rc + 1, Ab, Aa);
    }
    if (rc < nrows) row(0, rc, Aa, Ab);
}

}  // namespace qw
