// k_step2d.cuh -- fused coin + shift on the torus Z_Lx x Z_Ly, coin dimension 4.
//
// The 2D walk of Sec. 2.2 / Sec. 3 with U = S (C (x) I): coin 0 moves +x, 1 -x,
// 2 +y, 3 -y (moving shift), or the same moves into coin c xor 1 (flip-flop).
// A warp owns a row segment of 32*R sites (R per lane).  The coin is applied
// once per site at the source; the two y-moving coin planes are written
// straight into the neighbouring rows (aligned, coalesced stores), and the two
// x-moving planes cross lane boundaries with one warp shuffle each.  The first
// and last lane also evaluate the coin of the one site just outside the
// segment (periodic in x) so the segment edge needs no other warp.  Every
// amplitude is read once and written once: 4 planes in, 4 planes out.
//
// ADJ=1 applies U^dagger = (C^dagger (x) I) S^dagger in pull form: each plane
// is read from the neighbouring row / shuffled from the neighbouring lane, then
// C_v^dagger is applied at the site.
#pragma once
#include "qw_internal.cuh"

namespace qw {

// Per-site data the coin needs besides the amplitudes.
template <class R>
struct SiteCoin {
    Cx<R> e[4];   // CK_PHASE*: e^{i phi_{v,k}}
};

__device__ __forceinline__ void phase_of(const float *phi, int64_t v, SiteCoin<float> &sc) {
    float4 p = __ldg(reinterpret_cast<const float4 *>(phi) + v);
    float s, c;
    sincosf(p.x, &s, &c); sc.e[0] = {c, s};
    sincosf(p.y, &s, &c); sc.e[1] = {c, s};
    sincosf(p.z, &s, &c); sc.e[2] = {c, s};
    sincosf(p.w, &s, &c); sc.e[3] = {c, s};
}
__device__ __forceinline__ void phase_of(const float *phi, int64_t v, SiteCoin<double> &sc) {
    float4 p = __ldg(reinterpret_cast<const float4 *>(phi) + v);
    double s, c;
    sincos((double)p.x, &s, &c); sc.e[0] = {c, s};
    sincos((double)p.y, &s, &c); sc.e[1] = {c, s};
    sincos((double)p.z, &s, &c); sc.e[2] = {c, s};
    sincos((double)p.w, &s, &c); sc.e[3] = {c, s};
}
__device__ __forceinline__ void phase_of(const float *phi, int64_t v, SiteCoin<ff> &sc) {
    // phases are float inputs; the exponential is evaluated in double and split
    float4 p = __ldg(reinterpret_cast<const float4 *>(phi) + v);
    float a[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double s, c;
        sincos((double)a[k], &s, &c);
        float ch = (float)c, sh = (float)s;
        sc.e[k] = {{ch, (float)(c - (double)ch)}, {sh, (float)(s - (double)sh)}};
    }
}

template <int CK> __device__ __forceinline__ constexpr bool needs_phase() {
    return CK == CK_PHASE;
}

// p = C_v a  (d = 4)
template <int CK, class R>
__device__ __forceinline__ void coin4(const CoinP<R> &cp, const Cx<R> *__restrict__ m, const SiteCoin<R> &sc,
                                      const Cx<R> (&a)[4], Cx<R> (&p)[4]) {
    if (CK == CK_GROVER) {
        // G = (1/2) J - I: off-diagonal entries are the 1/2 (cp.re[1]).  p_r =
        // s/2 - a_r as one fused multiply-add: s/2 is exact, so this rounds
        // exactly as the separate multiply and subtraction would.
        Cx<R> s = cadd(cadd(a[0], a[1]), cadd(a[2], a[3]));
#pragma unroll
        for (int r = 0; r < 4; ++r) p[r] = rfma(cp.re[1], s, Cx<R>{-a[r].re, -a[r].im});
    } else if (CK == CK_HH) {
        Cx<R> u0 = cadd(a[0], a[1]), u1 = csub(a[0], a[1]);
        Cx<R> u2 = cadd(a[2], a[3]), u3 = csub(a[2], a[3]);
        R h = cp.re[0];  // every entry of H (x) H is +-1/2
        p[0] = rmul(h, cadd(u0, u2));
        p[1] = rmul(h, cadd(u1, u3));
        p[2] = rmul(h, csub(u0, u2));
        p[3] = rmul(h, csub(u1, u3));
    } else if (CK == CK_REAL) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            Cx<R> acc = rmul(cp.re[4 * r], a[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = rfma(cp.re[4 * r + c], a[c], acc);
            p[r] = acc;
        }
    } else if (CK == CK_COMPLEX || CK == CK_PHASE) {
        Cx<R> b[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = (CK == CK_PHASE) ? cmul(sc.e[c], a[c]) : a[c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            Cx<R> acc = cmul(Cx<R>{cp.re[4 * r], cp.im[4 * r]}, b[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = cfma(Cx<R>{cp.re[4 * r + c], cp.im[4 * r + c]}, b[c], acc);
            p[r] = acc;
        }
    } else {  // CK_PERSITE
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            Cx<R> acc = cmul(m[4 * r], a[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = cfma(m[4 * r + c], a[c], acc);
            p[r] = acc;
        }
    }
}

// a = C_v^dagger b  (d = 4)
template <int CK, class R>
__device__ __forceinline__ void coin4_adj(const CoinP<R> &cp, const Cx<R> *__restrict__ m, const SiteCoin<R> &sc,
                                          const Cx<R> (&b)[4], Cx<R> (&a)[4]) {
    if (CK == CK_GROVER || CK == CK_HH) {
        coin4<CK, R>(cp, m, sc, b, a);  // real symmetric: C^dagger = C
    } else if (CK == CK_REAL) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Cx<R> acc = rmul(cp.re[c], b[0]);
#pragma unroll
            for (int r = 1; r < 4; ++r) acc = rfma(cp.re[4 * r + c], b[r], acc);
            a[c] = acc;
        }
    } else if (CK == CK_COMPLEX || CK == CK_PHASE) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Cx<R> acc = conjmul(Cx<R>{cp.re[c], cp.im[c]}, b[0]);
#pragma unroll
            for (int r = 1; r < 4; ++r) acc = cadd(acc, conjmul(Cx<R>{cp.re[4 * r + c], cp.im[4 * r + c]}, b[r]));
            a[c] = (CK == CK_PHASE) ? conjmul(sc.e[c], acc) : acc;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Cx<R> acc = conjmul(m[c], b[0]);
#pragma unroll
            for (int r = 1; r < 4; ++r) acc = cadd(acc, conjmul(m[4 * r + c], b[r]));
            a[c] = acc;
        }
    }
}

template <int P, int CK>
__device__ __forceinline__ void site_coin(const float *phi, int64_t v, SiteCoin<typename St<P>::real> &sc) {
    if (needs_phase<CK>()) phase_of(phi, v, sc);
}

// Displacement of coin c: 0 +x, 1 -x, 2 +y, 3 -y; on the diagonal lattice
// (SH = 2) coin c = 2j+k moves by ((-1)^j, (-1)^k).
template <int SH> __device__ __forceinline__ int dir_dx(int c) {
    if (SH == 2) return (c >> 1) ? -1 : 1;
    return c == 0 ? 1 : (c == 1 ? -1 : 0);
}
template <int SH> __device__ __forceinline__ int dir_dy(int c) {
    if (SH == 2) return (c & 1) ? -1 : 1;
    return c == 2 ? 1 : (c == 3 ? -1 : 0);
}

// Ragged segment (fewer than 32R sites left in the row): one site per lane
// iteration in plain pull form, recomputing the source site's coin.
template <int P, int CK, int SH, int ADJ>
__device__ void step2d_site(View in, View out, int64_t nx, int64_t ny, int64_t x, int64_t y,
                            const CoinP<typename St<P>::real> &cp, const float *phi,
                            const Cx<typename St<P>::real> *coins, typename St<P>::real gain) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    const int64_t v = y * nx + x;
    if (!ADJ) {
#pragma unroll
        for (int co = 0; co < 4; ++co) {
            const int c = SH == 1 ? (co ^ 1) : co;  // coin that lands in plane co
            const int64_t ux = (x - dir_dx<SH>(c) + nx) % nx, uy = (y - dir_dy<SH>(c) + ny) % ny;
            const int64_t u = uy * nx + ux;
            C a[4], p[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = S::ld(in, k, u);
            SiteCoin<real> sc;
            site_coin<P, CK>(phi, u, sc);
            coin4<CK, real>(cp, coins + 16 * u, sc, a, p);
            S::st(out, co, v, rmul(gain, p[c]));
        }
    } else {
        C b[4], a[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t ux = (x + dir_dx<SH>(c) + nx) % nx, uy = (y + dir_dy<SH>(c) + ny) % ny;
            b[c] = S::ld(in, SH == 1 ? (c ^ 1) : c, uy * nx + ux);
        }
        SiteCoin<real> sc;
        site_coin<P, CK>(phi, v, sc);
        coin4_adj<CK, real>(cp, coins + 16 * v, sc, b, a);
#pragma unroll
        for (int c = 0; c < 4; ++c) S::st(out, c, v, rmul(gain, a[c]));
    }
}

// Warp gw runs row (r0 + gw / ng) mod ny, segment (g0 + gw mod ng) mod segs of
// that row (segments of 32R sites): the whole torus, or the rows and segments
// around the light-cone window of a localised state.
template <int P, int R, int CK, int SH, int ADJ>
__global__ void __launch_bounds__(128)
k_step2d(View in, View out, int64_t nx, int64_t ny, int64_t segs, int64_t r0, int64_t nr, int64_t g0, int64_t ng,
         int64_t nwarps, CoinP<typename St<P>::real> cp, const float *__restrict__ phi,
         const Cx<typename St<P>::real> *__restrict__ coins, typename St<P>::real gain) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= nwarps) return;  // uniform per warp
    const int64_t ry = gw / ng;
    int64_t y = r0 + ry, seg = g0 + (gw - ry * ng);
    if (y >= ny) y -= ny;
    if (seg >= segs) seg -= segs;
    const int64_t x0 = seg * (32 * R);
    const int64_t xs = x0 + lane * R;
    const int64_t row = y * nx;

    if (x0 + 32 * R > nx) {  // ragged tail of the row (uniform per warp)
#pragma unroll 1
        for (int i = 0; i < R; ++i)
            if (xs + i < nx) step2d_site<P, CK, SH, ADJ>(in, out, nx, ny, xs + i, y, cp, phi, coins, gain);
        return;
    }
    const int64_t yp = (y + 1 == ny) ? 0 : y + 1;
    const int64_t ym = (y == 0) ? ny - 1 : y - 1;
    const bool vec_ok = (row % S::VEC) == 0;  // lane sites are VEC-aligned within the row

    if (!ADJ) {
        C a[4][R], p[4][R];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (vec_ok) {
#pragma unroll
                for (int i = 0; i < R; i += S::VEC) S::ldv(in, c, row + xs + i, &a[c][i]);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) a[c][i] = S::ld(in, c, row + xs + i);
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            C ai[4] = {a[0][i], a[1][i], a[2][i], a[3][i]}, pi[4];
            SiteCoin<real> sc;
            site_coin<P, CK>(phi, row + xs + i, sc);
            coin4<CK, real>(cp, coins + 16 * (row + xs + i), sc, ai, pi);
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c][i] = pi[c];
        }
        if (!is_one(gain)) {
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) p[c][i] = rmul(gain, p[c][i]);
        }
        if constexpr (SH == 2) {
            // diagonal lattice: coins 0, 1 arrive from x-1, coins 2, 3 from x+1;
            // coins 0, 2 go to row y+1, coins 1, 3 to row y-1
            C ha = czero<real>(), hb = czero<real>();
            if (lane == 0 || lane == 31) {
                const int64_t xh = (lane == 0) ? (x0 == 0 ? nx - 1 : x0 - 1) : ((x0 + 32 * R) % nx);
                C ah[4], ph[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) ah[c] = S::ld(in, c, row + xh);
                SiteCoin<real> sc;
                site_coin<P, CK>(phi, row + xh, sc);
                coin4<CK, real>(cp, coins + 16 * (row + xh), sc, ah, ph);
                ha = rmul(gain, lane == 0 ? ph[0] : ph[2]);
                hb = rmul(gain, lane == 0 ? ph[1] : ph[3]);
            }
            C f0 = shfl_up(p[0][R - 1], 1), f1 = shfl_up(p[1][R - 1], 1);
            C f2 = shfl_down(p[2][0], 1), f3 = shfl_down(p[3][0], 1);
            if (lane == 0) { f0 = ha; f1 = hb; }
            if (lane == 31) { f2 = ha; f3 = hb; }
            C m0[R], m1[R], m2[R], m3[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                m0[i] = (i == 0) ? f0 : p[0][i - 1];
                m1[i] = (i == 0) ? f1 : p[1][i - 1];
                m2[i] = (i == R - 1) ? f2 : p[2][i + 1];
                m3[i] = (i == R - 1) ? f3 : p[3][i + 1];
            }
            if (vec_ok) {
#pragma unroll
                for (int i = 0; i < R; i += S::VEC) {
                    S::stv(out, 0, yp * nx + xs + i, &m0[i]);
                    S::stv(out, 1, ym * nx + xs + i, &m1[i]);
                    S::stv(out, 2, yp * nx + xs + i, &m2[i]);
                    S::stv(out, 3, ym * nx + xs + i, &m3[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    S::st(out, 0, yp * nx + xs + i, m0[i]);
                    S::st(out, 1, ym * nx + xs + i, m1[i]);
                    S::st(out, 2, yp * nx + xs + i, m2[i]);
                    S::st(out, 3, ym * nx + xs + i, m3[i]);
                }
            }
        } else {
        // coin 0 of the site left of the segment, coin 1 of the site right of it
        C halo = czero<real>();
        if (lane == 0 || lane == 31) {
            const int64_t xh = (lane == 0) ? (x0 == 0 ? nx - 1 : x0 - 1) : ((x0 + 32 * R) % nx);
            C ah[4], ph[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) ah[c] = S::ld(in, c, row + xh);
            SiteCoin<real> sc;
            site_coin<P, CK>(phi, row + xh, sc);
            coin4<CK, real>(cp, coins + 16 * (row + xh), sc, ah, ph);
            halo = rmul(gain, (lane == 0) ? ph[0] : ph[1]);
        }
        C fl = shfl_up(p[0][R - 1], 1);
        C fr = shfl_down(p[1][0], 1);
        if (lane == 0) fl = halo;
        if (lane == 31) fr = halo;
        C m0[R], m1[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            m0[i] = (i == 0) ? fl : p[0][i - 1];      // arrived from x-1 (coin 0 moves +x)
            m1[i] = (i == R - 1) ? fr : p[1][i + 1];  // arrived from x+1 (coin 1 moves -x)
        }
        const int o0 = SH ? 1 : 0, o1 = SH ? 0 : 1, o2 = SH ? 3 : 2, o3 = SH ? 2 : 3;
        if (vec_ok) {
#pragma unroll
            for (int i = 0; i < R; i += S::VEC) {
                S::stv(out, o0, row + xs + i, &m0[i]);
                S::stv(out, o1, row + xs + i, &m1[i]);
                S::stv(out, o2, yp * nx + xs + i, &p[2][i]);
                S::stv(out, o3, ym * nx + xs + i, &p[3][i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                S::st(out, o0, row + xs + i, m0[i]);
                S::st(out, o1, row + xs + i, m1[i]);
                S::st(out, o2, yp * nx + xs + i, p[2][i]);
                S::st(out, o3, ym * nx + xs + i, p[3][i]);
            }
        }
        }
    } else {
        // S^dagger: b_c(x, y) = psi_{src c}(x + e_c)
        C bb0[R], bb1[R], bb2[R], bb3[R];
        if constexpr (SH == 2) {
            // diagonal: b0 = psi0(x+1, y+1), b1 = psi1(x+1, y-1), b2 = psi2(x-1, y+1), b3 = psi3(x-1, y-1)
            C r0[R], r1[R], r2[R], r3[R];
            if (vec_ok) {
#pragma unroll
                for (int i = 0; i < R; i += S::VEC) {
                    S::ldv(in, 0, yp * nx + xs + i, &r0[i]);
                    S::ldv(in, 1, ym * nx + xs + i, &r1[i]);
                    S::ldv(in, 2, yp * nx + xs + i, &r2[i]);
                    S::ldv(in, 3, ym * nx + xs + i, &r3[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    r0[i] = S::ld(in, 0, yp * nx + xs + i);
                    r1[i] = S::ld(in, 1, ym * nx + xs + i);
                    r2[i] = S::ld(in, 2, yp * nx + xs + i);
                    r3[i] = S::ld(in, 3, ym * nx + xs + i);
                }
            }
            const int64_t xr = (x0 + 32 * R) % nx, xl = x0 == 0 ? nx - 1 : x0 - 1;
            C ha = czero<real>(), hb = czero<real>();
            if (lane == 31) { ha = S::ld(in, 0, yp * nx + xr); hb = S::ld(in, 1, ym * nx + xr); }
            if (lane == 0) { ha = S::ld(in, 2, yp * nx + xl); hb = S::ld(in, 3, ym * nx + xl); }
            C g0 = shfl_down(r0[0], 1), g1 = shfl_down(r1[0], 1);
            C g2 = shfl_up(r2[R - 1], 1), g3 = shfl_up(r3[R - 1], 1);
            if (lane == 31) { g0 = ha; g1 = hb; }
            if (lane == 0) { g2 = ha; g3 = hb; }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                bb0[i] = (i == R - 1) ? g0 : r0[i + 1];
                bb1[i] = (i == R - 1) ? g1 : r1[i + 1];
                bb2[i] = (i == 0) ? g2 : r2[i - 1];
                bb3[i] = (i == 0) ? g3 : r3[i - 1];
            }
        } else {
        const int s0 = SH ? 1 : 0, s1 = SH ? 0 : 1, s2 = SH ? 3 : 2, s3 = SH ? 2 : 3;
        C r0[R], r1[R], b2[R], b3[R];
        if (vec_ok) {
#pragma unroll
            for (int i = 0; i < R; i += S::VEC) {
                S::ldv(in, s0, row + xs + i, &r0[i]);
                S::ldv(in, s1, row + xs + i, &r1[i]);
                S::ldv(in, s2, yp * nx + xs + i, &b2[i]);
                S::ldv(in, s3, ym * nx + xs + i, &b3[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                r0[i] = S::ld(in, s0, row + xs + i);
                r1[i] = S::ld(in, s1, row + xs + i);
                b2[i] = S::ld(in, s2, yp * nx + xs + i);
                b3[i] = S::ld(in, s3, ym * nx + xs + i);
            }
        }
        C halo = czero<real>();
        if (lane == 31) halo = S::ld(in, s0, row + ((x0 + 32 * R) % nx));        // for b0 at the right edge
        if (lane == 0) halo = S::ld(in, s1, row + (x0 == 0 ? nx - 1 : x0 - 1));  // for b1 at the left edge
        C fr = shfl_down(r0[0], 1);
        C fl = shfl_up(r1[R - 1], 1);
        if (lane == 31) fr = halo;
        if (lane == 0) fl = halo;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            bb0[i] = (i == R - 1) ? fr : r0[i + 1];
            bb1[i] = (i == 0) ? fl : r1[i - 1];
            bb2[i] = b2[i];
            bb3[i] = b3[i];
        }
        }
        C res[4][R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            C bi[4] = {bb0[i], bb1[i], bb2[i], bb3[i]}, ai[4];
            SiteCoin<real> sc;
            site_coin<P, CK>(phi, row + xs + i, sc);
            coin4_adj<CK, real>(cp, coins + 16 * (row + xs + i), sc, bi, ai);
#pragma unroll
            for (int c = 0; c < 4; ++c) res[c][i] = is_one(gain) ? ai[c] : rmul(gain, ai[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (vec_ok) {
#pragma unroll
                for (int i = 0; i < R; i += S::VEC) S::stv(out, c, row + xs + i, &res[c][i]);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) S::st(out, c, row + xs + i, res[c][i]);
            }
        }
    }
}

}  // namespace qw
