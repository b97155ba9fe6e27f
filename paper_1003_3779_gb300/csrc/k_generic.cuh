// k_generic.cuh -- one walk step for any boundary and any broken-link mask.
//
// The slow, general path: one thread per site, pull form.  It serves the
// finite segment / line boundaries and random broken links of Sec. 3 (the RBL
// function: a closed link sends the amplitude back instead of across), and any
// coin kind the fast kernels do not specialise.  A closed link reflects: the
// amplitude stays on its site in the coin slot the closed link leaves empty
// (c xor 1 for the moving shift, c for the flip-flop shift), so S stays a
// permutation of basis states.  On the line boundary an amplitude crossing the
// lattice edge leaves the simulated window and is dropped.
#pragma once
#include "qw_internal.cuh"
#include "k_step2d.cuh"

namespace qw {

struct GenGeom {
    int ndim;
    int64_t nx, ny, ns;
    int shift, bc;
    const uint8_t *links;
    uint32_t rthr, rk0, rk1, rstep;   // links broken at random at this step (rthr 0: none)
};

// Word 0 of Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, SC 2011)
// for counter (c0, c1, c2, c3) and key (k0, k1): each round multiplies c0 and
// c2 by 0xD2511F53 and 0xCD9E8D57 and mixes the product halves with c1, c3 and
// the key, which then grows by (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(0xD2511F53u, c0), l0 = 0xD2511F53u * c0;
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c2), l1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0; c1 = l1; c2 = n2; c3 = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// Axis and sign of coin c: 1D coin 0 -> -x, coin 1 -> +x; 2D 0 +x, 1 -x, 2 +y, 3 -y.
__device__ __forceinline__ void coin_dir(int ndim, int c, int &axis, int &sgn) {
    if (ndim == 1) { axis = 0; sgn = c == 0 ? -1 : 1; }
    else { axis = c >> 1; sgn = (c & 1) ? -1 : 1; }
}

// The move of (x, y) along coin c: sets the neighbour, and returns the link
// state: 0 open, 1 closed (reflect), 2 absorbed (line boundary).
__device__ __forceinline__ int move_along(const GenGeom &g, int64_t x, int64_t y, int c,
                                          int64_t &nxo, int64_t &nyo) {
    int axis, sgn;
    coin_dir(g.ndim, c, axis, sgn);
    const int64_t n = axis == 0 ? g.nx : g.ny;
    const int64_t p = axis == 0 ? x : y;
    const int64_t lp = sgn > 0 ? p : (p == 0 ? n - 1 : p - 1);   // link (lp, lp+1)
    const bool edge = (lp == n - 1);
    bool closed = false;
    const int64_t lx = axis == 0 ? lp : x, ly = axis == 0 ? y : lp;
    if (g.links) closed = g.links[axis * g.ns + ly * g.nx + lx] != 0;
    if (!closed && g.rthr) {   // broken at random at this step (Sec. 3, the RBL function)
        const uint64_t v = (uint64_t)(ly * g.nx + lx);
        closed = philox_word0((uint32_t)v, (uint32_t)(v >> 32), g.rstep, (uint32_t)axis, g.rk0, g.rk1) < g.rthr;
    }
    if (edge && g.bc == QW_BC_SEGMENT) closed = true;
    int64_t q = p + sgn;
    q = q < 0 ? n - 1 : (q == n ? 0 : q);
    nxo = axis == 0 ? q : x;
    nyo = axis == 0 ? y : q;
    if (closed) return 1;
    if (edge && g.bc == QW_BC_LINE) return 2;
    return 0;
}

template <class R>
__device__ __forceinline__ void gen_phases(const float *phi, int64_t v, int d, Cx<R> *e);
template <>
__device__ __forceinline__ void gen_phases<float>(const float *phi, int64_t v, int d, Cx<float> *e) {
    for (int k = 0; k < d; ++k) { float s, c; sincosf(phi[v * d + k], &s, &c); e[k] = {c, s}; }
}
template <>
__device__ __forceinline__ void gen_phases<double>(const float *phi, int64_t v, int d, Cx<double> *e) {
    for (int k = 0; k < d; ++k) { double s, c; sincos((double)phi[v * d + k], &s, &c); e[k] = {c, s}; }
}
template <>
__device__ __forceinline__ void gen_phases<ff>(const float *phi, int64_t v, int d, Cx<ff> *e) {
    for (int k = 0; k < d; ++k) {
        double s, c;
        sincos((double)phi[v * d + k], &s, &c);
        float ch = (float)c, sh = (float)s;
        e[k] = {{ch, (float)(c - (double)ch)}, {sh, (float)(s - (double)sh)}};
    }
}

// Coin matrix entry C_v[r][k] for the generic path.
template <int CK, class R>
__device__ __forceinline__ Cx<R> gen_entry(const CoinP<R> &cp, const Cx<R> *coins, const Cx<R> *e,
                                           int d, int64_t v, int r, int k) {
    if (CK == CK_PERSITE) return coins[(v * d + r) * d + k];
    Cx<R> b{cp.re[r * d + k], cp.im[r * d + k]};
    if (CK == CK_PHASE) return cmul(b, e[k]);
    return b;
}

template <int P, int CK>
__global__ void __launch_bounds__(128)
k_step_generic(View in, View out, GenGeom g, int adjoint, CoinP<typename St<P>::real> cp,
               const Cx<typename St<P>::real> *__restrict__ coins, const float *__restrict__ phi,
               typename St<P>::real gain) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.ns) return;
    const int d = 2 * g.ndim;
    const int64_t x = v % g.nx, y = v / g.nx;
    C e[4];
    if (g.shift == 2) {   // diagonal lattice (periodic torus): coin c moves by d_c
        if (!adjoint) {
            for (int co = 0; co < 4; ++co) {
                const int64_t ux = (x - dir_dx<2>(co) + g.nx) % g.nx, uy = (y - dir_dy<2>(co) + g.ny) % g.ny;
                const int64_t u = uy * g.nx + ux;
                if (CK == CK_PHASE) gen_phases<real>(phi, u, d, e);
                C val = czero<real>();
                for (int k = 0; k < d; ++k) val = cfma(gen_entry<CK, real>(cp, coins, e, d, u, co, k), S::ld(in, k, u), val);
                S::st(out, co, v, rmul(gain, val));
            }
        } else {
            C b[4];
            for (int c = 0; c < 4; ++c) {
                const int64_t tx = (x + dir_dx<2>(c) + g.nx) % g.nx, ty = (y + dir_dy<2>(c) + g.ny) % g.ny;
                b[c] = S::ld(in, c, ty * g.nx + tx);
            }
            if (CK == CK_PHASE) gen_phases<real>(phi, v, d, e);
            for (int k = 0; k < d; ++k) {
                C acc = czero<real>();
                for (int r = 0; r < d; ++r) acc = cadd(acc, conjmul(gen_entry<CK, real>(cp, coins, e, d, v, r, k), b[r]));
                S::st(out, k, v, rmul(gain, acc));
            }
        }
        return;
    }
    if (!adjoint) {
        for (int co = 0; co < d; ++co) {
            // which (u, c) lands in (v, co)?
            int64_t ux, uy, u;
            int c, st;
            if (g.shift == QW_SHIFT_MOVING) {
                // the move into v along coin co starts at v - e_co; look at that link from v's side
                st = move_along(g, x, y, co ^ 1, ux, uy);  // coin co^1 points from v towards v - e_co
                c = co;
                if (st == 1) { ux = x; uy = y; c = co ^ 1; }
            } else {
                st = move_along(g, x, y, co, ux, uy);      // partner v + e_co sends coin co^1 into (v, co)
                c = co ^ 1;
                if (st == 1) { ux = x; uy = y; c = co; }
            }
            C val = czero<real>();
            if (st != 2) {
                u = uy * g.nx + ux;
                if (CK == CK_PHASE) gen_phases<real>(phi, u, d, e);
                for (int k = 0; k < d; ++k) val = cfma(gen_entry<CK, real>(cp, coins, e, d, u, c, k), S::ld(in, k, u), val);
            }
            S::st(out, co, v, rmul(gain, val));
        }
    } else {
        C b[4];
        for (int c = 0; c < d; ++c) {
            int64_t tx, ty;
            int st = move_along(g, x, y, c, tx, ty);
            if (st == 1) b[c] = S::ld(in, g.shift == QW_SHIFT_FLIPFLOP ? c : (c ^ 1), v);
            else if (st == 2) b[c] = czero<real>();
            else b[c] = S::ld(in, g.shift == QW_SHIFT_FLIPFLOP ? (c ^ 1) : c, ty * g.nx + tx);
        }
        if (CK == CK_PHASE) gen_phases<real>(phi, v, d, e);
        for (int k = 0; k < d; ++k) {
            C acc = czero<real>();
            for (int r = 0; r < d; ++r) acc = cadd(acc, conjmul(gen_entry<CK, real>(cp, coins, e, d, v, r, k), b[r]));
            S::st(out, k, v, rmul(gain, acc));
        }
    }
}

}  // namespace qw
