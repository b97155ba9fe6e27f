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
    // tiled kernels: block (bx, by) runs tile ((tx0 + bx) mod ntx, (ty0 + by) mod nty)
    // of the ntx x nty tiles of the lattice (all of them, or those around the
    // light-cone window of a localised state)
    int tx0, ntx, ty0, nty;
};

// Words 0 and 1 of Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, SC
// 2011) for counter (c0, c1, c2, c3) and key (k0, k1): each round multiplies c0
// and c2 by 0xD2511F53 and 0xCD9E8D57 and mixes the product halves with c1, c3
// and the key, which then grows by (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint2 philox_words01(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(0xD2511F53u, c0), l0 = 0xD2511F53u * c0;
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c2), l1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0; c1 = l1; c2 = n2; c3 = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint2(c0, c1);
}

// Is the link from (lx, ly) to its +axis neighbour broken at random at this
// step?  The site's two links share one draw: word `axis` below the threshold.
__device__ __forceinline__ bool random_closed(const GenGeom &g, int axis, int64_t lx, int64_t ly) {
    const uint64_t v = (uint64_t)(ly * g.nx + lx);
    const uint2 w = philox_words01((uint32_t)v, (uint32_t)(v >> 32), g.rstep, 0u, g.rk0, g.rk1);
    return (axis == 0 ? w.x : w.y) < g.rthr;
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
    if (!closed && g.rthr) closed = random_closed(g, axis, lx, ly);   // broken at random (Sec. 3, RBL)
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

// ---------------------------------------------------------------------------
// The common generic case in 2D tiles: forward step, moving or flip-flop shift,
// one global coin, per-site matrices or phase coins, any boundary, fixed and/or
// random link masks.  A block owns
// GT_X x gt_y<P>() sites.  It computes phi = C psi once for them and a one-site
// halo into shared memory, and the state of every link the tile needs once (a
// site's +x and +y links from one Philox draw), then each site pulls its four
// incoming amplitudes from shared memory.  Global coins of the Grover, H (x) H
// and real classes take their specialised form (as in the lattice kernels);
// other coins the same coin row, in the same order, as k_step_generic, which
// evaluates the coin row and the link again for every output.
constexpr int GT_X = 64, GT_THREADS = 256;
template <int P>
constexpr int gt_y() { return 8; }
// blocks per SM the register budget is sized for: 8 (all 64 warps) for 8-byte
// amplitudes and one global coin, whose 64 x 8 tile takes 21 KB of shared
// memory; 4 for 16-byte amplitudes and for per-site or phase coins (which need
// more than 32 registers)
template <int P, int CK>
constexpr int gt_min_blocks() {
    return (sizeof(Cx<typename St<P>::real>) > 8 || CK == CK_PERSITE || CK == CK_PHASE) ? 4 : 8;
}

// state of the link from (lx, ly) to its +axis neighbour: 0 open, 1 closed
// (reflect), 2 absorbed (line boundary); `rnd` is the site's random draw
__device__ __forceinline__ unsigned char link_state(const GenGeom &g, int axis, int lx, int ly, uint32_t rnd) {
    bool closed = false;
    if (g.links) closed = g.links[axis * g.ns + (int64_t)ly * g.nx + lx] != 0;
    if (g.rthr && rnd < g.rthr) closed = true;
    const bool edge = axis == 0 ? lx == g.nx - 1 : ly == g.ny - 1;
    if (edge && g.bc == QW_BC_SEGMENT) closed = true;
    if (closed) return 1;
    return (edge && g.bc == QW_BC_LINE) ? 2 : 0;
}

template <int P, int SHIFT, int CK>
__global__ void __launch_bounds__(GT_THREADS, gt_min_blocks<P, CK>())
k_step_generic_tile(View in, View out, GenGeom g, CoinP<typename St<P>::real> cp,
                    const Cx<typename St<P>::real> *__restrict__ coins, const float *__restrict__ phi,
                    typename St<P>::real gain) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    constexpr int GY = gt_y<P>();
    constexpr int EX = GT_X + 2, EY = GY + 2;
    __shared__ C ph[4][EY][EX];                        // phi of the tile and its halo
    __shared__ unsigned char ls[2][GY + 1][GT_X + 1];  // link states, owners from (x0 - 1, y0 - 1)
    const int nx = (int)g.nx, ny = (int)g.ny;          // both < 2^31 (launcher)
    int tx = g.tx0 + (int)blockIdx.x, ty = g.ty0 + (int)blockIdx.y;
    if (tx >= g.ntx) tx -= g.ntx;
    if (ty >= g.nty) ty -= g.nty;
    const int x0 = tx * GT_X, y0 = ty * GY;
    // item i of the tile and halo is (ex, ey) = (i mod EX, i div EX), advanced
    // by GT_THREADS items per round without a division
    constexpr int DX = GT_THREADS % EX, DY = GT_THREADS / EX;
    int ex = (int)threadIdx.x % EX, ey = (int)threadIdx.x / EX;
    for (int i = threadIdx.x; i < EX * EY; i += GT_THREADS, ex += DX, ey += DY) {
        if (ex >= EX) { ex -= EX; ++ey; }
        int gx = x0 - 1 + ex, gy = y0 - 1 + ey;       // in [-1, n + GT_X]: wrap
        if (gx < 0) gx += nx;
        while (gx >= nx) gx -= nx;                    // once, unless the lattice is narrower than a tile
        if (gy < 0) gy += ny;
        while (gy >= ny) gy -= ny;
        const int64_t u = (int64_t)gy * nx + gx;
        C a[4], e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = S::ld(in, k, u);
        if constexpr (CK == CK_GROVER || CK == CK_HH || CK == CK_REAL) {
            // a global coin of a class with fewer operations than a full complex
            // matrix (Grover: the vertex sum and one fused multiply-add per row)
            C p[4];
            SiteCoin<real> sc;
            coin4<CK, real>(cp, (const C *)nullptr, sc, a, p);
#pragma unroll
            for (int r = 0; r < 4; ++r) ph[r][ey][ex] = p[r];
        } else {
            if (CK == CK_PHASE) gen_phases<real>(phi, u, 4, e);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                C val = czero<real>();
#pragma unroll
                for (int k = 0; k < 4; ++k) val = cfma(gen_entry<CK, real>(cp, coins, e, 4, u, r, k), a[k], val);
                ph[r][ey][ex] = val;
            }
        }
        if (ex <= GT_X && ey <= GY) {
            uint2 rnd = make_uint2(0u, 0u);
            if (g.rthr) rnd = philox_words01((uint32_t)u, (uint32_t)((uint64_t)u >> 32), g.rstep, 0u, g.rk0, g.rk1);
            ls[0][ey][ex] = link_state(g, 0, gx, gy, rnd.x);
            ls[1][ey][ex] = link_state(g, 1, gx, gy, rnd.y);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GT_X * GY; i += GT_THREADS) {
        const int tx = i % GT_X, ty = i / GT_X;
        const int x = x0 + tx, y = y0 + ty;
        if (x >= nx || y >= ny) continue;
        const int ex = tx + 1, ey = ty + 1;
        const int64_t v = (int64_t)y * nx + x;
#pragma unroll
        for (int co = 0; co < 4; ++co) {
            // the neighbour that feeds (v, co) and the link to it, as in move_along
            int nbx, nby, st;
            if (SHIFT == QW_SHIFT_MOVING) {   // from v - e_co, same coin
                nbx = ex + (co == 0 ? -1 : (co == 1 ? 1 : 0));
                nby = ey + (co == 2 ? -1 : (co == 3 ? 1 : 0));
                st = co == 0 ? ls[0][ey][ex - 1] : (co == 1 ? ls[0][ey][ex] : (co == 2 ? ls[1][ey - 1][ex] : ls[1][ey][ex]));
            } else {                          // from v + e_co, coin co ^ 1
                nbx = ex + (co == 0 ? 1 : (co == 1 ? -1 : 0));
                nby = ey + (co == 2 ? 1 : (co == 3 ? -1 : 0));
                st = co == 0 ? ls[0][ey][ex] : (co == 1 ? ls[0][ey][ex - 1] : (co == 2 ? ls[1][ey][ex] : ls[1][ey - 1][ex]));
            }
            C val = czero<real>();
            if (st == 0) val = ph[SHIFT == QW_SHIFT_MOVING ? co : (co ^ 1)][nby][nbx];
            else if (st == 1) val = ph[SHIFT == QW_SHIFT_MOVING ? (co ^ 1) : co][ey][ex];
            S::st(out, co, v, rmul(gain, val));
        }
    }
}

// The same on the cycle: a block owns GT1_X sites, phi of them and a one-site
// halo in shared memory, the state of links x0 - 1 .. x0 + GT1_X - 1 once.
// 1D coins: 0 moves to x - 1, 1 to x + 1; a site's link (to x + 1) is word 0 of
// its draw.
constexpr int GT1_X = 1024;

template <int P, int SHIFT, int CK>
__global__ void __launch_bounds__(GT_THREADS)
k_step_generic_tile1d(View in, View out, GenGeom g, CoinP<typename St<P>::real> cp,
                      const Cx<typename St<P>::real> *__restrict__ coins, const float *__restrict__ phi,
                      typename St<P>::real gain) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    constexpr int EX = GT1_X + 2;
    __shared__ C ph[2][EX];
    __shared__ unsigned char ls[GT1_X + 1];      // links owned by x0 - 1 .. x0 + GT1_X - 1
    const int nx = (int)g.nx;                    // < 2^31 (launcher)
    int tx = g.tx0 + (int)blockIdx.x;
    if (tx >= g.ntx) tx -= g.ntx;
    const int x0 = tx * GT1_X;
    for (int ex = threadIdx.x; ex < EX; ex += GT_THREADS) {
        int gx = x0 - 1 + ex;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx % nx : gx);
        const C a0 = S::ld(in, 0, gx), a1 = S::ld(in, 1, gx);
        C e[2];
        if (CK == CK_PHASE) gen_phases<real>(phi, gx, 2, e);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            C val = czero<real>();
            val = cfma(gen_entry<CK, real>(cp, coins, e, 2, gx, r, 0), a0, val);
            val = cfma(gen_entry<CK, real>(cp, coins, e, 2, gx, r, 1), a1, val);
            ph[r][ex] = val;
        }
        if (ex <= GT1_X) {
            uint32_t rnd = 0u;
            if (g.rthr) rnd = philox_words01((uint32_t)gx, 0u, g.rstep, 0u, g.rk0, g.rk1).x;
            ls[ex] = link_state(g, 0, gx, 0, rnd);
        }
    }
    __syncthreads();
    for (int tx = threadIdx.x; tx < GT1_X; tx += GT_THREADS) {
        const int x = x0 + tx;
        if (x >= nx) break;
        const int ex = tx + 1;
#pragma unroll
        for (int co = 0; co < 2; ++co) {
            int nb, st;
            if (SHIFT == QW_SHIFT_MOVING) {   // from x + 1 (coin 0) or x - 1 (coin 1), same coin
                nb = co == 0 ? ex + 1 : ex - 1;
                st = co == 0 ? ls[ex] : ls[ex - 1];
            } else {                          // from x - 1 (coin 0) or x + 1 (coin 1), coin co ^ 1
                nb = co == 0 ? ex - 1 : ex + 1;
                st = co == 0 ? ls[ex - 1] : ls[ex];
            }
            C val = czero<real>();
            if (st == 0) val = ph[SHIFT == QW_SHIFT_MOVING ? co : (co ^ 1)][nb];
            else if (st == 1) val = ph[SHIFT == QW_SHIFT_MOVING ? (co ^ 1) : co][ex];
            S::st(out, co, x, rmul(gain, val));
        }
    }
}

}  // namespace qw
