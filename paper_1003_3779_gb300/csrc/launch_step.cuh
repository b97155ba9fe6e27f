// launch_step.cuh -- host-side launch of the step kernels for one precision.
// Included once per precision by step_<prec>.cu so the template instances of
// each precision compile in their own translation unit (in parallel).
#pragma once
#include "qw_internal.cuh"
#include "k_step1d.cuh"
#include "k_step2d.cuh"
#include "k_generic.cuh"
#include "k_window1d.cuh"

#include <algorithm>

namespace qw {

// Sites per lane compiled for the 1D kernel: two forward tiles, and the
// default tile used by the per-site coin and the adjoint.
template <int P> struct Tiles1D;
template <> struct Tiles1D<P_F32> { static constexpr int A = 8, B = 16, DEF = 16; };
template <> struct Tiles1D<P_BF16> { static constexpr int A = 8, B = 16, DEF = 16; };
template <> struct Tiles1D<P_F64> { static constexpr int A = 4, B = 8, DEF = 8; };
template <> struct Tiles1D<P_COMP> { static constexpr int A = 4, B = 8, DEF = 4; };

// Sites per lane of the 2D kernel (32 bytes of one plane per lane).
template <int P> struct Tile2D { static constexpr int R = 32 / St<P>::SLOT_BYTES < 1 ? 1 : 32 / St<P>::SLOT_BYTES; };
template <> struct Tile2D<P_COMP> { static constexpr int R = 4; };

template <int P, int CK, int FF, int ADJ>
static void go1d_k1(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    using real = typename St<P>::real;
    const int64_t nwarps = (a.n + 32 * St<P>::VEC - 1) / (32 * St<P>::VEC);
    const int64_t blocks = (nwarps + 7) / 8;
    k_step1d_k1<P, CK, FF, ADJ><<<(unsigned)blocks, 256, 0, s>>>(
        a.in, a.out, a.n, nwarps, cp, static_cast<const Cx<real> *>(a.coins),
        real_from_double<real>(a.pre0), real_from_double<real>(a.pre1),
        real_from_double<real>(a.post0), real_from_double<real>(a.post1));
}

template <int P, int ADJ>
static bool go1d_k1_kind(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    const bool ff = a.shift == QW_SHIFT_FLIPFLOP;
    switch (a.kind) {
        case CK_REAL: ff ? go1d_k1<P, CK_REAL, 1, ADJ>(a, cp, s) : go1d_k1<P, CK_REAL, 0, ADJ>(a, cp, s); return true;
        case CK_COMPLEX: ff ? go1d_k1<P, CK_COMPLEX, 1, ADJ>(a, cp, s) : go1d_k1<P, CK_COMPLEX, 0, ADJ>(a, cp, s); return true;
        case CK_PERSITE: ff ? go1d_k1<P, CK_PERSITE, 1, ADJ>(a, cp, s) : go1d_k1<P, CK_PERSITE, 0, ADJ>(a, cp, s); return true;
        case CK_SIGN_P: if (ff) return false; go1d_k1<P, CK_SIGN_P, 0, ADJ>(a, cp, s); return true;
        case CK_SIGN_M: if (ff) return false; go1d_k1<P, CK_SIGN_M, 0, ADJ>(a, cp, s); return true;
        default: return false;
    }
}

// Outputs per warp of the temporal-blocking kernel: a multiple of VEC with
// 32R >= W + 2K + VEC - 1 (the tile origin is rounded down to VEC).
template <int P>
inline int64_t outputs_per_warp(int R, int K) {
    constexpr int V = St<P>::VEC;
    return (32LL * R - 2LL * K - (V - 1)) / V * V;
}

template <int P, int R, int CK, int FF, int ADJ>
static void go1d(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    const int64_t W = outputs_per_warp<P>(R, a.K);
    const bool win = a.oend > a.obeg;   // a light-cone window, else the whole cycle
    const int64_t ob = win ? a.obeg : 0, oe = win ? a.oend : a.n;
    const int64_t nwarps = (oe - ob + W - 1) / W;
    const int64_t blocks = (nwarps + 3) / 4;
    k_step1d<P, R, CK, FF, ADJ><<<(unsigned)blocks, 128, 0, s>>>(
        a.in, a.out, a.n, a.K, W, ob, oe, nwarps, cp,
        static_cast<const Cx<typename St<P>::real> *>(a.coins),
        real_from_double<typename St<P>::real>(a.pre0), real_from_double<typename St<P>::real>(a.pre1),
        real_from_double<typename St<P>::real>(a.post0), real_from_double<typename St<P>::real>(a.post1));
}

template <int P, int R, int ADJ>
static bool go1d_kind(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    const bool ff = a.shift == QW_SHIFT_FLIPFLOP;
    switch (a.kind) {
        case CK_REAL: ff ? go1d<P, R, CK_REAL, 1, ADJ>(a, cp, s) : go1d<P, R, CK_REAL, 0, ADJ>(a, cp, s); return true;
        case CK_COMPLEX: ff ? go1d<P, R, CK_COMPLEX, 1, ADJ>(a, cp, s) : go1d<P, R, CK_COMPLEX, 0, ADJ>(a, cp, s); return true;
        case CK_SIGN_P: if (ff) return false; go1d<P, R, CK_SIGN_P, 0, ADJ>(a, cp, s); return true;
        case CK_SIGN_M: if (ff) return false; go1d<P, R, CK_SIGN_M, 0, ADJ>(a, cp, s); return true;
        default: return false;
    }
}

// Sites per lane compiled for the sweep kernel (R * SLOT_BYTES / 16 = 2..16
// sixteen-byte units per lane and plane); the double-float form has none.
// The larger tile halves the per-level overhead (edge hand-over, shuffles)
// per site and allows deeper k; the smaller one takes cycles that are a
// multiple of half its chunk.
template <int P> struct SweepTiles { static constexpr int A = 16, B = 32; };
template <> struct SweepTiles<P_F64> { static constexpr int A = 8, B = 8; };
template <> struct SweepTiles<P_COMP> { static constexpr int A = 0, B = 0; };

// The sites per lane a sweep plan with this tile runs on a cycle of n sites:
// the requested tile if it is compiled, else the larger tile when the cycle
// holds at least two of its chunks, else the smaller one.
template <int P>
int sweep_tile(int64_t n, int tile) {
    using T = SweepTiles<P>;
    if constexpr (T::A == 0) {
        return 0;
    } else {
        if (tile == T::A || tile == T::B) return tile;
        return n >= 2 * 32LL * T::B ? T::B : T::A;
    }
}

template <int P, int R, int CK, int FF, int ADJ>
static cudaError_t go1d_sweep(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    using real = typename St<P>::real;
    using SW = Sweep<P, R>;
    constexpr int warps = 4;
    const size_t smem = warps * SW::warp_bytes(a.K);
    auto kfn = k_step1d_sweep<P, R, CK, FF, ADJ>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // Segments sized so that the whole launch is one wave of resident warps:
    // every warp sweeps about the same number of chunks, and the one warm-up
    // chunk per segment is a small fraction of it.
    int nch = a.chunks;
    if (nch <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * warps, smem);
        const int64_t resident = (int64_t)std::max(1, sms) * std::max(1, per_sm) * warps;
        const int64_t chunks = (a.n + SW::B - 1) / SW::B;
        nch = (int)std::max<int64_t>(1, (chunks + resident - 1) / resident);
    }
    const int64_t nseg = ((a.n + SW::B - 1) / SW::B + nch - 1) / nch;
    const int64_t blocks = (nseg + warps - 1) / warps;
    kfn<<<(unsigned)blocks, 32 * warps, smem, s>>>(a.in, a.out, a.n, a.K, nch, nseg, cp,
                                                  real_from_double<real>(a.pre0), real_from_double<real>(a.pre1),
                                                  real_from_double<real>(a.post0), real_from_double<real>(a.post1));
    return cudaGetLastError();
}

template <int P, int R, int ADJ>
static cudaError_t go1d_sweep_kind(const Step1DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    const bool ff = a.shift == QW_SHIFT_FLIPFLOP;
    switch (a.kind) {
        case CK_REAL: return ff ? go1d_sweep<P, R, CK_REAL, 1, ADJ>(a, cp, s) : go1d_sweep<P, R, CK_REAL, 0, ADJ>(a, cp, s);
        case CK_COMPLEX: return ff ? go1d_sweep<P, R, CK_COMPLEX, 1, ADJ>(a, cp, s) : go1d_sweep<P, R, CK_COMPLEX, 0, ADJ>(a, cp, s);
        case CK_SIGN_P: return ff ? cudaErrorInvalidValue : go1d_sweep<P, R, CK_SIGN_P, 0, ADJ>(a, cp, s);
        case CK_SIGN_M: return ff ? cudaErrorInvalidValue : go1d_sweep<P, R, CK_SIGN_M, 0, ADJ>(a, cp, s);
        default: return cudaErrorInvalidValue;
    }
}

// Can the sweep kernel run this launch?  (n at least the chunk of the tile
// sweep_tile picks, 2 <= K < chunk / 2.)
template <int P>
bool sweep_ok(int64_t n, int K, int kind, int tile) {
    if (P == P_COMP || kind == CK_PERSITE || kind == CK_PHASE) return false;
    const int64_t B = 32LL * sweep_tile<P>(n, tile);
    return B > 0 && n >= B && K >= 2 && K <= B / 2 - 1;
}

// Largest K the 1D kernel accepts for tile R: at least half the tile is output.
inline int max_k_1d(int R) { return 8 * R; }

template <int P>
int tile1d_effective(int tile, int kind, int adj) {
    using T = Tiles1D<P>;
    if (adj || kind == CK_PERSITE) return T::DEF;
    return (tile == T::A || tile == T::B) ? tile : T::DEF;
}

template <int P>
cudaError_t step1d_t(const Step1DArgs &a0, const void *coinp, int adj, cudaStream_t s) {
    using T = Tiles1D<P>;
    const auto &cp = *static_cast<const CoinP<typename St<P>::real> *>(coinp);
    Step1DArgs a = a0;
    if (a.variant == 1) {   // time-skewed sweep
        if constexpr (P == P_COMP) {
            return cudaErrorInvalidValue;
        } else {
            using ST = SweepTiles<P>;
            if (!sweep_ok<P>(a.n, a.K, a.kind, a.tile)) return cudaErrorInvalidValue;
            if (sweep_tile<P>(a.n, a.tile) == ST::B)
                return adj ? go1d_sweep_kind<P, ST::B, 1>(a, cp, s) : go1d_sweep_kind<P, ST::B, 0>(a, cp, s);
            return adj ? go1d_sweep_kind<P, ST::A, 1>(a, cp, s) : go1d_sweep_kind<P, ST::A, 0>(a, cp, s);
        }
    }
    a.tile = tile1d_effective<P>(a.tile, a.kind, adj);
    if (a.K < 1 || a.K > max_k_1d(a.tile)) return cudaErrorInvalidValue;
    const bool ff = a.shift == QW_SHIFT_FLIPFLOP;
    if (a.K == 1 && a.oend <= a.obeg) {   // one step per launch over the whole cycle: the streaming kernel
        const bool ok = adj ? go1d_k1_kind<P, 1>(a, cp, s) : go1d_k1_kind<P, 0>(a, cp, s);
        return ok ? cudaGetLastError() : cudaErrorInvalidValue;
    }
    if (!adj) {
        if (a.kind == CK_PERSITE) {
            ff ? go1d<P, T::DEF, CK_PERSITE, 1, 0>(a, cp, s) : go1d<P, T::DEF, CK_PERSITE, 0, 0>(a, cp, s);
        } else if (a.tile == T::A) {
            if (!go1d_kind<P, T::A, 0>(a, cp, s)) return cudaErrorInvalidValue;
        } else {
            if (!go1d_kind<P, T::B, 0>(a, cp, s)) return cudaErrorInvalidValue;
        }
    } else {
        if (a.kind == CK_PERSITE) {
            ff ? go1d<P, T::DEF, CK_PERSITE, 1, 1>(a, cp, s) : go1d<P, T::DEF, CK_PERSITE, 0, 1>(a, cp, s);
        } else if (!go1d_kind<P, T::DEF, 1>(a, cp, s)) {
            return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <int P, int CK, int FF, int ADJ>
static void go2d(const Step2DArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    // per-site phase coins in FP32: two sites per lane, for more warps in flight
    // (the step is latency-bound at 1024^2: 17.7 against 20.5 us per step with four)
    constexpr int R = (CK == CK_PHASE && P == P_F32) ? 2 : Tile2D<P>::R;
    const int64_t segs = (a.nx + 32 * R - 1) / (32 * R);
    // Rows and row segments to run.  A warp reads its row and writes planes to
    // the rows above and below; x-moving planes arrive from the neighbouring
    // columns.  So a state supported on the box [bx0, bx0 + bw) x [by0, by0 + bh)
    // needs the rows and columns of the box widened by one on each side (the
    // adjoint pulls from the same neighbours): every other output is zero and
    // already zero in the output buffer.
    int64_t r0 = 0, nr = a.ny, g0 = 0, ng = segs;
    if (a.bw > 0) {
        if (a.bh + 2 < a.ny) { r0 = (a.by0 - 1 + a.ny) % a.ny; nr = a.bh + 2; }
        if (a.bw + 2 < a.nx) {
            // columns [c0, c0 + cw) modulo nx; the last segment of a row may be short
            const int64_t c0 = (a.bx0 - 1 + a.nx) % a.nx, cw = a.bw + 2, S = 32 * R;
            g0 = c0 / S;
            ng = c0 + cw <= a.nx ? (c0 + cw - 1) / S - g0 + 1 : (segs - g0) + (c0 + cw - a.nx - 1) / S + 1;
            ng = std::min<int64_t>(segs, ng);
        }
    }
    const int64_t nwarps = ng * nr;
    const int64_t blocks = (nwarps + 3) / 4;
    k_step2d<P, R, CK, FF, ADJ><<<(unsigned)blocks, 128, 0, s>>>(
        a.in, a.out, a.nx, a.ny, segs, r0, nr, g0, ng, nwarps, cp, a.phi,
        static_cast<const Cx<typename St<P>::real> *>(a.coins),
        real_from_double<typename St<P>::real>(a.gain));
}

template <int P, int CK>
static void go2d_ff(const Step2DArgs &a, const CoinP<typename St<P>::real> &cp, int adj, cudaStream_t s) {
    switch (a.shift) {
        case QW_SHIFT_FLIPFLOP: adj ? go2d<P, CK, 1, 1>(a, cp, s) : go2d<P, CK, 1, 0>(a, cp, s); break;
        case QW_SHIFT_DIAGONAL: adj ? go2d<P, CK, 2, 1>(a, cp, s) : go2d<P, CK, 2, 0>(a, cp, s); break;
        default: adj ? go2d<P, CK, 0, 1>(a, cp, s) : go2d<P, CK, 0, 0>(a, cp, s); break;
    }
}

// Does the fast 2D kernel of precision P handle this coin kind?
template <int P>
constexpr bool fast2d_has_phase() { return P == P_F32 || P == P_F64; }

template <int P>
cudaError_t step2d_t(const Step2DArgs &a, const void *coinp, int adj, cudaStream_t s) {
    const auto &cp = *static_cast<const CoinP<typename St<P>::real> *>(coinp);
    switch (a.kind) {
        case CK_REAL: go2d_ff<P, CK_REAL>(a, cp, adj, s); break;
        case CK_COMPLEX: go2d_ff<P, CK_COMPLEX>(a, cp, adj, s); break;
        case CK_GROVER: go2d_ff<P, CK_GROVER>(a, cp, adj, s); break;
        case CK_HH: go2d_ff<P, CK_HH>(a, cp, adj, s); break;
        case CK_PHASE:
            if constexpr (fast2d_has_phase<P>()) { go2d_ff<P, CK_PHASE>(a, cp, adj, s); break; }
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

// Tiles of T sites along an axis of n sites that hold the outputs of one step
// from a state supported on [c0, c0 + cw): that range widened by one site on
// each side (modulo n on the periodic lattice, cut at its ends otherwise).
// The last tile may be short.  cw = 0: every tile.
static inline void tile_range(int64_t c0, int64_t cw, int64_t n, int T, bool periodic, int &t0, int &nt) {
    const int64_t ntiles = (n + T - 1) / T;
    t0 = 0;
    nt = (int)ntiles;
    if (cw <= 0) return;
    int64_t a0, aw;
    if (periodic) {
        if (cw + 2 >= n) return;
        a0 = (c0 - 1 + n) % n;
        aw = cw + 2;
    } else {
        a0 = std::max<int64_t>(0, c0 - 1);
        aw = std::min<int64_t>(n, c0 + cw + 1) - a0;
    }
    t0 = (int)(a0 / T);
    const int64_t k = a0 + aw <= n ? (a0 + aw - 1) / T - t0 + 1 : (ntiles - t0) + (a0 + aw - n - 1) / T + 1;
    nt = (int)std::min<int64_t>(ntiles, k);
}

template <int P, int CK>
static void gogen(const StepGenericArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    GenGeom g{a.ndim, a.nx, a.ny, a.nx * a.ny, a.shift, a.bc, a.links, a.rthr, a.rk0, a.rk1, a.rstep, 0, 1, 0, 1};
    const int64_t blocks = (g.ns + 127) / 128;
    k_step_generic<P, CK><<<(unsigned)blocks, 128, 0, s>>>(
        a.in, a.out, g, a.adjoint, cp, static_cast<const Cx<typename St<P>::real> *>(a.coins), a.phi,
        real_from_double<typename St<P>::real>(a.gain));
}

// The tiled forms serve the forward step on the axis lattice (1D and 2D; any
// coin, boundary and links); the grid's y extent limits ny to 65535 tiles.
template <int P>
static bool generic_tile_ok(const StepGenericArgs &a) {
    if (a.adjoint || !(a.shift == QW_SHIFT_MOVING || a.shift == QW_SHIFT_FLIPFLOP) || a.nx >= (int64_t(1) << 30))
        return false;
    return a.ndim == 1 || (a.ny + gt_y<P>() - 1) / gt_y<P>() <= 65535;
}

template <int P, int CK>
static void gotile(const StepGenericArgs &a, const CoinP<typename St<P>::real> &cp, cudaStream_t s) {
    using real = typename St<P>::real;
    const bool per = a.bc == QW_BC_PERIODIC;
    GenGeom g{a.ndim, a.nx, a.ny, a.nx * a.ny, a.shift, a.bc, a.links, a.rthr, a.rk0, a.rk1, a.rstep, 0, 1, 0, 1};
    const auto gain = real_from_double<real>(a.gain);
    const auto *coins = static_cast<const Cx<real> *>(a.coins);
    if (a.ndim == 1) {
        if constexpr (CK == CK_COMPLEX || CK == CK_PERSITE || CK == CK_PHASE) {   // (the 1D tiles take these)
            tile_range(a.bx0, a.bw, a.nx, GT1_X, per, g.tx0, g.ntx);
            const unsigned grid = (unsigned)g.ntx;
            g.ntx = (int)((a.nx + GT1_X - 1) / GT1_X);
            if (a.shift == QW_SHIFT_MOVING)
                k_step_generic_tile1d<P, QW_SHIFT_MOVING, CK><<<grid, GT_THREADS, 0, s>>>(a.in, a.out, g, cp, coins, a.phi, gain);
            else
                k_step_generic_tile1d<P, QW_SHIFT_FLIPFLOP, CK><<<grid, GT_THREADS, 0, s>>>(a.in, a.out, g, cp, coins, a.phi, gain);
        }
        return;
    }
    int gx = 0, gy = 0;
    tile_range(a.bx0, a.bw, a.nx, GT_X, per, g.tx0, gx);
    tile_range(a.by0, a.bw > 0 ? a.bh : 0, a.ny, gt_y<P>(), per, g.ty0, gy);
    g.ntx = (int)((a.nx + GT_X - 1) / GT_X);
    g.nty = (int)((a.ny + gt_y<P>() - 1) / gt_y<P>());
    const dim3 grid((unsigned)gx, (unsigned)gy);
    if (a.shift == QW_SHIFT_MOVING)
        k_step_generic_tile<P, QW_SHIFT_MOVING, CK><<<grid, GT_THREADS, 0, s>>>(a.in, a.out, g, cp, coins, a.phi, gain);
    else
        k_step_generic_tile<P, QW_SHIFT_FLIPFLOP, CK><<<grid, GT_THREADS, 0, s>>>(a.in, a.out, g, cp, coins, a.phi, gain);
}

template <int P>
cudaError_t generic_t(const StepGenericArgs &a, const void *coinp, cudaStream_t s) {
    const auto &cp = *static_cast<const CoinP<typename St<P>::real> *>(coinp);
    if (generic_tile_ok<P>(a)) {
        const bool d2 = a.ndim == 2;   // the 2D tiles specialise the global coin classes
        switch (a.kind) {
            case CK_PERSITE: gotile<P, CK_PERSITE>(a, cp, s); break;
            case CK_PHASE: gotile<P, CK_PHASE>(a, cp, s); break;
            case CK_GROVER: d2 ? gotile<P, CK_GROVER>(a, cp, s) : gotile<P, CK_COMPLEX>(a, cp, s); break;
            case CK_HH: d2 ? gotile<P, CK_HH>(a, cp, s) : gotile<P, CK_COMPLEX>(a, cp, s); break;
            case CK_REAL: d2 ? gotile<P, CK_REAL>(a, cp, s) : gotile<P, CK_COMPLEX>(a, cp, s); break;
            default: gotile<P, CK_COMPLEX>(a, cp, s); break;   // other global coins as a full matrix
        }
        return cudaGetLastError();
    }
    switch (a.kind) {
        case CK_PERSITE: gogen<P, CK_PERSITE>(a, cp, s); break;
        case CK_PHASE: gogen<P, CK_PHASE>(a, cp, s); break;
        default: gogen<P, CK_COMPLEX>(a, cp, s); break;  // every global coin as a full matrix
    }
    return cudaGetLastError();
}

// The 1D window kernel (a clipped forward walk on the segment or the line,
// nsteps steps in one CTA); gains[i] is the drift gain of step i, a.rstep the
// random-link step of the first.  cudaErrorInvalidValue if the window after
// the steps is wider than win_capacity<P>() or nsteps is out of [1, WIN_MAX_STEPS].
template <int P, int CK, int SHIFT>
static cudaError_t gowin_shift(const StepGenericArgs &a, const CoinP<typename St<P>::real> &cp, const double *gains,
                               int nsteps, cudaStream_t s) {
    using real = typename St<P>::real;
    const int64_t w0 = std::max<int64_t>(0, a.bx0 - nsteps), w1 = std::min<int64_t>(a.nx, a.bx0 + a.bw + nsteps);
    const int64_t wn = w1 - w0;
    if (nsteps < 1 || nsteps > WIN_MAX_STEPS || wn < 1 || wn > win_capacity<P>() || a.bc == QW_BC_PERIODIC)
        return cudaErrorInvalidValue;
    GenGeom g{a.ndim, a.nx, a.ny, a.nx * a.ny, a.shift, a.bc, a.links, a.rthr, a.rk0, a.rk1, a.rstep, 0, 1, 0, 1};
    WinGains<real> gv{};
    for (int i = 0; i < nsteps; ++i) gv.v[i] = real_from_double<real>(gains[i]);
    const bool links = a.links != nullptr || a.rthr != 0;
    auto kfn = links ? k_step1d_window<P, SHIFT, CK, true> : k_step1d_window<P, SHIFT, CK, false>;
    // (set on every launch: the attribute is the current device's, and a launch runs up to 256 steps)
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WIN_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    kfn<<<1, WIN_THREADS, win_smem<P>(wn), s>>>(a.in, a.out, g, cp, static_cast<const Cx<real> *>(a.coins), a.phi,
                                                 (int)a.bx0, (int)a.bw, nsteps, (int)w0, (int)wn, gv);
    return cudaGetLastError();
}

template <int P, int CK>
static cudaError_t gowin(const StepGenericArgs &a, const CoinP<typename St<P>::real> &cp, const double *gains, int nsteps,
                         cudaStream_t s) {
    if (a.shift == QW_SHIFT_MOVING) return gowin_shift<P, CK, QW_SHIFT_MOVING>(a, cp, gains, nsteps, s);
    if (a.shift == QW_SHIFT_FLIPFLOP) return gowin_shift<P, CK, QW_SHIFT_FLIPFLOP>(a, cp, gains, nsteps, s);
    return cudaErrorInvalidValue;
}

template <int P>
cudaError_t window1d_t(const StepGenericArgs &a, const void *coinp, const double *gains, int nsteps, cudaStream_t s) {
    const auto &cp = *static_cast<const CoinP<typename St<P>::real> *>(coinp);
    if (a.ndim != 1 || a.adjoint || a.nx >= (int64_t(1) << 30)) return cudaErrorInvalidValue;
    switch (a.kind) {   // the coins of the 1D tiles: global coins as the full matrix
        case CK_PERSITE: return gowin<P, CK_PERSITE>(a, cp, gains, nsteps, s);
        case CK_PHASE: return gowin<P, CK_PHASE>(a, cp, gains, nsteps, s);
        default: return gowin<P, CK_COMPLEX>(a, cp, gains, nsteps, s);
    }
}

}  // namespace qw

// One translation unit per precision defines these entry points.
#define QW_DEFINE_STEP_LAUNCHERS(PREC, SUFFIX)                                                          \
    namespace qw {                                                                                      \
    cudaError_t launch_step1d_##SUFFIX(const Step1DArgs &a, const void *cp, int adj, cudaStream_t s) {  \
        return step1d_t<PREC>(a, cp, adj, s);                                                           \
    }                                                                                                   \
    cudaError_t launch_step2d_##SUFFIX(const Step2DArgs &a, const void *cp, int adj, cudaStream_t s) {  \
        return step2d_t<PREC>(a, cp, adj, s);                                                           \
    }                                                                                                   \
    cudaError_t launch_generic_##SUFFIX(const StepGenericArgs &a, const void *cp, cudaStream_t s) {     \
        return generic_t<PREC>(a, cp, s);                                                               \
    }                                                                                                   \
    cudaError_t launch_window1d_##SUFFIX(const StepGenericArgs &a, const void *cp, const double *gains,  \
                                         int nsteps, cudaStream_t s) {                                  \
        return window1d_t<PREC>(a, cp, gains, nsteps, s);                                               \
    }                                                                                                   \
    int64_t window1d_capacity_##SUFFIX() { return win_capacity<PREC>(); }                               \
    int tile1d_##SUFFIX(int tile, int kind, int adj) { return tile1d_effective<PREC>(tile, kind, adj); } \
    bool sweep_ok_##SUFFIX(int64_t n, int K, int kind, int tile) { return sweep_ok<PREC>(n, K, kind, tile); } \
    int sweep_tile_##SUFFIX(int64_t n, int tile) { return sweep_tile<PREC>(n, tile); }                   \
    }
