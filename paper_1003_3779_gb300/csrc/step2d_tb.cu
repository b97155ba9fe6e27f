// step2d_tb.cu -- launcher of the streaming temporal-blocking kernel on the torus.
#include <algorithm>

#include "qw_handle.h"
#include "k_step2d_tb.cuh"

namespace qw {

template <int KT, int CK, int FF>
static cudaError_t go2d_tb(const Step2DArgs &a, const CoinP<float> &cp, cudaStream_t s) {
    constexpr int R = 2;
    const int64_t W = 32 * R - 2 * KT;                 // output columns per strip
    const int64_t nstrips = (a.nx + W - 1) / W;
    // rows per warp: enough warps for about three waves of resident warps,
    // and at least 8 KT rows so the 2 KT rows of warm-up stay small
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t target = (int64_t)sms * 16 * 3;
    const int64_t want_chunks = std::max<int64_t>(1, (target + nstrips - 1) / nstrips);
    int64_t H = std::max<int64_t>(8 * KT, (a.ny + want_chunks - 1) / want_chunks);
    H = std::min<int64_t>(H, a.ny);
    const int64_t nchunks = (a.ny + H - 1) / H;
    const int64_t nwarps = nstrips * nchunks;
    const int64_t blocks = (nwarps + 3) / 4;
    k_step2d_tb<P_F32, KT, CK, FF><<<(unsigned)blocks, 128, step2d_tb_smem(), s>>>(a.in, a.out, a.nx, a.ny, W, nstrips,
                                                                                 H, nchunks, cp, (float)a.gain);
    return cudaGetLastError();
}

template <int KT>
static cudaError_t go2d_tb_kind(const Step2DArgs &a, const CoinP<float> &cp, cudaStream_t s) {
    const bool ff = a.shift == QW_SHIFT_FLIPFLOP;
    switch (a.kind) {
        case CK_REAL: return ff ? go2d_tb<KT, CK_REAL, 1>(a, cp, s) : go2d_tb<KT, CK_REAL, 0>(a, cp, s);
        case CK_COMPLEX: return ff ? go2d_tb<KT, CK_COMPLEX, 1>(a, cp, s) : go2d_tb<KT, CK_COMPLEX, 0>(a, cp, s);
        case CK_GROVER: return ff ? go2d_tb<KT, CK_GROVER, 1>(a, cp, s) : go2d_tb<KT, CK_GROVER, 0>(a, cp, s);
        case CK_HH: return ff ? go2d_tb<KT, CK_HH, 1>(a, cp, s) : go2d_tb<KT, CK_HH, 0>(a, cp, s);
        default: return cudaErrorInvalidValue;
    }
}

bool step2d_tb_ok(int prec, int kind, int K, int shift) {
    return prec == QW_F32 && (K == 4 || K == 8) && shift != QW_SHIFT_DIAGONAL &&
           (kind == CK_REAL || kind == CK_COMPLEX || kind == CK_GROVER || kind == CK_HH);
}

// K steps (K = 4 or 8) in one launch; the gain (drift correction) is applied
// once, to the launch's output.
cudaError_t launch_step2d_tb(const Step2DArgs &a, const void *coinp, cudaStream_t s) {
    const auto &cp = *static_cast<const CoinP<float> *>(coinp);
    switch (a.K) {
        case 4: return go2d_tb_kind<4>(a, cp, s);
        case 8: return go2d_tb_kind<8>(a, cp, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qw
