// step2d_tb.cu -- launcher of the streaming temporal-blocking kernel on the torus.
#include <algorithm>

#include "qw_handle.h"
#include "k_step2d_tb.cuh"

namespace qw {

template <int KT, int CK, int SH>
static cudaError_t go2d_tb(const Step2DArgs &a, const CoinP<float> &cp, cudaStream_t s) {
    constexpr int R = 2;
    const int64_t W = 32 * R - 2 * KT;                 // output columns per strip
    // the output box: the whole torus, or the support box widened by KT
    int64_t ox0 = 0, ow = a.nx, oy0 = 0, oh = a.ny;
    if (a.bw > 0) {
        if (a.bw + 2 * KT < a.nx) { ox0 = ((a.bx0 - KT) % a.nx + a.nx) % a.nx; ow = a.bw + 2 * KT; }
        if (a.bh + 2 * KT < a.ny) { oy0 = ((a.by0 - KT) % a.ny + a.ny) % a.ny; oh = a.bh + 2 * KT; }
    }
    const int64_t nstrips = (ow + W - 1) / W;
    constexpr size_t smem = step2d_tb_smem<KT, SH>();
    auto kern = k_step2d_tb<P_F32, KT, CK, SH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // Rows per warp.  Every warp of a launch does about the same work, so the
    // launch takes ceil(warps / resident warps) waves of (H + 2 KT) rows each;
    // pick the row chunk H (at least 8 KT rows, so the 2 KT rows of warm-up
    // stay small) that minimises that product: no last wave that runs nearly
    // empty.
    // resident warps of this instance (looked up once; every device here is the same part)
    static int64_t resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        resident = (int64_t)sms * per_sm * 4;
    }
    int64_t H = std::min<int64_t>(oh, 8 * KT), best = -1;
    for (int64_t nc = 1; nc <= (oh + 8 * KT - 1) / (8 * KT); ++nc) {
        const int64_t h = (oh + nc - 1) / nc;
        if (h < 8 * KT && nc > 1) break;
        const int64_t waves = (nstrips * nc + resident - 1) / resident;
        const int64_t cost = waves * (h + 2 * KT);
        if (best < 0 || cost < best) { best = cost; H = h; }
    }
    H = std::min<int64_t>(H, oh);
    const int64_t nchunks = (oh + H - 1) / H;
    const int64_t nwarps = nstrips * nchunks;
    const int64_t blocks = (nwarps + 3) / 4;
    kern<<<(unsigned)blocks, 128, smem, s>>>(a.in, a.out, a.nx, a.ny, ox0, ow, oy0, oh, W, nstrips, H, nchunks, cp,
                                             (float)a.gain);
    return cudaGetLastError();
}

template <int KT, int CK>
static cudaError_t go2d_tb_shift(const Step2DArgs &a, const CoinP<float> &cp, cudaStream_t s) {
    switch (a.shift) {
        case QW_SHIFT_MOVING: return go2d_tb<KT, CK, QW_SHIFT_MOVING>(a, cp, s);
        case QW_SHIFT_FLIPFLOP: return go2d_tb<KT, CK, QW_SHIFT_FLIPFLOP>(a, cp, s);
        case QW_SHIFT_DIAGONAL: return go2d_tb<KT, CK, QW_SHIFT_DIAGONAL>(a, cp, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int KT>
static cudaError_t go2d_tb_kind(const Step2DArgs &a, const CoinP<float> &cp, cudaStream_t s) {
    switch (a.kind) {
        case CK_REAL: return go2d_tb_shift<KT, CK_REAL>(a, cp, s);
        case CK_COMPLEX: return go2d_tb_shift<KT, CK_COMPLEX>(a, cp, s);
        case CK_GROVER: return go2d_tb_shift<KT, CK_GROVER>(a, cp, s);
        case CK_HH: return go2d_tb_shift<KT, CK_HH>(a, cp, s);
        default: return cudaErrorInvalidValue;
    }
}

bool step2d_tb_ok(int prec, int kind, int K, int shift) {
    return prec == QW_F32 && (K == 4 || K == 8) &&
           (shift == QW_SHIFT_MOVING || shift == QW_SHIFT_FLIPFLOP || shift == QW_SHIFT_DIAGONAL) &&
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
