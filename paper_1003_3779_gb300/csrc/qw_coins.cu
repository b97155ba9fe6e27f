// qw_coins.cu -- per-site coin set-up kernels.
//
// The coin flip transformation of Sec. 2.1 may differ from site to site
// (C = (C_v)_v).  The caller gives per-site matrices in double; they are
// rounded once to the compute precision here.  A phase coin
// C_v = B . diag(e^{i phi_{v,k}}) on the cycle is expanded to per-site matrices
// (the 1D kernels keep a site's matrix in registers for the whole launch).
#include "qw_handle.h"

namespace qw {

template <class R> __device__ __forceinline__ Cx<R> from_double(double re, double im);
template <> __device__ __forceinline__ Cx<float> from_double<float>(double re, double im) { return {(float)re, (float)im}; }
template <> __device__ __forceinline__ Cx<double> from_double<double>(double re, double im) { return {re, im}; }
template <> __device__ __forceinline__ Cx<ff> from_double<ff>(double re, double im) {
    float rh = (float)re, ih = (float)im;
    return {{rh, (float)(re - (double)rh)}, {ih, (float)(im - (double)ih)}};
}

template <class R>
__global__ void k_convert_coins(const double *src, Cx<R> *dst, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = from_double<R>(src[2 * i], src[2 * i + 1]);
}

// dst[(v*d + r)*d + k] = base[r][k] * e^{i phi[v*d + k]}, evaluated in double
template <class R>
__global__ void k_phase_coins(const double *base, const float *phi, Cx<R> *dst, int64_t ns, int d) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= ns) return;
    for (int k = 0; k < d; ++k) {
        double s, c;
        sincos((double)phi[v * d + k], &s, &c);
        for (int r = 0; r < d; ++r) {
            double br = base[2 * (r * d + k)], bi = base[2 * (r * d + k) + 1];
            dst[(v * d + r) * d + k] = from_double<R>(br * c - bi * s, br * s + bi * c);
        }
    }
}

cudaError_t launch_convert_coins(int prec, const double *src, void *dst, int64_t count, cudaStream_t s) {
    const unsigned b = (unsigned)((count + 255) / 256);
    if (count <= 0) return cudaSuccess;
    switch (prec) {
        case QW_F64: k_convert_coins<double><<<b, 256, 0, s>>>(src, (Cx<double> *)dst, count); break;
        case QW_F32_COMP: k_convert_coins<ff><<<b, 256, 0, s>>>(src, (Cx<ff> *)dst, count); break;
        default: k_convert_coins<float><<<b, 256, 0, s>>>(src, (Cx<float> *)dst, count); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_phase_coins(int prec, const double *base, const float *phi, void *dst, int64_t ns,
                               int d, cudaStream_t s) {
    const unsigned b = (unsigned)((ns + 255) / 256);
    switch (prec) {
        case QW_F64: k_phase_coins<double><<<b, 256, 0, s>>>(base, phi, (Cx<double> *)dst, ns, d); break;
        case QW_F32_COMP: k_phase_coins<ff><<<b, 256, 0, s>>>(base, phi, (Cx<ff> *)dst, ns, d); break;
        default: k_phase_coins<float><<<b, 256, 0, s>>>(base, phi, (Cx<float> *)dst, ns, d); break;
    }
    return cudaGetLastError();
}

}  // namespace qw
