// qw_noalloc.cu -- coin marginals and norm of a caller-owned state, with no
// device allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc.  A thread cannot
// allocate while another thread of the process holds a stream capture in the
// global capture mode (cudaMalloc then fails), an application whose own
// allocator has already reserved the device memory has none left to give, and
// a latency-critical path cannot afford cudaMalloc's implicit device
// synchronisation.  Such callers own the state, P and the norm and pass them in;
// the only extra memory, the per-block partial sums of the norm, lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
//
// The arithmetic is that of qw_probabilities: P(v) = sum_c |psi(v,c)|^2 per site,
// and the norm as a fixed-order sum of double partials.  The grid has
// ceil(nsites / NA_SITES_PER_BLOCK) blocks; each sums a strided set of sites
// (grid-stride loop) into one partial, then one warp adds the partials in
// block order.  The grid, and so the summation order, depends only on nsites.
#include <mutex>

#include "qw_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_SITES_PER_BLOCK = 8192;
constexpr int NA_MAX_BLOCKS = 16384;   // 128 KiB of scratch: up to 2^27 sites

// One partial sum per block.  Blocks overwrite their own slot on every call and
// the final sum reads only the slots of the current grid, so nothing needs
// clearing between calls; the array keeps the last call's values.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ void na_load(const void *amp, int c64, int64_t pitch, int c, int64_t i,
                                        double &re, double &im) {
    if (c64) {
        float2 a = reinterpret_cast<const float2 *>(amp)[c * pitch + i];
        re = a.x; im = a.y;
    } else {
        double2 a = reinterpret_cast<const double2 *>(amp)[c * pitch + i];
        re = a.x; im = a.y;
    }
}

template <int PF32>
__global__ void __launch_bounds__(NA_THREADS)
k_marginals_noalloc(const void *amp, int c64, int d, int64_t ns, void *P_out, double *partials) {
    __shared__ double sh[NA_THREADS / 32];
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < ns;
         v += (int64_t)gridDim.x * blockDim.x) {
        double p = 0.0;
        for (int c = 0; c < d; ++c) {
            double re, im;
            na_load(amp, c64, ns, c, v, re, im);
            p += re * re + im * im;
        }
        acc += p;
        if (P_out) {
            if (PF32) reinterpret_cast<float *>(P_out)[v] = (float)p;
            else reinterpret_cast<double *>(P_out)[v] = p;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < NA_THREADS / 32; ++i) b += sh[i];
        partials[blockIdx.x] = b;
    }
}

__global__ void k_sum_partials_noalloc(const double *partials, int n, double *out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && out) *out = v;
}

// Device address of the scratch array on the current device.  The array's
// name is only a host-side stand-in in host code, so the address is looked up
// once per device with that device current.  The same first call loads all
// three kernels of this file on the device (cudaFuncGetAttributes), so that a
// later call, with either P type, loads no module code.  The address is kept
// for the life of the process: after a cudaDeviceReset of that device, which
// invalidates every other handle of the library as well, it is stale.
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_marginals_noalloc<0>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_marginals_noalloc<1>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sum_partials_noalloc);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" qw_status qw_probabilities_noalloc(const void *amp, qw_cdtype dtype, int coin_dim, int64_t nsites,
                                              void *P_out, qw_rdtype pdtype, double *norm_out,
                                              void *cuda_stream) {
    if (!amp || nsites < 1 || (coin_dim != 2 && coin_dim != 4)) return QW_EINVAL;
    if ((dtype != QW_C128 && dtype != QW_C64) || (pdtype != QW_R64 && pdtype != QW_R32)) return QW_EINVAL;
    if (nsites > (int64_t)NA_MAX_BLOCKS * NA_SITES_PER_BLOCK) return QW_EINVAL;   // beyond the scratch array
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return QW_ECUDA; }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = (int)((nsites + NA_SITES_PER_BLOCK - 1) / NA_SITES_PER_BLOCK);
    if (pdtype == QW_R32)
        k_marginals_noalloc<1><<<blocks, NA_THREADS, 0, s>>>(amp, dtype == QW_C64, coin_dim, nsites, P_out, scratch);
    else
        k_marginals_noalloc<0><<<blocks, NA_THREADS, 0, s>>>(amp, dtype == QW_C64, coin_dim, nsites, P_out, scratch);
    k_sum_partials_noalloc<<<1, 32, 0, s>>>(scratch, blocks, norm_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? QW_OK : QW_ECUDA;
}
