// k_reduce.cu -- coin marginals, norm, and state import/export kernels.
//
// P(v) = sum_c |psi(v,c)|^2 is the per-site term of the normalisation of the
// walker state (Sec. 2.2, and the two-qubit state of Sec. 3).  The norm
// sum_v P(v) is accumulated in double: each thread sums a fixed, strided set of
// sites, a block reduces its threads with warp shuffles, and a second one-block
// kernel adds the per-block partials in block order.  The grid size is fixed,
// so the summation order, and hence every bit of the result, does not depend
// on timing.  For float amplitudes with a float P the per-site sum of squares
// is formed in float (one rounding of 2^-24 per site) and only the running
// norm is double: double arithmetic runs at a small fraction of the float rate
// on this part.
#include <algorithm>
#include <type_traits>

#include "qw_internal.cuh"

namespace qw {

static constexpr int RED_THREADS = 256;
static constexpr int RED_BLOCKS = 152 * 4;   // a multiple of the SM count

int marginal_blocks() { return RED_BLOCKS; }

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;
}

// Each thread handles VEC consecutive sites per iteration with vector loads.
template <int P, int PF32>
__global__ void __launch_bounds__(RED_THREADS)
k_marginals(View v, int64_t ns, void *P_out, double *partials) {
    using S = St<P>;
    using real = typename S::real;
    __shared__ double sh[RED_THREADS / 32];
    const int d = v.d;
    double acc = 0.0;
    const int64_t ngroups = (ns + S::VEC - 1) / S::VEC;
    for (int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gidx < ngroups;
         gidx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = gidx * S::VEC;
        double p[S::VEC];
#pragma unroll
        for (int k = 0; k < S::VEC; ++k) p[k] = 0.0;
        if constexpr (PF32 && std::is_same<real, float>::value) {
          if (i0 + S::VEC <= ns) {
            // float amplitudes and a float P: |psi|^2 per site in float (FP64 is
            // slow on this part), the VEC sites summed in float, one double add
            float pf[S::VEC], grp = 0.f;
#pragma unroll
            for (int k = 0; k < S::VEC; ++k) pf[k] = 0.f;
            for (int c = 0; c < d; ++c) {
                Cx<real> a[S::VEC];
                S::ldv(v, c, i0, a);
#pragma unroll
                for (int k = 0; k < S::VEC; ++k) pf[k] = __fmaf_rn((float)a[k].re, (float)a[k].re, __fmaf_rn((float)a[k].im, (float)a[k].im, pf[k]));
            }
#pragma unroll
            for (int k = 0; k < S::VEC; ++k) {
                grp += pf[k];
                if (P_out) reinterpret_cast<float *>(P_out)[i0 + k] = pf[k];
            }
            acc += (double)grp;
            continue;
          }
        }
        if (i0 + S::VEC <= ns) {
            for (int c = 0; c < d; ++c) {
                Cx<real> a[S::VEC];
                S::ldv(v, c, i0, a);
#pragma unroll
                for (int k = 0; k < S::VEC; ++k) p[k] += norm2d(a[k]);
            }
        } else {
            for (int c = 0; c < d; ++c)
                for (int k = 0; k < S::VEC; ++k)
                    if (i0 + k < ns) p[k] += norm2d(S::ld(v, c, i0 + k));
        }
#pragma unroll
        for (int k = 0; k < S::VEC; ++k) {
            if (i0 + k < ns) {
                acc += p[k];
                if (P_out) {
                    if (PF32) reinterpret_cast<float *>(P_out)[i0 + k] = (float)p[k];
                    else reinterpret_cast<double *>(P_out)[i0 + k] = p[k];
                }
            }
        }
    }
    double b = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void k_sum_partials(const double *partials, int n, double *out) {
    // one warp, lanes own fixed strided subsets, then a fixed shuffle tree
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
}

template <int P>
static cudaError_t marginals_t(View v, int64_t ns, void *P_out, int pf32, double *partials, int nblocks,
                               double *norm_dev, cudaStream_t s) {
    if (pf32) k_marginals<P, 1><<<nblocks, RED_THREADS, 0, s>>>(v, ns, P_out, partials);
    else k_marginals<P, 0><<<nblocks, RED_THREADS, 0, s>>>(v, ns, P_out, partials);
    k_sum_partials<<<1, 32, 0, s>>>(partials, nblocks, norm_dev);
    return cudaGetLastError();
}

cudaError_t launch_marginals(int prec, View v, int64_t ns, void *P, int p_f32, double *partials,
                             int nblocks, double *norm_dev, cudaStream_t s) {
    switch (prec) {
        case P_F64: return marginals_t<P_F64>(v, ns, P, p_f32, partials, nblocks, norm_dev, s);
        case P_F32: return marginals_t<P_F32>(v, ns, P, p_f32, partials, nblocks, norm_dev, s);
        case P_BF16: return marginals_t<P_BF16>(v, ns, P, p_f32, partials, nblocks, norm_dev, s);
        case P_COMP: return marginals_t<P_COMP>(v, ns, P, p_f32, partials, nblocks, norm_dev, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- support box
// Bounding box of the nonzero amplitudes of a state (any coin, any plane):
// box[0..1] the smallest and largest column, box[2..3] the smallest and
// largest row, as unsigned 64-bit values for the atomics; box[0] > box[1]
// means the state is zero.  It is the starting window of the light-cone
// clipping of a localised walk (the "line" computation window of Sec. 3,
// which starts at the walker's site and widens by one site per step).
//
// Work is split into tiles of SUP_THREADS consecutive sites of one row.
// Blocks run tiles in a probe order that starts with the first tile of row 0
// and the last tile of the last row: a dense state fills the box there, and
// every block that then finds the box full returns, so a dense state costs
// about one wave of tiles, a localised one a full read.
static constexpr int SUP_THREADS = 256;

__global__ void k_support_init(unsigned long long *box) {
    box[0] = ~0ull; box[1] = 0ull; box[2] = ~0ull; box[3] = 0ull;
}

template <int P>
__global__ void __launch_bounds__(SUP_THREADS)
k_support(View v, int64_t nx, int64_t ny, int64_t tiles_per_row, int64_t ntiles, unsigned long long *box) {
    using S = St<P>;
    const int lane = threadIdx.x & 31;
    for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        {   // the box already spans the lattice: nothing left to find
            const volatile unsigned long long *vb = box;
            if (vb[0] == 0ull && vb[1] == (unsigned long long)(nx - 1) && vb[2] == 0ull &&
                vb[3] == (unsigned long long)(ny - 1))
                return;
        }
        const int64_t t = ti == 0 ? 0 : (ti == 1 ? ntiles - 1 : ti - 1);   // probe order
        const int64_t y = t / tiles_per_row;
        const int64_t x = (t - y * tiles_per_row) * SUP_THREADS + threadIdx.x;
        bool nz = false;
        if (x < nx) {
            const int64_t i = y * nx + x;
            for (int c = 0; c < v.d; ++c) {
                const auto a = S::ld(v, c, i);
                // (a NaN compares unequal to zero too: it counts as nonzero)
                if constexpr (P == P_COMP)
                    nz = nz || a.re.hi != 0.f || a.im.hi != 0.f || a.re.lo != 0.f || a.im.lo != 0.f;
                else
                    nz = nz || a.re != 0 || a.im != 0;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (m && lane == 0) {
            const int64_t xw = x;   // lane 0's column; the warp's lowest / highest set lanes
            atomicMin(&box[0], (unsigned long long)(xw + (__ffs(m) - 1)));
            atomicMax(&box[1], (unsigned long long)(xw + (31 - __clz(m))));
            atomicMin(&box[2], (unsigned long long)y);
            atomicMax(&box[3], (unsigned long long)y);
        }
    }
}

cudaError_t launch_support(int prec, View v, int64_t nx, int64_t ny, unsigned long long *box, cudaStream_t s) {
    k_support_init<<<1, 1, 0, s>>>(box);
    const int64_t tpr = (nx + SUP_THREADS - 1) / SUP_THREADS, nt = tpr * ny;
    const unsigned grid = (unsigned)std::min<int64_t>(nt, 152 * 8);
    switch (prec) {
        case P_F64: k_support<P_F64><<<grid, SUP_THREADS, 0, s>>>(v, nx, ny, tpr, nt, box); break;
        case P_F32: k_support<P_F32><<<grid, SUP_THREADS, 0, s>>>(v, nx, ny, tpr, nt, box); break;
        case P_BF16: k_support<P_BF16><<<grid, SUP_THREADS, 0, s>>>(v, nx, ny, tpr, nt, box); break;
        case P_COMP: k_support<P_COMP><<<grid, SUP_THREADS, 0, s>>>(v, nx, ny, tpr, nt, box); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- import / export
// Caller layout: d dense planes of nsites complex numbers (complex128 or
// complex64).  One launch converts `count` sites of plane `plane`, starting at
// site `first`; `src`/`dst` point at the first of those sites.
template <int P>
__global__ void k_import(View dst, const void *src, int c64, int64_t first, int64_t count, int plane) {
    using real = typename St<P>::real;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double re, im;
    if (c64) {
        float2 a = reinterpret_cast<const float2 *>(src)[i];
        re = a.x; im = a.y;
    } else {
        double2 a = reinterpret_cast<const double2 *>(src)[i];
        re = a.x; im = a.y;
    }
    Cx<real> z;
    if constexpr (P == P_COMP) {
        float rh = (float)re, ih = (float)im;
        z = {{rh, (float)(re - (double)rh)}, {ih, (float)(im - (double)ih)}};
    } else {
        z = {(real)re, (real)im};
    }
    St<P>::st(dst, plane, first + i, z);
}

template <int P>
__global__ void k_export(View srcv, void *dst, int c64, int64_t first, int64_t count, int plane) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    auto z = St<P>::ld(srcv, plane, first + i);
    double re, im;
    if constexpr (P == P_COMP) {
        re = (double)z.re.hi + (double)z.re.lo;
        im = (double)z.im.hi + (double)z.im.lo;
    } else {
        re = (double)z.re; im = (double)z.im;
    }
    if (c64) reinterpret_cast<float2 *>(dst)[i] = make_float2((float)re, (float)im);
    else reinterpret_cast<double2 *>(dst)[i] = make_double2(re, im);
}

cudaError_t launch_import(int prec, View dst, int64_t nsites, const void *src, int src_c64,
                          int64_t first, int64_t count, int plane, cudaStream_t s) {
    (void)nsites;
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    switch (prec) {
        case P_F64: k_import<P_F64><<<blocks, 256, 0, s>>>(dst, src, src_c64, first, count, plane); break;
        case P_F32: k_import<P_F32><<<blocks, 256, 0, s>>>(dst, src, src_c64, first, count, plane); break;
        case P_BF16: k_import<P_BF16><<<blocks, 256, 0, s>>>(dst, src, src_c64, first, count, plane); break;
        case P_COMP: k_import<P_COMP><<<blocks, 256, 0, s>>>(dst, src, src_c64, first, count, plane); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export(int prec, View src, int64_t nsites, void *dst, int dst_c64,
                          int64_t first, int64_t count, int plane, cudaStream_t s) {
    (void)nsites;
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    switch (prec) {
        case P_F64: k_export<P_F64><<<blocks, 256, 0, s>>>(src, dst, dst_c64, first, count, plane); break;
        case P_F32: k_export<P_F32><<<blocks, 256, 0, s>>>(src, dst, dst_c64, first, count, plane); break;
        case P_BF16: k_export<P_BF16><<<blocks, 256, 0, s>>>(src, dst, dst_c64, first, count, plane); break;
        case P_COMP: k_export<P_COMP><<<blocks, 256, 0, s>>>(src, dst, dst_c64, first, count, plane); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qw
