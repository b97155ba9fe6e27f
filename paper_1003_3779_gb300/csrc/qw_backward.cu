// qw_backward.cu -- gradient of a region's probability mass with respect to the
// per-site coin phases, by the adjoint of the walk.
//
// Walk: psi_{t+1} = S C psi_t on the torus (Sec. 2.2 / Sec. 3, U = S (C (x) I)),
// with the per-site coin C_v = B diag(e^{i phi_{v,k}}) (phase first).
// Loss: L = sum_{v in R, c} |psi_T(v, c)|^2.  With lambda_T = 1_R psi_T and
// lambda_t = U^dagger lambda_{t+1}, differentiating D_v = diag(e^{i phi_v})
// (dD_v / dphi_{v,k} = i E_kk D_v) gives
//     dL/dphi_{v,k} = sum_t 2 Re( conj(a_t(v)_k) i b_t(v)_k ) = sum_t -2 Im(conj(a_k) b_k),
//     a_t = B^dagger S^dagger lambda_{t+1},   b_t = D_v psi_t = B^dagger S^dagger psi_{t+1}.
// So one backward step pulls both lambda_{t+1} and psi_{t+1} through S^dagger,
// applies B^dagger to both, adds the gradient term to a per-segment
// accumulator in the compute precision (flushed into the double gradient at the
// end of every segment of K steps), and emits
// lambda_t = D^dagger a and psi_t = D^dagger b.  psi_t is rebuilt from psi_{t+1}
// (the walk is unitary) instead of stored; it is re-seeded from a forward
// checkpoint every K steps, which bounds the drift of the reconstruction to K
// steps.
#include <algorithm>
#include <cmath>
#include <string>

#include "qw_handle.h"

namespace qw {

template <class R> __device__ __forceinline__ void expi(float a, Cx<R> &e);
template <> __device__ __forceinline__ void expi<float>(float a, Cx<float> &e) { float s, c; sincosf(a, &s, &c); e = {c, s}; }
template <> __device__ __forceinline__ void expi<double>(float a, Cx<double> &e) { double s, c; sincos((double)a, &s, &c); e = {c, s}; }

// One backward step on the torus, one thread per site.
template <int P, int FF, int GROVER>
__global__ void __launch_bounds__(256)
k_backward2d(View lam_in, View psi_in, View lam_out, View psi_out, int64_t nx, int64_t ny,
             CoinP<typename St<P>::real> cp, const float *__restrict__ phi, typename St<P>::real *__restrict__ gseg) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nx * ny) return;
    int64_t x, y;
    if (nx * ny < (int64_t(1) << 31)) {   // 32-bit division where it fits (uniform branch)
        x = (int)v % (int)nx;
        y = (int)v / (int)nx;
    } else {
        x = v % nx;
        y = v / nx;
    }
    const int64_t xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int64_t yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
    // S^dagger: field_c(v) <- field_{src c}(v + e_c); e_0 = +x, e_1 = -x, e_2 = +y, e_3 = -y
    const int64_t src[4] = {y * nx + xp, y * nx + xm, yp * nx + x, ym * nx + x};
    C mu[4], nu[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int pc = FF ? (c ^ 1) : c;
        mu[c] = S::ld(lam_in, pc, src[c]);
        nu[c] = S::ld(psi_in, pc, src[c]);
    }
    // a = B^dagger mu, b = B^dagger nu
    C a[4], b[4];
    if (GROVER) {   // real symmetric: B^dagger = B = (1/2) J - I
        C sm = cadd(cadd(mu[0], mu[1]), cadd(mu[2], mu[3]));
        C sn = cadd(cadd(nu[0], nu[1]), cadd(nu[2], nu[3]));
        sm = rmul(cp.re[1], sm);
        sn = rmul(cp.re[1], sn);
#pragma unroll
        for (int k = 0; k < 4; ++k) { a[k] = csub(sm, mu[k]); b[k] = csub(sn, nu[k]); }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            C aa = conjmul(C{cp.re[k], cp.im[k]}, mu[0]);
            C bb = conjmul(C{cp.re[k], cp.im[k]}, nu[0]);
#pragma unroll
            for (int r = 1; r < 4; ++r) {
                const C br{cp.re[4 * r + k], cp.im[4 * r + k]};
                aa = cadd(aa, conjmul(br, mu[r]));
                bb = cadd(bb, conjmul(br, nu[r]));
            }
            a[k] = aa;
            b[k] = bb;
        }
    }
    const float4 ph = reinterpret_cast<const float4 *>(phi)[v];
    const float pk[4] = {ph.x, ph.y, ph.z, ph.w};
    real g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // -2 Im(conj(a) b) in the compute precision; the segment's running sum
        // stays in that precision and is added into the double gradient once per
        // segment of K steps (double arithmetic is slow on this part)
        g[k] = (a[k].im * b[k].re - a[k].re * b[k].im) * (real)2;
        C e;
        expi<real>(pk[k], e);
        S::st(lam_out, k, v, conjmul(e, a[k]));
        S::st(psi_out, k, v, conjmul(e, b[k]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) gseg[4 * v + k] += g[k];
}

// grad += gseg (double), gseg = 0: the end of one segment of the adjoint sweep.
template <class R>
__global__ void k_flush_segment(R *__restrict__ gseg, double *__restrict__ grad, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    grad[i] += (double)gseg[i];
    gseg[i] = (R)0;
}

// lambda_T = 1_R psi_T, and per-block partial sums of |psi_T|^2 over R.
template <int P>
__global__ void __launch_bounds__(256)
k_seed_region(View psi, View lam, int64_t nx, int64_t ny, int64_t rx, int64_t ry, int64_t rw, int64_t rh,
              double *partials) {
    using S = St<P>;
    __shared__ double sh[8];
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nx * ny;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = v % nx, y = v / nx;
        const bool in = x >= rx && x < rx + rw && y >= ry && y < ry + rh;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            auto z = S::ld(psi, c, v);
            if (in) acc += norm2d(z);
            else z = czero<typename S::real>();
            S::st(lam, c, v, z);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += sh[i];
        partials[blockIdx.x] = b;
    }
}

__global__ void k_sum_blocks(const double *partials, int n, double *out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
}

template <int P>
static cudaError_t backward_step(const qw_walk *w, View lam_in, View psi_in, View lam_out, View psi_out,
                                 void *gseg_v) {
    auto *gseg = static_cast<typename St<P>::real *>(gseg_v);
    const auto &cp = *reinterpret_cast<const CoinP<typename St<P>::real> *>(w->coinp);
    const unsigned blocks = (unsigned)((w->ns + 255) / 256);
    bool grover = true;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            grover = grover && w->coin_host[2 * (4 * r + c)] == (r == c ? -0.5 : 0.5) &&
                     w->coin_host[2 * (4 * r + c) + 1] == 0.0;
    const bool ff = w->shift == QW_SHIFT_FLIPFLOP;
#define QW_BWD(FFV, GV) k_backward2d<P, FFV, GV><<<blocks, 256, 0, w->stream>>>(lam_in, psi_in, lam_out, psi_out, w->nx, w->ny, cp, w->phi_dev, gseg)
    if (ff) { if (grover) QW_BWD(1, 1); else QW_BWD(1, 0); }
    else { if (grover) QW_BWD(0, 1); else QW_BWD(0, 0); }
#undef QW_BWD
    return cudaGetLastError();
}

}  // namespace qw

using namespace qw;

extern "C" qw_status qw_backward(qw_walk *w, const int64_t rect[4], int64_t T, int64_t K, double *loss_out,
                                 double *grad_phi, int on_device) {
    if (!w) return QW_EINVAL;
    NvtxRange nvtx("qw_backward");
    if (!rect || !grad_phi || T < 0 || K < 1) return set_error(w, QW_EINVAL, "bad rect, grad buffer, T or K");
    if (w->ndim != 2) return set_error(w, QW_EUNSUPPORTED, "qw_backward is defined on the torus");
    if (w->kind != CK_PHASE) return set_error(w, QW_ESTATE, "qw_backward needs a phase coin (qw_set_coin_phases)");
    if (w->prec != QW_F32 && w->prec != QW_F64) return set_error(w, QW_EUNSUPPORTED, "qw_backward runs in FP32 or FP64");
    if (w->bc != QW_BC_PERIODIC || links_on(w)) return set_error(w, QW_EUNSUPPORTED, "qw_backward needs the periodic torus");
    if (rect[0] < 0 || rect[1] < 0 || rect[2] < 0 || rect[3] < 0 || rect[0] + rect[2] > w->nx || rect[1] + rect[3] > w->ny)
        return set_error(w, QW_EINVAL, "rect outside the lattice");

    const int64_t nseg = (T + K - 1) / K;
    const size_t sb = w->state_bytes;
    const size_t gbytes = sizeof(double) * 4 * (size_t)w->ns;
    const size_t segbytes = (w->prec == QW_F32 ? 4 : 8) * 4 * (size_t)w->ns;   // per-segment accumulator
    const size_t need = (size_t)(nseg + 1) * sb + 2 * sb + (on_device ? 0 : gbytes) + segbytes + 256;
    cudaError_t e;
    if (w->grad_scratch_bytes < need) {
        cudaStreamSynchronize(w->stream);
        cudaFree(w->grad_scratch);
        w->grad_scratch = nullptr;
        w->grad_scratch_bytes = 0;
        if ((e = dev_alloc(&w->grad_scratch, need)) != cudaSuccess) return cuda_error(w, e, "gradient scratch");
        w->grad_scratch_bytes = need;
    }
    char *base = static_cast<char *>(w->grad_scratch);
    auto ckpt = [&](int64_t s) { return View{base + s * sb, w->pitch, w->d}; };
    View lam[2] = {View{base + (nseg + 1) * sb, w->pitch, w->d}, View{base + (nseg + 2) * sb, w->pitch, w->d}};
    double *grad = on_device ? grad_phi : reinterpret_cast<double *>(base + (nseg + 3) * sb);
    void *gseg = base + (nseg + 3) * sb + (on_device ? 0 : gbytes);

    // forward with a checkpoint every K steps
    e = cudaMemcpyAsync(ckpt(0).p, w->buf[w->cur], sb, cudaMemcpyDeviceToDevice, w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "checkpoint");
    for (int64_t s = 0; s < nseg; ++s) {
        qw_status st = run_steps(w, std::min(K, T - s * K), 0);
        if (st != QW_OK) return st;
        if ((e = cudaMemcpyAsync(ckpt(s + 1).p, w->buf[w->cur], sb, cudaMemcpyDeviceToDevice, w->stream)) != cudaSuccess)
            return cuda_error(w, e, "checkpoint");
    }

    // lambda_T and the loss
    const int nb = marginal_blocks();
    if (w->prec == QW_F32)
        k_seed_region<P_F32><<<nb, 256, 0, w->stream>>>(ckpt(nseg), lam[0], w->nx, w->ny, rect[0], rect[1], rect[2], rect[3], w->partials);
    else
        k_seed_region<P_F64><<<nb, 256, 0, w->stream>>>(ckpt(nseg), lam[0], w->nx, w->ny, rect[0], rect[1], rect[2], rect[3], w->partials);
    k_sum_blocks<<<1, 32, 0, w->stream>>>(w->partials, nb, w->norm_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(w, e, "region seed");
    if ((e = cudaMemsetAsync(grad, 0, gbytes, w->stream)) != cudaSuccess) return cuda_error(w, e, "gradient clear");
    if ((e = cudaMemsetAsync(gseg, 0, segbytes, w->stream)) != cudaSuccess) return cuda_error(w, e, "gradient clear");

    // backward, segment by segment, psi re-seeded from the checkpoint at each boundary
    int li = 0;
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t t_hi = std::min((s + 1) * K, T), t_lo = s * K;
        View psi_in = ckpt(s + 1);
        int pi = 0;
        for (int64_t t = t_hi - 1; t >= t_lo; --t) {
            View psi_out = view_of(w, pi);
            e = w->prec == QW_F32 ? backward_step<P_F32>(w, lam[li], psi_in, lam[li ^ 1], psi_out, gseg)
                                  : backward_step<P_F64>(w, lam[li], psi_in, lam[li ^ 1], psi_out, gseg);
            if (e != cudaSuccess) return cuda_error(w, e, "backward step");
            li ^= 1;
            psi_in = psi_out;
            pi ^= 1;
        }
        const int64_t n4 = 4 * w->ns;
        const unsigned fb = (unsigned)((n4 + 255) / 256);
        if (w->prec == QW_F32) k_flush_segment<float><<<fb, 256, 0, w->stream>>>(static_cast<float *>(gseg), grad, n4);
        else k_flush_segment<double><<<fb, 256, 0, w->stream>>>(static_cast<double *>(gseg), grad, n4);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(w, e, "segment flush");
    }

    // leave the walk at psi_T; hand out the gradient and the loss (the sweep
    // used the walk's other buffer as scratch: it is no longer zero outside
    // the support box)
    w->next_clear = false;
    e = cudaMemcpyAsync(w->buf[w->cur], ckpt(nseg).p, sb, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(grad_phi, grad, gbytes, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(w->host_scalar, w->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess && (loss_out || !on_device)) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return cuda_error(w, e, "gradient readout");
    if (loss_out) *loss_out = *w->host_scalar;
    return QW_OK;
}
