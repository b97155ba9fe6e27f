// qw_graph.cu -- the coined walk on a general graph (Sec. 2.1).
//
// The local space of vertex v has one basis state |v, e> per edge e at v, so
// the state is one amplitude per (vertex, edge end): an arc.  Arc form: the
// arcs of v are off[v] .. off[v+1]-1 (its coin slots), and partner[a] is the
// arc at the other end of a's edge.  One step is U = S (I (x) C):
//
//   phi(a) = sum_j C_v[i][j] psi(off[v] + j)      (a = off[v] + i, coin at v)
//   psi'(partner[a]) = phi(a)                     (S|v,e> = |v',e>)
//
// and the adjoint U^dagger = (I (x) C^dagger) S, since S is an involution:
//
//   psi'(a) = sum_j conj(C_v[j][i]) psi(partner[off[v] + j]).
//
// There is no locality to block over in a general graph, so each step is one
// pass over the arcs, bound by HBM: one thread per arc, which reads its
// vertex's amplitudes (neighbouring threads share them through L1) and writes
// one amplitude.  Two forms of the forward step:
//   push (variant 0): thread a reads its own vertex (coalesced) and writes
//     psi'(partner[a]) (a scattered 8 or 16 B store);
//   pull (variant 1): thread a reads the vertex of partner[a] (a scattered
//     read of that vertex's arcs) and writes psi'(a) (coalesced).
// On a graph whose arcs are ordered with locality (lattices) both stream; on a
// random graph the scattered side costs whole 32-byte sectors at random DRAM
// addresses.  Two more forms route the permutation through L2 instead, in two
// passes, as a radix-sort scatter does:
//   pass 1 computes phi with coalesced reads and writes it into destination
//     buckets (each bucket covers GR_WINDOW bytes of the output): a tile of
//     GR_TILE arcs is ordered by bucket in shared memory first, so the writes
//     leave as contiguous runs;
//   pass 2 moves each bucket to its final places, which all lie in one window
//     small enough to stay in L2: scattered writes (variant 2) or gathered
//     reads (variant 3) hit L2, and DRAM sees whole lines.
// On graphs of degree 2 or 4 the gather form runs the gather of one step and
// the bucketing of the next as one pass (the state stays bucketed between the
// steps of a call): T steps take T + 1 passes, not 2T, and psi is written and
// read back once per call instead of once per step.
// Which form is fastest for a graph is measured (qw_gwalk_autotune).
//
// Regular graphs of degree 2 or 4 find an arc's vertex by division; others
// read it from a per-arc vertex index.  The Grover coin (2/d) J - I needs the
// vertex sum of the amplitudes; vertices of degree above GR_HEAVY get it from
// a one-block-per-vertex pre-pass instead of every arc summing d values.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qw_handle.h"

namespace qw {

static constexpr int GR_THREADS = 256;
static constexpr int GR_HEAVY = 32;
static constexpr int GR_RED_BLOCKS = 152 * 4;
static constexpr int GR_TILE = 2048;                       // arcs per block of the bucketing pass (1024..4096 swept)
static constexpr size_t GR_WINDOW = size_t(16) << 20;      // output bytes per bucket

template <class R>
struct GraphArgs {
    int A;                     // number of arcs
    const int *src;            // vertex of each arc (irregular graphs)
    const int *off;            // first arc of each vertex, nvert + 1 entries
    const int *partner;        // the shift: arc at the other end of the edge
    const Cx<R> *coins;        // uniform: one d x d; per vertex: concatenated blocks
    const long long *coff;     // per vertex: first entry of the vertex's block
    const Cx<R> *vsum;         // Grover: amplitude sums of the heavy vertices
};

template <int DR, class R>
__device__ __forceinline__ void vertex_of(const GraphArgs<R> &g, int a, int &v, int &o, int &d) {
    if constexpr (DR > 0) {
        v = a / DR;
        o = v * DR;
        d = DR;
    } else {
        v = __ldg(g.src + a);
        o = __ldg(g.off + v);
        d = __ldg(g.off + v + 1) - o;
    }
}

// Row i of the coin at v applied to the vertex's amplitudes x_j: x_j =
// psi(o + j) for the forward step, psi(partner[o + j]) for the adjoint, whose
// coin is C_v^dagger (row i of C^dagger = conjugated column i of C).
template <int MODE, int DR, int ADJ, class R>
__device__ __forceinline__ Cx<R> coin_row(const GraphArgs<R> &g, const Cx<R> *__restrict__ in, int v, int o, int d,
                                          int i) {
    auto x = [&](int k) -> Cx<R> { return ADJ ? in[__ldg(g.partner + k)] : in[k]; };
    if constexpr (MODE == QW_GCOIN_GROVER) {
        Cx<R> s{R(0), R(0)};
        if (DR == 0 && d > GR_HEAVY) {
            s = g.vsum[v];
        } else {
            for (int j = 0; j < d; ++j) s = cadd(s, x(o + j));
        }
        return csub(rmul(R(2) / R(d), s), x(o + i));
    } else {
        const Cx<R> *C = MODE == QW_GCOIN_UNIFORM ? g.coins : g.coins + g.coff[v];
        Cx<R> acc{R(0), R(0)};
        for (int j = 0; j < d; ++j) {
            if (ADJ) acc = cadd(acc, conjmul(C[j * d + i], x(o + j)));
            else acc = cfma(C[i * d + j], x(o + j), acc);
        }
        return acc;
    }
}

// Row i of the coin at v applied to amplitudes already in registers (regular
// graphs of degree DR, forward step).
template <int MODE, int DR, class R>
__device__ __forceinline__ Cx<R> coin_row_reg(const GraphArgs<R> &g, const Cx<R> (&x)[DR], int v, int i) {
    if constexpr (MODE == QW_GCOIN_GROVER) {
        Cx<R> s{R(0), R(0)};
#pragma unroll
        for (int j = 0; j < DR; ++j) s = cadd(s, x[j]);
        return csub(rmul(R(2) / R(DR), s), x[i]);
    } else {
        const Cx<R> *C = MODE == QW_GCOIN_UNIFORM ? g.coins : g.coins + g.coff[v];
        Cx<R> acc{R(0), R(0)};
#pragma unroll
        for (int j = 0; j < DR; ++j) acc = cfma(C[i * DR + j], x[j], acc);
        return acc;
    }
}

// the DR amplitudes of vertex v with 16-byte loads (the vertex starts on a
// multiple of DR * sizeof(Cx<R>) >= 16 bytes)
template <int DR, class R>
__device__ __forceinline__ void load_vertex(const Cx<R> *__restrict__ in, int v, Cx<R> (&x)[DR]) {
    if constexpr (sizeof(R) == 4) {
        const float4 *p = reinterpret_cast<const float4 *>(in + v * DR);
#pragma unroll
        for (int j = 0; j < DR / 2; ++j) {
            const float4 q = p[j];
            x[2 * j] = Cx<R>{q.x, q.y};
            x[2 * j + 1] = Cx<R>{q.z, q.w};
        }
    } else {
        const double2 *p = reinterpret_cast<const double2 *>(in + v * DR);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const double2 q = p[j];
            x[j] = Cx<R>{q.x, q.y};
        }
    }
}

// forward, push: psi'(partner[a]) = row i of C_v applied to psi at v
template <class R, int MODE, int DR>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_push(GraphArgs<R> g, const Cx<R> *__restrict__ in, Cx<R> *__restrict__ out) {
    const long long a64 = (long long)blockIdx.x * GR_THREADS + threadIdx.x;   // A < 2^31: 64-bit before the check
    if (a64 >= g.A) return;
    const int a = (int)a64;
    int v, o, d;
    vertex_of<DR>(g, a, v, o, d);
    out[__ldg(g.partner + a)] = coin_row<MODE, DR, 0>(g, in, v, o, d, a - o);
}

// forward, pull: psi'(a) = phi(partner[a]), computed at the partner's vertex
template <class R, int MODE, int DR>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_pull(GraphArgs<R> g, const Cx<R> *__restrict__ in, Cx<R> *__restrict__ out) {
    const long long a64 = (long long)blockIdx.x * GR_THREADS + threadIdx.x;
    if (a64 >= g.A) return;
    const int a = (int)a64;
    const int b = __ldg(g.partner + a);
    int v, o, d;
    vertex_of<DR>(g, b, v, o, d);
    out[a] = coin_row<MODE, DR, 0>(g, in, v, o, d, b - o);
}

// adjoint: psi'(a) = row i of C_v^dagger applied to (S psi) at v
template <class R, int MODE, int DR>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_adjoint(GraphArgs<R> g, const Cx<R> *__restrict__ in, Cx<R> *__restrict__ out) {
    const long long a64 = (long long)blockIdx.x * GR_THREADS + threadIdx.x;
    if (a64 >= g.A) return;
    const int a = (int)a64;
    int v, o, d;
    vertex_of<DR>(g, a, v, o, d);
    out[a] = coin_row<MODE, DR, 1>(g, in, v, o, d, a - o);
}

// two-pass forward, pass 1: phi of the tile's arcs, ordered by destination
// bucket in shared memory (lpos: the arc's place in that order), then written
// to its bucket slots (gsl: the slot of each place), contiguous per bucket
template <class R, int MODE, int DR>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_bucket(GraphArgs<R> g, const Cx<R> *__restrict__ in, const unsigned short *__restrict__ lpos,
               const int *__restrict__ gsl, Cx<R> *__restrict__ tmp) {
    __shared__ Cx<R> sm[GR_TILE];
    const int base = blockIdx.x * GR_TILE;   // < A: the grid has ceil(A / GR_TILE) blocks
    const int n = min(GR_TILE, g.A - base);
    if constexpr (DR > 0) {
        // a thread per vertex: one vector load of its DR amplitudes (GR_TILE is
        // a multiple of DR, so tiles hold whole vertices)
        for (int vv = threadIdx.x; vv < n / DR; vv += GR_THREADS) {
            const int v = base / DR + vv;
            Cx<R> x[DR];
            load_vertex<DR>(in, v, x);
#pragma unroll
            for (int i = 0; i < DR; ++i) sm[lpos[v * DR + i]] = coin_row_reg<MODE, DR>(g, x, v, i);
        }
    } else {
        for (int i = threadIdx.x; i < n; i += GR_THREADS) {
            const int a = base + i;
            int v, o, d;
            vertex_of<DR>(g, a, v, o, d);
            sm[lpos[a]] = coin_row<MODE, DR, 0>(g, in, v, o, d, a - o);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += GR_THREADS) tmp[__ldcs(gsl + base + j)] = sm[j];
}

// pass 2, scatter form: slot s of the bucketed phi goes to arc dst[s]
template <class R>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_scatter(int A, const int *__restrict__ dst, const Cx<R> *__restrict__ tmp, Cx<R> *__restrict__ out) {
    const long long s = (long long)blockIdx.x * GR_THREADS + threadIdx.x;
    if (s < A) out[__ldg(dst + s)] = tmp[s];
}

// pass 2, gather form: arc a takes bucketed slot srcs[a].  Bucket w holds
// exactly the values bound for the arcs of window w, so its slots are the same
// index range; each thread asks L2 for the slot one window ahead of its arc
// (pf), so that the next window's bucket is read from DRAM in order while this
// window's random reads hit L2.  The index and output streams are marked
// evict-first to leave L2 to the buckets.
static constexpr int GR_GATHER = 4;   // arcs per thread of the gather pass (loads in flight; 4 measured
                                      // fastest of 1..16 at 2^28 arcs: more fill the load queue)

// L2-only load (the random reads of the gather pass gain nothing from L1)
__device__ __forceinline__ Cx<float> ldcg(const Cx<float> *p) {
    const float2 q = __ldcg(reinterpret_cast<const float2 *>(p));
    return Cx<float>{q.x, q.y};
}
__device__ __forceinline__ Cx<double> ldcg(const Cx<double> *p) {
    const double2 q = __ldcg(reinterpret_cast<const double2 *>(p));
    return Cx<double>{q.x, q.y};
}

template <class R>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_gather(int A, const int *__restrict__ srcs, const Cx<R> *__restrict__ tmp, Cx<R> *__restrict__ out, int pf) {
    const long long a0 = (long long)blockIdx.x * (GR_THREADS * GR_GATHER) + threadIdx.x;
    int sl[GR_GATHER];
    Cx<R> v[GR_GATHER];
#pragma unroll
    for (int k = 0; k < GR_GATHER; ++k) {
        const long long a = a0 + k * GR_THREADS;
        if (a < A) {
            if (pf > 0 && a < (long long)A - pf) asm volatile("prefetch.global.L2 [%0];" ::"l"(tmp + a + pf));
            sl[k] = __ldcs(srcs + a);
        }
    }
#pragma unroll
    for (int k = 0; k < GR_GATHER; ++k)
        if (a0 + k * GR_THREADS < A) v[k] = ldcg(tmp + sl[k]);
#pragma unroll
    for (int k = 0; k < GR_GATHER; ++k) {
        const long long a = a0 + k * GR_THREADS;
        if (a >= A) continue;
        if constexpr (sizeof(R) == 4) {
            __stcs(reinterpret_cast<float2 *>(out + a), make_float2(v[k].re, v[k].im));
        } else {
            __stcs(reinterpret_cast<double2 *>(out + a), make_double2(v[k].re, v[k].im));
        }
    }
}

// Steps t and t + 1 of the gather form fused, on regular graphs: a thread per
// vertex gathers psi_t of the vertex's arcs from the bucketed phi of step t - 1
// (the same L2-resident window reads as k_graph_gather), applies the coin of
// step t, and the tile is bucketed for the next gather as in k_graph_bucket.
// psi_t itself never goes to memory; the values that reach the coin are the
// ones the two separate passes would store and reload, so the result is the
// same to the bit.  GF_GATHERS gathers in flight per thread per round (swept
// at 2^28 arcs: 256 threads x 4 gathers 1.80 ms per step; x 8 gathers 1.99;
// 128 threads x 8 or 16 gathers 2.04 / 2.21; 8 blocks per SM forced: 1.79).
static constexpr int GF_THREADS = 256, GF_GATHERS = 4, GF_MIN_BLOCKS = 1;
template <class R, int MODE, int DR>
__global__ void __launch_bounds__(GF_THREADS, GF_MIN_BLOCKS)
k_graph_gather_bucket(GraphArgs<R> g, const Cx<R> *__restrict__ tin, const int *__restrict__ srcs,
                      const unsigned short *__restrict__ lpos, const int *__restrict__ gsl, Cx<R> *__restrict__ tout,
                      int pf) {
    static_assert(DR == 2 || DR == 4, "regular graphs of degree 2 or 4");
    constexpr int UV = GF_GATHERS / DR;      // vertices per thread per round
    __shared__ Cx<R> sm[GR_TILE];
    const int base = blockIdx.x * GR_TILE;   // < A: the grid has ceil(A / GR_TILE) blocks
    const int n = min(GR_TILE, g.A - base);  // a multiple of DR (GR_TILE is, and so is A)
    const int nv = n / DR;
    for (int v0 = threadIdx.x; v0 < nv; v0 += GF_THREADS * UV) {
        int sl[UV][DR];
        Cx<R> x[UV][DR];
#pragma unroll
        for (int u = 0; u < UV; ++u) {
            const int vv = v0 + u * GF_THREADS;
            if (vv >= nv) continue;
            const long long a = (long long)base + (long long)vv * DR;   // first arc of the vertex
            if (pf > 0 && a < (long long)g.A - pf) asm volatile("prefetch.global.L2 [%0];" ::"l"(tin + a + pf));
            if constexpr (DR == 4) {
                const int4 q = __ldcs(reinterpret_cast<const int4 *>(srcs + a));
                sl[u][0] = q.x; sl[u][1] = q.y; sl[u][2] = q.z; sl[u][3] = q.w;
            } else {
                const int2 q = __ldcs(reinterpret_cast<const int2 *>(srcs + a));
                sl[u][0] = q.x; sl[u][1] = q.y;
            }
        }
#pragma unroll
        for (int u = 0; u < UV; ++u) {
            if (v0 + u * GF_THREADS >= nv) continue;
#pragma unroll
            for (int i = 0; i < DR; ++i) x[u][i] = ldcg(tin + sl[u][i]);
        }
#pragma unroll
        for (int u = 0; u < UV; ++u) {
            const int vv = v0 + u * GF_THREADS;
            if (vv >= nv) continue;
            const int v = base / DR + vv;
#pragma unroll
            for (int i = 0; i < DR; ++i) sm[lpos[v * DR + i]] = coin_row_reg<MODE, DR>(g, x[u], v, i);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += GF_THREADS) tout[__ldcs(gsl + base + j)] = sm[j];
}

// Grover pre-pass: the amplitude sum of each heavy vertex (of psi, or of S psi
// for the adjoint), one block per vertex, threads over fixed strided arcs, then
// a fixed shuffle / shared-memory tree: the same bits on every run.
template <class R, int ADJ>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_heavy(GraphArgs<R> g, const int *__restrict__ heavy, int nheavy, const Cx<R> *__restrict__ in,
              Cx<R> *__restrict__ vsum) {
    __shared__ R sh[2][GR_THREADS / 32];
    for (int h = blockIdx.x; h < nheavy; h += gridDim.x) {
        const int v = heavy[h];
        const int o = g.off[v], d = g.off[v + 1] - o;
        Cx<R> s{R(0), R(0)};
        for (int j = threadIdx.x; j < d; j += GR_THREADS) s = cadd(s, ADJ ? in[g.partner[o + j]] : in[o + j]);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            s.re += __shfl_down_sync(0xffffffffu, s.re, m);
            s.im += __shfl_down_sync(0xffffffffu, s.im, m);
        }
        if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s.re; sh[1][threadIdx.x >> 5] = s.im; }
        __syncthreads();
        if (threadIdx.x == 0) {
            Cx<R> t{R(0), R(0)};
            for (int w = 0; w < GR_THREADS / 32; ++w) { t.re += sh[0][w]; t.im += sh[1][w]; }
            vsum[v] = t;
        }
        __syncthreads();
    }
}

// P(v) = sum over the arcs of v of |psi(a)|^2 (in the compute precision), and
// the norm in double over a fixed grid: per-thread strided vertices, a block
// tree, then one warp over the block partials in order.
template <class R, class PO>
__global__ void __launch_bounds__(GR_THREADS)
k_graph_marginals(const int *__restrict__ off, int nvert, const Cx<R> *__restrict__ psi, PO *P, double *partials) {
    __shared__ double sh[GR_THREADS / 32];
    double acc = 0.0;
    for (long long v = (long long)blockIdx.x * GR_THREADS + threadIdx.x; v < nvert; v += (long long)gridDim.x * GR_THREADS) {
        R p = R(0);
        for (int a = off[v]; a < off[v + 1]; ++a) p += psi[a].re * psi[a].re + psi[a].im * psi[a].im;
        if (P) P[v] = (PO)p;
        acc += (double)p;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < GR_THREADS / 32; ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_graph_norm(const double *partials, int n, double *out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += partials[i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_down_sync(0xffffffffu, v, m);
    if (threadIdx.x == 0) *out = v;
}

// element conversion between caller and compute precision
template <class RI, class RO>
__global__ void k_graph_convert(const Cx<RI> *__restrict__ in, Cx<RO> *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)GR_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * GR_THREADS)
        out[i] = Cx<RO>{(RO)in[i].re, (RO)in[i].im};
}

}  // namespace qw

using namespace qw;

struct qw_gwalk {
    int64_t nvert = 0;
    int A = 0;
    int prec = QW_F32;
    int dreg = 0;                 // common degree when every vertex has it, else 0
    int maxdeg = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> deg;         // host copy of the degrees
    int *off_dev = nullptr, *src_dev = nullptr, *partner_dev = nullptr;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    int mode = QW_GCOIN_GROVER;
    void *coins_dev = nullptr;
    size_t coins_bytes = 0;
    long long *coff_dev = nullptr;
    int *heavy_dev = nullptr;
    int nheavy = 0;
    void *vsum_dev = nullptr;
    double *partials = nullptr, *norm_dev = nullptr;
    void *p_dev = nullptr;
    size_t p_bytes = 0;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    int variant = -1;             // -1: default (push)
    // two-pass forms: bucket order of each tile, bucket slot of each tile
    // place, final arc of each slot (scatter) / slot of each arc (gather)
    unsigned short *lpos_dev = nullptr;
    int *gsl_dev = nullptr, *dst_dev = nullptr, *slot_dev = nullptr;
    void *tmp_dev = nullptr;
    size_t window = GR_WINDOW;    // output bytes per bucket
    int window_arcs = 0;          // arcs per bucket of the built tables
    std::string err;
};

namespace {

qw_status gfail(qw_gwalk *g, qw_status st, const std::string &m) {
    if (g) g->err = m;
    return st;
}

qw_status gcuda(qw_gwalk *g, cudaError_t e, const char *where) {
    (void)cudaGetLastError();
    return gfail(g, e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA,
                 std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

size_t amp_bytes(const qw_gwalk *g) { return g->prec == QW_F64 ? 16 : 8; }

qw_status ensure_staging(qw_gwalk *g, size_t bytes) {
    if (g->staging_bytes >= bytes) return QW_OK;
    if (g->staging) { cudaStreamSynchronize(g->stream); cudaFree(g->staging); g->staging = nullptr; g->staging_bytes = 0; }
    cudaError_t e = dev_alloc(&g->staging, bytes);
    if (e != cudaSuccess) return gcuda(g, e, "graph staging allocation");
    g->staging_bytes = bytes;
    return QW_OK;
}

template <class R>
GraphArgs<R> args_of(const qw_gwalk *g) {
    GraphArgs<R> a{};
    a.A = g->A;
    a.src = g->src_dev;
    a.off = g->off_dev;
    a.partner = g->partner_dev;
    a.coins = static_cast<const Cx<R> *>(g->coins_dev);
    a.coff = g->coff_dev;
    a.vsum = static_cast<const Cx<R> *>(g->vsum_dev);
    return a;
}

// kernel: 0 push, 1 pull, 2 adjoint
template <class R, int MODE, int DR>
cudaError_t launch_mode_dr(const GraphArgs<R> &a, int kernel, const Cx<R> *in, Cx<R> *out, cudaStream_t s) {
    const unsigned blocks = (unsigned)(((long long)a.A + GR_THREADS - 1) / GR_THREADS);
    if (kernel == 0) k_graph_push<R, MODE, DR><<<blocks, GR_THREADS, 0, s>>>(a, in, out);
    else if (kernel == 1) k_graph_pull<R, MODE, DR><<<blocks, GR_THREADS, 0, s>>>(a, in, out);
    else k_graph_adjoint<R, MODE, DR><<<blocks, GR_THREADS, 0, s>>>(a, in, out);
    return cudaGetLastError();
}

template <class R, int MODE, int DR>
cudaError_t launch_bucket_dr(const GraphArgs<R> &a, const qw_gwalk *g, const Cx<R> *in) {
    const unsigned tiles = (unsigned)(((long long)a.A + GR_TILE - 1) / GR_TILE);
    k_graph_bucket<R, MODE, DR><<<tiles, GR_THREADS, 0, g->stream>>>(a, in, g->lpos_dev, g->gsl_dev,
                                                                       static_cast<Cx<R> *>(g->tmp_dev));
    return cudaGetLastError();
}

template <class R, int MODE>
cudaError_t launch_bucket(const qw_gwalk *g, const GraphArgs<R> &a, const Cx<R> *in) {
    if (g->dreg == 2) return launch_bucket_dr<R, MODE, 2>(a, g, in);
    if (g->dreg == 4) return launch_bucket_dr<R, MODE, 4>(a, g, in);
    return launch_bucket_dr<R, MODE, 0>(a, g, in);
}

template <class R, int MODE>
cudaError_t launch_mode(const qw_gwalk *g, const GraphArgs<R> &a, int kernel, const Cx<R> *in, Cx<R> *out) {
    if (g->dreg == 2) return launch_mode_dr<R, MODE, 2>(a, kernel, in, out, g->stream);
    if (g->dreg == 4) return launch_mode_dr<R, MODE, 4>(a, kernel, in, out, g->stream);
    return launch_mode_dr<R, MODE, 0>(a, kernel, in, out, g->stream);
}

template <class R>
cudaError_t graph_step(qw_gwalk *g, int kernel) {
    if (g->A == 0) return cudaSuccess;
    GraphArgs<R> a = args_of<R>(g);
    const Cx<R> *in = static_cast<const Cx<R> *>(g->buf[g->cur]);
    Cx<R> *out = static_cast<Cx<R> *>(g->buf[g->cur ^ 1]);
    if (g->mode == QW_GCOIN_GROVER && g->nheavy && g->dreg != 2 && g->dreg != 4) {
        const int blocks = std::min(g->nheavy, 152 * 8);
        if (kernel == 2)
            k_graph_heavy<R, 1><<<blocks, GR_THREADS, 0, g->stream>>>(a, g->heavy_dev, g->nheavy, in, (Cx<R> *)g->vsum_dev);
        else
            k_graph_heavy<R, 0><<<blocks, GR_THREADS, 0, g->stream>>>(a, g->heavy_dev, g->nheavy, in, (Cx<R> *)g->vsum_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (kernel >= 3) {   // two-pass forms
        cudaError_t e;
        switch (g->mode) {
            case QW_GCOIN_GROVER: e = launch_bucket<R, QW_GCOIN_GROVER>(g, a, in); break;
            case QW_GCOIN_UNIFORM: e = launch_bucket<R, QW_GCOIN_UNIFORM>(g, a, in); break;
            default: e = launch_bucket<R, QW_GCOIN_PER_VERTEX>(g, a, in); break;
        }
        if (e != cudaSuccess) return e;
        const unsigned blocks = (unsigned)(((long long)a.A + GR_THREADS - 1) / GR_THREADS);
        const Cx<R> *tmp = static_cast<const Cx<R> *>(g->tmp_dev);
        if (kernel == 3) k_graph_scatter<R><<<blocks, GR_THREADS, 0, g->stream>>>(a.A, g->dst_dev, tmp, out);
        else
            k_graph_gather<R><<<(unsigned)(((long long)a.A + GR_THREADS * GR_GATHER - 1) / (GR_THREADS * GR_GATHER)), GR_THREADS, 0,
                                g->stream>>>(a.A, g->slot_dev, tmp, out, g->window_arcs);
        return cudaGetLastError();
    }
    switch (g->mode) {
        case QW_GCOIN_GROVER: return launch_mode<R, QW_GCOIN_GROVER>(g, a, kernel, in, out);
        case QW_GCOIN_UNIFORM: return launch_mode<R, QW_GCOIN_UNIFORM>(g, a, kernel, in, out);
        default: return launch_mode<R, QW_GCOIN_PER_VERTEX>(g, a, kernel, in, out);
    }
}

// The tables of the two-pass forms, built on the host once per graph: the
// destination bucket of arc a is partner[a] / W (W arcs per GR_WINDOW bytes);
// slots are bucket-major, then tile, then arc order; within a tile the arcs
// are ordered by bucket (a counting sort), so each tile's run for a bucket is
// contiguous both in shared memory and in the slot array.
qw_status ensure_two_pass(qw_gwalk *g) {
    if (g->tmp_dev) return QW_OK;
    const int A = g->A;
    std::vector<int> partner((size_t)A);
    if (A) {
        cudaError_t e = cudaMemcpyAsync(partner.data(), g->partner_dev, sizeof(int) * (size_t)A, cudaMemcpyDeviceToHost,
                                        g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return gcuda(g, e, "two-pass tables");
    }
    const int64_t W = std::max<int64_t>(1, (int64_t)(g->window / amp_bytes(g)));
    const int nb = (int)((A + W - 1) / W);
    g->window_arcs = (int)std::min<int64_t>(W, A);
    std::vector<int64_t> bstart((size_t)nb + 1, 0);
    for (int a = 0; a < A; ++a) ++bstart[(size_t)(partner[(size_t)a] / W) + 1];
    for (int b = 0; b < nb; ++b) bstart[(size_t)b + 1] += bstart[(size_t)b];
    std::vector<int64_t> ptr(bstart.begin(), bstart.end() - 1);
    std::vector<unsigned short> lpos((size_t)A);
    std::vector<int> gsl((size_t)A), dst((size_t)A), slot((size_t)A);
    std::vector<int> lcnt((size_t)nb), lstart((size_t)nb);
    for (int64_t base = 0; base < A; base += GR_TILE) {
        const int n = (int)std::min<int64_t>(GR_TILE, A - base);
        std::fill(lcnt.begin(), lcnt.end(), 0);
        for (int i = 0; i < n; ++i) ++lcnt[(size_t)(partner[(size_t)(base + i)] / W)];
        int acc = 0;
        for (int b = 0; b < nb; ++b) { lstart[(size_t)b] = acc; acc += lcnt[(size_t)b]; }
        for (int i = 0; i < n; ++i) {
            const int a = (int)(base + i);
            const int b = (int)(partner[(size_t)a] / W);
            const int place = lstart[(size_t)b]++;
            const int s = (int)ptr[(size_t)b]++;
            lpos[(size_t)a] = (unsigned short)place;
            gsl[(size_t)(base + place)] = s;
            dst[(size_t)s] = partner[(size_t)a];
            slot[(size_t)partner[(size_t)a]] = s;
        }
    }
    const size_t n4 = sizeof(int) * (size_t)std::max(A, 1);
    cudaError_t e = dev_alloc((void **)&g->lpos_dev, sizeof(unsigned short) * (size_t)std::max(A, 1));
    if (e == cudaSuccess) e = dev_alloc((void **)&g->gsl_dev, n4);
    if (e == cudaSuccess) e = dev_alloc((void **)&g->dst_dev, n4);
    if (e == cudaSuccess) e = dev_alloc((void **)&g->slot_dev, n4);
    if (e == cudaSuccess) e = dev_alloc(&g->tmp_dev, (size_t)std::max(A, 1) * amp_bytes(g));
    if (e == cudaSuccess && A) {
        e = cudaMemcpyAsync(g->lpos_dev, lpos.data(), sizeof(unsigned short) * A, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->gsl_dev, gsl.data(), sizeof(int) * (size_t)A, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->dst_dev, dst.data(), sizeof(int) * (size_t)A, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->slot_dev, slot.data(), sizeof(int) * (size_t)A, cudaMemcpyHostToDevice, g->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        for (void *p : {(void *)g->lpos_dev, (void *)g->gsl_dev, (void *)g->dst_dev, (void *)g->slot_dev, g->tmp_dev})
            if (p) cudaFree(p);
        g->lpos_dev = nullptr; g->gsl_dev = g->dst_dev = g->slot_dev = nullptr; g->tmp_dev = nullptr;
        return gcuda(g, e, "two-pass tables");
    }
    return QW_OK;
}

template <class R, int MODE>
cudaError_t launch_gather_bucket(const qw_gwalk *g, const GraphArgs<R> &a, const Cx<R> *tin, Cx<R> *tout) {
    const unsigned tiles = (unsigned)(((long long)a.A + GR_TILE - 1) / GR_TILE);
    if (g->dreg == 2)
        k_graph_gather_bucket<R, MODE, 2><<<tiles, GF_THREADS, 0, g->stream>>>(a, tin, g->slot_dev, g->lpos_dev,
                                                                               g->gsl_dev, tout, g->window_arcs);
    else
        k_graph_gather_bucket<R, MODE, 4><<<tiles, GF_THREADS, 0, g->stream>>>(a, tin, g->slot_dev, g->lpos_dev,
                                                                               g->gsl_dev, tout, g->window_arcs);
    return cudaGetLastError();
}

// T >= 2 forward steps of the gather form on a regular graph of degree 2 or 4:
// one bucketing pass from psi, T - 1 fused gather + bucketing passes, one
// gather into the other state buffer.  The bucketed phi alternates between the
// two-pass scratch and the input state buffer, which the first pass has
// consumed.
template <class R>
cudaError_t graph_steps_fused(qw_gwalk *g, int64_t T) {
    GraphArgs<R> a = args_of<R>(g);
    Cx<R> *in = static_cast<Cx<R> *>(g->buf[g->cur]);
    Cx<R> *out = static_cast<Cx<R> *>(g->buf[g->cur ^ 1]);
    Cx<R> *x[2] = {static_cast<Cx<R> *>(g->tmp_dev), in};
    cudaError_t e;
    switch (g->mode) {
        case QW_GCOIN_GROVER: e = launch_bucket<R, QW_GCOIN_GROVER>(g, a, in); break;
        case QW_GCOIN_UNIFORM: e = launch_bucket<R, QW_GCOIN_UNIFORM>(g, a, in); break;
        default: e = launch_bucket<R, QW_GCOIN_PER_VERTEX>(g, a, in); break;
    }
    for (int64_t t = 1; t < T && e == cudaSuccess; ++t) {
        const Cx<R> *tin = x[(t - 1) & 1];
        Cx<R> *tout = x[t & 1];
        switch (g->mode) {
            case QW_GCOIN_GROVER: e = launch_gather_bucket<R, QW_GCOIN_GROVER>(g, a, tin, tout); break;
            case QW_GCOIN_UNIFORM: e = launch_gather_bucket<R, QW_GCOIN_UNIFORM>(g, a, tin, tout); break;
            default: e = launch_gather_bucket<R, QW_GCOIN_PER_VERTEX>(g, a, tin, tout); break;
        }
    }
    if (e != cudaSuccess) return e;
    k_graph_gather<R><<<(unsigned)(((long long)a.A + GR_THREADS * GR_GATHER - 1) / (GR_THREADS * GR_GATHER)), GR_THREADS,
                        0, g->stream>>>(a.A, g->slot_dev, x[(T - 1) & 1], out, g->window_arcs);
    return cudaGetLastError();
}

qw_status run_graph(qw_gwalk *g, int64_t T, int adj) {
    if (T < 0) return gfail(g, QW_EINVAL, "T must be >= 0");
    const int kernel = adj ? 2 : (g->variant <= 0 ? 0 : (g->variant == 1 ? 1 : g->variant + 1));
    if (kernel == 4 && T >= 2 && g->A > 0 && (g->dreg == 2 || g->dreg == 4)) {
        cudaError_t e = g->prec == QW_F64 ? graph_steps_fused<double>(g, T) : graph_steps_fused<float>(g, T);
        if (e != cudaSuccess) return gcuda(g, e, "graph step launch");
        g->cur ^= 1;
        return QW_OK;
    }
    for (int64_t t = 0; t < T; ++t) {
        cudaError_t e = g->prec == QW_F64 ? graph_step<double>(g, kernel) : graph_step<float>(g, kernel);
        if (e != cudaSuccess) return gcuda(g, e, "graph step launch");
        g->cur ^= 1;
    }
    return QW_OK;
}

template <class RI, class RO>
cudaError_t convert(const void *in, void *out, long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const long long want = (n + GR_THREADS - 1) / GR_THREADS;
    const unsigned blocks = (unsigned)std::min<long long>(want, 152 * 16);
    k_graph_convert<RI, RO><<<blocks, GR_THREADS, 0, s>>>(static_cast<const Cx<RI> *>(in), static_cast<Cx<RO> *>(out), n);
    return cudaGetLastError();
}

// doubles (re/im) -> compute precision, device to device
cudaError_t from_doubles(const qw_gwalk *g, const void *in, void *out, long long n) {
    if (g->prec == QW_F64)
        return cudaMemcpyAsync(out, in, (size_t)n * 16, cudaMemcpyDeviceToDevice, g->stream);
    return convert<double, float>(in, out, n, g->stream);
}

void free_all(qw_gwalk *g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : {(void *)g->off_dev, (void *)g->src_dev, (void *)g->partner_dev, g->buf[0], g->buf[1], g->coins_dev,
                    (void *)g->coff_dev, (void *)g->heavy_dev, g->vsum_dev, (void *)g->partials, (void *)g->norm_dev,
                    g->p_dev, g->staging, (void *)g->lpos_dev, (void *)g->gsl_dev, (void *)g->dst_dev,
                    (void *)g->slot_dev, g->tmp_dev})
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

qw_status qw_graph_arcs(int64_t nvert, int64_t nedges, const int64_t *edges, int64_t *off, int64_t *partner) {
    if (nvert < 1 || nedges < 0 || !off || (nedges && (!edges || !partner))) return QW_EINVAL;
    for (int64_t k = 0; k < 2 * nedges; ++k)
        if (edges[k] < 0 || edges[k] >= nvert) return QW_EINVAL;
    // count the edge ends at each vertex, prefix-sum into first arcs, then hand
    // out slots in list order and pair the two ends of every edge
    std::vector<int64_t> next((size_t)nvert + 1, 0);
    for (int64_t k = 0; k < 2 * nedges; ++k) ++next[(size_t)edges[k] + 1];
    for (int64_t v = 0; v < nvert; ++v) next[(size_t)v + 1] += next[(size_t)v];
    std::memcpy(off, next.data(), sizeof(int64_t) * ((size_t)nvert + 1));
    for (int64_t e = 0; e < nedges; ++e) {
        const int64_t a = next[(size_t)edges[2 * e]]++;
        const int64_t b = next[(size_t)edges[2 * e + 1]]++;
        partner[a] = b;
        partner[b] = a;
    }
    return QW_OK;
}

qw_status qw_gwalk_create(int64_t nvert, const int64_t *off, const int64_t *partner, qw_precision prec,
                          void *cuda_stream, qw_gwalk **out) {
    if (!out) return QW_EINVAL;
    *out = nullptr;
    if (nvert < 1 || !off) return QW_EINVAL;
    if (prec != QW_F32 && prec != QW_F64) return QW_EUNSUPPORTED;
    if (nvert >= (int64_t(1) << 31) || off[nvert] >= (int64_t(1) << 31)) return QW_EUNSUPPORTED;
    if (off[0] != 0) return QW_EINVAL;
    for (int64_t v = 0; v < nvert; ++v)
        if (off[v + 1] < off[v]) return QW_EINVAL;
    const int64_t A = off[nvert];
    if (A && !partner) return QW_EINVAL;
    for (int64_t a = 0; a < A; ++a)
        if (partner[a] < 0 || partner[a] >= A || partner[partner[a]] != a) return QW_EINVAL;

    qw_gwalk *g = new (std::nothrow) qw_gwalk();
    if (!g) return QW_ENOMEM;
    g->nvert = nvert;
    g->A = (int)A;
    g->prec = prec;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->deg.resize((size_t)nvert);
    std::vector<int> offi((size_t)nvert + 1), heavy;
    for (int64_t v = 0; v <= nvert; ++v) offi[(size_t)v] = (int)off[v];
    for (int64_t v = 0; v < nvert; ++v) {
        const int d = (int)(off[v + 1] - off[v]);
        g->deg[(size_t)v] = d;
        g->maxdeg = std::max(g->maxdeg, d);
        if (d > GR_HEAVY) heavy.push_back((int)v);
    }
    g->dreg = g->deg[0];
    for (int64_t v = 1; v < nvert; ++v)
        if (g->deg[(size_t)v] != g->dreg) { g->dreg = 0; break; }
    const bool need_src = g->dreg != 2 && g->dreg != 4;
    std::vector<int> pi((size_t)A), src(need_src ? (size_t)A : 0);
    for (int64_t a = 0; a < A; ++a) pi[(size_t)a] = (int)partner[a];
    if (need_src)
        for (int64_t v = 0; v < nvert; ++v)
            for (int64_t a = off[v]; a < off[v + 1]; ++a) src[(size_t)a] = (int)v;
    g->nheavy = (int)heavy.size();

    const size_t sb = (size_t)std::max<int64_t>(A, 1) * amp_bytes(g);
    cudaError_t e = dev_alloc((void **)&g->off_dev, sizeof(int) * offi.size());
    if (e == cudaSuccess) e = dev_alloc((void **)&g->partner_dev, sizeof(int) * std::max<size_t>(pi.size(), 1));
    if (e == cudaSuccess && need_src) e = dev_alloc((void **)&g->src_dev, sizeof(int) * std::max<size_t>(src.size(), 1));
    if (e == cudaSuccess) e = dev_alloc(&g->buf[0], sb);
    if (e == cudaSuccess) e = dev_alloc(&g->buf[1], sb);
    if (e == cudaSuccess) e = dev_alloc((void **)&g->partials, sizeof(double) * GR_RED_BLOCKS);
    if (e == cudaSuccess) e = dev_alloc((void **)&g->norm_dev, sizeof(double));
    if (e == cudaSuccess && g->nheavy) e = dev_alloc((void **)&g->heavy_dev, sizeof(int) * heavy.size());
    if (e == cudaSuccess && g->nheavy) e = dev_alloc(&g->vsum_dev, (size_t)nvert * amp_bytes(g));
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->off_dev, offi.data(), sizeof(int) * offi.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && A)
        e = cudaMemcpyAsync(g->partner_dev, pi.data(), sizeof(int) * pi.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && need_src && A)
        e = cudaMemcpyAsync(g->src_dev, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && g->nheavy)
        e = cudaMemcpyAsync(g->heavy_dev, heavy.data(), sizeof(int) * heavy.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->buf[0], 0, sb, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);   // the host vectors go out of scope
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        const qw_status st = e == cudaErrorMemoryAllocation ? QW_ENOMEM : QW_ECUDA;
        free_all(g);
        delete g;
        return st;
    }
    *out = g;
    return QW_OK;
}

qw_status qw_gwalk_destroy(qw_gwalk *g) {
    if (!g) return QW_OK;
    free_all(g);
    delete g;
    return QW_OK;
}

const char *qw_gwalk_last_error(const qw_gwalk *g) { return g ? g->err.c_str() : "null handle"; }

int64_t qw_gwalk_narcs(const qw_gwalk *g) { return g ? g->A : -1; }

qw_status qw_gwalk_set_coin(qw_gwalk *g, qw_gcoin mode, const double *coins, int on_device) {
    if (!g) return QW_EINVAL;
    if (mode == QW_GCOIN_GROVER) { g->mode = mode; return QW_OK; }
    if (mode != QW_GCOIN_UNIFORM && mode != QW_GCOIN_PER_VERTEX) return gfail(g, QW_EINVAL, "unknown coin mode");
    if (!coins) return gfail(g, QW_EINVAL, "coins is NULL");
    long long n = 0;
    std::vector<long long> coff;
    if (mode == QW_GCOIN_UNIFORM) {
        if (g->dreg == 0) return gfail(g, QW_EINVAL, "a uniform coin needs a regular graph");
        n = (long long)g->dreg * g->dreg;
    } else {
        coff.resize((size_t)g->nvert);
        for (int64_t v = 0; v < g->nvert; ++v) {
            coff[(size_t)v] = n;
            n += (long long)g->deg[(size_t)v] * g->deg[(size_t)v];
        }
    }
    const size_t want = (size_t)std::max<long long>(n, 1) * amp_bytes(g);
    cudaError_t e = cudaSuccess;
    if (g->coins_bytes < want) {
        cudaStreamSynchronize(g->stream);
        cudaFree(g->coins_dev);
        g->coins_dev = nullptr;
        g->coins_bytes = 0;
        if ((e = dev_alloc(&g->coins_dev, want)) != cudaSuccess) return gcuda(g, e, "graph coin allocation");
        g->coins_bytes = want;
    }
    if (mode == QW_GCOIN_PER_VERTEX && !g->coff_dev) {
        if ((e = dev_alloc((void **)&g->coff_dev, sizeof(long long) * coff.size())) != cudaSuccess)
            return gcuda(g, e, "graph coin offsets");
        e = cudaMemcpyAsync(g->coff_dev, coff.data(), sizeof(long long) * coff.size(), cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return gcuda(g, e, "graph coin offsets");
    }
    if (n) {
        const void *src = coins;
        if (!on_device) {
            qw_status st = ensure_staging(g, (size_t)n * 16);
            if (st != QW_OK) return st;
            if ((e = cudaMemcpyAsync(g->staging, coins, (size_t)n * 16, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
                return gcuda(g, e, "graph coin copy");
            src = g->staging;
        }
        if ((e = from_doubles(g, src, g->coins_dev, n)) != cudaSuccess) return gcuda(g, e, "graph coin conversion");
        if (!on_device && (e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return gcuda(g, e, "graph coin copy");
    }
    g->mode = mode;
    return QW_OK;
}

qw_status qw_gwalk_set_state(qw_gwalk *g, const void *amp, qw_cdtype dtype, int on_device) {
    if (!g) return QW_EINVAL;
    if (!amp || (dtype != QW_C128 && dtype != QW_C64)) return gfail(g, QW_EINVAL, "bad state buffer or dtype");
    const long long n = g->A;
    const size_t eb = dtype == QW_C128 ? 16 : 8;
    const bool same = (g->prec == QW_F64) == (dtype == QW_C128);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    if (n == 0) return QW_OK;
    if (same) {
        e = cudaMemcpyAsync(g->buf[g->cur], amp, (size_t)n * eb, kind, g->stream);
    } else {
        const void *src = amp;
        if (!on_device) {
            qw_status st = ensure_staging(g, (size_t)n * eb);
            if (st != QW_OK) return st;
            e = cudaMemcpyAsync(g->staging, amp, (size_t)n * eb, kind, g->stream);
            src = g->staging;
        }
        if (e == cudaSuccess)
            e = dtype == QW_C128 ? convert<double, float>(src, g->buf[g->cur], n, g->stream)
                                 : convert<float, double>(src, g->buf[g->cur], n, g->stream);
    }
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return gcuda(g, e, "graph state upload");
    return QW_OK;
}

qw_status qw_gwalk_get_state(qw_gwalk *g, void *amp_out, qw_cdtype dtype, int on_device) {
    if (!g) return QW_EINVAL;
    if (!amp_out || (dtype != QW_C128 && dtype != QW_C64)) return gfail(g, QW_EINVAL, "bad state buffer or dtype");
    const long long n = g->A;
    const size_t eb = dtype == QW_C128 ? 16 : 8;
    const bool same = (g->prec == QW_F64) == (dtype == QW_C128);
    cudaError_t e = cudaSuccess;
    if (n == 0) return QW_OK;
    if (same) {
        e = cudaMemcpyAsync(amp_out, g->buf[g->cur], (size_t)n * eb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            g->stream);
    } else {
        void *dst = amp_out;
        if (!on_device) {
            qw_status st = ensure_staging(g, (size_t)n * eb);
            if (st != QW_OK) return st;
            dst = g->staging;
        }
        e = dtype == QW_C128 ? convert<float, double>(g->buf[g->cur], dst, n, g->stream)
                             : convert<double, float>(g->buf[g->cur], dst, n, g->stream);
        if (e == cudaSuccess && !on_device)
            e = cudaMemcpyAsync(amp_out, g->staging, (size_t)n * eb, cudaMemcpyDeviceToHost, g->stream);
    }
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return gcuda(g, e, "graph state download");
    return QW_OK;
}

qw_status qw_gwalk_step(qw_gwalk *g, int64_t T) {
    if (!g) return QW_EINVAL;
    NvtxRange nvtx("qw_gwalk_step");
    return run_graph(g, T, 0);
}

qw_status qw_gwalk_step_adjoint(qw_gwalk *g, int64_t T) {
    if (!g) return QW_EINVAL;
    NvtxRange nvtx("qw_gwalk_step_adjoint");
    return run_graph(g, T, 1);
}

qw_status qw_gwalk_probabilities(qw_gwalk *g, void *P_out, qw_rdtype pdtype, int on_device, double *norm_out) {
    if (!g) return QW_EINVAL;
    if (pdtype != QW_R64 && pdtype != QW_R32) return gfail(g, QW_EINVAL, "bad probability dtype");
    const size_t pb = (size_t)g->nvert * (pdtype == QW_R32 ? 4 : 8);
    void *pdst = nullptr;
    cudaError_t e = cudaSuccess;
    if (P_out) {
        if (on_device) {
            pdst = P_out;
        } else {
            if (g->p_bytes < pb) {
                cudaStreamSynchronize(g->stream);
                cudaFree(g->p_dev);
                g->p_dev = nullptr;
                g->p_bytes = 0;
                if ((e = dev_alloc(&g->p_dev, pb)) != cudaSuccess) return gcuda(g, e, "graph probability buffer");
                g->p_bytes = pb;
            }
            pdst = g->p_dev;
        }
    }
    const int nv = (int)g->nvert;
    const bool f64 = g->prec == QW_F64;
    if (pdtype == QW_R32) {
        if (f64) k_graph_marginals<double, float><<<GR_RED_BLOCKS, GR_THREADS, 0, g->stream>>>(
                     g->off_dev, nv, (const Cx<double> *)g->buf[g->cur], (float *)pdst, g->partials);
        else k_graph_marginals<float, float><<<GR_RED_BLOCKS, GR_THREADS, 0, g->stream>>>(
                 g->off_dev, nv, (const Cx<float> *)g->buf[g->cur], (float *)pdst, g->partials);
    } else {
        if (f64) k_graph_marginals<double, double><<<GR_RED_BLOCKS, GR_THREADS, 0, g->stream>>>(
                     g->off_dev, nv, (const Cx<double> *)g->buf[g->cur], (double *)pdst, g->partials);
        else k_graph_marginals<float, double><<<GR_RED_BLOCKS, GR_THREADS, 0, g->stream>>>(
                 g->off_dev, nv, (const Cx<float> *)g->buf[g->cur], (double *)pdst, g->partials);
    }
    k_graph_norm<<<1, 32, 0, g->stream>>>(g->partials, GR_RED_BLOCKS, g->norm_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return gcuda(g, e, "graph marginals launch");
    if (P_out && !on_device)
        if ((e = cudaMemcpyAsync(P_out, pdst, pb, cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess)
            return gcuda(g, e, "graph probability download");
    if (norm_out) {
        if ((e = cudaMemcpyAsync(norm_out, g->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess)
            return gcuda(g, e, "graph norm download");
    }
    if ((norm_out || (P_out && !on_device)) && (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
        return gcuda(g, e, "graph probabilities");
    return QW_OK;
}

qw_status qw_gwalk_set_variant(qw_gwalk *g, int variant) {
    if (!g) return QW_EINVAL;
    if (variant < -1 || variant > 3)
        return gfail(g, QW_EINVAL, "variant must be -1 (default), 0 (push), 1 (pull), 2 or 3 (two-pass)");
    if (variant >= 2) {
        qw_status st = ensure_two_pass(g);
        if (st != QW_OK) return st;
    }
    g->variant = variant;
    return QW_OK;
}

qw_status qw_gwalk_set_window(qw_gwalk *g, size_t bytes) {
    if (!g) return QW_EINVAL;
    if (bytes < amp_bytes(g)) return gfail(g, QW_EINVAL, "the window must hold at least one amplitude");
    if (bytes == g->window) return QW_OK;
    cudaStreamSynchronize(g->stream);
    for (void *p : {(void *)g->lpos_dev, (void *)g->gsl_dev, (void *)g->dst_dev, (void *)g->slot_dev, g->tmp_dev})
        if (p) cudaFree(p);
    g->lpos_dev = nullptr; g->gsl_dev = g->dst_dev = g->slot_dev = nullptr; g->tmp_dev = nullptr;
    g->window = bytes;
    if (g->variant >= 2) return ensure_two_pass(g);
    return QW_OK;
}

qw_status qw_gwalk_get_variant(const qw_gwalk *g, int *variant) {
    if (!g || !variant) return QW_EINVAL;
    *variant = g->variant < 0 ? 0 : g->variant;
    return QW_OK;
}

qw_status qw_gwalk_autotune(qw_gwalk *g, char *report, size_t report_len) {
    if (!g) return QW_EINVAL;
    // time a few steps of each forward form on the current state and keep the
    // faster; the state is saved first and put back afterwards
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const size_t sb = (size_t)g->A * amp_bytes(g);
    qw_status st = ensure_staging(g, std::max<size_t>(sb, 16));
    if (st != QW_OK) return st;
    cudaError_t e = cudaMemcpyAsync(g->staging, g->buf[g->cur], sb, cudaMemcpyDeviceToDevice, g->stream);
    float ms[4] = {0.f, 0.f, 0.f, 0.f};
    const int saved = g->variant;
    // the two-pass forms only where their tables fit (they are built once)
    const int nvar = (e == cudaSuccess && ensure_two_pass(g) == QW_OK) ? 4 : 2;
    for (int v = 0; v < nvar && e == cudaSuccess; ++v) {
        g->variant = v;
        if (run_graph(g, 2, 0) != QW_OK) { e = cudaErrorLaunchFailure; break; }
        cudaEventRecord(e0, g->stream);
        if (run_graph(g, 6, 0) != QW_OK) { e = cudaErrorLaunchFailure; break; }
        cudaEventRecord(e1, g->stream);
        if ((e = cudaEventSynchronize(e1)) == cudaSuccess) cudaEventElapsedTime(&ms[v], e0, e1);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->buf[g->cur], g->staging, sb, cudaMemcpyDeviceToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) { g->variant = saved; return gcuda(g, e, "graph autotune"); }
    int best = 0;
    for (int v = 1; v < nvar; ++v)
        if (ms[v] < ms[best]) best = v;
    g->variant = best;
    if (report && report_len) {
        std::snprintf(report, report_len,
                      "{\"push_ms_per_step\": %.6f, \"pull_ms_per_step\": %.6f, \"two_pass_scatter_ms_per_step\": %.6f, "
                      "\"two_pass_gather_ms_per_step\": %.6f, \"variant\": %d}",
                      ms[0] / 6, ms[1] / 6, nvar > 2 ? ms[2] / 6 : -1.0, nvar > 2 ? ms[3] / 6 : -1.0, g->variant);
    }
    return QW_OK;
}

qw_status qw_gwalk_synchronize(qw_gwalk *g) {
    if (!g) return QW_EINVAL;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    return e == cudaSuccess ? QW_OK : gcuda(g, e, "graph synchronize");
}

}  // extern "C"
