// k_window1d.cuh -- many generic steps of a 1D walk whose light cone is still
// narrow, in one CTA: the line computation window of Sec. 3 (a walker started
// at MP steps only the sites [l_i, r_i] its light cone has reached, which
// widen by one site per step on each side and stop at the ends of the line).
//
// On the segment and the line such a window is a few thousand sites for
// hundreds of steps, so a launch per step costs far more than the step.  One
// CTA keeps the window's state in shared memory, in the walk's storage format,
// and runs up to WIN_MAX_STEPS steps with a barrier between the coin phase and
// the shift phase of each.  Each step is the one k_step_generic_tile1d makes:
// the same coin row per site (gen_entry), the same link states (link_state,
// with the step's Philox draw), the same pull rule and the same drift gain, so
// the state after the launch equals that of the per-step launches bit for bit.
// Sites outside the support box are zero and stay zero until the box reaches
// them; the window is the box after the launch's steps.
#pragma once
#include "k_generic.cuh"

namespace qw {

constexpr int WIN_THREADS = 1024;
constexpr int WIN_MAX_STEPS = 256;               // steps per launch
constexpr size_t WIN_SMEM_BYTES = 200 * 1024;   // dynamic shared memory of the window CTA

// drift gains of the launch's steps, in the compute real
template <class R>
struct WinGains {
    R v[WIN_MAX_STEPS];
};

// Shared-memory layout for a window of wn sites: phi of sites w0 - 1 .. w0 + wn
// (2 coin values each), the state (d = 2 coins, SLOTS_PER_COIN slots each, of
// SLOT_BYTES per site) and one link-state byte per owner w0 - 1 .. w0 + wn - 1.
template <int P>
constexpr size_t win_ph_bytes(int64_t wn) { return ((size_t)2 * (wn + 2) * sizeof(Cx<typename St<P>::real>) + 15) / 16 * 16; }
template <int P>
constexpr size_t win_state_bytes(int64_t wn) {
    return ((size_t)2 * St<P>::SLOTS_PER_COIN * St<P>::SLOT_BYTES * wn + 15) / 16 * 16;
}
template <int P>
constexpr size_t win_smem(int64_t wn) { return win_ph_bytes<P>(wn) + win_state_bytes<P>(wn) + (size_t)wn + 2; }
// the widest window that fits WIN_SMEM_BYTES
template <int P>
constexpr int64_t win_capacity() {
    int64_t wn = (int64_t)(WIN_SMEM_BYTES / (2 * sizeof(Cx<typename St<P>::real>) +
                                            2 * St<P>::SLOTS_PER_COIN * St<P>::SLOT_BYTES + 1));
    while (wn > 0 && win_smem<P>(wn) > WIN_SMEM_BYTES) --wn;
    return wn;
}

// nsteps forward steps of the walk on the segment or the line (no wrap): the
// input's support box is [b0, b0 + bw); the window [w0, w0 + wn) is that box
// after nsteps steps (cut at the ends), read from `in` and written to `out`.
// LINKS: fixed or random broken links, whose states are drawn per step into
// shared memory; without them a link is open unless it is the edge link
// (owned by site n - 1, and seen by site 0 from its left), whose state is the
// boundary's, so nothing is stored.
template <int P, int SHIFT, int CK, bool LINKS>
__global__ void __launch_bounds__(WIN_THREADS)
k_step1d_window(View in, View out, GenGeom g, CoinP<typename St<P>::real> cp,
                const Cx<typename St<P>::real> *__restrict__ coins, const float *__restrict__ phi, int b0, int bw,
                int nsteps, int w0, int wn, WinGains<typename St<P>::real> gains) {
    using real = typename St<P>::real;
    using S = St<P>;
    using C = Cx<real>;
    extern __shared__ __align__(16) unsigned char wsm[];
    C *ph0 = reinterpret_cast<C *>(wsm);                  // phi, coin 0, of site w0 - 1 + i at i
    C *ph1 = ph0 + (wn + 2);                              // coin 1
    const View sv{wsm + win_ph_bytes<P>(wn), (int64_t)wn, 2};   // the window's state, site w0 + i at i
    unsigned char *ls = wsm + win_ph_bytes<P>(wn) + win_state_bytes<P>(wn);   // owner w0 - 1 + i at i
    const int n = (int)g.nx;                              // < 2^30 (launcher)
    const int nt = (int)blockDim.x;
    // the edge link's state without broken links: reflecting (segment) or absorbing (line)
    const unsigned char edge = g.bc == QW_BC_SEGMENT ? 1 : 2;

    for (int i = threadIdx.x; i < wn; i += nt) {
#pragma unroll
        for (int c = 0; c < 2; ++c) S::st(sv, c, i, S::ld(in, c, (int64_t)w0 + i));
    }
    __syncthreads();
    for (int t = 0; t < nsteps; ++t) {
        // outputs of this step: the box after it
        const int o0 = max(0, b0 - (t + 1)), o1 = min(n, b0 + bw + t + 1);
        const uint32_t rstep = g.rstep + (uint32_t)t;
        // phase 1: phi of sites o0 - 1 .. o1 (zero off the lattice and outside
        // the window, where the state is zero) and, with broken links, the links
        // owned by o0 - 1 .. o1 - 1
        for (int x = o0 - 1 + (int)threadIdx.x; x <= o1; x += nt) {
            const int i = x - w0 + 1;
            C v0 = czero<real>(), v1 = czero<real>();
            if (x >= 0 && x < n && x >= w0 && x < w0 + wn) {
                const C a0 = S::ld(sv, 0, x - w0), a1 = S::ld(sv, 1, x - w0);
                C e[2];
                if (CK == CK_PHASE) gen_phases<real>(phi, x, 2, e);
                v0 = cfma(gen_entry<CK, real>(cp, coins, e, 2, x, 0, 0), a0, v0);
                v0 = cfma(gen_entry<CK, real>(cp, coins, e, 2, x, 0, 1), a1, v0);
                v1 = cfma(gen_entry<CK, real>(cp, coins, e, 2, x, 1, 0), a0, v1);
                v1 = cfma(gen_entry<CK, real>(cp, coins, e, 2, x, 1, 1), a1, v1);
            }
            ph0[i] = v0;
            ph1[i] = v1;
            if (LINKS && x < o1) {
                // site 0's left link is the edge link, owned by site n - 1
                const int owner = x < 0 ? n - 1 : x;
                uint32_t rnd = 0u;
                if (g.rthr) rnd = philox_words01((uint32_t)owner, 0u, rstep, 0u, g.rk0, g.rk1).x;
                ls[i] = link_state(g, 0, owner, 0, rnd);
            }
        }
        __syncthreads();
        // phase 2: each output site pulls its two amplitudes (as the 1D tile)
        const real gain = gains.v[t];
        for (int x = o0 + (int)threadIdx.x; x < o1; x += nt) {
            const int ex = x - w0 + 1;
            // states of the links to the right (owned by x) and to the left (owned by x - 1)
            const int sr = LINKS ? ls[ex] : (x == n - 1 ? edge : 0);
            const int sl = LINKS ? ls[ex - 1] : (x == 0 ? edge : 0);
            C out2[2];
#pragma unroll
            for (int co = 0; co < 2; ++co) {
                int nb, st;
                if (SHIFT == QW_SHIFT_MOVING) {   // from x + 1 (coin 0) or x - 1 (coin 1), same coin
                    nb = co == 0 ? ex + 1 : ex - 1;
                    st = co == 0 ? sr : sl;
                } else {                          // from x - 1 (coin 0) or x + 1 (coin 1), coin co ^ 1
                    nb = co == 0 ? ex - 1 : ex + 1;
                    st = co == 0 ? sl : sr;
                }
                const int from = SHIFT == QW_SHIFT_MOVING ? co : (co ^ 1);   // coin of the arriving value
                C val = czero<real>();
                if (st == 0) val = from == 0 ? ph0[nb] : ph1[nb];
                else if (st == 1) val = from == 0 ? ph1[ex] : ph0[ex];   // reflected: the other coin of x
                out2[co] = rmul(gain, val);
            }
            S::st(sv, 0, x - w0, out2[0]);
            S::st(sv, 1, x - w0, out2[1]);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < wn; i += nt) {
#pragma unroll
        for (int c = 0; c < 2; ++c) S::st(out, c, (int64_t)w0 + i, S::ld(sv, c, i));
    }
}

}  // namespace qw
