/*
 * qw_oracle.c -- plain, slow, FP64 CPU oracle for the discrete-time coined
 * quantum walk on the cycle Z_N (coin dim 2), the torus Z_Lx x Z_Ly
 * (coin dim 4) and a general graph (coin dim = vertex degree, Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this file.  It shares no
 * code, header, table or helper with the CUDA library; it is written directly
 * from the definitions in Sawerwain & Gielerak, "GPGPU based simulations for
 * one and two dimensional quantum walks" (arXiv:1003.3779):
 *
 *   Sec. 2.1   coin flip transformation C_v acting on the local space of v,
 *              one-step operator U = S (I (x) C), shift S|v,e> = |v',e>.
 *   Sec. 2.2   Z^1 walk on l2(Z) (x) C^2, Z^2 walk on l2(Z^2) (x) C^4,
 *              normalised amplitudes (sum of |alpha|^2 equals 1).
 *   Sec. 3     U = S (C (x) I) restated for the 2D state with two coin
 *              qubits, shift operator (eq. "shift operator"), random broken
 *              links (the RBL function), segment vs. line boundary.
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *   - state: d coin-major planes, plane c holds nsites complex amplitudes
 *     (re, im interleaved doubles), site index v = x (1D) or v = y*Lx + x (2D);
 *   - 1D directions: coin 0 moves x -> x-1, coin 1 moves x -> x+1;
 *   - 2D directions: coin 0: +x, 1: -x, 2: +y, 3: -y;
 *   - moving shift:    S|v,c> = |v + e_c, c>
 *     flip-flop shift: S|v,c> = |v + e_c, c xor 1>
 *     diagonal lattice (2D, Sec. 3 Fig. 1(c)): each coin qubit drives one axis,
 *     coin c = 2j+k moves by ((-1)^j, (-1)^k): S|v,c> = |v + d_c, c>
 *     (periodic torus only, no broken links)
 *   - a closed link (RBL) reflects: the amplitude stays on its site and
 *     takes the one coin slot the closed link leaves empty, which keeps S a
 *     permutation of basis states: S|v,c> = |v, c xor 1> for the moving
 *     shift, S|v,c> = |v, c> for the flip-flop shift (whose open move already
 *     flips the coin); a link that crosses the lattice edge is periodic (bc 0),
 *     closed (bc 1, "segment") or absorbing (bc 2, "line": the amplitude
 *     leaves the finite window of the infinite lattice and is dropped);
 *   - coin modes: 0 one global d x d matrix; 1 one matrix per site;
 *     2 per-site phases, C_v = B . diag(exp(i phi_{v,k})) (phase first).
 *
 * Every step is the push form of the definition: first the coin at every
 * site, phi_v = C_v psi_v, then every amplitude is sent along the shift map.
 * The adjoint step applies the transpose of the same map, then C_v^dagger.
 * No blocking, fusion or reordering beyond that.  Floating point: IEEE
 * double, compiled with -ffp-contract=off.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef double complex cplx;

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

/* Lattice description shared by the routines below. */
typedef struct {
    int ndim;          /* 1 or 2 */
    int64_t nx, ny;    /* extent in x and y (ny = 1 in 1D) */
    int64_t nsites;    /* nx * ny */
    int d;             /* coin dimension: 2 (1D) or 4 (2D) */
    int shift;         /* 0 moving, 1 flip-flop, 2 diagonal lattice (2D) */
    int bc;            /* 0 periodic, 1 segment (reflect), 2 line (absorb) */
    const uint8_t *closed; /* NULL, or ndim*nsites link flags (RBL) */
    int coin_mode;     /* 0 global, 1 per-site matrices, 2 per-site phases */
    const double *coin;/* complex, row-major d x d (mode 0 and 2) or nsites*d*d */
    const double *phi; /* nsites*d reals (mode 2) */
} lattice;

static int lattice_init(lattice *L, int ndim, const int64_t *dims, int shift,
                        int bc, const uint8_t *closed, int coin_mode,
                        const double *coin, const double *phi)
{
    if (ndim != 1 && ndim != 2) return OR_EINVAL;
    if (!dims || dims[0] < 1 || (ndim == 2 && dims[1] < 1)) return OR_EINVAL;
    if (shift < 0 || shift > 2) return OR_EINVAL;
    if (shift == 2 && (ndim != 2 || bc != 0 || closed)) return OR_EINVAL;
    if (bc < 0 || bc > 2) return OR_EINVAL;
    if (coin_mode < 0 || coin_mode > 2 || !coin) return OR_EINVAL;
    if (coin_mode == 2 && !phi) return OR_EINVAL;
    L->ndim = ndim;
    L->nx = dims[0];
    L->ny = ndim == 2 ? dims[1] : 1;
    L->nsites = L->nx * L->ny;
    L->d = 2 * ndim;
    L->shift = shift;
    L->bc = bc;
    L->closed = closed;
    L->coin_mode = coin_mode;
    L->coin = coin;
    L->phi = phi;
    return OR_OK;
}

/* Coin C_v as a d x d complex matrix, row-major (Sec. 2.1: the coin flip
 * transformation C_v acts on the local space of site v). */
static void coin_at(const lattice *L, int64_t v, cplx *C)
{
    const int d = L->d;
    const double *m = L->coin;
    if (L->coin_mode == 1) m += (size_t)v * d * d * 2;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c)
            C[r * d + c] = m[2 * (r * d + c)] + I * m[2 * (r * d + c) + 1];
    if (L->coin_mode == 2) {
        /* C_v = B . diag(e^{i phi_{v,k}}): column k of B times e^{i phi_{v,k}} */
        for (int c = 0; c < d; ++c) {
            double a = L->phi[(size_t)v * d + c];
            cplx e = cos(a) + I * sin(a);
            for (int r = 0; r < d; ++r) C[r * d + c] = C[r * d + c] * e;
        }
    }
}

/* Where the shift sends the basis state |v, c>.  Returns 1 and sets
 * (*vo, *co) when the amplitude lands somewhere, 0 when it is absorbed
 * (line boundary).  Directions: 1D coin 0 -> x-1, coin 1 -> x+1; 2D coin 0
 * +x, 1 -x, 2 +y, 3 -y.  The link used by a move from (x,y) in direction +x
 * is x-link (x,y); in direction -x it is x-link (x-1,y); same for y.  The
 * x-links occupy closed[0 .. nsites), the y-links closed[nsites .. 2 nsites). */
static int shift_map(const lattice *L, int64_t v, int c, int64_t *vo, int *co)
{
    int64_t x = v % L->nx, y = v / L->nx;
    if (L->shift == 2) {   /* diagonal lattice: coin c = 2j+k moves by ((-1)^j, (-1)^k) */
        int64_t dx = (c >> 1) ? -1 : 1, dy = (c & 1) ? -1 : 1;
        int64_t xn = (x + dx + L->nx) % L->nx, yn = (y + dy + L->ny) % L->ny;
        *vo = yn * L->nx + xn;
        *co = c;
        return 1;
    }
    int axis, sgn;
    if (L->ndim == 1) { axis = 0; sgn = (c == 0) ? -1 : +1; }
    else { axis = c >> 1; sgn = (c & 1) ? -1 : +1; }
    int64_t n = axis == 0 ? L->nx : L->ny;
    int64_t p = axis == 0 ? x : y;
    /* the link between p and p+1 is indexed by p; moving -1 uses link p-1 */
    int64_t lp = sgn > 0 ? p : (p - 1 + n) % n;
    int64_t lx = axis == 0 ? lp : x, ly = axis == 0 ? y : lp;
    int closed = 0;
    if (L->closed) closed = L->closed[(size_t)axis * L->nsites + ly * L->nx + lx] != 0;
    int crosses_edge = (lp == n - 1);   /* link (n-1) -- 0 wraps the lattice */
    if (crosses_edge && L->bc == 1) closed = 1;
    if (closed) { *vo = v; *co = L->shift == 1 ? c : (c ^ 1); return 1; }
    if (crosses_edge && L->bc == 2) return 0;
    int64_t q = (p + sgn + n) % n;
    if (axis == 0) x = q; else y = q;
    *vo = y * L->nx + x;
    *co = L->shift == 1 ? (c ^ 1) : c;
    return 1;
}

static void load_state(const lattice *L, const double *psi, cplx *s)
{
    for (int c = 0; c < L->d; ++c)
        for (int64_t v = 0; v < L->nsites; ++v) {
            const double *p = psi + 2 * ((size_t)c * L->nsites + v);
            s[(size_t)v * L->d + c] = p[0] + I * p[1];
        }
}

static void store_state(const lattice *L, const cplx *s, double *psi)
{
    for (int c = 0; c < L->d; ++c)
        for (int64_t v = 0; v < L->nsites; ++v) {
            double *p = psi + 2 * ((size_t)c * L->nsites + v);
            cplx a = s[(size_t)v * L->d + c];
            p[0] = creal(a);
            p[1] = cimag(a);
        }
}

/* One step of U = S (I (x) C) (Sec. 2.1).  in/out are site-major d-vectors. */
static void step_forward(const lattice *L, const cplx *in, cplx *out)
{
    const int d = L->d;
    memset(out, 0, sizeof(cplx) * (size_t)L->nsites * d);
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < L->nsites; ++v) {
        cplx C[16], phi[4];
        coin_at(L, v, C);
        for (int r = 0; r < d; ++r) {
            cplx acc = 0;
            for (int c = 0; c < d; ++c) acc += C[r * d + c] * in[(size_t)v * d + c];
            phi[r] = acc;
        }
        /* the shift is a bijection of basis states (or drops an amplitude),
         * so every target slot receives from exactly one source: no races */
        for (int c = 0; c < d; ++c) {
            int64_t vo; int co;
            if (shift_map(L, v, c, &vo, &co)) out[(size_t)vo * d + co] = phi[c];
        }
    }
}

/* One step of U^dagger = (I (x) C^dagger) S^dagger: S^dagger gathers along
 * the same map that S scatters along, then each site applies C_v^dagger. */
static void step_adjoint(const lattice *L, const cplx *in, cplx *out)
{
    const int d = L->d;
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < L->nsites; ++v) {
        cplx C[16], g[4];
        for (int c = 0; c < d; ++c) {
            int64_t vo; int co;
            g[c] = shift_map(L, v, c, &vo, &co) ? in[(size_t)vo * d + co] : 0;
        }
        coin_at(L, v, C);
        for (int r = 0; r < d; ++r) {
            cplx acc = 0;
            for (int c = 0; c < d; ++c) acc += conj(C[c * d + r]) * g[c];
            out[(size_t)v * d + r] = acc;
        }
    }
}

/* psi_out = U^T psi_in (adjoint = 0) or (U^dagger)^T psi_in (adjoint = 1).
 * psi_in and psi_out: d coin-major planes of nsites complex doubles; they may
 * alias.  closed: NULL or ndim*nsites link flags; closed_per_step != 0 means
 * closed holds T consecutive such masks, mask t used by step t (for the
 * adjoint run, step t applies the adjoint of forward step T-1-t). */
int oracle_evolve(int ndim, const int64_t *dims, int shift, int bc,
                  const uint8_t *closed, int closed_per_step,
                  int coin_mode, const double *coin, const double *phi,
                  const double *psi_in, int64_t T, int adjoint, double *psi_out)
{
    lattice L;
    int st = lattice_init(&L, ndim, dims, shift, bc, closed, coin_mode, coin, phi);
    if (st) return st;
    if (T < 0 || !psi_in || !psi_out) return OR_EINVAL;
    size_t n = (size_t)L.nsites * L.d;
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n);
    if (!a || !b) { free(a); free(b); return OR_ENOMEM; }
    load_state(&L, psi_in, a);
    for (int64_t t = 0; t < T; ++t) {
        if (closed && closed_per_step) {
            int64_t m = adjoint ? (T - 1 - t) : t;
            L.closed = closed + (size_t)m * ndim * L.nsites;
        }
        if (adjoint) step_adjoint(&L, a, b); else step_forward(&L, a, b);
        cplx *tmp = a; a = b; b = tmp;
    }
    store_state(&L, a, psi_out);
    free(a); free(b);
    return OR_OK;
}

/* P(v) = sum_c |psi(v,c)|^2 (the normalisation sums of Sec. 2.2, per site),
 * norm = sum_v P(v) with Neumaier-compensated summation in site order. */
int oracle_probabilities(int ndim, const int64_t *dims, const double *psi,
                         double *P, double *norm)
{
    if ((ndim != 1 && ndim != 2) || !dims || !psi) return OR_EINVAL;
    int64_t ns = dims[0] * (ndim == 2 ? dims[1] : 1);
    int d = 2 * ndim;
    double s = 0.0, comp = 0.0;
    for (int64_t v = 0; v < ns; ++v) {
        double p = 0.0;
        for (int c = 0; c < d; ++c) {
            const double *a = psi + 2 * ((size_t)c * ns + v);
            p += a[0] * a[0] + a[1] * a[1];
        }
        if (P) P[v] = p;
        double t = s + p;
        if (fabs(s) >= fabs(p)) comp += (s - t) + p; else comp += (p - t) + s;
        s = t;
    }
    if (norm) *norm = s + comp;
    return OR_OK;
}

/* Gradient of the region mass L = sum_{v in R, c} |psi_T(v,c)|^2 with respect
 * to the per-site coin phases phi_{v,k}, for C_v = B . diag(e^{i phi_{v,k}})
 * on the 2D torus (coin mode 2).  Stored-trajectory form: psi_0 .. psi_T are
 * all kept.  With lambda_T = 1_R psi_T and lambda_t = U^dagger lambda_{t+1}:
 *     a_t = B^dagger S^dagger lambda_{t+1}  (at site v),
 *     b_t = diag(e^{i phi_v}) psi_t(v),
 *     dL/dphi_{v,k} = sum_t -2 Im( conj(a_t[k]) b_t[k] ).
 * rect = {x0, y0, w, h}: the sites x0 <= x < x0+w, y0 <= y < y0+h.
 * grad: nsites*d doubles, site-major (grad[v*d + k]). */
int oracle_region_grad(const int64_t *dims, int shift, const double *base,
                       const double *phi, const double *psi0, int64_t T,
                       const int64_t *rect, double *loss, double *grad)
{
    lattice L;
    int st = lattice_init(&L, 2, dims, shift, 0, NULL, 2, base, phi);
    if (st) return st;
    if (T < 0 || !psi0 || !rect || !grad) return OR_EINVAL;
    if (rect[0] < 0 || rect[1] < 0 || rect[2] < 0 || rect[3] < 0 ||
        rect[0] + rect[2] > L.nx || rect[1] + rect[3] > L.ny) return OR_EINVAL;
    const int d = 4;
    size_t n = (size_t)L.nsites * d;
    cplx *traj = malloc(sizeof(cplx) * n * (size_t)(T + 1));
    cplx *lam = malloc(sizeof(cplx) * n), *nxt = malloc(sizeof(cplx) * n);
    if (!traj || !lam || !nxt) { free(traj); free(lam); free(nxt); return OR_ENOMEM; }
    load_state(&L, psi0, traj);
    for (int64_t t = 0; t < T; ++t) step_forward(&L, traj + n * t, traj + n * (t + 1));

    const cplx *psiT = traj + n * T;
    double l = 0.0;
    memset(lam, 0, sizeof(cplx) * n);
    for (int64_t y = rect[1]; y < rect[1] + rect[3]; ++y)
        for (int64_t x = rect[0]; x < rect[0] + rect[2]; ++x) {
            int64_t v = y * L.nx + x;
            for (int c = 0; c < d; ++c) {
                cplx a = psiT[(size_t)v * d + c];
                lam[(size_t)v * d + c] = a;
                l += creal(a) * creal(a) + cimag(a) * cimag(a);
            }
        }
    if (loss) *loss = l;
    memset(grad, 0, sizeof(double) * n);

    cplx B[16];
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c)
            B[r * d + c] = base[2 * (r * d + c)] + I * base[2 * (r * d + c) + 1];

    for (int64_t t = T - 1; t >= 0; --t) {
        const cplx *psit = traj + n * t;
        for (int64_t v = 0; v < L.nsites; ++v) {
            cplx mu[4], a[4];
            for (int c = 0; c < d; ++c) {
                int64_t vo; int co;
                mu[c] = shift_map(&L, v, c, &vo, &co) ? lam[(size_t)vo * d + co] : 0;
            }
            for (int r = 0; r < d; ++r) {
                cplx acc = 0;
                for (int c = 0; c < d; ++c) acc += conj(B[c * d + r]) * mu[c];
                a[r] = acc;
            }
            for (int k = 0; k < d; ++k) {
                double ph = phi[(size_t)v * d + k];
                cplx e = cos(ph) + I * sin(ph);
                cplx b = e * psit[(size_t)v * d + k];
                grad[(size_t)v * d + k] += -2.0 * cimag(conj(a[k]) * b);
                nxt[(size_t)v * d + k] = conj(e) * a[k];
            }
        }
        cplx *tmp = lam; lam = nxt; nxt = tmp;
    }
    free(traj); free(lam); free(nxt);
    return OR_OK;
}

/* Number of threads the OpenMP build runs with (1 without OpenMP). */
/* ---------------------------------------------------------------------------
 * Random broken links resampled at every step (Sec. 3: the RBL function, a
 * link that breaks at random).  The randomness is a counter-based generator,
 * Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), written here from that definition:
 * a round maps the counter (c0, c1, c2, c3) with the key (k0, k1) to
 * (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), where hi
 * and lo are the halves of the 64-bit products with M0 = 0xD2511F53 and
 * M1 = 0xCD9E8D57, and the key grows by (0x9E3779B9, 0xBB67AE85) before every
 * round after the first.
 *
 * The two links a site owns (to its +x and +y neighbours) share one draw:
 * link (axis, site) is closed at step t when word `axis` of Philox(counter =
 * (site low 32 bits, site high 32 bits, t, 0), key = (seed low, seed high))
 * is below the threshold (the closing probability times 2^32).
 */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The closed-link masks of steps t0 .. t0+T-1: out holds T masks of ndim*nsites
 * flags in the layout oracle_evolve takes (x-links, then y-links). */
int oracle_link_masks(int ndim, const int64_t *dims, uint64_t seed, uint32_t threshold,
                      int64_t t0, int64_t T, uint8_t *out)
{
    if ((ndim != 1 && ndim != 2) || !dims || T < 0 || !out) return OR_EINVAL;
    int64_t ns = dims[0] * (ndim == 2 ? dims[1] : 1);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t t = 0; t < T; ++t)
        for (int64_t v = 0; v < ns; ++v) {
            uint32_t ctr[4] = {(uint32_t)v, (uint32_t)((uint64_t)v >> 32), (uint32_t)(t0 + t), 0};
            uint32_t r[4];
            oracle_philox4x32_10(ctr, key, r);
            for (int axis = 0; axis < ndim; ++axis)
                out[((size_t)t * ndim + axis) * ns + v] = r[axis] < threshold;
        }
    return OR_OK;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ graphs
 * The discrete-time walk on a general graph G = (V, E) (Sec. 2.1).  The local
 * space of vertex v is spanned by one basis state |v, e> per edge e at v, so
 * the global space has one basis state per (vertex, edge-end) pair: an "arc".
 * Arc form used here: the arcs of vertex v are off[v] .. off[v+1]-1 in a fixed
 * slot order, and partner[a] is the arc |v', e> at the other end of the same
 * edge e = {v, v'} (a loop contributes two arcs at v, partners of each other).
 * The shift S|v,e> = |v',e> is then |a> -> |partner[a]>, an involution, and the
 * coin C_v acts on the d(v) arcs of v.  One step is U = S (I (x) C).
 *
 * Coin modes: 0 Grover, C_v = (2/d(v)) J - I on every vertex (the standard coin
 * of graph walks; J the all-ones matrix); 1 one d(v) x d(v) matrix per vertex,
 * concatenated in vertex order, row-major, interleaved re/im doubles.
 */

/* Build the arc form from an edge list (pairs of vertex indices).  Slots of a
 * vertex follow the order in which its edge ends appear in the list: edge i
 * = (u, w) gives u the arc of end 0 and w the arc of end 1 (both at u for a
 * loop, end 0 first).  off: nvert+1 entries; partner: 2*nedges entries. */
int oracle_graph_arcs(int64_t nvert, int64_t nedges, const int64_t *edges, int64_t *off, int64_t *partner)
{
    if (nvert < 1 || nedges < 0 || (nedges && !edges) || !off || (nedges && !partner)) return OR_EINVAL;
    for (int64_t i = 0; i < 2 * nedges; ++i)
        if (edges[i] < 0 || edges[i] >= nvert) return OR_EINVAL;
    int64_t *deg = calloc((size_t)nvert, sizeof(int64_t));
    int64_t *arc = malloc(sizeof(int64_t) * (size_t)(2 * nedges + 1));
    if (!deg || !arc) { free(deg); free(arc); return OR_ENOMEM; }
    /* each edge end, in list order, takes the next free slot of its vertex */
    for (int64_t i = 0; i < 2 * nedges; ++i) arc[i] = deg[edges[i]]++;
    off[0] = 0;
    for (int64_t v = 0; v < nvert; ++v) off[v + 1] = off[v] + deg[v];
    for (int64_t i = 0; i < 2 * nedges; ++i) arc[i] += off[edges[i]];
    for (int64_t e = 0; e < nedges; ++e) {
        partner[arc[2 * e]] = arc[2 * e + 1];
        partner[arc[2 * e + 1]] = arc[2 * e];
    }
    free(deg); free(arc);
    return OR_OK;
}

typedef struct {
    int64_t nvert, narcs;
    const int64_t *off, *partner;
    int coin_mode;
    const cplx *coins;        /* mode 1 */
    int64_t *coin_at;         /* mode 1: first entry of vertex v's matrix */
} graph;

static int graph_init(graph *G, int64_t nvert, const int64_t *off, const int64_t *partner,
                      int coin_mode, const double *coins)
{
    if (nvert < 1 || !off || off[0] != 0 || (coin_mode != 0 && coin_mode != 1) || (coin_mode == 1 && !coins))
        return OR_EINVAL;
    for (int64_t v = 0; v < nvert; ++v)
        if (off[v + 1] < off[v]) return OR_EINVAL;
    G->nvert = nvert;
    G->narcs = off[nvert];
    G->off = off;
    G->partner = partner;
    G->coin_mode = coin_mode;
    G->coins = (const cplx *)coins;
    G->coin_at = NULL;
    if (G->narcs && !partner) return OR_EINVAL;
    /* S must be a permutation of the arcs that is its own inverse */
    for (int64_t a = 0; a < G->narcs; ++a)
        if (partner[a] < 0 || partner[a] >= G->narcs || partner[partner[a]] != a) return OR_EINVAL;
    if (coin_mode == 1) {
        G->coin_at = malloc(sizeof(int64_t) * (size_t)nvert);
        if (!G->coin_at) return OR_ENOMEM;
        int64_t k = 0;
        for (int64_t v = 0; v < nvert; ++v) {
            int64_t d = off[v + 1] - off[v];
            G->coin_at[v] = k;
            k += d * d;
        }
    }
    return OR_OK;
}

/* entry (r, c) of C_v */
static cplx graph_coin(const graph *G, int64_t v, int64_t r, int64_t c)
{
    int64_t d = G->off[v + 1] - G->off[v];
    if (G->coin_mode == 0) return (r == c ? -1.0 : 0.0) + 2.0 / (double)d;
    return G->coins[G->coin_at[v] + r * d + c];
}

/* U = S (I (x) C): phi = C_v psi on each vertex, then phi(a) moves to partner[a] */
static void graph_step_forward(const graph *G, const cplx *in, cplx *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < G->nvert; ++v) {
        const int64_t o = G->off[v], d = G->off[v + 1] - o;
        for (int64_t r = 0; r < d; ++r) {
            cplx phi = 0;
            for (int64_t c = 0; c < d; ++c) phi += graph_coin(G, v, r, c) * in[o + c];
            out[G->partner[o + r]] = phi;   /* partner is a bijection: no races */
        }
    }
}

/* U^dagger = (I (x) C^dagger) S^dagger, and S^dagger = S (an involution) */
static void graph_step_adjoint(const graph *G, const cplx *in, cplx *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < G->nvert; ++v) {
        const int64_t o = G->off[v], d = G->off[v + 1] - o;
        for (int64_t r = 0; r < d; ++r) {
            cplx acc = 0;
            for (int64_t c = 0; c < d; ++c) acc += conj(graph_coin(G, v, c, r)) * in[G->partner[o + c]];
            out[o + r] = acc;
        }
    }
}

/* psi_out = U^T psi_in (or (U^dagger)^T); psi: narcs complex doubles in arc
 * order.  psi_in and psi_out may alias. */
int oracle_graph_evolve(int64_t nvert, const int64_t *off, const int64_t *partner, int coin_mode,
                        const double *coins, const double *psi_in, int64_t T, int adjoint, double *psi_out)
{
    graph G = {0};
    int st = graph_init(&G, nvert, off, partner, coin_mode, coins);
    if (st) { free(G.coin_at); return st; }
    if (T < 0 || (G.narcs && (!psi_in || !psi_out))) { free(G.coin_at); return OR_EINVAL; }
    size_t n = (size_t)G.narcs;
    cplx *a = malloc(sizeof(cplx) * (n ? n : 1)), *b = malloc(sizeof(cplx) * (n ? n : 1));
    if (!a || !b) { free(a); free(b); free(G.coin_at); return OR_ENOMEM; }
    if (n) memcpy(a, psi_in, sizeof(cplx) * n);
    for (int64_t t = 0; t < T; ++t) {
        if (adjoint) graph_step_adjoint(&G, a, b); else graph_step_forward(&G, a, b);
        cplx *tmp = a; a = b; b = tmp;
    }
    if (n) memcpy(psi_out, a, sizeof(cplx) * n);
    free(a); free(b); free(G.coin_at);
    return OR_OK;
}

/* P(v) = sum over the arcs of v of |psi(a)|^2, norm = sum_v P(v) (Neumaier
 * compensated, vertex order). */
int oracle_graph_probabilities(int64_t nvert, const int64_t *off, const double *psi, double *P, double *norm)
{
    if (nvert < 1 || !off || !psi || !P) return OR_EINVAL;
    const cplx *s = (const cplx *)psi;
    double sum = 0.0, comp = 0.0;
    for (int64_t v = 0; v < nvert; ++v) {
        double p = 0.0;
        for (int64_t a = off[v]; a < off[v + 1]; ++a) p += creal(s[a]) * creal(s[a]) + cimag(s[a]) * cimag(s[a]);
        P[v] = p;
        double t = sum + p;
        comp += fabs(sum) >= fabs(p) ? (sum - t) + p : (p - t) + sum;
        sum = t;
    }
    if (norm) *norm = sum + comp;
    return OR_OK;
}
