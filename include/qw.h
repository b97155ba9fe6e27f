/*
 * qw.h -- C ABI of the GB300 (sm_103a) discrete-time coined quantum-walk library.
 *
 * The operation is the one-step walk operator of Sawerwain & Gielerak,
 * "GPGPU based simulations for one and two dimensional quantum walks"
 * (arXiv:1003.3779):
 *
 *   U = S (I (x) C)                      (Sec. 2.1, restated as S (C (x) I) in Sec. 3)
 *   C = (C_v)_v  unitary coin on the coin register of each site v   (Sec. 2.1)
 *   S |v, e> = |v', e>  moves the walker along the edge its coin names (Sec. 2.1)
 *
 * on the lattice Z^1 (here the cycle Z_N, coin space C^2, Sec. 2.2) and Z^2
 * (here the torus Z_Lx x Z_Ly, coin space C^4 = two coin qubits, Sec. 2.2 and
 * the two-qubit state of Sec. 3).  Probabilities are the coin marginals
 * P(v) = sum_c |psi(v,c)|^2, whose sum is the normalisation of Sec. 2.2.
 *
 * Conventions used by every call:
 *   - coin basis / directions: 1D coin 0 moves x -> x-1, coin 1 moves x -> x+1;
 *     2D coin 0: +x, 1: -x, 2: +y, 3: -y.  (The paper's own labelling of the
 *     2D shift equation in Sec. 3 is a permutation of this basis.)
 *   - moving shift:    S|v,c> = |v + e_c, c>;
 *     flip-flop shift: S|v,c> = |v + e_c, c xor 1>;
 *     diagonal lattice (2D): S|v,c> = |v + d_c, c>, d_c = ((-1)^j, (-1)^k), c = 2j+k.
 *   - a closed link (broken link, Sec. 3 "RBL") reflects: the amplitude stays
 *     on its site, in coin c xor 1 (moving) or c (flip-flop).
 *   - state layout seen by callers: d coin-major planes of nsites complex
 *     numbers, re/im interleaved; site index v = x (1D) or v = y*Lx + x (2D).
 *     Inside the library the planes are padded; callers never see the padding.
 *   - coins are row-major d x d complex matrices, re/im interleaved doubles;
 *     C_v acts as phi(v)[r] = sum_c C_v[r][c] psi(v)[c].
 *
 * Ownership: a handle owns all of its device memory.  Pointers passed in are
 * borrowed for the duration of the call only and are never freed by the
 * library; device pointers may come from any allocator (e.g. torch tensors).
 * Streams: every call is ordered on the handle's CUDA stream.  Calls that
 * write to host memory or return a host scalar (norm, loss) synchronise the
 * stream before returning; all others are asynchronous.
 * Errors: every call returns a qw_status and never aborts or traps.  After an
 * error the handle stays valid; qw_last_error() holds a message.  A CUDA
 * error is reported as QW_ECUDA.  The state is never renormalised.
 * Threads: a handle may be used by one host thread at a time.
 */
#ifndef QW_H
#define QW_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qw_walk qw_walk;     /* opaque, library-owned */
typedef struct qw_batch qw_batch;   /* opaque, library-owned */

typedef enum {
    QW_OK = 0,
    QW_EINVAL = 1,        /* bad argument (null pointer, size, enum value) */
    QW_ENOMEM = 2,        /* device or host allocation failed */
    QW_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    QW_ESTATE = 4,        /* call not valid in the handle's current state */
    QW_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    QW_EUNSUPPORTED = 6   /* valid request this build does not implement */
} qw_status;

typedef enum {
    QW_BC_PERIODIC = 0,   /* cycle / torus */
    QW_BC_SEGMENT = 1,    /* finite segment: the links across the edge are closed (Sec. 3, Fig. 2 "segment") */
    QW_BC_LINE = 2        /* finite window of the infinite line: amplitude crossing the edge is dropped (Sec. 3 "line") */
} qw_boundary;

/* Shift S (Sec. 2.1, Sec. 3).  QW_SHIFT_DIAGONAL is the diagonal lattice of
 * Sec. 3 (Fig. 1(c)) on the torus: each coin qubit drives one axis, coin
 * c = 2j+k moves the walker by ((-1)^j, (-1)^k); 2D, periodic, no broken links. */
typedef enum { QW_SHIFT_MOVING = 0, QW_SHIFT_FLIPFLOP = 1, QW_SHIFT_DIAGONAL = 2 } qw_shift;

/* Storage / arithmetic of the state.  QW_F64: double storage and arithmetic.
 * QW_F32: float.  QW_F32_BF16STORE: bfloat16 storage, float arithmetic (one
 * rounding to bf16 per HBM round trip).  QW_F32_COMP: each amplitude is an
 * unevaluated float pair hi+lo, arithmetic in double-float (TwoSum /
 * TwoProduct), about 44 significant bits. */
typedef enum { QW_F64 = 0, QW_F32 = 1, QW_F32_BF16STORE = 2, QW_F32_COMP = 3 } qw_precision;

/* Element type of caller-side state buffers. */
typedef enum { QW_C128 = 0, QW_C64 = 1 } qw_cdtype;
/* Element type of caller-side real buffers (probabilities). */
typedef enum { QW_R64 = 0, QW_R32 = 1 } qw_rdtype;

/* ---------------------------------------------------------------- walks */

/* Create a walk on the cycle (ndim=1, dims[0]=N, coin_dim=2) or the torus
 * (ndim=2, dims={Lx, Ly}, coin_dim=4), Sec. 2.2.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream).  The coin starts as the identity, the state
 * as all zeros.  Allocates two state buffers on the current device.
 * QW_EINVAL for ndim not 1/2, coin_dim != 2*ndim, a dimension < 1, or an
 * unknown enum; QW_ENOMEM if the device allocation fails. */
qw_status qw_create(int ndim, const int64_t *dims, int coin_dim, qw_boundary bc,
                    qw_shift shift, qw_precision prec, void *cuda_stream,
                    qw_walk **out);

/* Release every resource of the handle (NULL is accepted). */
qw_status qw_destroy(qw_walk *w);

/* Coin flip transformation (Sec. 2.1).  per_site = 0: `coin` holds one d x d
 * matrix (2*d*d doubles); per_site = 1: nsites matrices, site-major.
 * on_device selects whether `coin` is a host or device pointer.  Unitarity is
 * the caller's responsibility (the walk is linear either way). */
qw_status qw_set_coin(qw_walk *w, const double *coin, int per_site, int on_device);

/* Per-site phase coin C_v = base . diag(e^{i phi_{v,k}}) (the phase acts
 * first).  base: one d x d matrix (host doubles, 2*d*d).  phi: nsites*d reals,
 * site-major (phi[v*d + k]), float, host or device (on_device).  The phases are
 * copied; later changes to the caller's buffer have no effect. */
qw_status qw_set_coin_phases(qw_walk *w, const double *base, const float *phi, int on_device);

/* Broken links (Sec. 3, RBL).  closed: ndim*nsites bytes, nonzero = closed;
 * bytes [0, nsites) are the links from (x,y) to (x+1,y), bytes
 * [nsites, 2 nsites) (2D only) the links from (x,y) to (x,y+1).  NULL clears
 * all.  Host or device (on_device). */
qw_status qw_set_links(qw_walk *w, const uint8_t *closed, int on_device);

/* Links broken at random afresh at every step (Sec. 3, RBL resampled per
 * step), on top of the fixed mask of qw_set_links.  The link of axis a
 * (0: x, 1: y) at link site v = y*nx + x (the link from v to its +a
 * neighbour) is closed during step t when word a of Philox4x32-10 (Salmon et
 * al., SC 2011) with counter (v mod 2^32, v >> 32, t mod 2^32, 0) and key
 * (seed mod 2^32, seed >> 32) is below floor(p * 2^32) (capped at 2^32 - 1).  p in [0, 1]; p = 0 turns it
 * off.  `step` is the index t of the next forward step: qw_step uses t and
 * counts up, qw_step_adjoint counts down and then uses t, so a forward run
 * followed by its adjoint retraces the same masks.  QW_EINVAL for p outside
 * [0, 1]; QW_EUNSUPPORTED on the diagonal lattice.  The walk then runs the
 * generic kernel, and qw_backward is rejected. */
qw_status qw_set_link_noise(qw_walk *w, double p, uint64_t seed, int64_t step);

/* Index of the next forward step of the random links (see qw_set_link_noise). */
qw_status qw_get_link_step(const qw_walk *w, int64_t *step);

/* Replace the state: amp holds d coin-major planes of nsites complex numbers
 * of type dtype (host or device).  Converted to the walk's precision on the
 * device (QW_F32_COMP keeps the rounding residue of a QW_C128 input). */
qw_status qw_set_state(qw_walk *w, const void *amp, qw_cdtype dtype, int on_device);

/* Copy the state out in the same layout (converted to dtype). */
qw_status qw_get_state(qw_walk *w, void *amp_out, qw_cdtype dtype, int on_device);

/* Apply U^T (T >= 0; T = 0 does nothing).  Runs ceil(T/k) fused kernels, each
 * advancing k steps per HBM round trip (temporal blocking), k from the plan. */
qw_status qw_step(qw_walk *w, int64_t T);

/* Apply (U^dagger)^T: the walk run backward. */
qw_status qw_step_adjoint(qw_walk *w, int64_t T);

/* Coin marginals P(v) = sum_c |psi(v,c)|^2 into P_out (nsites values of type
 * pdtype, host or device; may be NULL) and the total norm sum_v P(v),
 * accumulated in double in a fixed order (bitwise reproducible), into
 * *norm_out (host; may be NULL).  Synchronises when norm_out is given or
 * P_out is a host pointer. */
qw_status qw_probabilities(qw_walk *w, void *P_out, qw_rdtype pdtype, int on_device,
                           double *norm_out);

/* Run `count` independent walks of T steps from host states, the way a
 * server would: the result is what qw_set_state(host), qw_step(T) and
 * qw_probabilities(host) give for each input in turn, bit for bit, but the
 * copy of state i+1 in and of the marginals of state i-1 out overlap the
 * steps of state i (two copy streams, a third state buffer that the call
 * allocates once).  Input i starts at amp_in + i*in_stride bytes, in the
 * layout of qw_set_state; dtype must match the precision (QW_C64 for QW_F32,
 * QW_C128 for QW_F64; else QW_EUNSUPPORTED).  P of run i goes to
 * P_out + i*p_stride bytes (nsites values of pdtype), its norm to norms_out[i]
 * (may be NULL; any host memory: the norms are copied once, at the end).  A stride of 0 reuses one buffer for every run (the last
 * run's P remains).  Host buffers should be pinned for the copies to overlap.
 * Synchronous: returns when every P is on the host; the walk's state is then
 * the last run's final state. */
qw_status qw_run_host_batch(qw_walk *w, int count, const void *amp_in, int64_t in_stride, qw_cdtype dtype,
                            int64_t T, void *P_out, int64_t p_stride, qw_rdtype pdtype, double *norms_out);

/* Execution plan of qw_step: temporal depth k (steps per kernel, >= 1) and
 * tile (sites per thread in 1D, 0 = library default).  k = 0 restores the
 * default / tuned plan.  QW_EINVAL for a combination the kernels reject. */
qw_status qw_set_plan(qw_walk *w, int depth_k, int tile);
qw_status qw_get_plan(const qw_walk *w, int *depth_k, int *tile);

/* The same with the 1D kernel variant: 0 = independent warp tiles (each warp
 * recomputes a halo of k sites on both sides), 1 = time-skewed sweep (a warp
 * walks a segment chunk by chunk in a frame that slides one site per step and
 * hands two values per step to the next chunk; no halo except one warm-up
 * chunk per segment).  For variant 1, tile is the sites per lane: 16 or 32 in
 * FP32 / BF16 (chunks of 512 or 1024 sites), 8 in FP64 (256 sites); 0 picks
 * the larger tile when the cycle holds two of its chunks.  Variant 1 needs the
 * periodic cycle, N at least one chunk (any N: the last chunk wraps round), a
 * global coin, FP32 / BF16 / FP64 and k < chunk / 2, else QW_EINVAL.
 * qw_set_plan selects variant 0. */
qw_status qw_set_plan_ex(qw_walk *w, int depth_k, int tile, int variant);
qw_status qw_get_plan_ex(const qw_walk *w, int *depth_k, int *tile, int *variant);

/* Time the candidate plans on this walk (CUDA events on the walk's stream,
 * reading the current state, writing only the scratch buffer, so the state is
 * unchanged) and keep the fastest.  Results are cached per (lattice shape,
 * precision, coin kind) in memory and, if the environment variable
 * QW_TUNE_CACHE names a file, in that JSON file.  report (may be NULL)
 * receives a one-line JSON summary, truncated to report_len bytes. */
qw_status qw_autotune(qw_walk *w, char *report, size_t report_len);

/* Light-cone clipping (the computation window of the paper's line walk,
 * Sec. 3: a walker started at one site is stepped only on the window
 * [MP - ES - i, MP + ES + i] its light cone has reached after i steps; the
 * complexity analysis of Sec. 3.1 counts (2i + 1)^2 sites in 2D).  With
 * clipping on (the default), qw_set_state searches the bounding box of the
 * state's nonzero amplitudes on the GPU, and every step kernel then runs only
 * on that box widened by its steps, until the box covers the lattice: on the
 * cycle and the torus the box wraps; on the segment and the line it stops at
 * the ends (with broken links too), and in 1D, while the box after the next
 * steps fits one CTA's shared memory (about 6200 sites in FP32), up to 256
 * steps run in one launch with the state on chip (qw_describe's path
 * "k_step1d_window").  The adjoint with a boundary or broken
 * links, and per-site coins on the torus, run kernels that step the whole
 * lattice; the box still widens with them.  The first qw_step or
 * qw_step_adjoint after qw_set_state waits for the search (not for other
 * queued work); while the walk's stream is being captured into a CUDA graph
 * nothing waits: the search is skipped and the steps run on the whole lattice.  A dense state costs about one wave of the search.  Every
 * amplitude equals that of stepping the whole lattice with the same plan, bit
 * for bit (a zero may differ in sign).  on = 0 turns it off
 * (the current state is then stepped in full); on = 1 takes effect at the next
 * qw_set_state.  qw_describe reports the box ("support": [x0, w, y0, h],
 * columns [x0, x0 + w) and rows [y0, y0 + h) modulo the lattice, "full" or
 * "pending"). */
qw_status qw_set_clipping(qw_walk *w, int on);

/* One-line JSON description of the handle: lattice, precision, the coin kind
 * the kernels specialise on ("real", "complex", "grover", "hadamard2",
 * "per_site", "phase", "hadamard_class"), the plan (k, tile), which kernel
 * family runs the step and the bytes of one state buffer.  Truncated to len. */
qw_status qw_describe(const qw_walk *w, char *buf, size_t len);

/* Number of sites (N or Lx*Ly). */
int64_t qw_nsites(const qw_walk *w);

/* Wait for all work queued on the walk's stream. */
qw_status qw_synchronize(qw_walk *w);

/* Gradient of the region mass L = sum_{v in rect, c} |psi_T(v,c)|^2 with
 * respect to the per-site coin phases phi_{v,k} set by qw_set_coin_phases
 * (2D torus only), starting from the current state.  rect = {x0, y0, w, h}:
 * x0 <= x < x0+w, y0 <= y < y0+h, inside the lattice.  Runs T forward steps
 * storing psi every K steps (checkpoints), then walks back with U^dagger,
 * re-seeding psi from the checkpoint at each segment boundary so FP32 drift
 * is bounded by K steps, and accumulates
 *     dL/dphi_{v,k} = sum_t -2 Im( conj(a_t(v)_k) (D_v psi_t(v))_k ),
 *     a_t = B^dagger S^dagger lambda_{t+1},  lambda_T = 1_rect psi_T,
 * in double.  grad_phi: nsites*d doubles, site-major (host or device).
 * *loss_out (host, may be NULL) receives L.  The walk's state is left at psi_T.
 * QW_ESTATE if no phase coin is set. */
qw_status qw_backward(qw_walk *w, const int64_t rect[4], int64_t T, int64_t K,
                      double *loss_out, double *grad_phi, int on_device);

/* Coin marginals and norm of a state the caller owns, without allocating any
 * memory: the same P(v) = sum_c |psi(v,c)|^2 and fixed-order double norm as
 * qw_probabilities, for callers that cannot call cudaMalloc -- a thread that
 * runs while another thread holds a global-mode stream capture (cudaMalloc
 * fails then), an application whose own allocator has already reserved the
 * device memory, or a latency-critical path that cannot take cudaMalloc's
 * implicit device synchronisation.  The paper has no counterpart.
 *
 * amp: device pointer, coin_dim dense coin-major planes of nsites complex
 * numbers (QW_C64 or QW_C128), element-aligned.  P_out: device pointer to
 * nsites values of pdtype, or NULL.  norm_out: device pointer to one double,
 * or NULL.  Everything is enqueued on cuda_stream; nothing synchronises.
 *
 * Scratch: one double per 8192 sites in a fixed array inside the library
 * (16384 doubles = 128 KiB, held by every GPU that loads the library until the
 * process exits), so nsites is limited to 16384 * 8192 = 2^27; larger sizes,
 * a NULL amp, nsites < 1, a coin_dim other than 2 or 4, or an unknown dtype
 * return QW_EINVAL before anything is launched.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with the device
 * current) and loads the entry point's three kernels on that device; make that
 * first call before any stream capture.  The address is kept until the process
 * exits (a cudaDeviceReset makes it stale, with every other handle of this
 * library).  All calls share the array: each call overwrites the slots it
 * uses, so nothing needs clearing, but two calls that overlap on the GPU
 * (different streams, or different host threads) race on it and must be
 * ordered by the caller.
 * Returns QW_ECUDA if the lookup or a launch fails. */
qw_status qw_probabilities_noalloc(const void *amp, qw_cdtype dtype, int coin_dim, int64_t nsites,
                                   void *P_out, qw_rdtype pdtype, double *norm_out,
                                   void *cuda_stream);

/* ---------------------------------------------------------------- graphs */

/* The walk on a general graph G = (V, E) (Sec. 2.1).  The local space of
 * vertex v has one basis state |v, e> per edge e at v; the state holds one
 * complex amplitude per such (vertex, edge end) pair, an "arc".  Arc form of
 * a graph: the arcs of vertex v are off[v] .. off[v+1]-1 (its coin slots, in
 * a fixed order), and partner[a] is the arc |v', e> at the other end of a's
 * edge e = {v, v'}; a loop gives v two arcs that are each other's partner.
 * One step is U = S (I (x) C):
 *   phi(a) = sum_j C_v[i][j] psi(off[v] + j)   for a = off[v] + i,
 *   psi'(partner[a]) = phi(a)                  (S|v,e> = |v',e>).
 * On the cycle or torus with the lattice's coin slots as arc slots this is
 * the flip-flop lattice walk. */
typedef struct qw_gwalk qw_gwalk;   /* opaque, library-owned */

/* Coins of a graph walk: QW_GCOIN_GROVER, C_v = (2/d(v)) J - I at every vertex
 * (J all ones; no matrix is passed); QW_GCOIN_UNIFORM, one d x d matrix for a
 * graph whose vertices all have degree d; QW_GCOIN_PER_VERTEX, one d(v) x d(v)
 * matrix per vertex, concatenated in vertex order. */
typedef enum { QW_GCOIN_GROVER = 0, QW_GCOIN_UNIFORM = 1, QW_GCOIN_PER_VERTEX = 2 } qw_gcoin;

/* Arc form from an edge list (host memory): edges holds nedges pairs (u, w) of
 * vertex indices in [0, nvert).  Each vertex's slots follow the order in which
 * its edge ends appear in the list (end u of pair k before end w).  off:
 * nvert + 1 entries, partner: 2*nedges entries, written by the call.
 * QW_EINVAL for a vertex index out of range. */
qw_status qw_graph_arcs(int64_t nvert, int64_t nedges, const int64_t *edges, int64_t *off, int64_t *partner);

/* Create a graph walk (nvert >= 1 vertices, arcs off[nvert] < 2^31) from the
 * arc form in host memory (copied; the caller keeps its arrays).  The state
 * starts at zero and the coin is Grover.  prec: QW_F64 or QW_F32 (others
 * QW_EUNSUPPORTED).  QW_EINVAL when off is not non-decreasing from 0 or
 * partner is not an involution of [0, off[nvert]).  Device memory: two state
 * buffers (A amplitudes each), off, partner and, for graphs that are not
 * regular of degree 2 or 4, the vertex of each arc (4 bytes per arc). */
qw_status qw_gwalk_create(int64_t nvert, const int64_t *off, const int64_t *partner, qw_precision prec,
                          void *cuda_stream, qw_gwalk **out);
qw_status qw_gwalk_destroy(qw_gwalk *g);

/* Set the coin (see qw_gcoin).  coins: row-major complex doubles (re/im),
 * d*d entries (uniform) or sum_v d(v)^2 entries (per vertex), host or device
 * (on_device); NULL for Grover.  QW_EINVAL for a uniform coin on a graph that
 * is not regular. */
qw_status qw_gwalk_set_coin(qw_gwalk *g, qw_gcoin mode, const double *coins, int on_device);

/* Replace / read the state: off[nvert] complex amplitudes in arc order, of
 * type dtype, host or device (on_device). */
qw_status qw_gwalk_set_state(qw_gwalk *g, const void *amp, qw_cdtype dtype, int on_device);
qw_status qw_gwalk_get_state(qw_gwalk *g, void *amp_out, qw_cdtype dtype, int on_device);

/* Apply U^T, or (U^dagger)^T = ((I (x) C^dagger) S)^T.  One kernel per step
 * (plus, for the Grover coin, a pre-pass over the vertices of degree > 32). */
qw_status qw_gwalk_step(qw_gwalk *g, int64_t T);
qw_status qw_gwalk_step_adjoint(qw_gwalk *g, int64_t T);

/* P(v) = sum over the arcs of v of |psi(a)|^2 (nvert values of type pdtype,
 * host or device; may be NULL) and the norm sum_v P(v), accumulated in double
 * in a fixed order, into *norm_out (host; may be NULL). */
qw_status qw_gwalk_probabilities(qw_gwalk *g, void *P_out, qw_rdtype pdtype, int on_device, double *norm_out);

/* Form of the forward step: 0 push (each arc's thread reads its own vertex and
 * writes the partner arc), 1 pull (reads the partner's vertex, writes its own
 * arc), 2 and 3 two passes through L2-sized destination buckets (the first
 * computes the coin and writes bucket runs, the second permutes within one
 * L2-resident window by scattered writes (2) or gathered reads (3)); -1
 * restores the default (push).  Every form gives the same bits.  Forms 2 and 3
 * build tables on first use (host work O(arcs); device memory 14 bytes per arc
 * plus one more state buffer).  On graphs of degree 2 or 4, a qw_gwalk_step
 * call of T >= 2 steps in form 3 fuses each step's gather with the next
 * step's coin and bucketing (T + 1 passes); it uses the input state buffer as
 * scratch, so a launch error in that call leaves no valid state. */
qw_status qw_gwalk_set_variant(qw_gwalk *g, int variant);

/* Output bytes each destination bucket of forms 2 and 3 covers (default
 * 16 MiB, an eighth of L2); the tables are rebuilt.  QW_EINVAL below one
 * amplitude. */
qw_status qw_gwalk_set_window(qw_gwalk *g, size_t bytes);
qw_status qw_gwalk_get_variant(const qw_gwalk *g, int *variant);

/* Time the forms on the current state (which is saved and restored), keep
 * the fastest, and write a JSON report. */
qw_status qw_gwalk_autotune(qw_gwalk *g, char *report, size_t report_len);

qw_status qw_gwalk_synchronize(qw_gwalk *g);
int64_t qw_gwalk_narcs(const qw_gwalk *g);   /* -1 for NULL */
const char *qw_gwalk_last_error(const qw_gwalk *g);

/* ---------------------------------------------------------------- batches */

/* A batch of independent 1D walks on cycles (Sec. 2.2), walk i with N[i]
 * sites, T[i] steps, its own 2x2 coin (coins + 8*i: row-major complex), and the
 * localised initial state |x0[i]> (x) (coin_state[0]|0> + coin_state[1]|1>)
 * (coin_state: 2 complex = 4 doubles).  prec: QW_F32 or QW_F32_BF16STORE
 * (state storage; arithmetic is float), or QW_F32_COMP (double-float: the
 * state, the coin and the arithmetic carry a hi + lo pair of floats, ~48 bits;
 * for walks whose coin entries lie within ~2^-20 of +-1, where float rounding
 * is biased; warp tiles of 8 sites per lane, variant 0 only, k <= 64);
 * anything else QW_EUNSUPPORTED.  All arrays are host pointers; QW_EINVAL for
 * N < 1, T < 0 or x0 outside [0, N).  Device memory: two state buffers for all
 * walks (ping-pong; the double-float form holds twice the planes), their
 * probabilities (float) and norms.  The default kernel of the float forms
 * (variant 1 of qw_batch_set_plan_ex) sweeps each walk's light cone
 * [x0 - t, x0 + t] only; the state outside it stays exactly zero. */
qw_status qw_batch_create(int nwalks, const int64_t *N, const int64_t *T,
                          const double *coins, const int64_t *x0,
                          const double *coin_state, qw_precision prec,
                          void *cuda_stream, qw_batch **out);

/* Run every walk of the batch from its initial state for its own T[i] steps
 * (one persistent kernel launch, replayed from a CUDA graph after the first
 * call) and compute each walk's probabilities.  Repeated calls start again
 * from the initial states. */
qw_status qw_batch_step(qw_batch *b);

/* Temporal depth k (steps per round, 1..128; default 96) of the batched
 * kernel; the tile is fixed at 16 sites per lane (double-float: 1..64, default
 * 32, 8 sites per lane).  Changing k re-captures the graph. */
qw_status qw_batch_set_plan(qw_batch *b, int depth_k);
qw_status qw_batch_get_plan(const qw_batch *b, int *depth_k, int *tile);

/* The same with the kernel variant: 0 = warp register tiles, each
 * recomputing a halo of k sites on both sides, tiles outside the light cone
 * skipped; 1 = time-skewed window sweep (the sweep of qw_set_plan_ex variant 1
 * over the chunks that cover a walk's light cone, no halo; over the whole
 * cycle with warm-up chunks once the cone nearly covers it).  Both give the
 * same results up to rounding order.  QW_EINVAL for another variant;
 * QW_EUNSUPPORTED for variant 1 on a double-float batch. */
qw_status qw_batch_set_plan_ex(qw_batch *b, int depth_k, int variant);
qw_status qw_batch_get_plan_ex(const qw_batch *b, int *depth_k, int *tile, int *variant);

/* Work split of variant 1: the n walks with the most light-cone work
 * sum_{t<T} min(N, 2t+1) (site-steps) are each shared by the four warps of a
 * CTA (segments with warm-up chunks, a barrier between passes), which
 * shortens the longest walks, the critical path; every other walk is swept by
 * one warp alone.  n is clamped to [0, nwalks]; the default is nwalks / 16.
 * Results do not depend on it.  QW_EINVAL for n < 0; re-captures the graph.
 * qw_batch_cta_walks returns n (-1 for a null handle). */
qw_status qw_batch_set_cta_walks(qw_batch *b, int n);
int qw_batch_cta_walks(const qw_batch *b);

/* Time the batch for k in {8, ..., 128} and both variants (each timing runs
 * the whole batch from its initial states) and keep the fastest; report as
 * for qw_autotune. */
qw_status qw_batch_autotune(qw_batch *b, char *report, size_t report_len);

/* Probabilities of all walks, concatenated in walk order (walk i starts at
 * sum_{j<i} N[j]), float, host or device; norms (host, may be NULL): nwalks
 * doubles, the sum of each walk's P.  Synchronises. */
qw_status qw_batch_probabilities(qw_batch *b, float *P_concat, int on_device, double *norms);

/* Final state of walk i (2 planes of N[i] complex, dtype, host pointer). */
qw_status qw_batch_get_state(qw_batch *b, int walk, void *amp_out, qw_cdtype dtype);

qw_status qw_batch_destroy(qw_batch *b);

/* ---------------------------------------------------------------- misc */

const char *qw_status_string(qw_status s);
const char *qw_last_error(const qw_walk *w);
const char *qw_batch_last_error(const qw_batch *b);
/* Version string of the library ("qw <major>.<minor> sm_103a"). */
const char *qw_version(void);

/* Bounded-wait self test: launches one kernel that waits on a device flag that
 * nothing sets, giving up after `spins` polls; returns QW_ETIMEOUT when the
 * wait gave up (the expected outcome) and leaves the context usable.  Exists
 * so failure detection can be tested without hanging a GPU. */
qw_status qw_debug_bounded_wait(int64_t spins, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QW_H */
