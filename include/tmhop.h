/*
 * tmhop.h -- C ABI of the GB300 (sm_103a) library for the even-odd
 * preconditioned Wilson twisted-mass operator.
 *
 * The operator is the one whose hopping matrix the tmLQCD suite optimises
 * (arXiv:1311.4521, introduction and Sec. 2: "Hopping_Matrix", full- and half-spinor
 * kernels, "Dirac matrix inversion" by the inverter), in the standard
 * hopping-parameter form:
 *
 *   Dhop psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
 *   H_eo, H_oe  = Dhop from odd to even / even to odd sites
 *   Q_tm        = gamma5 [ (1 + i mut gamma5) - kappa^2 H_eo (1 + i mut gamma5)^-1 H_oe ],
 *                 mut = 2 kappa mu
 *
 * in the chiral gamma basis (gamma5 = diag(1,1,-1,-1)); direction 0 is
 * time.  A hop that wraps around the lattice in direction mu is multiplied
 * by bc[mu] (+1 periodic, -1 antiperiodic).
 *
 * Conventions for every entry point:
 *   - dims[4] = {Lx, Ly, Lz, Lt}; every extent even and >= 2, else
 *     TM_ERR_ARG.  Sites are lex = x + Lx*(y + Ly*(z + Lz*t)); parity
 *     (x+y+z+t) mod 2; a one-parity field holds its Vh = V/2 sites at index
 *     lex/2.
 *   - Pointers named *_dev are device memory of the context's device,
 *     owned by the caller, 16-byte aligned, and not overlapping unless
 *     stated; a null or misaligned field pointer gives TM_ERR_ARG (the
 *     kernels use 16-byte vector accesses).  Host pointers are named
 *     *_host.
 *   - "Packed" spinor fields are the library's storage of one parity in a
 *     given precision (component-major, see tm_spinor_bytes); they are
 *     produced by tm_spinor_pack and read back by tm_spinor_unpack.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous unless stated.  Arguments are validated
 *     on the host before anything is launched.
 *   - Errors are returned as tm_status, never thrown; tm_last_error gives
 *     the message of the most recent failure on that context.
 */
#ifndef TMHOP_H
#define TMHOP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tm_ctx tm_ctx;
typedef struct tm_gauge tm_gauge;

typedef enum {
    TM_OK = 0,
    TM_ERR_ARG = 1,            /* invalid argument (null pointer, odd extent, bad enum ...) */
    TM_ERR_CUDA = 2,           /* a CUDA runtime call failed; message in tm_last_error */
    TM_ERR_NOT_CONVERGED = 3,  /* solver reached maxiter; x holds the last iterate */
    TM_ERR_NONFINITE = 4,      /* NaN or Inf met in a residual norm */
    TM_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    TM_ERR_UNSUPPORTED = 6     /* valid but not implemented combination */
} tm_status;

/* Storage precisions.  TM_F64X stores each FP64 value as a pair of FP32
 * numbers (hi, lo; about 48 significant bits) and computes with double-float
 * arithmetic on the FP32 units, which on GB300 issue 64 times as many FMAs
 * per clock as the FP64 units; results agree with FP64 to ~1e-14. */
typedef enum { TM_F64 = 0, TM_F32 = 1, TM_F16 = 2, TM_F64X = 3 } tm_prec;

enum { TM_EO = 0,   /* output even sites, input odd sites: H_eo */
       TM_OE = 1 }; /* output odd sites, input even sites: H_oe */

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (which becomes current).  The
 * context owns scratch buffers and tuning results; one context serves one
 * host thread at a time. */
tm_status tm_ctx_create(tm_ctx **ctx, int device);
void tm_ctx_destroy(tm_ctx *ctx);
/* Message of the last failure on ctx (never NULL; "" if none). */
const char *tm_last_error(const tm_ctx *ctx);
const char *tm_status_string(tm_status s);
/* Tracing hook for timing individual kernels with CUDA events.  While
 * events != NULL, each later multi-kernel call records events[k] (cudaEvent_t
 * values created by the caller) on its stream at its kernel boundaries:
 * tm_Qtm records events[0] before its first launch, events[1] between its
 * two launches and events[2] after the second.  nevents must be >= 3.
 * Pass events = NULL to stop.  The array is copied; the events are not
 * owned by the library. */
tm_status tm_ctx_trace(tm_ctx *ctx, void *const *events, int nevents);

/* Turns timing-based selection of launch configurations on (default) or
 * off.  With it on, the first batched call for a new batch shape runs a few
 * candidate configurations of its hop launch and keeps the fastest for the
 * context's lifetime; off, a fixed configuration is used. */
tm_status tm_ctx_set_autotune(tm_ctx *ctx, int on);

/* Fixes the configuration of the batched hop (tm_Qtm_batch,
 * tm_cg_QdagQ_batch) instead of letting the autotuner choose it.  code % 10
 * is the pass width: 1 links streamed from memory, work items (tile, rhs);
 * 0 the same with the right-hand sides of a tile on consecutive CTAs, so
 * that they share the links through L2; 2 or 4 the tile's links staged in
 * shared memory once and applied to 2 or 4 right-hand sides at a time.
 * code / 10 + 1 is the number of right-hand sides each thread computes (2:
 * one link load for both and twice the neighbour loads in flight; FP32 and
 * FP16 storage only).  Code 100 is the staged hop of tm_Qtm_batch: boxes of
 * 8 x 2 x 2 x 2 half-sites whose neighbour spinors (for every right-hand
 * side) and links are copied into shared memory by TMA tensor copies, one
 * persistent CTA per SM, for TM_F32 (12 or 18 reals) and TM_F16 (12)
 * handles on lattices with Lx a multiple of 16 when some lattice of the
 * batch has at least two right-hand sides; it builds, once per gauge handle,
 * a site-complete copy of the links (the 8 links of every site: 1152 bytes
 * per even-odd site pair for TM_F32 handles, which keeps all 18 reals,
 * twice the handle's link bytes for TM_F16; freed with the handle).  Valid codes: 0, 1, 2, 4, 10, 12, 14, 100; a code that a
 * storage format or call does not have (2, 10, 12, 14 for TM_F64 and
 * TM_F64X, e.g. the FP64 reliable updates of a mixed-precision batched
 * solve; 100 outside tm_Qtm_batch) is ignored there, and the autotuner
 * configures that launch.  cap: at most this many persistent CTAs (0: one
 * per work item; for code 100 one per SM).  code = -1 returns to the
 * autotuner. */
tm_status tm_ctx_set_batch_config(tm_ctx *ctx, int code, unsigned cap);

/* Synchronises the device and reports whether a kernel of this context gave
 * up a bounded wait since the last check (the staged batched hop waits on
 * shared-memory barriers for its tensor copies, each wait limited to about
 * a second of SM clock): TM_ERR_CUDA with a message then, else TM_OK.  The
 * flag is cleared by the check. */
tm_status tm_ctx_check(tm_ctx *ctx);

/* Test of the bounded-wait path: enqueues on `stream` one CTA whose thread
 * waits on a shared-memory barrier that nothing completes.  The wait gives
 * up after its limit (about a second), records that in the context's device
 * status and the kernel returns; tm_ctx_check then reports TM_ERR_CUDA and
 * clears it.  The context stays usable. */
tm_status tm_ctx_selftest_wait(tm_ctx *ctx, void *stream);

/* Text report of the launch configurations the context has chosen so far,
 * one line per batch shape: "<key> nrb=<pass width> cap=<CTA cap> ms3=<time
 * of three launches at selection> band=<1: tiles in z bands, t within a
 * band; 0: lexicographic tiles>", and one per lattice tuned by
 * tm_gauge_tune: "hop/<cache key> map=<map> ms=<per launch> linear128_ms=<the
 * default map's> gain=<ratio> candidates=<n>" (or "map=<map> (cache)").  Writes at most size bytes including the
 * terminating NUL (truncating) and returns the size the full report needs;
 * buf may be NULL to ask for that size. */
size_t tm_ctx_tune_report(const tm_ctx *ctx, char *buf, size_t size);

/* File in which tm_gauge_tune keeps its choices, one line "<key> <map>
 * <ms>" per lattice, keyed by "<GPU name>|<Lx>x<Ly>x<Lz>x<Lt>|prec<p>|recon<r>
 * |nrhs1" (NULL or "": no file).  The batched hop (tm_Qtm_batch,
 * tm_cg_QdagQ_batch) keeps its tuned configuration there too, one line
 * "<GPU name>|bhop/<prec>/<recon>/<Vh>x<nrhs>[/...][/staged] code<c>-cap<n>
 * <ms>" per batch shape.  A context starts with the path in the
 * environment variable TMHOP_TUNE_CACHE, if set.  With a cache file and
 * autotuning on, tm_gauge_create gives a new handle the cached map of its
 * lattice and a batch whose shape has an entry runs its configuration
 * without timing candidates. */
tm_status tm_ctx_set_tune_cache(tm_ctx *ctx, const char *path);

/* ---- fields --------------------------------------------------------------- */

/* Bytes of one packed one-parity spinor field of Vh sites in precision prec:
 *   TM_F64: 12 arrays of Vh double2 (one per spin-colour component)   192*Vh
 *   TM_F32:  6 arrays of Vh float4  (two components each)              96*Vh
 *   TM_F16:  3 arrays of Vh x 8 halves (four components each, scaled by
 *            the site norm) followed by Vh floats (the site norm = max |re|,|im|) 52*Vh
 *   TM_F64X: 12 arrays of Vh float4 (re.hi, re.lo, im.hi, im.lo)       192*Vh
 * Returns 0 for an invalid prec. */
size_t tm_spinor_bytes(long vh, int prec);

/* Packs Vh spinors given as complex double [Vh][4][3] (re, im interleaved)
 * into the packed layout of precision prec.  in_dev and out_dev must not
 * overlap. */
tm_status tm_spinor_pack(tm_ctx *ctx, long vh, const double *in_dev, void *out_dev, int prec, void *stream);
/* Inverse of tm_spinor_pack: packed field -> complex double [Vh][4][3]. */
tm_status tm_spinor_unpack(tm_ctx *ctx, long vh, const void *in_dev, double *out_dev, int prec, void *stream);

/* ---- gauge field -------------------------------------------------------- */

/* Builds the library's storage of a gauge field from U_dev, complex double
 * [4][V][3][3] (mu = 0 is time, then x, y, z; row-major 3x3).  prec is the
 * storage precision; reconstruct 18 stores all nine complex entries, 12
 * stores two rows and rebuilds the third as conj(row0 x row1), which is
 * exact for SU(3) links only (TM_F16 requires 12; TM_F64X stores every
 * complex entry as a float4 of hi/lo pairs).  bc[mu] in {+1,-1} is
 * the boundary sign of direction mu.  The handle owns its device memory
 * and keeps no reference to U_dev.  Synchronous with respect to stream. */
tm_status tm_gauge_create(tm_ctx *ctx, const int dims[4], const double *U_dev, int prec, int reconstruct,
                          const int bc[4], void *stream, tm_gauge **out);
void tm_gauge_destroy(tm_gauge *g);
/* Bytes of device memory held by the handle's link storage. */
size_t tm_gauge_bytes(const tm_gauge *g);

/* Site-to-thread maps of the hop launches (tm_hopping_eo, tm_Qtm, tm_force,
 * tm_solve_eo) on the handle's lattice.  "linear<B>" gives CTAs of B threads
 * consecutive even-odd sites (whole rows along x, then y, z, t); "box<a>x<b>
 * x<c>x<d>" gives each CTA a box of a x b x c x d sites along (x half-row,
 * y, z, t), a..d powers of two dividing (Lx/2, Ly, Lz, Lt), 32 to 128 sites.
 * The analogue of the paper's hopping-order index and thread-distribution
 * studies (Secs. 2.2, 2.3): every map computes every site with the same
 * arithmetic, so outputs are bit-identical whatever the map; only the
 * memory access order, and with it the time, changes.  Default: linear128.
 *
 * tm_gauge_tune chooses the map: with a cache entry for the lattice (see
 * tm_ctx_set_tune_cache) it takes that; otherwise, with autotuning on, it
 * times the linear maps of 128 and 64 threads and every box of 64 or 128
 * sites with at least 4 sites along the half-row and at most 8 along y, z, t
 * (each: median of three rounds of two launches of the even-output hop with
 * the fused Q_tm update), keeps the fastest and appends it to the cache file;
 * with autotuning off it sets linear128.  It uses the context's workspace
 * and synchronises `stream`, so call it outside stream capture.
 * tm_gauge_set_map sets a map by name (TM_ERR_ARG if it does not fit the
 * lattice); tm_gauge_map writes the current map's name (like
 * tm_ctx_tune_report: at most size bytes, returns the size needed). */
tm_status tm_gauge_tune(tm_ctx *ctx, tm_gauge *U, void *stream);
tm_status tm_gauge_set_map(tm_ctx *ctx, tm_gauge *U, const char *name);
size_t tm_gauge_map(const tm_gauge *U, char *buf, size_t size);

/* ---- operator ------------------------------------------------------------ */

/* out = H psi for dir TM_EO (H_eo: odd in, even out) or TM_OE (H_oe: even
 * in, odd out).  dagger != 0 applies the adjoint hop Dhop^dagger between
 * the same parities instead: for TM_EO that is H_oe^dagger = gamma5 H_eo
 * gamma5, the hop with its two spin projectors (1 -+ gamma_mu) swapped;
 * for TM_OE it is H_eo^dagger.  Fields are packed in the gauge handle's
 * precision; out and in must not overlap. */
tm_status tm_hopping_eo(tm_ctx *ctx, const tm_gauge *U, void *out_dev, const void *in_dev, int dir, int dagger,
                        void *stream);

/* out_e = Q_tm(sign*mu) in_e on even sites, packed in the gauge handle's
 * precision.  sign = +1 gives Q(mu), sign = -1 gives Q(-mu) = Q(mu)^dagger.
 * Two launches: tmp_o = (1 + i mut gamma5)^-1 H_oe in_e into a scratch odd
 * field owned by ctx, then the fused even update.  out_e and in_e must not
 * overlap. */
tm_status tm_Qtm(tm_ctx *ctx, const tm_gauge *U, void *out_e_dev, const void *in_e_dev, double kappa, double mu,
                 int sign, void *stream);

/* The non-degenerate twisted-mass doublet (the mass-split flavour doublet
 * of the tmLQCD suite, whose operators the paper's introduction lists):
 * on an even-site doublet (in_s, in_c),
 *   (out_s, out_c) = Q_nd (in_s, in_c),  Q_nd = gamma5 (A - kappa^2 H_eo A^-1 H_oe),
 *   A = 1 + i mubar gamma5 tau3 - epsbar tau1 (site-local, spin x flavour),
 *   mubar = 2 kappa sign mu_sigma, epsbar = 2 kappa mu_delta,
 * the hops acting on each flavour alone.  sign = -1 gives Q_nd(-mu_sigma,
 * mu_delta) = Q_nd(mu_sigma, mu_delta)^dagger; mu_delta = 0 gives
 * (Q_tm(mu) in_s, Q_tm(-mu) in_c).  Both flavours of a site are hopped by
 * one thread with one load of each link; A^-1 = (1 - i mubar gamma5 tau3 +
 * epsbar tau1) / (1 + mubar^2 - epsbar^2) and A are fused into the two
 * launches like tm_Qtm's site-local factors.  Fields are packed in U's
 * precision (TM_F64, TM_F32 or TM_F16; TM_F64X: TM_ERR_UNSUPPORTED); the
 * outputs must differ from each other and from the inputs; a singular A
 * (epsbar^2 = 1 + mubar^2) gives TM_ERR_ARG.  Two odd temporaries live in
 * ctx's scratch.  Traced like tm_Qtm (events 0, 1, 2). */
tm_status tm_Qnd(tm_ctx *ctx, const tm_gauge *U, void *out_s_dev, void *out_c_dev, const void *in_s_dev,
                 const void *in_c_dev, double kappa, double mu_sigma, double mu_delta, int sign, void *stream);

/* The clover-improved twisted-mass operator (the Sheikholeslami-Wohlert
 * term; the paper's introduction lists the suite's operators):
 *   M_sw = 1 - kappa Dhop + T + i mut gamma5,  mut = 2 kappa mu,
 *   T(x) = c_sw kappa i sum_{mu<nu} sigma_munu F_munu(x),  sigma_munu = (i/2)[gamma_mu, gamma_nu],
 *   F_munu(x) = (Q_munu(x) - Q_munu(x)^dag) / 8, Q_munu(x) the sum of the four
 *   plaquettes of the (mu, nu) plane that start and end at x (links periodic),
 *   Q_sw = gamma5 (A_ee - kappa^2 H_eo A_oo^-1 H_oe) on even sites, A = 1 + T + i mut gamma5.
 * tm_clover_create computes, from the canonical links U_dev (complex double
 * [4][V][3][3], the same field U was made from), the two 6x6 chirality blocks
 * of A on every site for both signs of mu: A itself on even sites and
 * -kappa^2 A^-1 on odd sites (FP64 arithmetic, stored in U's precision;
 * TM_F64 and TM_F32 only).  kappa, mu and c_sw are fixed at creation; a
 * singular site matrix gives TM_ERR_ARG.  Synchronous with respect to
 * stream.  The handle owns its device memory (tm_clover_bytes: 4 x 36
 * complex numbers per site). */
typedef struct tm_clover tm_clover;
tm_status tm_clover_create(tm_ctx *ctx, const tm_gauge *U, const double *U_dev, double csw, double kappa, double mu,
                           void *stream, tm_clover **out);
void tm_clover_destroy(tm_clover *C);
size_t tm_clover_bytes(const tm_clover *C);

/* out_e = Q_sw(sign * mu) in_e with the kappa, mu and c_sw of C (sign = -1
 * gives Q_sw(-mu) = Q_sw(mu)^dagger; c_sw = 0 gives tm_Qtm).  Two launches
 * like tm_Qtm, the blocks applied in their epilogues; the odd temporary
 * lives in ctx's scratch.  Traced like tm_Qtm. */
tm_status tm_Qsw(tm_ctx *ctx, const tm_gauge *U, const tm_clover *C, void *out_e_dev, const void *in_e_dev, int sign,
                 void *stream);

/* ---- solver ------------------------------------------------------------- */

/* Parameters of tm_cg_QdagQ. */
typedef struct {
    double kappa, mu;      /* operator parameters of Q_tm (mu is the twisted mass, mut = 2 kappa mu) */
    double tol;            /* target true relative residual |b - Q^dag Q x|_2 / |b|_2, checked in FP64 */
    int maxiter;           /* iteration limit (counted in inner CG iterations) */
    int reliable_every;    /* iterations per segment between host checks; with a reduced-precision
                              inner solver also the longest stretch without a reliable update */
    int use_graph;         /* nonzero: capture one segment as a CUDA graph and replay it */
    double reliable_delta; /* reduced-precision inner solver: FP64 reliable update (x += y,
                              r = b - Q^dag Q x in FP64) as soon as the recursive |r| has fallen
                              below reliable_delta times its largest value since the previous
                              one (delta < 1; 0: only every reliable_every iterations; negative:
                              automatic, sqrt of the inner format's unit roundoff and at least
                              1e-3, i.e. 1e-3 for TM_F32 and 0.022 for TM_F16) */
} tm_cg_params;

/* Results of tm_cg_QdagQ. */
typedef struct {
    int iters;             /* inner CG iterations performed */
    int reliable_updates;  /* FP64 residual recomputations (reliable updates and final checks) */
    double true_relres;    /* final |b - Q^dag Q x| / |b| computed in FP64 */
    double seconds;        /* wall time of the solve, host clock, from entry to the final synchronisation */
    int status;            /* tm_status of the solve */
} tm_cg_info;

/* Solves Q^dag Q x = b on the even sites by conjugate gradients, the
 * inversion the tmLQCD inverter performs (the paper's Sec. 3 samples it;
 * Q^dag Q = Q(-mu) Q(mu) is Hermitian positive definite for mu != 0).
 *
 * U_hi is an FP64 or FP64X gauge handle; x_dev (in: initial guess, out:
 * solution) and b_dev are even fields packed in U_hi's precision.  U_lo
 * selects the inner solver: NULL, U_hi or another handle of U_hi's precision
 * gives a plain CG in that precision, checked against the FP64 true
 * residual whenever the recursive residual reaches tol; an FP32 or FP16
 * handle gives a mixed-precision CG whose vectors are stored in that
 * precision with FP32 arithmetic; its solution increments are accumulated
 * (in FP32) and added to x in FP64 at each reliable update, where the
 * residual is recomputed in FP64 and replaces the recursive one (the
 * search direction is kept).  Inner products are reduced in FP64, in a fixed order
 * (bit-reproducible).  Convergence is declared only on the FP64 true
 * residual.  Returns TM_OK, TM_ERR_NOT_CONVERGED (x holds the last iterate)
 * or TM_ERR_NONFINITE; info (may be NULL) receives the statistics.
 * Synchronous: returns after the solve has finished on `stream`.  Scratch
 * fields are owned by ctx. */
tm_status tm_cg_QdagQ(tm_ctx *ctx, const tm_gauge *U_hi, const tm_gauge *U_lo, void *x_dev, const void *b_dev,
                      const tm_cg_params *params, tm_cg_info *info, void *stream);

/* Solves the full-lattice system M x = b, M = 1 - kappa Dhop + i mut gamma5,
 * by even-odd preconditioning: bhat_e = b_e + kappa H_eo M_oo^-1 b_o, CG on
 * Q^dag Q x_e = Q^dag gamma5 bhat_e (tm_cg_QdagQ with the same U_hi, U_lo
 * and params; x_e in: initial guess), then x_o = M_oo^-1 (b_o + kappa H_oe
 * x_e).  All four fields are packed FP64 (even: x_e, b_e; odd: x_o, b_o),
 * pairwise distinct.  info and the return value are those of the even-site
 * solve; its tolerance applies to the Q^dag Q system.  Synchronous. */
tm_status tm_solve_eo(tm_ctx *ctx, const tm_gauge *U_hi, const tm_gauge *U_lo, void *x_e, void *x_o, const void *b_e,
                      const void *b_o, const tm_cg_params *params, tm_cg_info *info, void *stream);

/* ---- adjoint: force and gradient ---------------------------------------- */

enum { TM_FORCE_SU3 = 0,    /* F in su(3): U -> exp(eps T) U changes S by eps <T, F>, <A,B> = -2 tr(AB) */
       TM_FORCE_GRAD = 1 }; /* G = dS/dRe U + i dS/dIm U, the gradient w.r.t. the complex link entries */

/* Fermion force of the action S = phi^dag (Q^dag Q)^-1 phi given the
 * solution X = (Q^dag Q)^-1 phi, the derivative the HMC integration needs
 * (the paper's Sec. 2.4 "fermionic derivative").  X_e_dev is a packed even
 * field in U's precision; F_dev receives complex double [4][V][3][3] in the
 * canonical gauge layout: for TM_FORCE_SU3 the traceless anti-Hermitian
 * F_mu(x) = -kappa^2 s TA(U M1 - M2 U^dag), for TM_FORCE_GRAD the complex
 * gradient 2 kappa^2 s (M1^dag + M2), with M1, M2 the spin-summed outer
 * products of the projected fields at the two ends of the link and s its
 * boundary sign.  Three hop launches (Y = Q X and the two odd fields) and
 * one launch with one thread per link, which writes every link exactly once
 * (no atomics).  Scratch is owned by ctx. */
tm_status tm_force(tm_ctx *ctx, const tm_gauge *U, double *F_dev, const void *X_e_dev, double kappa, double mu,
                   int mode, void *stream);

/* Link gradients of the linear operators, for backpropagation through them:
 * G_dev (complex double [4][V][3][3], the canonical gauge layout) receives
 * the gradient with respect to the complex link entries (dL = Re tr(G^dag dU)
 * summed over links, the convention of tm_force's TM_FORCE_GRAD) of
 *   TM_GRAD_QTM     Re <Y, Q_tm(sign*mu) X>    X, Y even fields
 *   TM_GRAD_HOP_EO  Re <Y, H_eo X>             X odd, Y even
 *   TM_GRAD_HOP_OE  Re <Y, H_oe X>             X even, Y odd
 * (<a, b> = sum conj(a) b), fields packed in U's precision.  With Y the
 * upstream gradient of an operator's output and X its input this is the
 * operator's vector-Jacobian product with respect to U.  Computed by the
 * force kernels (one thread per link, no atomics) after at most two hop
 * launches; the temporaries live in ctx's workspace.  kappa and mu are
 * used by TM_GRAD_QTM only. */
enum { TM_GRAD_QTM = 0, TM_GRAD_HOP_EO = 1, TM_GRAD_HOP_OE = 2 };
tm_status tm_link_grad(tm_ctx *ctx, const tm_gauge *U, double *G_dev, const void *X_dev, const void *Y_dev, int op,
                       double kappa, double mu, int sign, void *stream);

/* ---- host-resident fields --------------------------------------------------- */

/* Q_tm (sign as in tm_Qtm) on n one-parity fields in host memory:
 * out_host[k] = Q in_host[k], each a complex double [Vh][4][3] array (the
 * layout tm_spinor_pack reads).  The fields go through two device staging
 * slots in U's storage precision, pipelined: field k+1 is copied to the
 * device and packed on one copy stream owned by the context, field k-1
 * unpacked and copied back on the other, while field k is multiplied on
 * `stream`.
 * Host buffers should be pinned (cudaHostAlloc, cudaHostRegister) for the
 * copies to overlap the kernels; pageable memory works but serialises.  No
 * output may be one of the inputs or overlap one (an output that is an input
 * gives TM_ERR_ARG).  Inputs may repeat, and so may outputs: the results are
 * copied back in field order on one stream, so an output buffer given for
 * several fields ends up holding the result of the last of them.
 * Synchronous: returns when every output is in host memory.  Device memory:
 * two slots of two canonical and two packed fields, kept by the context
 * (grow-only), plus tm_Qtm's scratch.  The paper has no counterpart; this is
 * the entry point for callers whose data is in host memory. */
tm_status tm_Qtm_host(tm_ctx *ctx, const tm_gauge *U, int n, double *const *out_host, const double *const *in_host,
                      double kappa, double mu, int sign, void *stream);

/* How tm_force_ex assembles the per-link force.  Every link's force has two
 * parts, one from each hop that uses the link; the paper (Sec. 2.4) weighs
 * updating a shared derivative field with "atomic" directives against
 * per-site "halo memory" with a second accumulation loop.
 *   TM_FORCE_OWNER  one thread per link computes both parts (tm_force)
 *   TM_FORCE_ATOMIC one thread per site pushes the forward part of its 4
 *                   links and the backward part of the 4 links ending there
 *                   with FP64 atomic adds into F (zeroed first); with two
 *                   addends per entry the result does not depend on order
 *   TM_FORCE_HALO   the same pushes into two private buffers, then a second
 *                   pass F = forward + backward (no atomics, more traffic) */
enum { TM_FORCE_OWNER = 0, TM_FORCE_ATOMIC = 1, TM_FORCE_HALO = 2 };

/* tm_force with a choice of scheme (the push schemes for TM_F64 and TM_F32
 * handles only; TM_ERR_UNSUPPORTED otherwise).  Same result up to rounding;
 * TM_FORCE_ATOMIC and TM_FORCE_HALO agree bit for bit. */
tm_status tm_force_ex(tm_ctx *ctx, const tm_gauge *U, double *F_dev, const void *X_e_dev, double kappa, double mu,
                      int mode, int scheme, void *stream);

/* ---- batches ------------------------------------------------------------ */

/* Q_tm(sign*mu) applied to nsys even fields (out_e[k] = Q in_e[k] with gauge
 * U[k]) with one launch per hop for the whole batch.  Systems that share a
 * gauge handle pointer are several right-hand sides of one lattice: the
 * links of each site are read once and applied to all of them.  Systems on
 * different handles may have different lattice sizes.  All handles must
 * have the same precision and reconstruction.  Every output buffer belongs
 * to one system and is none of the inputs (TM_ERR_ARG); inputs may repeat.
 * The batch's device tables
 * and odd temporaries are owned by ctx.  Asynchronous on `stream` like
 * tm_Qtm: the first call for a batch (its handles, field pointers, lattice
 * sizes and stream) uploads its tables and, for a new batch shape, times
 * launch configurations (both synchronise the stream); a repeated call with
 * the same batch only launches.  Batched calls on one ctx that overlap on
 * different streams are not supported (the ctx synchronises the previous
 * stream when the stream changes). */
tm_status tm_Qtm_batch(tm_ctx *ctx, int nsys, const tm_gauge *const *U, void *const *out_e, const void *const *in_e,
                       double kappa, double mu, int sign, void *stream);

/* Solves the nsys systems Q^dag Q x[k] = b[k] at once, each step of the
 * iteration one launch over all of them (systems sharing U_hi[k] reuse its
 * links as in tm_Qtm_batch).  U_hi[k] are FP64 handles; U_lo (may be NULL)
 * gives each system's inner handle (NULL or U_lo[k] == U_hi[k]: FP64 inner
 * solver); systems sharing U_hi need the same U_lo; all inner handles need
 * the same precision.  Every system uses the reliable-update scheme of
 * tm_cg_QdagQ with its own scalars and stops on its own FP64 true residual;
 * params are shared.  Every x[k] belongs to one system and is none of the
 * b (TM_ERR_ARG); sources may repeat.  info[k] receives system k's
 * statistics (seconds is the batch's wall time).  Returns TM_OK if every
 * system converged, else TM_ERR_NONFINITE or TM_ERR_NOT_CONVERGED. */
tm_status tm_cg_QdagQ_batch(tm_ctx *ctx, int nsys, const tm_gauge *const *U_hi, const tm_gauge *const *U_lo,
                            void *const *x_dev, const void *const *b_dev, const tm_cg_params *params,
                            tm_cg_info *info, void *stream);

/* ---- slabs: the operator on a lattice cut along time, one slab per GPU ------ */

/* The paper's Sec. 2.5 splits the hopping matrix of a lattice distributed
 * over MPI processes into the "surface" (sites whose neighbours live on
 * another process) and the "body", sends the projected half-spinors of the
 * surface and overlaps that communication with the body loop.  Here a
 * lattice Lx x Ly x Lz x Lt is cut along t into slabs of even extent Lt_s >= 2
 * (each starting at an even global t, so local and global parities agree),
 * one per GPU.  A slab is an ordinary local lattice: its gauge handle is made
 * by tm_gauge_create from the slab's own links U[4][Vs][3][3] (including U_0
 * of its top time slice, which points into the next slab); its fields are
 * packed one-parity fields of the slab.  Only the hops across the slab's two
 * time faces need data from the neighbouring slabs, 12 reals per face site:
 *   lower face (t = 0) of the INPUT field, sent to the previous slab:
 *       the upper pair of (1 -+ gamma_0) psi, for that slab's forward hops;
 *   upper face (t = Lt_s-1), sent to the next slab: U_0^dag times the upper
 *       pair of (1 +- gamma_0) psi, for that slab's backward hops.
 * A face holds the (Lx Ly Lz / 2) sites of one time slice and parity,
 * component-major in FP64 (TM_F64 handles) or FP32 (TM_F32, TM_F16), and
 * occupies tm_slab_face_bytes(U) bytes.  Supported storage: TM_F64, TM_F32,
 * TM_F16 (TM_F64X gives 0 / TM_ERR_UNSUPPORTED). */
enum { TM_SLAB_INTERIOR = 1,   /* output sites with 1 <= t <= Lt_s-2 (no face data needed) */
       TM_SLAB_BOUNDARY = 2,   /* output sites with t = 0 or t = Lt_s-1 (read the received faces) */
       TM_SLAB_ALL = 3 };
enum { TM_SLAB_HOP = 0,        /* out = H in (plain hop, H_eo or H_oe, or its adjoint with dagger) */
       TM_SLAB_QTM_A = 1,      /* out_o = -kappa^2 (1 + i mut gamma5)^-1 H_oe in_e: first stage of Q_tm */
       TM_SLAB_QTM_B = 2 };    /* out_e = gamma5 [(1 + i mut gamma5) x_e + H_eo in_o]: second stage */

/* Bytes of one face of a slab with gauge handle U (0 if unsupported). */
size_t tm_slab_face_bytes(const tm_gauge *U);

/* Writes the two faces of the input field in_dev of the hop `dir` (TM_OE:
 * in is even; TM_EO: in is odd) with the projectors of the plain or the
 * adjoint hop (dagger): send_lower_dev for the previous slab, send_upper_dev
 * for the next one.  Asynchronous on `stream`. */
tm_status tm_slab_pack(tm_ctx *ctx, const tm_gauge *U, const void *in_dev, int dir, int dagger, void *send_lower_dev,
                       void *send_upper_dev, void *stream);

/* The hop of the slab for the output sites in `region`: op TM_SLAB_HOP
 * gives out = H in (dagger as in tm_hopping_eo); TM_SLAB_QTM_A (dir TM_OE)
 * and TM_SLAB_QTM_B (dir TM_EO, x_dev the even input of Q_tm) are the two
 * stages of Q_tm(sign*mu) as in tm_Qtm, so that stage A, the face exchange
 * of its output and stage B give Q_tm on the whole lattice.  recv_lower_dev
 * holds the previous slab's upper face, recv_upper_dev the next slab's lower
 * face (both needed for TM_SLAB_BOUNDARY); sign_lower / sign_upper (+1 or
 * -1) multiply the hops through the lower / upper face (the boundary sign
 * of the global time direction for the slabs at its ends, else +1); the
 * slab's own bc[0] is not used for those hops.  The interior region reads
 * no face, so its launch may run while the faces are in transit.
 * Asynchronous on `stream`. */
tm_status tm_slab_hop(tm_ctx *ctx, const tm_gauge *U, void *out_dev, const void *in_dev, const void *recv_lower_dev,
                      const void *recv_upper_dev, int dir, int dagger, int region, int op, double kappa, double mu,
                      int sign, const void *x_dev, int sign_lower, int sign_upper, void *stream);

/* ---- measurement and field utilities -------------------------------------- */

/* Measures the fused multiply-add throughput of the device in precision prec
 * (TM_F64 or TM_F32): 8 CTAs of 256 threads per SM, each thread running 8
 * independent FMA chains for about 10 ms; the best of three timed launches
 * (CUDA events on `stream`, after one warm-up launch) at 2 flop per FMA is
 * written to *tflops (host memory) in TFLOP/s.  It is the arithmetic peak the
 * FP64 operator, which on this GPU is bound by its FP64 units rather than by
 * memory, is measured against.  The paper has no counterpart (its machines
 * were measured against their own nominal peaks).  Synchronous; allocates
 * nothing. */
tm_status tm_probe_fma(tm_ctx *ctx, int prec, double *tflops, void *stream);

/* out_dev[0] + i out_dev[1] = <a, b> = sum over the Vh sites and 12
 * spin-colour components of conj(a) b, for two packed one-parity fields of
 * precision prec, accumulated in FP64 (the global inner product of the
 * paper's Sec. 3, "scalar_prod_r", on one GPU).  The summation order depends
 * only on Vh and the device's SM count, so repeated calls give identical
 * bits.  out_dev is device memory holding two doubles, 8-byte aligned.
 * Asynchronous on `stream`; the partial sums live in a buffer owned by ctx
 * (grow-only), so calls on one ctx must not overlap on different streams. */
tm_status tm_spinor_dot(tm_ctx *ctx, long vh, const void *a_dev, const void *b_dev, int prec, double *out_dev,
                        void *stream);

/* z[k] <- c * alpha * z[k] for the n complex doubles at z_dev (re, im
 * interleaved, 16-byte aligned), with alpha = *alpha_dev read on the device
 * (a scalar the caller keeps in device memory, e.g. an upstream gradient) or
 * alpha = 1 when alpha_dev is NULL.  Asynchronous on `stream`. */
tm_status tm_scale_complex(tm_ctx *ctx, size_t n, double *z_dev, const double *alpha_dev, double c, void *stream);

/* Bytes of device memory the context holds at this moment (its scratch,
 * solver workspace, staging slots, batch tables and reduction buffer; gauge
 * handles are counted by tm_gauge_bytes).  0 for a context that has not yet
 * allocated anything. */
size_t tm_ctx_device_bytes(const tm_ctx *ctx);

/* Size in bytes of the static device array behind tm_Qtm_noalloc: room for
 * one odd-parity field of up to 174,762 sites in TM_F64 (e.g. 24^3x24),
 * 349,525 in TM_F32 (24^3x48) or 645,277 in TM_F16 (32^3x32 and below).
 * Every GPU that loads this library holds it until the process exits. */
#define TM_QTM_NOALLOC_MAX_BYTES (32u << 20)

/* Same operator and arguments as tm_Qtm, for callers that cannot let the
 * library allocate device memory (a framework that owns all device memory
 * through its own pool, a plugin with a fixed memory budget, a loop that
 * cannot take the device synchronisation an allocation may cause).  The
 * paper has no counterpart; this is an interface addition.  The odd
 * temporary lives in a static device array of TM_QTM_NOALLOC_MAX_BYTES
 * bytes instead of the context's scratch buffer, and the call makes no
 * cudaMalloc or cudaFree.  The gauge handle and the fields are still the
 * caller's, created beforehand.  Lattices whose odd temporary
 * (tm_spinor_bytes(V/2, prec)) exceeds the array are rejected with
 * TM_ERR_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device made current for the
 * lookup) and caches it for the life of the process; make that first call
 * before any stream capture.  The cached address belongs to the device's
 * primary context: after a cudaDeviceReset every object of this library
 * (contexts, gauge handles, and this address) is invalid and must not be
 * used again.  All calls on a device share the one array, which keeps the
 * last call's contents; calls that overlap on the GPU race on it.  With
 * tm_ctx_trace on, records the same three events as tm_Qtm. */
tm_status tm_Qtm_noalloc(tm_ctx *ctx, const tm_gauge *U, void *out_e_dev, const void *in_e_dev, double kappa,
                         double mu, int sign, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TMHOP_H */
