// tm_cg.cu -- conjugate gradients on Q^dag Q: plain FP64 and mixed precision
// with FP64 reliable updates.
//
// The tmLQCD inverter spends its time in repeated hopping-matrix calls and
// in global scalar products (scalar_prod_r), whose reductions and thread
// management the paper measures as overhead (Sec. 3).  Here every scalar of
// the iteration lives in device memory: each reduction is fused into the
// kernel that produces its operand (<p, Q^dag Q p> = |Q p|^2 in the launch
// that writes Q p; the vector update and |r|^2 in the launch that computes
// Q^dag Q p, which is therefore never stored), finished by the last block
// to arrive in a fixed order (bit-reproducible, no atomics on the values),
// and alpha, beta and the stopping test are computed there too.  The host
// only synchronises once per segment of `reliable_every` iterations; the
// segment itself is a CUDA graph, the GPU analogue of launching the threads
// once at solver level with orphaned directives.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "tm_cg.cuh"
#include "tm_internal.h"

namespace twm {

// Block sum of v; the block's partial goes to partials[blockIdx.x] and the
// last block to arrive sums all partials in index order and finishes `op`.
// Every thread of the block must call this.
template <int BLOCK>
__device__ void reduce_finish(double v, double *partials, CgScalars *s, int op)
{
    __shared__ double sh[BLOCK / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            partials[blockIdx.x] = v;
            __threadfence();
            unsigned t = atomicAdd(&s->ticket, 1u);
            last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = 0.0;
    const volatile double *vp = partials;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += BLOCK) acc += vp[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __syncthreads();
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            cg_finish(op, acc, s);
            s->ticket = 0;
        }
    }
}

constexpr int HOP_BLOCK = 128;
constexpr int LA_BLOCK = 256;

// Hop with the twisted-mass epilogue.  MODE HOP_NORM also reduces |out|^2
// into pAp; MODE HOP_UPDATE is the last hop of Q^dag Q p: instead of storing
// its result Ap it applies the CG update at once, y += alpha p and
// r -= alpha Ap (y in precision PY), and reduces |r|^2 into rr_new, so Ap is
// never written to memory and read back.
enum { HOP_PLAIN = 0, HOP_NORM = 1, HOP_UPDATE = 2 };

template <int P, int RECON, int MODE>
__global__ void __launch_bounds__(HOP_BLOCK, TM_HOP_MINB(P)) k_cg_hop(Geom g, int p, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                                      const void *__restrict__ in, void *__restrict__ out,
                                                      const void *__restrict__ x, Coef k, void *__restrict__ y,
                                                      void *__restrict__ r, const void *__restrict__ pdir,
                                                      double *partials, CgScalars *s, int gate)
{
    using R = typename SpinorIO<P>::R;
    constexpr int PY = P == F16 ? F32 : P;
    using RY = typename SpinorIO<PY>::R;
    if (gated(s, gate)) return;
    unsigned i = blockIdx.x * HOP_BLOCK + threadIdx.x;
    double nrm = 0.0;
    if (i < g.vh) {
        Spinor<R> acc, o;
        hop_site<P, RECON, false>(g, p, i, links, in, acc);
        if (x) {
            Spinor<R> xs;
            SpinorIO<P>::load(x, g.vh, i, xs);
            epilogue(k, acc, &xs, o);
        } else {
            epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
        }
        if (MODE == HOP_UPDATE) {
            const double alpha = s->alpha;
            Spinor<R> pv, rv;
            Spinor<RY> yv;
            SpinorIO<P>::load(pdir, g.vh, i, pv);
            SpinorIO<P>::load(r, g.vh, i, rv);
            SpinorIO<PY>::load(y, g.vh, i, yv);
            const R a = to_R<R>(alpha);
            const RY ay = to_R<RY>(alpha);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    yv[sp][c].re += ay * RY(pv[sp][c].re);
                    yv[sp][c].im += ay * RY(pv[sp][c].im);
                    rv[sp][c].re -= a * o[sp][c].re;
                    rv[sp][c].im -= a * o[sp][c].im;
                }
            SpinorIO<PY>::store(y, g.vh, i, yv);
            SpinorIO<P>::store(r, g.vh, i, rv);
            nrm = norm2(rv);
        } else {
            SpinorIO<P>::store(out, g.vh, i, o);
            if (MODE == HOP_NORM) nrm = norm2(o);
        }
    }
    if (MODE != HOP_PLAIN) reduce_finish<HOP_BLOCK>(nrm, partials, s, MODE == HOP_NORM ? FIN_PAP : FIN_RR_UPDATE);
}

// p = r + beta p with beta = rr_new / rr (restart: p = r); then rr = rr_new.
template <int P>
__global__ void __launch_bounds__(LA_BLOCK, (P == F64 || P == F64X) ? 3 : 4) k_cg_pupdate(unsigned vh, void *p, const void *r, double *partials,
                                                         CgScalars *s, int skip, int restart)
{
    using R = typename SpinorIO<P>::R;
    if (skip && s->done) return;
    const double beta = restart ? 0.0 : s->rr_new / s->rr;
    unsigned i = blockIdx.x * LA_BLOCK + threadIdx.x;
    if (i < vh) {
        Spinor<R> rv, pv;
        SpinorIO<P>::load(r, vh, i, rv);
        if (!restart) {
            SpinorIO<P>::load(p, vh, i, pv);
            const R b = to_R<R>(beta);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rv[sp][c].re += b * pv[sp][c].re;
                    rv[sp][c].im += b * pv[sp][c].im;
                }
        }
        SpinorIO<P>::store(p, vh, i, rv);
    }
    reduce_finish<LA_BLOCK>(0.0, partials, s, FIN_ROLL);
}

// x += y (x in the high precision PH), y = 0.
template <int PH, int PY>
__global__ void __launch_bounds__(LA_BLOCK, 4) k_cg_accum(unsigned vh, void *x, void *y, const CgScalars *s, int gate)
{
    using RH = typename SpinorIO<PH>::R;
    using RY = typename SpinorIO<PY>::R;
    if (gated(s, gate)) return;
    unsigned i = blockIdx.x * LA_BLOCK + threadIdx.x;
    if (i >= vh) return;
    Spinor<RH> xv;
    Spinor<RY> yv, z;
    SpinorIO<PH>::load(x, vh, i, xv);
    SpinorIO<PY>::load(y, vh, i, yv);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xv[sp][c].re += cvt<RH>(yv[sp][c].re);
            xv[sp][c].im += cvt<RH>(yv[sp][c].im);
            z[sp][c] = {RY(0), RY(0)};
        }
    SpinorIO<PH>::store(x, vh, i, xv);
    SpinorIO<PY>::store(y, vh, i, z);
}

// res = b - Ax (high precision PH, may alias Ax); r_lo = res in precision P if given; |res|^2 -> op.
template <int PH, int P>
__global__ void __launch_bounds__(LA_BLOCK, 3) k_cg_residual(unsigned vh, const void *b, const void *Ax, void *res,
                                                             void *r_lo, double *partials, CgScalars *s, int op, int gate)
{
    using RH = typename SpinorIO<PH>::R;
    using R = typename SpinorIO<P>::R;
    if (gated(s, gate)) return;
    unsigned i = blockIdx.x * LA_BLOCK + threadIdx.x;
    double nrm = 0.0;
    if (i < vh) {
        Spinor<RH> bv, av;
        SpinorIO<PH>::load(b, vh, i, bv);
        SpinorIO<PH>::load(Ax, vh, i, av);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bv[sp][c].re -= av[sp][c].re;
                bv[sp][c].im -= av[sp][c].im;
            }
        if (res) SpinorIO<PH>::store(res, vh, i, bv);
        if (r_lo) {
            Spinor<R> lo;
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) lo[sp][c] = {cvt<R>(bv[sp][c].re), cvt<R>(bv[sp][c].im)};
            SpinorIO<P>::store(r_lo, vh, i, lo);
        }
        nrm = norm2(bv);
    }
    reduce_finish<LA_BLOCK>(nrm, partials, s, op);
}

// |v|^2 of a high-precision field -> op.
template <int PH>
__global__ void __launch_bounds__(LA_BLOCK, 4) k_cg_norm(unsigned vh, const void *v, double *partials, CgScalars *s, int op)
{
    unsigned i = blockIdx.x * LA_BLOCK + threadIdx.x;
    double nrm = 0.0;
    if (i < vh) {
        Spinor<typename SpinorIO<PH>::R> a;
        SpinorIO<PH>::load(v, vh, i, a);
        nrm = norm2(a);
    }
    reduce_finish<LA_BLOCK>(nrm, partials, s, op);
}

template <int P>
__global__ void __launch_bounds__(LA_BLOCK, 4) k_cg_zero(unsigned vh, void *v)
{
    using R = typename SpinorIO<P>::R;
    unsigned i = blockIdx.x * LA_BLOCK + threadIdx.x;
    if (i >= vh) return;
    Spinor<R> z;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) z[sp][c] = {R(0), R(0)};
    SpinorIO<P>::store(v, vh, i, z);
}

// ------------------------------------------------------------------ host side
namespace {

struct Work {
    unsigned vh;
    int PH;             // high precision of x, b and the true residual (F64 or F64X)
    int P, PY;          // inner storage precision, solution-increment precision
    bool mixed;
    // FP64 fields
    void *x, *b, *ax, *t_hi, *q_hi, *r_hi;
    // inner fields (precision P), y in PY
    void *r, *p, *q, *t, *y;
    double *partials;
    CgScalars *s;
};

unsigned blocks(unsigned vh, int b) { return (vh + b - 1) / b; }

template <int P, int RECON>
cudaError_t hop_launch(const tm_gauge *U, int parity, const void *in, void *out, const void *x, const Coef &k, int mode,
                       const Work &w, int gate, cudaStream_t st)
{
    using V = typename LinkIO<P, RECON>::V;
    const V *l = static_cast<const V *>(U->links);
    unsigned grid = blocks(U->geom.vh, HOP_BLOCK);
    auto kern = mode == HOP_UPDATE ? k_cg_hop<P, RECON, HOP_UPDATE>
                                   : mode == HOP_NORM ? k_cg_hop<P, RECON, HOP_NORM> : k_cg_hop<P, RECON, HOP_PLAIN>;
    kern<<<grid, HOP_BLOCK, 0, st>>>(U->geom, parity, l, in, out, x, k, w.y, w.r, w.p, w.partials, w.s, gate);
    return cudaGetLastError();
}

cudaError_t hop(const tm_gauge *U, int parity, const void *in, void *out, const void *x, const Coef &k, int mode,
                const Work &w, int gate, cudaStream_t st)
{
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: return hop_launch<F64, 18>(U, parity, in, out, x, k, mode, w, gate, st);
    case F64 * 100 + 12: return hop_launch<F64, 12>(U, parity, in, out, x, k, mode, w, gate, st);
    case F32 * 100 + 18: return hop_launch<F32, 18>(U, parity, in, out, x, k, mode, w, gate, st);
    case F32 * 100 + 12: return hop_launch<F32, 12>(U, parity, in, out, x, k, mode, w, gate, st);
    case F16 * 100 + 12: return hop_launch<F16, 12>(U, parity, in, out, x, k, mode, w, gate, st);
    case F64X * 100 + 18: return hop_launch<F64X, 18>(U, parity, in, out, x, k, mode, w, gate, st);
    case F64X * 100 + 12: return hop_launch<F64X, 12>(U, parity, in, out, x, k, mode, w, gate, st);
    }
    return cudaErrorInvalidValue;
}

// out = Q(-mu) Q(mu) in with temporaries t (odd) and q (even).  With
// `iterate` (the CG iteration, in = p): the second launch also reduces
// |Q p|^2 into pAp and alpha, and the last one applies the CG update instead
// of writing out (which may then be null).
cudaError_t qdagq(const tm_gauge *U, double kappa, double mu, const void *in, void *out, void *t, void *q,
                  bool iterate, const Work &w, int gate, cudaStream_t st)
{
    double mut = 2.0 * kappa * mu;
    cudaError_t e = hop(U, 1, in, t, nullptr, coef_qtm_a_scaled(kappa, mut), HOP_PLAIN, w, gate, st);
    if (e == cudaSuccess) e = hop(U, 0, t, q, in, coef_qtm_b_unit(mut), iterate ? HOP_NORM : HOP_PLAIN, w, gate, st);
    if (e == cudaSuccess) e = hop(U, 1, q, t, nullptr, coef_qtm_a_scaled(kappa, -mut), HOP_PLAIN, w, gate, st);
    if (e == cudaSuccess) e = hop(U, 0, t, out, q, coef_qtm_b_unit(-mut), iterate ? HOP_UPDATE : HOP_PLAIN, w, gate, st);
    return e;
}

cudaError_t pupdate(const Work &w, int skip, int restart, cudaStream_t st)
{
    unsigned g = blocks(w.vh, LA_BLOCK);
    if (w.P == F64) k_cg_pupdate<F64><<<g, LA_BLOCK, 0, st>>>(w.vh, w.p, w.r, w.partials, w.s, skip, restart);
    else if (w.P == F64X) k_cg_pupdate<F64X><<<g, LA_BLOCK, 0, st>>>(w.vh, w.p, w.r, w.partials, w.s, skip, restart);
    else if (w.P == F32) k_cg_pupdate<F32><<<g, LA_BLOCK, 0, st>>>(w.vh, w.p, w.r, w.partials, w.s, skip, restart);
    else k_cg_pupdate<F16><<<g, LA_BLOCK, 0, st>>>(w.vh, w.p, w.r, w.partials, w.s, skip, restart);
    return cudaGetLastError();
}

template <int PH>
cudaError_t residual_h(const Work &w, void *res, void *r_lo, int op, int gate, cudaStream_t st)
{
    unsigned g = blocks(w.vh, LA_BLOCK);
    const int P = r_lo ? w.P : PH;
    if (P == PH)
        k_cg_residual<PH, PH><<<g, LA_BLOCK, 0, st>>>(w.vh, w.b, w.ax, res, r_lo, w.partials, w.s, op, gate);
    else if (P == F32)
        k_cg_residual<PH, F32><<<g, LA_BLOCK, 0, st>>>(w.vh, w.b, w.ax, res, r_lo, w.partials, w.s, op, gate);
    else if (P == F16)
        k_cg_residual<PH, F16><<<g, LA_BLOCK, 0, st>>>(w.vh, w.b, w.ax, res, r_lo, w.partials, w.s, op, gate);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t residual(const Work &w, void *res, void *r_lo, int op, int gate, cudaStream_t st)
{
    return w.PH == F64X ? residual_h<F64X>(w, res, r_lo, op, gate, st) : residual_h<F64>(w, res, r_lo, op, gate, st);
}

cudaError_t zero(unsigned vh, int P, void *v, cudaStream_t st)
{
    unsigned g = blocks(vh, LA_BLOCK);
    if (P == F64) k_cg_zero<F64><<<g, LA_BLOCK, 0, st>>>(vh, v);
    else if (P == F64X) k_cg_zero<F64X><<<g, LA_BLOCK, 0, st>>>(vh, v);
    else if (P == F32) k_cg_zero<F32><<<g, LA_BLOCK, 0, st>>>(vh, v);
    else k_cg_zero<F16><<<g, LA_BLOCK, 0, st>>>(vh, v);
    return cudaGetLastError();
}

cudaError_t accum(const Work &w, int gate, cudaStream_t st)
{
    unsigned g = blocks(w.vh, LA_BLOCK);
    if (w.PH == F64X) k_cg_accum<F64X, F32><<<g, LA_BLOCK, 0, st>>>(w.vh, w.x, w.y, w.s, gate);
    else k_cg_accum<F64, F32><<<g, LA_BLOCK, 0, st>>>(w.vh, w.x, w.y, w.s, gate);
    return cudaGetLastError();
}

struct Solver {
    const tm_gauge *Uh, *Ul;
    double kappa, mu;
    Work w;

    // One inner iteration.  In mixed precision every iteration carries the
    // reliable-update kernels, gated on the device flag the update sets.
    cudaError_t iteration(cudaStream_t st) const
    {
        cudaError_t e = qdagq(Ul, kappa, mu, w.p, nullptr, w.t, w.q, true, w, 1, st);
        if (e == cudaSuccess && w.mixed) {
            e = accum(w, 2, st);
            if (e == cudaSuccess) e = qdagq(Uh, kappa, mu, w.x, w.ax, w.t_hi, w.q_hi, false, w, 2, st);
            if (e == cudaSuccess) e = residual(w, nullptr, w.r, FIN_RR_TRUE, 2, st);
        }
        if (e == cudaSuccess) e = pupdate(w, 1, 0, st);
        return e;
    }

    cudaError_t segment(int n, cudaStream_t st) const
    {
        cudaError_t e = cudaSuccess;
        for (int j = 0; j < n && e == cudaSuccess; ++j) e = iteration(st);
        return e;
    }

    // ax = Q^dag Q x in FP64, then |b - ax|^2 -> op (and r_lo / res if given).
    cudaError_t true_residual(void *res, void *r_lo, int op, cudaStream_t st) const
    {
        cudaError_t e = qdagq(Uh, kappa, mu, w.x, w.ax, w.t_hi, w.q_hi, false, w, 0, st);
        if (e == cudaSuccess) e = residual(w, res, r_lo, op, 0, st);
        return e;
    }
};

}  // namespace
}  // namespace twm

using namespace twm;


static tm_status cg_cuda(tm_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) ctx->err = std::string("tm_cg_QdagQ: ") + where + ": " + cudaGetErrorString(e);
    return TM_ERR_CUDA;
}

tm_status tm_ctx_workspace(tm_ctx *ctx, size_t bytes, void **ptr)
{
    if (ctx->ws_bytes < bytes) {
        if (ctx->ws) {
            cudaError_t e = cudaFree(ctx->ws);
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
            if (e != cudaSuccess) return cg_cuda(ctx, e, "cudaFree(workspace)");
        }
        cudaError_t e = cudaMalloc(&ctx->ws, bytes);
        if (e != cudaSuccess) return cg_cuda(ctx, e, "cudaMalloc(workspace)");
        ctx->ws_bytes = bytes;
    }
    *ptr = ctx->ws;
    return TM_OK;
}

extern "C" tm_status tm_cg_QdagQ(tm_ctx *ctx, const tm_gauge *U_hi, const tm_gauge *U_lo, void *x_dev,
                                 const void *b_dev, const tm_cg_params *prm, tm_cg_info *info, void *stream)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!ctx) return TM_ERR_ARG;
    if (!U_hi || bad_ptr(x_dev) || bad_ptr(b_dev) || !prm) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ: null or misaligned pointer");
    if (U_hi->prec != TM_F64 && U_hi->prec != TM_F64X)
        return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ: U_hi must be an FP64 or FP64X handle");
    if (!U_lo) U_lo = U_hi;
    if (memcmp(U_lo->dims, U_hi->dims, sizeof U_hi->dims) || memcmp(U_lo->bc, U_hi->bc, sizeof U_hi->bc))
        return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ: U_hi and U_lo describe different lattices");
    if (!(prm->tol > 0.0) || prm->maxiter < 0 || prm->reliable_every < 1 || !(prm->reliable_delta < 1.0))
        return tm_fail(ctx, TM_ERR_ARG,
                       "tm_cg_QdagQ: need tol > 0, maxiter >= 0, reliable_every >= 1, reliable_delta < 1");
    if (x_dev == b_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ: x and b must not overlap");

    Solver S;
    S.Uh = U_hi;
    S.Ul = U_lo;
    S.kappa = prm->kappa;
    S.mu = prm->mu;
    Work &w = S.w;
    w.vh = U_hi->geom.vh;
    w.PH = U_hi->prec;
    w.mixed = U_lo->prec == TM_F32 || U_lo->prec == TM_F16;
    w.P = w.mixed ? U_lo->prec : w.PH;
    w.PY = w.P == F16 ? F32 : w.P;
    if (!w.mixed) S.Ul = U_hi;

    // workspace: FP64 ax, t_hi, q_hi (+ r in plain mode), inner r, p, q, t, y, partials, scalars
    const size_t f64 = spinor_bytes(w.vh, w.PH), flo = spinor_bytes(w.vh, w.P), fy = spinor_bytes(w.vh, w.PY);
    const size_t nblk = blocks(w.vh, 128) + 1;
    size_t need = 3 * align256(f64) + 4 * align256(flo) + (w.mixed ? align256(fy) : 0) + align256(nblk * sizeof(double)) + align256(sizeof(CgScalars));
    void *base = nullptr;
    tm_status st = tm_ctx_workspace(ctx, need, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    auto take = [&](size_t n) { void *p = c; c += align256(n); return p; };
    w.x = x_dev;
    w.b = const_cast<void *>(b_dev);
    w.ax = take(f64);
    w.t_hi = take(f64);
    w.q_hi = take(f64);
    w.r = take(flo);
    w.p = take(flo);
    w.q = take(flo);
    w.t = take(flo);
    w.y = w.mixed ? take(fy) : x_dev;   // plain FP64: the update adds straight into x
    w.r_hi = w.r;
    w.partials = static_cast<double *>(take(nblk * sizeof(double)));
    w.s = static_cast<CgScalars *>(take(sizeof(CgScalars)));

    cudaStream_t s = (cudaStream_t)stream;
    tm_cg_info inf{};
    CgScalars h{};
    h.tol2 = prm->tol * prm->tol;
    h.maxiter = prm->maxiter;
    {
        const double d = w.mixed ? reliable_delta_for(prm->reliable_delta, w.P) : 0.0;
        h.delta2 = d * d;
    }
    h.every = prm->reliable_every;
    h.mixed = w.mixed ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(w.s, &h, sizeof h, cudaMemcpyHostToDevice, s);
    // |b|^2, then r = b - Q^dag Q x in FP64 (the inner residual r is its rounded copy)
    if (e == cudaSuccess) {
        if (w.PH == F64X) k_cg_norm<F64X><<<blocks(w.vh, LA_BLOCK), LA_BLOCK, 0, s>>>(w.vh, w.b, w.partials, w.s, FIN_BB);
        else k_cg_norm<F64><<<blocks(w.vh, LA_BLOCK), LA_BLOCK, 0, s>>>(w.vh, w.b, w.partials, w.s, FIN_BB);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = S.true_residual(nullptr, w.r, FIN_RR_TRUE, s);
    if (e == cudaSuccess) e = pupdate(w, 0, 1, s);   // p = r, rr = |r|^2 (ends the solve if already converged)
    if (e == cudaSuccess && w.mixed) e = zero(w.vh, w.PY, w.y, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.s, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cg_cuda(ctx, e, "setup");

    const int K = prm->reliable_every;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    if (prm->use_graph) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = S.segment(K, cap);
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            if (cap) cudaStreamDestroy(cap);
            return cg_cuda(ctx, e, "graph capture");
        }
    }

    const double target = h.tol2 * h.bb;
    bool converged = !(h.rr_true > target);
    tm_status result = TM_OK;
    int stalled = 0;
    while (!converged && h.status == TM_OK && h.iters < prm->maxiter) {
        const int before = h.iters;
        e = exec ? cudaGraphLaunch(exec, s) : S.segment(K, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.s, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        if (h.status != TM_OK) break;
        // a segment that performed no iteration twice in a row (breakdown) ends the solve
        stalled = h.iters == before ? stalled + 1 : 0;
        if (stalled >= 2) break;
        if (w.mixed) {
            // every FP64 residual recomputation happened inside the segment
            converged = h.done && h.rr_true <= target;
            if (h.done) break;
        } else if (h.done) {
            e = S.true_residual(w.ax, nullptr, FIN_RR_CHECK, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.s, sizeof h, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            converged = h.rr_true <= target;
            if (!converged && h.iters < prm->maxiter) {
                // recursive residual below target, true residual above: aim lower and go on
                double stop = h.stop_rr * 0.25;
                int zero_flag = 0;
                e = cudaMemcpyAsync(&w.s->stop_rr, &stop, sizeof(double), cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(&w.s->done, &zero_flag, sizeof(int), cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) break;
            }
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cg_cuda(ctx, e, "iteration");

    // plain FP64 mode that stopped on maxiter: report the true residual of the last iterate
    if (!w.mixed && !converged && h.status == TM_OK) {
        e = S.true_residual(w.ax, nullptr, FIN_RR_CHECK, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, w.s, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cg_cuda(ctx, e, "final residual");
    }
    if (h.status != TM_OK || !std::isfinite(h.rr_true)) result = TM_ERR_NONFINITE;
    else if (!converged) result = TM_ERR_NOT_CONVERGED;
    inf.iters = h.iters;
    inf.reliable_updates = h.nreliable;
    inf.true_relres = h.bb > 0 ? std::sqrt(h.rr_true / h.bb) : 0.0;
    inf.status = result;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) *info = inf;
    if (result == TM_ERR_NONFINITE) ctx->err = "tm_cg_QdagQ: non-finite residual";
    if (result == TM_ERR_NOT_CONVERGED) ctx->err = "tm_cg_QdagQ: maxiter reached";
    return result;
}
