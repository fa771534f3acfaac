// tm_force.cu -- the fermion force of S = phi^dag (Q^dag Q)^-1 phi and the
// complex gradient dS/dU.  Default assembly: one thread per link, no
// atomics: every link is written by exactly one thread, so the race the
// paper discusses for the HMC derivative (Sec. 2.4: atomic updates of the
// derivative field) cannot occur.  The two push schemes of that discussion
// (atomic adds, and private buffers summed in a second pass) are built
// beside it for comparison.
#include <string>

#include "tm_force.cuh"
#include "tm_internal.h"

namespace twm {

template <int P, int RECON>
__global__ void __launch_bounds__(128) k_force(Geom g, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                               const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                               double kappa2, int mode, double *F)
{
    // the 8 (parity, direction) slices of one tile of sites are consecutive
    // blocks, so the spinors that neighbouring slices share come from L2
    const int slice = blockIdx.x & 7;
    const unsigned i = (blockIdx.x >> 3) * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const int p = slice >> 2, mu = slice & 3;   // uniform per block
    switch (mu) {
    case 0: force_site<P, RECON, 0>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F); break;
    case 1: force_site<P, RECON, 1>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F); break;
    case 2: force_site<P, RECON, 2>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F); break;
    default: force_site<P, RECON, 3>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F); break;
    }
}

template <int P, int RECON>
static cudaError_t force_launch(const tm_gauge *U, const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                double kappa2, int mode, double *F, cudaStream_t s)
{
    const unsigned grid = 8 * ((U->geom.vh + 127) / 128);
    k_force<P, RECON><<<grid, 128, 0, s>>>(U->geom, static_cast<const typename LinkIO<P, RECON>::V *>(U->links), Xe,
                                          Ye, Zo, Bo, kappa2, mode, F);
    return cudaGetLastError();
}

// ---- push schemes (the comparison of Sec. 2.4: atomics vs "halo memory")
// One thread per site y; for each direction it computes the forward part of
// link (mu, y) and the backward part of link (mu, y - mu).  Every link thus
// has two writers: its base and its tip.
enum { PUSH_ATOMIC = 1, PUSH_HALO = 2 };

template <int P, int RECON, int MU, int SCHEME>
__device__ __forceinline__ void push_site(const Geom &g, int p, unsigned i, const typename LinkIO<P, RECON>::V *links,
                                          const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                          double kappa2, int mode, double *F, double *Hf, double *Hb)
{
    using R = typename SpinorIO<P>::R;
    using L = LinkIO<P, RECON>;
    Nbrs n;
    neighbours(g, p, i, n);
    // fields at y: L(y) (own), R at the two neighbours
    Spinor<R> Ly, Rf, Rb;
    const void *Rnb = p == 0 ? Zo : Xe;  // R on the other parity
    if (p == 0) {
        SpinorIO<P>::load(Ye, g.vh, i, Ly);
        apply_g5(Ly);
    } else {
        SpinorIO<P>::load(Bo, g.vh, i, Ly);
    }
    SpinorIO<P>::load(Rnb, g.vh, n.fwd[MU], Rf);
    SpinorIO<P>::load(Rnb, g.vh, n.bwd[MU], Rb);
    Link<R> uf, ub;
    L::load(links + size_t(4 * p + MU) * L::NCHUNK * g.vh, g.vh, i, uf);
    L::load(links + size_t(4 * (1 - p) + MU) * L::NCHUNK * g.vh, g.vh, n.bwd[MU], ub);
    const R sf = (n.wf[MU] && g.anti[MU]) ? R(-1) : R(1);
    const R sb = (n.wb[MU] && g.anti[MU]) ? R(-1) : R(1);
    Mat<R> mf, mb;
    force_part_fwd<MU>(uf, Rf, Ly, to_R<R>(kappa2), sf, mode, mf);
    force_part_bwd<MU>(ub, Rb, Ly, to_R<R>(kappa2), sb, mode, mb);
    const size_t V = 2 * size_t(g.vh);
    const size_t lf = size_t(MU) * V + lex_of(g, p, i);              // link (mu, y)
    const size_t lb = size_t(MU) * V + lex_of(g, 1 - p, n.bwd[MU]);  // link (mu, y - mu)
    if (SCHEME == PUSH_ATOMIC) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int k = 6 * a + 2 * b;
                atomicAdd(F + lf * 18 + k, double(mf[a][b].re));
                atomicAdd(F + lf * 18 + k + 1, double(mf[a][b].im));
                atomicAdd(F + lb * 18 + k, double(mb[a][b].re));
                atomicAdd(F + lb * 18 + k + 1, double(mb[a][b].im));
            }
    } else {
        store_mat(Hf + lf * 18, mf);
        store_mat(Hb + lb * 18, mb);
    }
}

template <int P, int RECON, int SCHEME>
__global__ void __launch_bounds__(128) k_force_push(Geom g, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                                    const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                                    double kappa2, int mode, double *F, double *Hf, double *Hb)
{
    const int slice = blockIdx.x & 7;   // as in k_force
    const unsigned i = (blockIdx.x >> 3) * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const int p = slice >> 2, mu = slice & 3;
    switch (mu) {
    case 0: push_site<P, RECON, 0, SCHEME>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb); break;
    case 1: push_site<P, RECON, 1, SCHEME>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb); break;
    case 2: push_site<P, RECON, 2, SCHEME>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb); break;
    default: push_site<P, RECON, 3, SCHEME>(g, p, i, links, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb); break;
    }
}

// Second pass of the halo-memory scheme: F = Hf + Hb, element by element.
__global__ void __launch_bounds__(256) k_force_halo_sum(size_t n, const double *Hf, const double *Hb, double *F)
{
    const size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    if (k < n) F[k] = Hf[k] + Hb[k];
}

template <int P, int RECON>
static cudaError_t force_push_launch(const tm_gauge *U, const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                     double kappa2, int mode, int scheme, double *F, double *Hf, double *Hb,
                                     cudaStream_t s)
{
    const unsigned grid = 8 * ((U->geom.vh + 127) / 128);
    const auto *l = static_cast<const typename LinkIO<P, RECON>::V *>(U->links);
    if (scheme == PUSH_ATOMIC)
        k_force_push<P, RECON, PUSH_ATOMIC><<<grid, 128, 0, s>>>(U->geom, l, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb);
    else
        k_force_push<P, RECON, PUSH_HALO><<<grid, 128, 0, s>>>(U->geom, l, Xe, Ye, Zo, Bo, kappa2, mode, F, Hf, Hb);
    return cudaGetLastError();
}

// out = gamma5 in on a packed field (spins 2 and 3 negated)
template <int P>
__global__ void __launch_bounds__(256) k_gamma5(unsigned vh, const void *__restrict__ in, void *__restrict__ out)
{
    using R = typename SpinorIO<P>::R;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    Spinor<R> s;
    SpinorIO<P>::load(in, vh, i, s);
    apply_g5(s);
    SpinorIO<P>::store(out, vh, i, s);
}

static cudaError_t launch_gamma5(unsigned vh, int prec, const void *in, void *out, cudaStream_t s)
{
    if (vh == 0) return cudaSuccess;
    const unsigned grid = (vh + 255) / 256;
    if (prec == F64) k_gamma5<F64><<<grid, 256, 0, s>>>(vh, in, out);
    else if (prec == F64X) k_gamma5<F64X><<<grid, 256, 0, s>>>(vh, in, out);
    else if (prec == F32) k_gamma5<F32><<<grid, 256, 0, s>>>(vh, in, out);
    else k_gamma5<F16><<<grid, 256, 0, s>>>(vh, in, out);
    return cudaGetLastError();
}

// The owner-scheme link kernel for every storage format.
static cudaError_t force_owner(const tm_gauge *U, const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                               double kappa2, int mode, double *F, cudaStream_t s)
{
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: return force_launch<F64, 18>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F64 * 100 + 12: return force_launch<F64, 12>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F32 * 100 + 18: return force_launch<F32, 18>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F32 * 100 + 12: return force_launch<F32, 12>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F16 * 100 + 12: return force_launch<F16, 12>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F64X * 100 + 18: return force_launch<F64X, 18>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    case F64X * 100 + 12: return force_launch<F64X, 12>(U, Xe, Ye, Zo, Bo, kappa2, mode, F, s);
    }
    return cudaErrorInvalidValue;
}

// gamma5 (1 + i mut gamma5) / (1 + mut^2): upper (1 + i mut) d, lower -(1 - i mut) d
Coef coef_force_b(double mut)
{
    double d = 1.0 / (1.0 + mut * mut);
    return Coef{d, mut * d, -d, mut * d, 0, 0, 0, 0};
}

}  // namespace twm

using namespace twm;

extern "C" tm_status tm_force_ex(tm_ctx *ctx, const tm_gauge *U, double *F_dev, const void *X_e_dev, double kappa,
                                 double mu, int mode, int scheme, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(F_dev) || bad_ptr(X_e_dev)) {
        ctx->err = "tm_force: null or misaligned pointer";
        return TM_ERR_ARG;
    }
    if (mode != TM_FORCE_SU3 && mode != TM_FORCE_GRAD) {
        ctx->err = "tm_force: mode must be TM_FORCE_SU3 or TM_FORCE_GRAD";
        return TM_ERR_ARG;
    }
    if (scheme != TM_FORCE_OWNER && scheme != TM_FORCE_ATOMIC && scheme != TM_FORCE_HALO) {
        ctx->err = "tm_force_ex: scheme must be TM_FORCE_OWNER, TM_FORCE_ATOMIC or TM_FORCE_HALO";
        return TM_ERR_ARG;
    }
    if (scheme != TM_FORCE_OWNER && U->prec != TM_F64 && U->prec != TM_F32) {
        ctx->err = "tm_force_ex: the push schemes are built for TM_F64 and TM_F32 handles";
        return TM_ERR_UNSUPPORTED;
    }
    const unsigned vh = U->geom.vh;
    const size_t fb = align256(spinor_bytes(vh, U->prec));
    const size_t nF = size_t(4) * 2 * vh * 18;   // doubles in one force field
    const size_t hb = scheme == TM_FORCE_HALO ? align256(nF * sizeof(double)) : 0;
    void *base = nullptr;
    tm_status st = tm_ctx_workspace(ctx, 3 * fb + 2 * hb, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    void *Ye = c, *Zo = c + fb, *Bo = c + 2 * fb;
    double *Hf = hb ? reinterpret_cast<double *>(c + 3 * fb) : nullptr;
    double *Hb = hb ? reinterpret_cast<double *>(c + 3 * fb + hb) : nullptr;
    const double mut = 2.0 * kappa * mu;
    cudaStream_t s = (cudaStream_t)stream;
    // Z = M_oo^-1 H_oe X, Y = Q X, B = gamma5 (M_oo^-1)^dag H_oe Y
    cudaError_t e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, X_e_dev, Zo, nullptr,
                               coef_qtm_a(mut), s, U->map);
    if (e == cudaSuccess)
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, Zo, Ye, X_e_dev, coef_qtm_b(kappa, mut), s, U->map);
    if (e == cudaSuccess)
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, Ye, Bo, nullptr, coef_force_b(mut), s, U->map);
    const double k2 = kappa * kappa;
    if (e == cudaSuccess && scheme == TM_FORCE_OWNER) {
        switch (U->prec * 100 + U->recon) {
        case F64 * 100 + 18: e = force_launch<F64, 18>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F64 * 100 + 12: e = force_launch<F64, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F32 * 100 + 18: e = force_launch<F32, 18>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F32 * 100 + 12: e = force_launch<F32, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F16 * 100 + 12: e = force_launch<F16, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F64X * 100 + 18: e = force_launch<F64X, 18>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        case F64X * 100 + 12: e = force_launch<F64X, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, F_dev, s); break;
        default: e = cudaErrorInvalidValue;
        }
    } else if (e == cudaSuccess) {
        const int sch = scheme == TM_FORCE_ATOMIC ? PUSH_ATOMIC : PUSH_HALO;
        if (scheme == TM_FORCE_ATOMIC) e = cudaMemsetAsync(F_dev, 0, nF * sizeof(double), s);
        if (e == cudaSuccess) {
            switch (U->prec * 100 + U->recon) {
            case F64 * 100 + 18: e = force_push_launch<F64, 18>(U, X_e_dev, Ye, Zo, Bo, k2, mode, sch, F_dev, Hf, Hb, s); break;
            case F64 * 100 + 12: e = force_push_launch<F64, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, sch, F_dev, Hf, Hb, s); break;
            case F32 * 100 + 18: e = force_push_launch<F32, 18>(U, X_e_dev, Ye, Zo, Bo, k2, mode, sch, F_dev, Hf, Hb, s); break;
            case F32 * 100 + 12: e = force_push_launch<F32, 12>(U, X_e_dev, Ye, Zo, Bo, k2, mode, sch, F_dev, Hf, Hb, s); break;
            default: e = cudaErrorInvalidValue;
            }
        }
        if (e == cudaSuccess && scheme == TM_FORCE_HALO) {
            k_force_halo_sum<<<unsigned((nF + 255) / 256), 256, 0, s>>>(nF, Hf, Hb, F_dev);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        ctx->err = std::string("tm_force: ") + cudaGetErrorString(e);
        return TM_ERR_CUDA;
    }
    return TM_OK;
}

extern "C" tm_status tm_force(tm_ctx *ctx, const tm_gauge *U, double *F_dev, const void *X_e_dev, double kappa,
                              double mu, int mode, void *stream)
{
    return tm_force_ex(ctx, U, F_dev, X_e_dev, kappa, mu, mode, TM_FORCE_OWNER, stream);
}

// The link gradient of a bilinear form: the force kernel computes, for any
// full-lattice fields R = (Xe on even, Zo on odd) and L = (gamma5 Ye on
// even, Bo on odd), the gradient of 2 k Re(L^dag Dhop(U) R) with respect to
// the complex link entries (k its kappa2 argument).
//   Q_tm:  Re <Y, Q X> = -kappa^2 Re(L^dag dDhop R) with Z = M_oo^-1 H_oe X and
//          B = gamma5 (M_oo^-1)^dag H_oe Y (the same fields as for the force),
//          so k = -kappa^2 / 2;
//   H_eo:  Re <Y, H_eo X> with R = (0, X), L = (Y, 0): Ye = gamma5 Y, k = 1/2;
//   H_oe:  Re <Y, H_oe X> with R = (X, 0), L = (0, Y): Bo = Y, k = 1/2.
extern "C" tm_status tm_link_grad(tm_ctx *ctx, const tm_gauge *U, double *G_dev, const void *X_dev, const void *Y_dev,
                                  int op, double kappa, double mu, int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(G_dev) || bad_ptr(X_dev) || bad_ptr(Y_dev))
        return tm_fail(ctx, TM_ERR_ARG, "tm_link_grad: null or misaligned pointer");
    if (op != TM_GRAD_QTM && op != TM_GRAD_HOP_EO && op != TM_GRAD_HOP_OE)
        return tm_fail(ctx, TM_ERR_ARG, "tm_link_grad: op must be TM_GRAD_QTM, TM_GRAD_HOP_EO or TM_GRAD_HOP_OE");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_link_grad: sign must be +1 or -1");
    const unsigned vh = U->geom.vh;
    const size_t fb = align256(spinor_bytes(vh, U->prec));
    void *base = nullptr;
    tm_status st = tm_ctx_workspace(ctx, 2 * fb, &base);
    if (st != TM_OK) return st;
    char *w0 = static_cast<char *>(base), *w1 = w0 + fb;
    cudaStream_t s = (cudaStream_t)stream;
    const void *Xe, *Ye, *Zo, *Bo;
    double k2;
    cudaError_t e = cudaSuccess;
    if (op == TM_GRAD_QTM) {
        const double mut = 2.0 * kappa * mu * sign;
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, X_dev, w0, nullptr, coef_qtm_a(mut), s, U->map);
        if (e == cudaSuccess)
            e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, Y_dev, w1, nullptr, coef_force_b(mut), s,
                           U->map);
        Xe = X_dev, Ye = Y_dev, Zo = w0, Bo = w1;
        k2 = -0.5 * kappa * kappa;
    } else if (op == TM_GRAD_HOP_EO) {
        e = cudaMemsetAsync(w0, 0, fb, s);   // zeros for the unused halves of R and L
        if (e == cudaSuccess) e = launch_gamma5(vh, U->prec, Y_dev, w1, s);
        Xe = w0, Ye = w1, Zo = X_dev, Bo = w0;
        k2 = 0.5;
    } else {
        e = cudaMemsetAsync(w0, 0, fb, s);
        Xe = X_dev, Ye = w0, Zo = w0, Bo = Y_dev;
        k2 = 0.5;
    }
    if (e == cudaSuccess) e = force_owner(U, Xe, Ye, Zo, Bo, k2, TM_FORCE_GRAD, G_dev, s);
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_link_grad: ") + cudaGetErrorString(e));
    return TM_OK;
}
