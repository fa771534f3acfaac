// tm_force.cu -- the fermion force of S = phi^dag (Q^dag Q)^-1 phi and the
// complex gradient dS/dU, one thread per link, no atomics: every link is
// written by exactly one thread, so the race the paper discusses for the
// HMC derivative (Sec. 2.4: atomic updates of the derivative field) cannot
// occur.
#include <string>

#include "tm_force.cuh"
#include "tm_internal.h"

namespace twm {

template <int P, int RECON>
__global__ void __launch_bounds__(128) k_force(Geom g, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                               const void *Xe, const void *Ye, const void *Zo, const void *Bo,
                                               double kappa2, int mode, double *F)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const int p = blockIdx.y >> 2, mu = blockIdx.y & 3;   // uniform per block
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
    dim3 grid((U->geom.vh + 127) / 128, 8);
    k_force<P, RECON><<<grid, 128, 0, s>>>(U->geom, static_cast<const typename LinkIO<P, RECON>::V *>(U->links), Xe,
                                          Ye, Zo, Bo, kappa2, mode, F);
    return cudaGetLastError();
}

// gamma5 (1 + i mut gamma5) / (1 + mut^2): upper (1 + i mut) d, lower -(1 - i mut) d
Coef coef_force_b(double mut)
{
    double d = 1.0 / (1.0 + mut * mut);
    return Coef{d, mut * d, -d, mut * d, 0, 0, 0, 0};
}

}  // namespace twm

using namespace twm;

extern "C" tm_status tm_force(tm_ctx *ctx, const tm_gauge *U, double *F_dev, const void *X_e_dev, double kappa,
                              double mu, int mode, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || !F_dev || !X_e_dev) {
        ctx->err = "tm_force: null pointer";
        return TM_ERR_ARG;
    }
    if (mode != TM_FORCE_SU3 && mode != TM_FORCE_GRAD) {
        ctx->err = "tm_force: mode must be TM_FORCE_SU3 or TM_FORCE_GRAD";
        return TM_ERR_ARG;
    }
    const unsigned vh = U->geom.vh;
    const size_t fb = (spinor_bytes(vh, U->prec) + 255) & ~size_t(255);
    void *base = nullptr;
    tm_status st = tm_ctx_workspace(ctx, 3 * fb, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    void *Ye = c, *Zo = c + fb, *Bo = c + 2 * fb;
    const double mut = 2.0 * kappa * mu;
    cudaStream_t s = (cudaStream_t)stream;
    // Z = M_oo^-1 H_oe X, Y = Q X, B = gamma5 (M_oo^-1)^dag H_oe Y
    cudaError_t e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, X_e_dev, Zo, nullptr,
                               coef_qtm_a(mut), s, 128);
    if (e == cudaSuccess)
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, Zo, Ye, X_e_dev, coef_qtm_b(kappa, mut), s, 128);
    if (e == cudaSuccess)
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, Ye, Bo, nullptr, coef_force_b(mut), s, 128);
    if (e == cudaSuccess) {
        const double k2 = kappa * kappa;
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
    }
    if (e != cudaSuccess) {
        ctx->err = std::string("tm_force: ") + cudaGetErrorString(e);
        return TM_ERR_CUDA;
    }
    return TM_OK;
}
