// tm_solve.cu -- the full-lattice Wilson twisted-mass solve M x = b by even-odd
// preconditioning: the steps on either side of the CG on the even sites.
//
//   [M_ee M_eo] [x_e]   [b_e]      M_ee = M_oo = 1 + i mut gamma5,
//   [M_oe M_oo] [x_o] = [b_o],     M_eo = -kappa H_eo, M_oe = -kappa H_oe.
//
// The Schur complement gives (M_ee - M_eo M_oo^-1 M_oe) x_e = bhat_e with
// bhat_e = b_e - M_eo M_oo^-1 b_o = b_e + kappa H_eo M_oo^-1 b_o, i.e.
// Q x_e = gamma5 bhat_e with Q = gamma5 (M_ee - M_eo M_oo^-1 M_oe), solved as
// Q^dag Q x_e = Q^dag gamma5 bhat_e; then x_o = M_oo^-1 (b_o - M_oe x_e)
// = M_oo^-1 (b_o + kappa H_oe x_e).
#include <string>

#include "tm_internal.h"

namespace twm {

// out = a in on one parity (a per spin half): the site-local factors of M.
template <int P>
__global__ void __launch_bounds__(256) k_site_scale(unsigned vh, const void *in, void *out, Coef k)
{
    using R = typename SpinorIO<P>::R;
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    Spinor<R> s, o;
    SpinorIO<P>::load(in, vh, i, s);
    epilogue(k, s, static_cast<const Spinor<R> *>(nullptr), o);
    SpinorIO<P>::store(out, vh, i, o);
}

}  // namespace twm

using namespace twm;

extern "C" tm_status tm_solve_eo(tm_ctx *ctx, const tm_gauge *U_hi, const tm_gauge *U_lo, void *x_e, void *x_o,
                                 const void *b_e, const void *b_o, const tm_cg_params *prm, tm_cg_info *info,
                                 void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U_hi || bad_ptr(x_e) || bad_ptr(x_o) || bad_ptr(b_e) || bad_ptr(b_o) || !prm) {
        ctx->err = "tm_solve_eo: null or misaligned pointer";
        return TM_ERR_ARG;
    }
    if (U_hi->prec != TM_F64) {
        ctx->err = "tm_solve_eo: U_hi must be an FP64 handle";
        return TM_ERR_ARG;
    }
    if (x_e == x_o || x_e == b_e || x_e == b_o || x_o == b_e || x_o == b_o) {
        ctx->err = "tm_solve_eo: x and b fields must not overlap";
        return TM_ERR_ARG;
    }
    const Geom &g = U_hi->geom;
    const size_t fb = align256(spinor_bytes(g.vh, F64));
    void *base = nullptr;
    tm_status st = tm_ctx_scratch(ctx, 3 * fb, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    void *t_o = c, *c_e = c + fb, *src = c + 2 * fb;
    const double kappa = prm->kappa, mut = 2.0 * prm->kappa * prm->mu, d = 1.0 / (1.0 + mut * mut);
    cudaStream_t s = (cudaStream_t)stream;
    // t_o = M_oo^-1 b_o
    k_site_scale<F64><<<(g.vh + 255) / 256, 256, 0, s>>>(g.vh, b_o, t_o, coef_qtm_a(mut));
    cudaError_t e = cudaGetLastError();
    // c_e = gamma5 (b_e + kappa H_eo t_o)
    if (e == cudaSuccess)
        e = launch_hop(g, F64, U_hi->recon, false, TM_EO, U_hi->links, t_o, c_e, b_e,
                       Coef{kappa, 0, -kappa, 0, 1, 0, -1, 0}, s, U_hi->map);
    // src = Q(-mu) c_e = Q^dag gamma5 bhat_e
    if (e == cudaSuccess)
        e = launch_hop(g, F64, U_hi->recon, false, TM_OE, U_hi->links, c_e, t_o, nullptr, coef_qtm_a_scaled(kappa, -mut), s, U_hi->map);
    if (e == cudaSuccess)
        e = launch_hop(g, F64, U_hi->recon, false, TM_EO, U_hi->links, t_o, src, c_e, coef_qtm_b_unit(-mut), s, U_hi->map);
    if (e != cudaSuccess) {
        ctx->err = std::string("tm_solve_eo: source: ") + cudaGetErrorString(e);
        return TM_ERR_CUDA;
    }
    tm_status cg = tm_cg_QdagQ(ctx, U_hi, U_lo, x_e, src, prm, info, stream);
    if (cg != TM_OK && cg != TM_ERR_NOT_CONVERGED) return cg;
    // x_o = M_oo^-1 (b_o + kappa H_oe x_e)
    e = launch_hop(g, F64, U_hi->recon, false, TM_OE, U_hi->links, x_e, x_o, b_o,
                   Coef{kappa * d, -kappa * mut * d, kappa * d, kappa * mut * d, d, -mut * d, d, mut * d}, s, U_hi->map);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ctx->err = std::string("tm_solve_eo: reconstruction: ") + cudaGetErrorString(e);
        return TM_ERR_CUDA;
    }
    return cg;
}
