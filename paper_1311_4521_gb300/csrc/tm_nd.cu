// tm_nd.cu -- the non-degenerate twisted-mass doublet (the mass-split
// strange-charm doublet of Frezzotti and Rossi, one of the operators the
// tmLQCD suite applies; the paper's introduction lists the suite's
// operators).  On a flavour doublet (psi_s, psi_c):
//
//   M_nd = (1 - kappa Dhop) x 1_f + i mubar gamma5 x tau3 - epsbar 1 x tau1,
//   mubar = 2 kappa mu_sigma, epsbar = 2 kappa mu_delta,
//   Q_nd = gamma5 (A - kappa^2 H_eo A^-1 H_oe),  A = M_ee = M_oo,
//   A^-1 = (1 - i mubar gamma5 tau3 + epsbar tau1) / (1 + mubar^2 - epsbar^2).
//
// The hops act on each flavour alone, so both flavours of a site are hopped
// by one thread with one load of each link (hop_site_src_pair); the
// site-local flavour mixing is fused into the two launches as in tm_Qtm:
// launch A writes t = -kappa^2 A^-1 H_oe psi on odd sites, launch B writes
// gamma5 (A psi + H_eo t) on even sites.  In the chiral basis (gamma5 = +1
// on spins 0, 1 and -1 on spins 2, 3) every factor is a complex number per
// spin half and flavour.
#include <cmath>
#include <string>

#include "tm_internal.h"

namespace twm {

// Resident CTAs per SM the pair hop is compiled for.  Measured on 32^3x64
// (Q_nd, FP32-12 / FP16-12): 3 CTAs (168 registers) 0.342 / 0.277 ms, 4 (128
// registers, 16 bytes of spills) 0.332 / 0.255 ms, 2 0.407 / 0.277 ms.  One
// thread per (site, flavour) instead, the flavours on adjacent lanes sharing
// each link load and mixed by shuffles, was slower at every occupancy
// (0.359-0.384 / 0.291-0.298 ms): the pair form's single link load and
// reconstruction per site outweigh its lower occupancy.
#ifndef TM_ND_MINB_F64
#define TM_ND_MINB_F64 1
#endif
#ifndef TM_ND_MINB_F32
#define TM_ND_MINB_F32 4
#endif
#define TM_ND_MINB(P) ((P) == F64 ? TM_ND_MINB_F64 : TM_ND_MINB_F32)

// The doublet's site-local coefficients, in double and rounded once to float.
struct NdCoef {
    // launch A: a = c (1 - i mubar), b = c (1 + i mubar), e = c epsbar with c = -kappa^2 / D
    // launch B: p = 1 + i mubar, m = 1 - i mubar, f = epsbar
    double d[10];  // a.re a.im b.re b.im e  p.re p.im m.re m.im f
    float f[10];
    TM_HD double get(int k, double) const { return d[k]; }
    TM_HD float get(int k, float) const { return f[k]; }
};

template <typename R> TM_HD cpx<R> cscale(cpx<R> a, cpx<R> b) { return a * b; }

// acc + s * v for a real s
template <typename R> TM_HD cpx<R> rmadd(R s, cpx<R> v, cpx<R> acc) { return {acc.re + s * v.re, acc.im + s * v.im}; }

template <int P, int RECON, bool STAGE_B>
__global__ void __launch_bounds__(128, TM_ND_MINB(P))
    k_nd(Geom g, int p, const typename LinkIO<P, RECON>::V *__restrict__ links, const void *__restrict__ in_s,
         const void *__restrict__ in_c, void *__restrict__ out_s, void *__restrict__ out_c,
         const void *__restrict__ x_s, const void *__restrict__ x_c, NdCoef k)
{
    using R = typename SpinorIO<P>::R;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    Nbrs n;
    neighbours(g, p, i, n);
    GlobalLinks<P, RECON> src{links, g.vh, i, p};
    Spinor<R> hs, hc, os, oc;
    hop_site_src_pair<P, false>(g, n, src, in_s, in_c, hs, hc);
    const R z = R(0);
    if (!STAGE_B) {
        const cpx<R> a = {k.get(0, z), k.get(1, z)}, b = {k.get(2, z), k.get(3, z)};
        const R e = k.get(4, z);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cpx<R> fs = sp < 2 ? a : b, fc = sp < 2 ? b : a;   // (1 -+ i mubar gamma5) on s, c
                os[sp][c] = rmadd(e, hc[sp][c], cscale(fs, hs[sp][c]));
                oc[sp][c] = rmadd(e, hs[sp][c], cscale(fc, hc[sp][c]));
            }
    } else {
        Spinor<R> xs, xc;
        SpinorIO<P>::load(x_s, g.vh, i, xs);
        SpinorIO<P>::load(x_c, g.vh, i, xc);
        const cpx<R> pl = {k.get(5, z), k.get(6, z)}, mi = {k.get(7, z), k.get(8, z)};
        const R f = k.get(9, z);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // A x: s gets (1 + i mubar gamma5) x_s - epsbar x_c, c gets (1 - i mubar gamma5) x_c - epsbar x_s
                const cpx<R> fs = sp < 2 ? pl : mi, fc = sp < 2 ? mi : pl;
                cpx<R> vs = rmadd(-f, xc[sp][c], cmadd(fs, xs[sp][c], hs[sp][c]));
                cpx<R> vc = rmadd(-f, xs[sp][c], cmadd(fc, xc[sp][c], hc[sp][c]));
                os[sp][c] = sp < 2 ? vs : -vs;   // the outer gamma5
                oc[sp][c] = sp < 2 ? vc : -vc;
            }
    }
    SpinorIO<P>::store(out_s, g.vh, i, os);
    SpinorIO<P>::store(out_c, g.vh, i, oc);
}

template <int P, int RECON>
cudaError_t nd_launch(const tm_gauge *U, bool stage_b, const void *in_s, const void *in_c, void *out_s, void *out_c,
                      const void *x_s, const void *x_c, const NdCoef &k, cudaStream_t s)
{
    using V = typename LinkIO<P, RECON>::V;
    const Geom &g = U->geom;
    const unsigned grid = (g.vh + 127) / 128;
    const V *l = static_cast<const V *>(U->links);
    if (stage_b) k_nd<P, RECON, true><<<grid, 128, 0, s>>>(g, 0, l, in_s, in_c, out_s, out_c, x_s, x_c, k);
    else k_nd<P, RECON, false><<<grid, 128, 0, s>>>(g, 1, l, in_s, in_c, out_s, out_c, x_s, x_c, k);
    return cudaGetLastError();
}

cudaError_t nd_dispatch(const tm_gauge *U, bool stage_b, const void *in_s, const void *in_c, void *out_s, void *out_c,
                        const void *x_s, const void *x_c, const NdCoef &k, cudaStream_t s)
{
    if (U->geom.vh == 0) return cudaSuccess;
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: return nd_launch<F64, 18>(U, stage_b, in_s, in_c, out_s, out_c, x_s, x_c, k, s);
    case F64 * 100 + 12: return nd_launch<F64, 12>(U, stage_b, in_s, in_c, out_s, out_c, x_s, x_c, k, s);
    case F32 * 100 + 18: return nd_launch<F32, 18>(U, stage_b, in_s, in_c, out_s, out_c, x_s, x_c, k, s);
    case F32 * 100 + 12: return nd_launch<F32, 12>(U, stage_b, in_s, in_c, out_s, out_c, x_s, x_c, k, s);
    case F16 * 100 + 12: return nd_launch<F16, 12>(U, stage_b, in_s, in_c, out_s, out_c, x_s, x_c, k, s);
    }
    return cudaErrorInvalidValue;
}

NdCoef nd_coef(double kappa, double mubar, double epsbar)
{
    const double D = 1.0 + mubar * mubar - epsbar * epsbar, c = -kappa * kappa / D;
    NdCoef k;
    const double v[10] = {c, -c * mubar, c, c * mubar, c * epsbar, 1.0, mubar, 1.0, -mubar, epsbar};
    for (int j = 0; j < 10; ++j) {
        k.d[j] = v[j];
        k.f[j] = float(v[j]);
    }
    return k;
}

}  // namespace twm

using namespace twm;

extern "C" tm_status tm_Qnd(tm_ctx *ctx, const tm_gauge *U, void *out_s_dev, void *out_c_dev, const void *in_s_dev,
                            const void *in_c_dev, double kappa, double mu_sigma, double mu_delta, int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(out_s_dev) || bad_ptr(out_c_dev) || bad_ptr(in_s_dev) || bad_ptr(in_c_dev))
        return tm_fail(ctx, TM_ERR_ARG, "tm_Qnd: null or misaligned pointer");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_Qnd: sign must be +1 or -1");
    if (out_s_dev == out_c_dev || out_s_dev == in_s_dev || out_s_dev == in_c_dev || out_c_dev == in_s_dev ||
        out_c_dev == in_c_dev)
        return tm_fail(ctx, TM_ERR_ARG, "tm_Qnd: the outputs must differ from each other and from the inputs");
    if (U->prec != TM_F64 && U->prec != TM_F32 && U->prec != TM_F16)
        return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_Qnd: TM_F64, TM_F32 and TM_F16 handles only");
    const double mubar = 2.0 * kappa * mu_sigma * sign, epsbar = 2.0 * kappa * mu_delta;
    const double D = 1.0 + mubar * mubar - epsbar * epsbar;
    if (!(std::fabs(D) > 1e-12)) return tm_fail(ctx, TM_ERR_ARG, "tm_Qnd: M_oo is singular (epsbar^2 = 1 + mubar^2)");
    const size_t fb = align256(spinor_bytes(U->geom.vh, U->prec));
    void *base = nullptr;
    tm_status st = tm_ctx_scratch(ctx, 2 * fb, &base);
    if (st != TM_OK) return st;
    char *t = static_cast<char *>(base);
    const NdCoef k = nd_coef(kappa, mubar, epsbar);
    cudaStream_t s = (cudaStream_t)stream;
    tm_trace_mark(ctx, 0, s);
    cudaError_t e = nd_dispatch(U, false, in_s_dev, in_c_dev, t, t + fb, nullptr, nullptr, k, s);
    if (e == cudaSuccess) {
        tm_trace_mark(ctx, 1, s);
        e = nd_dispatch(U, true, t, t + fb, out_s_dev, out_c_dev, in_s_dev, in_c_dev, k, s);
    }
    if (e == cudaSuccess) tm_trace_mark(ctx, 2, s);
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qnd: ") + cudaGetErrorString(e));
    return TM_OK;
}
