// tm_slab.cu -- the hopping matrix on one time slab of a lattice that is cut
// along t into slabs, one per GPU: the surface/body split with overlapped
// communication of the paper's Sec. 2.5, on GPUs.
//
// A slab is an ordinary local lattice (its gauge handle is created from the
// slab's own links with tm_gauge_create), whose hops across its two time
// faces reach sites of the neighbouring slabs.  Only those hops need data
// from elsewhere, and only as projected half-spinors (12 reals per face
// site):
//   - the output sites on the upper face (t = Lt-1) hop forward to the
//     lower face (t = 0) of the next slab: (1 -+ gamma_0) U_0(x) psi(x+t).
//     The next slab projects its own t = 0 sites, (1 -+ gamma_0) psi, and
//     sends the upper pairs; the receiver multiplies by its own U_0(x).
//   - the output sites on the lower face (t = 0) hop backward to the upper
//     face of the previous slab: (1 +- gamma_0) U_0(x-t)^dag psi(x-t).  The
//     link U_0(x-t) belongs to the previous slab, which projects, multiplies
//     by U_0^dag and sends the product; the receiver only accumulates it.
// tm_slab_pack writes both faces of an input field; the caller moves them
// (cudaMemcpyAsync between GPUs or within one, NCCL send/recv between
// processes); tm_slab_hop runs the interior sites (all neighbours local:
// 1 <= t <= Lt-2, a contiguous index range since the even-odd index is
// t-major) and the face sites (reading the received faces) as separate
// launches, so that the interior work overlaps the exchange.
//
// Within a slab the local neighbour arithmetic wraps periodically in t; for
// a face site that wrapped index minus (Lt-1) x (sites per time slice and
// parity) is its position in the received face, so no extra index table is
// needed.  The sign of a hop through a face (the antiperiodic boundary, for
// the faces that close the global time direction) is given per face.
#include <cstdio>
#include <string>

#include "tm_internal.h"

namespace twm {

// One face: the 12 reals of Half<R> for `nf` face sites, component-major
// (FP64: 6 double2 arrays; FP32: 3 float4 arrays of two complex each).
template <typename R> struct FaceIO;

template <> struct FaceIO<double> {
    static constexpr size_t BYTES_PER_SITE = 96;
    TM_HD static void load(const void *base, unsigned nf, unsigned j, Half<double> &h)
    {
        const double2 *b = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 v = ld_keep(b + size_t(k) * nf + j);
            h[k / 3][k % 3] = {v.x, v.y};
        }
    }
    TM_HD static void store(void *base, unsigned nf, unsigned j, const Half<double> &h)
    {
        double2 *b = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) b[size_t(k) * nf + j] = make_double2(h[k / 3][k % 3].re, h[k / 3][k % 3].im);
    }
};

template <> struct FaceIO<float> {
    static constexpr size_t BYTES_PER_SITE = 48;
    TM_HD static void load(const void *base, unsigned nf, unsigned j, Half<float> &h)
    {
        const float4 *b = static_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = ld_keep(b + size_t(k) * nf + j);
            h[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            h[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
    }
    TM_HD static void store(void *base, unsigned nf, unsigned j, const Half<float> &h)
    {
        float4 *b = static_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cpx<float> &a = h[(2 * k) / 3][(2 * k) % 3];
            const cpx<float> &c = h[(2 * k + 1) / 3][(2 * k + 1) % 3];
            b[size_t(k) * nf + j] = make_float4(a.re, a.im, c.re, c.im);
        }
    }
};

// Faces of the input field of parity q: thread j < st writes the lower face
// (site j, t = 0: the projection the previous slab's forward hops need),
// thread st + j the upper face (site (Lt-1) st + j: U_0^dag times the
// projection, what the next slab's backward hops need).
template <int P, int RECON, bool DAG>
__global__ void __launch_bounds__(128) k_slab_pack(Geom g, int q, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                                   const void *__restrict__ in, void *lower, void *upper)
{
    using R = typename SpinorIO<P>::R;
    using L = LinkIO<P, RECON>;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_0 of the receiving hop
    constexpr int SB = -SF;
    const unsigned k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * g.st) return;
    Spinor<R> s;
    Half<R> h;
    if (k < g.st) {
        SpinorIO<P>::load(in, g.vh, k, s);
        project<0, SF>(s, h);
        FaceIO<R>::store(lower, g.st, k, h);
    } else {
        const unsigned j = k - g.st, i = unsigned(g.lt - 1) * g.st + j;
        SpinorIO<P>::load(in, g.vh, i, s);
        project<0, SB>(s, h);
        Link<R> u;
        Half<R> r;
        L::load(links + size_t(4 * q + 0) * L::NCHUNK * g.vh, g.vh, i, u);   // U_0 of site i, towards the next slab
        link_mul<true>(u, h, r);
        FaceIO<R>::store(upper, g.st, j, r);
    }
}

// The interior output sites st <= i < (Lt-1) st: every neighbour is local.
template <int P, int RECON, bool DAG, bool HASX>
__global__ void __launch_bounds__(128, TM_HOP_MINB(P))
    k_slab_interior(Geom g, int p, const typename LinkIO<P, RECON>::V *__restrict__ links, const void *__restrict__ in,
                    void *__restrict__ out, const void *__restrict__ x, Coef k)
{
    using R = typename SpinorIO<P>::R;
    const unsigned i = g.st + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= unsigned(g.lt - 1) * g.st) return;
    Spinor<R> acc, o;
    hop_site<P, RECON, DAG>(g, p, i, links, in, acc);
    if (HASX) {
        Spinor<R> xs;
        SpinorIO<P>::load(x, g.vh, i, xs);
        epilogue(k, acc, &xs, o);
    } else {
        epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
    }
    SpinorIO<P>::store(out, g.vh, i, o);
}

// The face output sites (t = 0 and t = Lt-1; all sites when Lt = 2): the
// spatial hops and the t hops that stay in the slab as in the interior, the
// t hops through a face from the received faces, with the face's sign.
template <int P, int RECON, bool DAG, bool HASX>
__global__ void __launch_bounds__(128, TM_HOP_MINB(P))
    k_slab_boundary(Geom g, int p, const typename LinkIO<P, RECON>::V *__restrict__ links, const void *__restrict__ in,
                    void *__restrict__ out, const void *__restrict__ x, const void *__restrict__ recv_lower,
                    const void *__restrict__ recv_upper, int neg_lower, int neg_upper, Coef k)
{
    using R = typename SpinorIO<P>::R;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const unsigned kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= 2 * g.st) return;
    const unsigned top = unsigned(g.lt - 1) * g.st;
    const unsigned i = kk < g.st ? kk : top + (kk - g.st);
    Nbrs n;
    neighbours(g, p, i, n);
    GlobalLinks<P, RECON> src{links, g.vh, i, p};
    Spinor<R> acc, o;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = {R(0), R(0)};
    if (n.wf[0]) {   // t = Lt-1: forward neighbour on the next slab's lower face
        Half<R> h, r;
        Link<R> u;
        FaceIO<R>::load(recv_upper, g.st, n.fwd[0], h);   // the wrapped index is the face index
        src.template fwd<0>(n, u);
        link_mul<false>(u, h, r);
        accumulate<0, SF>(r, neg_upper ? R(-1) : R(1), acc);
    } else {
        hop_fwd<P, DAG, 0>(g, n, src, in, acc);
    }
    if (n.wb[0]) {   // t = 0: backward neighbour on the previous slab's upper face, already multiplied
        Half<R> r;
        FaceIO<R>::load(recv_lower, g.st, n.bwd[0] - top, r);
        accumulate<0, SB>(r, neg_lower ? R(-1) : R(1), acc);
    } else {
        hop_bwd<P, DAG, 0>(g, n, src, in, acc);
    }
    hop_dir<P, DAG, 1>(g, n, src, in, acc);
    hop_dir<P, DAG, 2>(g, n, src, in, acc);
    hop_dir<P, DAG, 3>(g, n, src, in, acc);
    if (HASX) {
        Spinor<R> xs;
        SpinorIO<P>::load(x, g.vh, i, xs);
        epilogue(k, acc, &xs, o);
    } else {
        epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
    }
    SpinorIO<P>::store(out, g.vh, i, o);
}

template <int P, int RECON>
cudaError_t slab_pack(const tm_gauge *U, int q, bool dag, const void *in, void *lower, void *upper, cudaStream_t s)
{
    using V = typename LinkIO<P, RECON>::V;
    const unsigned n = 2 * U->geom.st, grid = (n + 127) / 128;
    const V *l = static_cast<const V *>(U->links);
    if (dag) k_slab_pack<P, RECON, true><<<grid, 128, 0, s>>>(U->geom, q, l, in, lower, upper);
    else k_slab_pack<P, RECON, false><<<grid, 128, 0, s>>>(U->geom, q, l, in, lower, upper);
    return cudaGetLastError();
}

template <int P, int RECON, bool DAG>
cudaError_t slab_hop_dag(const tm_gauge *U, int p, void *out, const void *in, const void *x, const void *rl,
                         const void *ru, int neg_l, int neg_u, int region, const Coef &k, cudaStream_t s)
{
    using V = typename LinkIO<P, RECON>::V;
    const Geom &g = U->geom;
    const V *l = static_cast<const V *>(U->links);
    if ((region & TM_SLAB_INTERIOR) && g.lt > 2) {
        const unsigned n = unsigned(g.lt - 2) * g.st, grid = (n + 127) / 128;
        if (x) k_slab_interior<P, RECON, DAG, true><<<grid, 128, 0, s>>>(g, p, l, in, out, x, k);
        else k_slab_interior<P, RECON, DAG, false><<<grid, 128, 0, s>>>(g, p, l, in, out, x, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (region & TM_SLAB_BOUNDARY) {
        const unsigned n = 2 * g.st, grid = (n + 127) / 128;
        if (x) k_slab_boundary<P, RECON, DAG, true><<<grid, 128, 0, s>>>(g, p, l, in, out, x, rl, ru, neg_l, neg_u, k);
        else k_slab_boundary<P, RECON, DAG, false><<<grid, 128, 0, s>>>(g, p, l, in, out, x, rl, ru, neg_l, neg_u, k);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

template <int P, int RECON>
cudaError_t slab_hop(const tm_gauge *U, bool dag, int p, void *out, const void *in, const void *x, const void *rl,
                     const void *ru, int neg_l, int neg_u, int region, const Coef &k, cudaStream_t s)
{
    return dag ? slab_hop_dag<P, RECON, true>(U, p, out, in, x, rl, ru, neg_l, neg_u, region, k, s)
               : slab_hop_dag<P, RECON, false>(U, p, out, in, x, rl, ru, neg_l, neg_u, region, k, s);
}

size_t face_bytes_per_site(int prec) { return prec == F64 ? FaceIO<double>::BYTES_PER_SITE : FaceIO<float>::BYTES_PER_SITE; }

bool slab_supported(const tm_gauge *U) { return U->prec == F64 || U->prec == F32 || U->prec == F16; }

}  // namespace twm

using namespace twm;

extern "C" {

size_t tm_slab_face_bytes(const tm_gauge *U)
{
    if (!U || !slab_supported(U)) return 0;
    return face_bytes_per_site(U->prec) * U->geom.st;
}

tm_status tm_slab_pack(tm_ctx *ctx, const tm_gauge *U, const void *in_dev, int dir, int dagger, void *send_lower_dev,
                       void *send_upper_dev, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(in_dev) || bad_ptr(send_lower_dev) || bad_ptr(send_upper_dev))
        return tm_fail(ctx, TM_ERR_ARG, "tm_slab_pack: null or misaligned pointer");
    if (dir != TM_EO && dir != TM_OE) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_pack: dir must be TM_EO or TM_OE");
    if (!slab_supported(U)) return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_slab_pack: slabs support TM_F64, TM_F32, TM_F16");
    if (send_lower_dev == send_upper_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_pack: the two faces must differ");
    const int q = dir == TM_EO ? 1 : 0;   // parity of the input field
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    const bool dag = dagger != 0;
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: e = slab_pack<F64, 18>(U, q, dag, in_dev, send_lower_dev, send_upper_dev, s); break;
    case F64 * 100 + 12: e = slab_pack<F64, 12>(U, q, dag, in_dev, send_lower_dev, send_upper_dev, s); break;
    case F32 * 100 + 18: e = slab_pack<F32, 18>(U, q, dag, in_dev, send_lower_dev, send_upper_dev, s); break;
    case F32 * 100 + 12: e = slab_pack<F32, 12>(U, q, dag, in_dev, send_lower_dev, send_upper_dev, s); break;
    case F16 * 100 + 12: e = slab_pack<F16, 12>(U, q, dag, in_dev, send_lower_dev, send_upper_dev, s); break;
    default: return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_slab_pack: unsupported storage");
    }
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_slab_pack: ") + cudaGetErrorString(e));
    return TM_OK;
}

tm_status tm_slab_hop(tm_ctx *ctx, const tm_gauge *U, void *out_dev, const void *in_dev, const void *recv_lower_dev,
                      const void *recv_upper_dev, int dir, int dagger, int region, int op, double kappa, double mu,
                      int sign, const void *x_dev, int sign_lower, int sign_upper, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(out_dev) || bad_ptr(in_dev)) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: null or misaligned pointer");
    if (out_dev == in_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: out and in must not overlap");
    if (dir != TM_EO && dir != TM_OE) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: dir must be TM_EO or TM_OE");
    if (region < TM_SLAB_INTERIOR || region > TM_SLAB_ALL) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: bad region");
    if ((region & TM_SLAB_BOUNDARY) && (bad_ptr(recv_lower_dev) || bad_ptr(recv_upper_dev)))
        return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: the face sites need both received faces");
    if ((sign_lower != 1 && sign_lower != -1) || (sign_upper != 1 && sign_upper != -1))
        return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: face signs must be +1 or -1");
    if (!slab_supported(U)) return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_slab_hop: slabs support TM_F64, TM_F32, TM_F16");
    Coef k = coef_plain();
    const void *x = nullptr;
    if (op == TM_SLAB_QTM_A || op == TM_SLAB_QTM_B) {
        if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: sign must be +1 or -1");
        if (dagger) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: the Q_tm stages take dagger = 0 (use sign = -1)");
        const double mut = 2.0 * kappa * mu * sign;
        if (op == TM_SLAB_QTM_A) {
            if (dir != TM_OE) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: TM_SLAB_QTM_A is the odd-output stage (TM_OE)");
            k = coef_qtm_a_scaled(kappa, mut);
        } else {
            if (dir != TM_EO) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: TM_SLAB_QTM_B is the even-output stage (TM_EO)");
            if (bad_ptr(x_dev) || x_dev == out_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: TM_SLAB_QTM_B needs x_dev (the even input)");
            k = coef_qtm_b_unit(mut);
            x = x_dev;
        }
    } else if (op != TM_SLAB_HOP) {
        return tm_fail(ctx, TM_ERR_ARG, "tm_slab_hop: op must be TM_SLAB_HOP, TM_SLAB_QTM_A or TM_SLAB_QTM_B");
    }
    const int p = dir == TM_EO ? 0 : 1;   // parity of the output sites
    const bool dag = dagger != 0;
    const int nl = sign_lower < 0, nu = sign_upper < 0;
    cudaStream_t s = (cudaStream_t)stream;
    const void *rl = recv_lower_dev, *ru = recv_upper_dev;
    cudaError_t e;
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: e = slab_hop<F64, 18>(U, dag, p, out_dev, in_dev, x, rl, ru, nl, nu, region, k, s); break;
    case F64 * 100 + 12: e = slab_hop<F64, 12>(U, dag, p, out_dev, in_dev, x, rl, ru, nl, nu, region, k, s); break;
    case F32 * 100 + 18: e = slab_hop<F32, 18>(U, dag, p, out_dev, in_dev, x, rl, ru, nl, nu, region, k, s); break;
    case F32 * 100 + 12: e = slab_hop<F32, 12>(U, dag, p, out_dev, in_dev, x, rl, ru, nl, nu, region, k, s); break;
    case F16 * 100 + 12: e = slab_hop<F16, 12>(U, dag, p, out_dev, in_dev, x, rl, ru, nl, nu, region, k, s); break;
    default: return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_slab_hop: unsupported storage");
    }
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_slab_hop: ") + cudaGetErrorString(e));
    return TM_OK;
}

}  // extern "C"
