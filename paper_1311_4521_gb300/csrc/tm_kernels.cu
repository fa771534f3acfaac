// tm_kernels.cu -- hopping-matrix kernels with fused twisted-mass epilogues,
// and the layout conversions between the canonical complex-double layouts
// and the packed component-major storage.
#include "tm_internal.h"

namespace twm {

bool make_geom(const int dims[4], const int bc[4], Geom &g)
{
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2 || (dims[d] & 1)) return false;
    double V = double(dims[0]) * dims[1] * dims[2] * dims[3];
    if (V >= 2147483648.0) return false;
    g.lx = dims[0];
    g.ly = dims[1];
    g.lz = dims[2];
    g.lt = dims[3];
    g.hx = dims[0] / 2;
    g.vh = unsigned(V / 2);
    g.sy = unsigned(g.hx);
    g.sz = g.sy * unsigned(g.ly);
    g.st = g.sz * unsigned(g.lz);
    for (int m = 0; m < 4; ++m) g.anti[m] = bc ? (bc[m] < 0) : 0;
    geom_set_divisors(g);
    return true;
}

Coef coef_plain() { return Coef{1, 0, 1, 0, 0, 0, 0, 0}; }

Coef coef_qtm_a(double mut)
{
    double d = 1.0 / (1.0 + mut * mut);
    // (1 - i mut) / (1 + mut^2) on spins 0,1 and (1 + i mut) / (1 + mut^2) on spins 2,3
    return Coef{d, -mut * d, d, mut * d, 0, 0, 0, 0};
}

Coef coef_qtm_b(double kappa, double mut)
{
    double k2 = kappa * kappa;
    // upper: -k2 hop + (1 + i mut) x ; lower: -( -k2 hop + (1 - i mut) x )
    return Coef{-k2, 0, k2, 0, 1.0, mut, -1.0, mut};
}

// The same pair with -kappa^2 moved into the first launch: it writes
// -kappa^2 M_oo^-1 H_oe x, and the second launch adds the hop of that with
// the coefficients +1 (upper) and -1 (lower), a sign instead of a multiply.
Coef coef_qtm_a_scaled(double kappa, double mut)
{
    double d = -kappa * kappa / (1.0 + mut * mut);
    return Coef{d, -mut * d, d, mut * d, 0, 0, 0, 0};
}

Coef coef_qtm_b_unit(double mut)
{
    Coef c{1.0, 0, -1.0, 0, 1.0, mut, -1.0, mut};
    c.unit = 1;
    return c;
}

// ------------------------------------------------------------------ hop
template <int P, int RECON, bool DAG, bool HASX>
__global__ void __launch_bounds__(128, TM_HOP_MINB(P)) k_hop(Geom g, int p, const typename LinkIO<P, RECON>::V *__restrict__ links,
                                             const void *__restrict__ in, void *__restrict__ out,
                                             const void *__restrict__ x, Coef k, SiteMap m)
{
    using R = typename SpinorIO<P>::R;
    const unsigned i = map_site(g, m, blockIdx.x, threadIdx.x);
    if (i >= g.vh) return;
    Spinor<R> acc, o;
    hop_site<P, RECON, DAG>(g, p, i, links, in, acc);
    if (HASX) {
        Spinor<R> xs;
        if constexpr (P == F16) {   // the re-read input's site norm folded into its coefficients
            const R xn = SpinorIO<P>::load_raw(x, g.vh, i, xs);
            epilogue(k, acc, &xs, o, xn);
        } else {
            SpinorIO<P>::load(x, g.vh, i, xs);
            epilogue(k, acc, &xs, o);
        }
    } else {
        epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
    }
    SpinorIO<P>::store(out, g.vh, i, o);
}

// The two Q_tm launches of tm_Qtm_host for FP64 handles, on the caller's
// canonical layout: launch A (PI = F64C) gathers its input from it, launch B
// re-reads it as x (PX = F64C) and writes its result in it (PO = F64C); the
// odd temporary between them stays component-major.  The per-site
// arithmetic is the hop's, so results equal tm_Qtm's on packed fields.
template <int PI, int PX, int PO, int RECON, bool HASX>
__global__ void __launch_bounds__(128, TM_HOP_MINB(F64))
    k_hop_io(Geom g, int p, const typename LinkIO<F64, RECON>::V *__restrict__ links, const void *__restrict__ in,
             void *__restrict__ out, const void *__restrict__ x, Coef k, SiteMap m)
{
    const unsigned i = map_site(g, m, blockIdx.x, threadIdx.x);
    if (i >= g.vh) return;
    Nbrs n;
    neighbours(g, p, i, n);
    GlobalLinks<F64, RECON> src{links, g.vh, i, p};
    Spinor<double> acc, o;
    hop_site_src<PI, false>(g, n, src, in, acc);
    if (HASX) {
        Spinor<double> xs;
        SpinorIO<PX>::load(x, g.vh, i, xs);
        epilogue(k, acc, &xs, o);
    } else {
        epilogue(k, acc, static_cast<const Spinor<double> *>(nullptr), o);
    }
    SpinorIO<PO>::store(out, g.vh, i, o);
}

template <int RECON>
static cudaError_t qtm_canonical(bool stage_b, const Geom &g, const SiteMap &m, const void *links,
                                 const double *in_can, void *tmp, double *out_can, const Coef &k, cudaStream_t s)
{
    using V = typename LinkIO<F64, RECON>::V;
    const V *l = static_cast<const V *>(links);
    const unsigned grid = map_grid(g, m);
    if (!stage_b) k_hop_io<F64C, F64, F64, RECON, false><<<grid, m.block, 0, s>>>(g, 1, l, in_can, tmp, nullptr, k, m);
    else k_hop_io<F64, F64C, F64C, RECON, true><<<grid, m.block, 0, s>>>(g, 0, l, tmp, out_can, in_can, k, m);
    return cudaGetLastError();
}

cudaError_t launch_qtm_canonical(bool stage_b, const Geom &g, int recon, const SiteMap &m, const void *links,
                                 const double *in_can, void *tmp, double *out_can, const Coef &k, cudaStream_t s)
{
    if (g.vh == 0) return cudaSuccess;
    if (recon == 18) return qtm_canonical<18>(stage_b, g, m, links, in_can, tmp, out_can, k, s);
    if (recon == 12) return qtm_canonical<12>(stage_b, g, m, links, in_can, tmp, out_can, k, s);
    return cudaErrorInvalidValue;
}

template <int P, int RECON>
static cudaError_t hop_dispatch(const Geom &g, bool dag, int p, const void *links, const void *in, void *out,
                                const void *x, const Coef &k, cudaStream_t s, const SiteMap &m)
{
    using V = typename LinkIO<P, RECON>::V;
    const V *l = static_cast<const V *>(links);
    const unsigned grid = map_grid(g, m);
    auto kern = dag ? (x ? k_hop<P, RECON, true, true> : k_hop<P, RECON, true, false>)
                    : (x ? k_hop<P, RECON, false, true> : k_hop<P, RECON, false, false>);
    kern<<<grid, m.block, 0, s>>>(g, p, l, in, out, x, k, m);
    return cudaGetLastError();
}

cudaError_t launch_hop(const Geom &g, int prec, int recon, bool dag, int out_parity, const void *links,
                       const void *in, void *out, const void *x, const Coef &k, cudaStream_t s, const SiteMap &m)
{
    if (g.vh == 0) return cudaSuccess;
    if (prec == F64 && recon == 18) return hop_dispatch<F64, 18>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F64 && recon == 12) return hop_dispatch<F64, 12>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F32 && recon == 18) return hop_dispatch<F32, 18>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F32 && recon == 12) return hop_dispatch<F32, 12>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F16 && recon == 12) return hop_dispatch<F16, 12>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F64X && recon == 18) return hop_dispatch<F64X, 18>(g, dag, out_parity, links, in, out, x, k, s, m);
    if (prec == F64X && recon == 12) return hop_dispatch<F64X, 12>(g, dag, out_parity, links, in, out, x, k, s, m);
    return cudaErrorInvalidValue;
}

cudaError_t launch_hop(const Geom &g, int prec, int recon, bool dag, int out_parity, const void *links,
                       const void *in, void *out, const void *x, const Coef &k, cudaStream_t s, int block)
{
    return launch_hop(g, prec, recon, dag, out_parity, links, in, out, x, k, s, linear_map(unsigned(block)));
}

// ------------------------------------------------------------------ layouts
int link_nchunk(int prec, int recon)
{
    if (prec == F64 || prec == F64X) return recon == 18 ? 9 : 6;
    if (prec == F32) return recon == 18 ? 9 : 3;
    if (prec == F16 && recon == 12) return 3;
    return 0;
}

size_t link_chunk_bytes(int prec, int recon)
{
    if (prec == F64 || prec == F64X) return 16;
    if (prec == F32) return recon == 18 ? 8 : 16;
    if (prec == F16) return 8;
    return 0;
}

// One thread per (mu, lexicographic site) of the canonical U[mu][lex][3][3].
template <int P, int RECON>
__global__ void k_pack_gauge(Geom g, const double *__restrict__ U, typename LinkIO<P, RECON>::V *links)
{
    unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long V = 2ull * g.vh;
    if (idx >= 4 * V) return;
    int mu = int(idx / V);
    unsigned lex = unsigned(idx % V);
    unsigned x = lex % g.lx, r = lex / g.lx;
    unsigned y = r % g.ly;
    r /= g.ly;
    unsigned z = r % g.lz, t = r / g.lz;
    int p = (x + y + z + t) & 1;
    double m[18];
    for (int k = 0; k < 18; ++k) m[k] = U[idx * 18 + k];
    using L = LinkIO<P, RECON>;
    L::store(links + size_t(4 * p + mu) * L::NCHUNK * g.vh, g.vh, lex >> 1, m);
}

cudaError_t launch_pack_gauge(const Geom &g, int prec, int recon, const double *U, void *links, cudaStream_t s)
{
    unsigned long long n = 8ull * g.vh;
    unsigned grid = unsigned((n + 255) / 256);
#define TM_PACK(P, RC)                                                                                   \
    if (prec == P && recon == RC) {                                                                      \
        k_pack_gauge<P, RC><<<grid, 256, 0, s>>>(g, U, static_cast<typename LinkIO<P, RC>::V *>(links)); \
        return cudaGetLastError();                                                                       \
    }
    TM_PACK(F64, 18)
    TM_PACK(F64, 12)
    TM_PACK(F32, 18)
    TM_PACK(F32, 12)
    TM_PACK(F16, 12)
    TM_PACK(F64X, 18)
    TM_PACK(F64X, 12)
#undef TM_PACK
    return cudaErrorInvalidValue;
}

template <int P>
__global__ void k_pack_spinor(unsigned vh, const double *__restrict__ in, void *out)
{
    using R = typename SpinorIO<P>::R;
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    Spinor<R> s;
    for (int c = 0; c < 12; ++c) s[c / 3][c % 3] = {to_R<R>(in[size_t(i) * 24 + 2 * c]), to_R<R>(in[size_t(i) * 24 + 2 * c + 1])};
    SpinorIO<P>::store(out, vh, i, s);
}

template <int P>
__global__ void k_unpack_spinor(unsigned vh, const void *in, double *__restrict__ out)
{
    using R = typename SpinorIO<P>::R;
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    Spinor<R> s;
    SpinorIO<P>::load(in, vh, i, s);
    for (int c = 0; c < 12; ++c) {
        out[size_t(i) * 24 + 2 * c] = double(s[c / 3][c % 3].re);
        out[size_t(i) * 24 + 2 * c + 1] = double(s[c / 3][c % 3].im);
    }
}

cudaError_t launch_pack_spinor(unsigned vh, int prec, const double *in, void *out, cudaStream_t s)
{
    if (vh == 0) return cudaSuccess;
    unsigned grid = (vh + 127) / 128;
    if (prec == F64) k_pack_spinor<F64><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F64X) k_pack_spinor<F64X><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F32) k_pack_spinor<F32><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F16) k_pack_spinor<F16><<<grid, 128, 0, s>>>(vh, in, out);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_unpack_spinor(unsigned vh, int prec, const void *in, double *out, cudaStream_t s)
{
    if (vh == 0) return cudaSuccess;
    unsigned grid = (vh + 127) / 128;
    if (prec == F64) k_unpack_spinor<F64><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F64X) k_unpack_spinor<F64X><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F32) k_unpack_spinor<F32><<<grid, 128, 0, s>>>(vh, in, out);
    else if (prec == F16) k_unpack_spinor<F16><<<grid, 128, 0, s>>>(vh, in, out);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace twm
