// tm_clover.cu -- the clover-improved twisted-mass operator (the
// Sheikholeslami-Wohlert term, one of the operators of the tmLQCD suite
// that the paper's introduction lists):
//
//   M_sw = 1 - kappa Dhop + T + i mut gamma5,
//   T(x) = c_sw kappa i sum_{mu<nu} sigma_munu F_munu(x),
//   sigma_munu = (i/2)[gamma_mu, gamma_nu],  F_munu = (Q_munu - Q_munu^dag)/8,
//   Q_munu(x) = sum of the four plaquettes of the (mu, nu) plane at x,
//   Q_sw = gamma5 (A_ee - kappa^2 H_eo A_oo^-1 H_oe),  A = 1 + T + i mut gamma5.
//
// In the chiral basis sigma_munu is block diagonal (spins 0,1 and 2,3), so A
// is two 6x6 blocks per site (spin within the chirality x colour), with the
// twist i mut on the first and -i mut on the second.  tm_clover_create
// computes F from the links once (one thread per site, FP64) and stores,
// for each sign of mu, the even sites' blocks A and the odd sites' blocks
// -kappa^2 A^-1 (inverted by Gauss-Jordan elimination with partial
// pivoting in FP64), component-major like the spinors.  tm_Qsw then runs
// the two hop launches of Q_tm with the blocks in the epilogues: launch A
// writes t = -kappa^2 A_oo^-1 H_oe psi, launch B gamma5 (A_ee psi + H_eo t).
#include <cmath>
#include <cstring>
#include <string>

#include "tm_internal.h"

struct tm_clover {
    int prec = 0;
    unsigned vh = 0;
    double csw = 0, kappa = 0, mu = 0;
    void *blocks = nullptr;   // [sign +,-][parity][chirality][36 entries][Vh] complex, in prec
    size_t bytes = 0;
};

namespace twm {

// c_sw kappa i s_munu for the 6 planes and 2 chiralities: the 2x2 spin blocks of
// the clover term's plane coefficients (s_munu the chirality blocks of sigma_munu).
struct CloverSpin {
    double re[6][2][2][2], im[6][2][2][2];   // [plane][chirality][a][b]
};

struct C3 {
    cpx<double> m[3][3];
};

__device__ __forceinline__ C3 load_link(const double *U, size_t V, int mu, size_t x, bool dag)
{
    C3 r;
    const double2 *p = reinterpret_cast<const double2 *>(U) + (size_t(mu) * V + x) * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double2 v = p[dag ? b * 3 + a : a * 3 + b];
            r.m[a][b] = {v.x, dag ? -v.y : v.y};
        }
    return r;
}

__device__ __forceinline__ C3 mul(const C3 &A, const C3 &B)
{
    C3 r;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<double> acc = {0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = cmadd(A.m[a][k], B.m[k][b], acc);
            r.m[a][b] = acc;
        }
    return r;
}

__device__ __forceinline__ size_t lex_of4(const Geom &g, const int c[4])
{
    return size_t(c[1]) + size_t(g.lx) * (c[2] + size_t(g.ly) * (c[3] + size_t(g.lz) * c[0]));
}

__device__ __forceinline__ size_t shifted(const Geom &g, const int c0[4], int mu, int smu, int nu, int snu)
{
    int c[4] = {c0[0], c0[1], c0[2], c0[3]};
    const int ext[4] = {g.lt, g.lx, g.ly, g.lz};
    c[mu] = (c[mu] + smu + ext[mu]) % ext[mu];
    c[nu] = (c[nu] + snu + ext[nu]) % ext[nu];
    return lex_of4(g, c);
}

__device__ __forceinline__ void put2(double2 *p, double re, double im) { *p = make_double2(re, im); }
__device__ __forceinline__ void put2(float2 *p, double re, double im) { *p = make_float2(float(re), float(im)); }

// Solves B X = I for a 6x6 complex B in place; returns false if a pivot vanishes.
__device__ bool invert6(cpx<double> (&B)[6][6], cpx<double> (&X)[6][6])
{
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) X[r][c] = {r == c ? 1.0 : 0.0, 0.0};
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = B[c][c].re * B[c][c].re + B[c][c].im * B[c][c].im;
        for (int r = c + 1; r < 6; ++r) {
            const double v = B[r][c].re * B[r][c].re + B[r][c].im * B[r][c].im;
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 1e-200)) return false;
        for (int k = 0; k < 6; ++k) {
            const cpx<double> t = B[c][k];
            B[c][k] = B[piv][k];
            B[piv][k] = t;
            const cpx<double> u = X[c][k];
            X[c][k] = X[piv][k];
            X[piv][k] = u;
        }
        // 1 / pivot
        const cpx<double> p = B[c][c];
        const double n = p.re * p.re + p.im * p.im;
        const cpx<double> inv = {p.re / n, -p.im / n};
        for (int k = 0; k < 6; ++k) {
            B[c][k] = inv * B[c][k];
            X[c][k] = inv * X[c][k];
        }
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const cpx<double> f = B[r][c];
            for (int k = 0; k < 6; ++k) {
                B[r][k] = B[r][k] - f * B[c][k];
                X[r][k] = X[r][k] - f * X[c][k];
            }
        }
    }
    return true;
}

// One thread per lexicographic site: the clover term's two 6x6 blocks from
// the links, then for each sign of mu the stored block (even sites: A;
// odd sites: -kappa^2 A^-1).
template <typename T2>
__global__ void __launch_bounds__(64) k_clover_setup(Geom g, const double *__restrict__ U, CloverSpin cs, double mut,
                                                     double kappa2, T2 *blocks, int *singular)
{
    const size_t V = 2 * size_t(g.vh);
    const size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    if (x >= V) return;
    int c[4];
    {
        size_t r = x;
        c[1] = int(r % g.lx);
        r /= g.lx;
        c[2] = int(r % g.ly);
        r /= g.ly;
        c[3] = int(r % g.lz);
        c[0] = int(r / g.lz);
    }
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const size_t i = x / 2;
    cpx<double> T[2][6][6];
#pragma unroll
    for (int h = 0; h < 2; ++h)
        for (int r = 0; r < 6; ++r)
            for (int q = 0; q < 6; ++q) T[h][r][q] = {0.0, 0.0};
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            const size_t xpm = shifted(g, c, mu, 1, nu, 0), xmm = shifted(g, c, mu, -1, nu, 0);
            const size_t xpn = shifted(g, c, mu, 0, nu, 1), xmn = shifted(g, c, mu, 0, nu, -1);
            const size_t xmm_pn = shifted(g, c, mu, -1, nu, 1), xmm_mn = shifted(g, c, mu, -1, nu, -1);
            const size_t xpm_mn = shifted(g, c, mu, 1, nu, -1);
            // the four plaquettes at x, each oriented mu before nu
            C3 Q = mul(mul(load_link(U, V, mu, x, false), load_link(U, V, nu, xpm, false)),
                       mul(load_link(U, V, mu, xpn, true), load_link(U, V, nu, x, true)));
            C3 P = mul(mul(load_link(U, V, nu, x, false), load_link(U, V, mu, xmm_pn, true)),
                       mul(load_link(U, V, nu, xmm, true), load_link(U, V, mu, xmm, false)));
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + P.m[a][b];
            P = mul(mul(load_link(U, V, mu, xmm, true), load_link(U, V, nu, xmm_mn, true)),
                    mul(load_link(U, V, mu, xmm_mn, false), load_link(U, V, nu, xmn, false)));
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + P.m[a][b];
            P = mul(mul(load_link(U, V, nu, xmn, true), load_link(U, V, mu, xmn, false)),
                    mul(load_link(U, V, nu, xpm_mn, false), load_link(U, V, mu, x, true)));
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + P.m[a][b];
            // F = (Q - Q^dag) / 8, added with the plane's spin coefficients
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const cpx<double> f = {(Q.m[a][b].re - Q.m[b][a].re) * 0.125, (Q.m[a][b].im + Q.m[b][a].im) * 0.125};
                    for (int h = 0; h < 2; ++h)
                        for (int s1 = 0; s1 < 2; ++s1)
                            for (int s2 = 0; s2 < 2; ++s2) {
                                const cpx<double> w = {cs.re[plane][h][s1][s2], cs.im[plane][h][s1][s2]};
                                T[h][s1 * 3 + a][s2 * 3 + b] = cmadd(w, f, T[h][s1 * 3 + a][s2 * 3 + b]);
                            }
                }
        }
    for (int sg = 0; sg < 2; ++sg) {   // sign of mu: +, -
        const double tw = sg == 0 ? mut : -mut;
        for (int h = 0; h < 2; ++h) {
            cpx<double> B[6][6], X[6][6];
            for (int r = 0; r < 6; ++r)
                for (int q = 0; q < 6; ++q) {
                    B[r][q] = T[h][r][q];
                    if (r == q) B[r][q] = {B[r][q].re + 1.0, B[r][q].im + (h == 0 ? tw : -tw)};
                }
            T2 *dst = blocks + ((size_t(sg) * 2 + p) * 2 + h) * 36 * g.vh;
            if (p == 0) {
                for (int k = 0; k < 36; ++k) put2(dst + size_t(k) * g.vh + i, B[k / 6][k % 6].re, B[k / 6][k % 6].im);
            } else {
                if (!invert6(B, X)) {
                    atomicExch(singular, 1);
                    continue;
                }
                for (int k = 0; k < 36; ++k)
                    put2(dst + size_t(k) * g.vh + i, -kappa2 * X[k / 6][k % 6].re, -kappa2 * X[k / 6][k % 6].im);
            }
        }
    }
}

template <typename R> struct BlockIO;
template <> struct BlockIO<double> {
    using T2 = double2;
};
template <> struct BlockIO<float> {
    using T2 = float2;
};

// The two launches of Q_sw.  STAGE_B = false: out = (-kappa^2 A_oo^-1) H_oe in
// on odd sites; true: out = gamma5 (A_ee x + H_eo in) on even sites.
template <int P, int RECON, bool STAGE_B>
__global__ void __launch_bounds__(128, P == F64 ? 2 : 4)
    k_sw(Geom g, const typename LinkIO<P, RECON>::V *__restrict__ links, const void *__restrict__ in,
         void *__restrict__ out, const void *__restrict__ x, const typename BlockIO<typename SpinorIO<P>::R>::T2 *blk)
{
    using R = typename SpinorIO<P>::R;
    const int p = STAGE_B ? 0 : 1;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    Spinor<R> acc, v, o;
    hop_site<P, RECON, false>(g, p, i, links, in, acc);
    if (STAGE_B) SpinorIO<P>::load(x, g.vh, i, v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        cpx<R> w[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) w[r] = STAGE_B ? acc[2 * h + r / 3][r % 3] : cpx<R>{R(0), R(0)};
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const auto e = blk[(size_t(h) * 36 + r * 6 + q) * g.vh + i];
                const cpx<R> src = STAGE_B ? v[2 * h + q / 3][q % 3] : acc[2 * h + q / 3][q % 3];
                w[r] = cmadd(cpx<R>{R(e.x), R(e.y)}, src, w[r]);
            }
#pragma unroll
        for (int r = 0; r < 6; ++r) o[2 * h + r / 3][r % 3] = (STAGE_B && h == 1) ? -w[r] : w[r];   // gamma5 in B
    }
    SpinorIO<P>::store(out, g.vh, i, o);
}

template <int P, int RECON>
cudaError_t sw_launch(const tm_gauge *U, const tm_clover *C, bool stage_b, int sign, const void *in, void *out,
                      const void *x, cudaStream_t s)
{
    using R = typename SpinorIO<P>::R;
    using T2 = typename BlockIO<R>::T2;
    using V = typename LinkIO<P, RECON>::V;
    const Geom &g = U->geom;
    const unsigned grid = (g.vh + 127) / 128;
    const T2 *blk = static_cast<const T2 *>(C->blocks) + ((size_t(sign > 0 ? 0 : 1) * 2 + (stage_b ? 0 : 1)) * 2) * 36 * g.vh;
    const V *l = static_cast<const V *>(U->links);
    if (stage_b) k_sw<P, RECON, true><<<grid, 128, 0, s>>>(g, l, in, out, x, blk);
    else k_sw<P, RECON, false><<<grid, 128, 0, s>>>(g, l, in, out, x, blk);
    return cudaGetLastError();
}

cudaError_t sw_dispatch(const tm_gauge *U, const tm_clover *C, bool stage_b, int sign, const void *in, void *out,
                        const void *x, cudaStream_t s)
{
    if (U->geom.vh == 0) return cudaSuccess;
    switch (U->prec * 100 + U->recon) {
    case F64 * 100 + 18: return sw_launch<F64, 18>(U, C, stage_b, sign, in, out, x, s);
    case F64 * 100 + 12: return sw_launch<F64, 12>(U, C, stage_b, sign, in, out, x, s);
    case F32 * 100 + 18: return sw_launch<F32, 18>(U, C, stage_b, sign, in, out, x, s);
    case F32 * 100 + 12: return sw_launch<F32, 12>(U, C, stage_b, sign, in, out, x, s);
    }
    return cudaErrorInvalidValue;
}

// c_sw kappa i s_munu per plane (mu < nu) and chirality, from the chiral gamma basis.
CloverSpin clover_spin(double csw, double kappa)
{
    typedef cpx<double> z;
    z gm[4][4][4] = {};
    auto set = [&](int mu, int a, int b, z v) { gm[mu][a][b] = v; };
    // gamma_0 = [[0, -1], [-1, 0]]; gamma_k = [[0, -i s_k], [i s_k, 0]]
    set(0, 0, 2, {-1, 0}), set(0, 1, 3, {-1, 0}), set(0, 2, 0, {-1, 0}), set(0, 3, 1, {-1, 0});
    const z s[3][2][2] = {{{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},
                          {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},
                          {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}}};
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const z v = s[k][a][b];
                gm[k + 1][a][2 + b] = {v.im, -v.re};    // -i v
                gm[k + 1][2 + a][b] = {-v.im, v.re};    //  i v
            }
    CloverSpin cs{};
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane)
            for (int h = 0; h < 2; ++h)
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        // sigma = (i/2)[g_mu, g_nu]; coefficient c_sw kappa i sigma = -(c_sw kappa / 2) [g_mu, g_nu]
                        z com = {0, 0};
                        const int A = 2 * h + a, Bi = 2 * h + b;
                        for (int k = 0; k < 4; ++k)
                            com = com + gm[mu][A][k] * gm[nu][k][Bi] - gm[nu][A][k] * gm[mu][k][Bi];
                        cs.re[plane][h][a][b] = -0.5 * csw * kappa * com.re;
                        cs.im[plane][h][a][b] = -0.5 * csw * kappa * com.im;
                    }
    return cs;
}

}  // namespace twm

using namespace twm;

extern "C" {

tm_status tm_clover_create(tm_ctx *ctx, const tm_gauge *U, const double *U_dev, double csw, double kappa, double mu,
                           void *stream, tm_clover **out)
{
    if (!ctx) return TM_ERR_ARG;
    if (!out || !U || bad_ptr(U_dev)) return tm_fail(ctx, TM_ERR_ARG, "tm_clover_create: null or misaligned pointer");
    *out = nullptr;
    if (U->prec != TM_F64 && U->prec != TM_F32)
        return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_clover_create: TM_F64 and TM_F32 handles only");
    const Geom &g = U->geom;
    const size_t es = U->prec == TM_F64 ? sizeof(double2) : sizeof(float2);
    tm_clover *C = new tm_clover;
    C->prec = U->prec;
    C->vh = g.vh;
    C->csw = csw;
    C->kappa = kappa;
    C->mu = mu;
    C->bytes = size_t(2) * 2 * 2 * 36 * g.vh * es;
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&C->blocks, C->bytes);
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess && g.vh > 0) {
        const CloverSpin cs = clover_spin(csw, kappa);
        const unsigned grid = unsigned((2 * size_t(g.vh) + 63) / 64);
        const double mut = 2.0 * kappa * mu;
        if (U->prec == TM_F64)
            k_clover_setup<double2><<<grid, 64, 0, s>>>(g, U_dev, cs, mut, kappa * kappa, static_cast<double2 *>(C->blocks), flag);
        else
            k_clover_setup<float2><<<grid, 64, 0, s>>>(g, U_dev, cs, mut, kappa * kappa, static_cast<float2 *>(C->blocks), flag);
        e = cudaGetLastError();
    }
    int singular = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&singular, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess || singular) {
        if (C->blocks) cudaFree(C->blocks);
        delete C;
        if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_clover_create: ") + cudaGetErrorString(e));
        return tm_fail(ctx, TM_ERR_ARG, "tm_clover_create: a site matrix 1 + T + i mut gamma5 is singular");
    }
    *out = C;
    return TM_OK;
}

void tm_clover_destroy(tm_clover *C)
{
    if (!C) return;
    if (C->blocks) cudaFree(C->blocks);
    delete C;
}

size_t tm_clover_bytes(const tm_clover *C) { return C ? C->bytes : 0; }

tm_status tm_Qsw(tm_ctx *ctx, const tm_gauge *U, const tm_clover *C, void *out_e_dev, const void *in_e_dev, int sign,
                 void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || !C || bad_ptr(out_e_dev) || bad_ptr(in_e_dev)) return tm_fail(ctx, TM_ERR_ARG, "tm_Qsw: null or misaligned pointer");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_Qsw: sign must be +1 or -1");
    if (out_e_dev == in_e_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_Qsw: out and in must not overlap");
    if (C->prec != U->prec || C->vh != U->geom.vh)
        return tm_fail(ctx, TM_ERR_ARG, "tm_Qsw: the clover handle was made for another gauge handle");
    void *tmp = nullptr;
    tm_status st = tm_ctx_scratch(ctx, spinor_bytes(U->geom.vh, U->prec), &tmp);
    if (st != TM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    tm_trace_mark(ctx, 0, s);
    cudaError_t e = sw_dispatch(U, C, false, sign, in_e_dev, tmp, nullptr, s);
    if (e == cudaSuccess) {
        tm_trace_mark(ctx, 1, s);
        e = sw_dispatch(U, C, true, sign, tmp, out_e_dev, in_e_dev, s);
    }
    if (e == cudaSuccess) tm_trace_mark(ctx, 2, s);
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qsw: ") + cudaGetErrorString(e));
    return TM_OK;
}

}  // extern "C"
