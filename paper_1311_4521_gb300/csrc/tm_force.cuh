// tm_force.cuh -- per-link fermion force of S = phi^dag (Q^dag Q)^-1 phi.
//
// With X = (Q^dag Q)^-1 phi and Y = Q X, a change dU of one link changes the
// action by dS = -2 Re(Y^dag dQ X), and with
// dQ = -kappa^2 gamma5 (dH_eo M_oo^-1 H_oe + H_eo M_oo^-1 dH_oe)
// this is dS = 2 kappa^2 Re(L^dag dDhop R) for the full-lattice fields
//     R = X on even sites,  Z = M_oo^-1 H_oe X on odd sites,
//     L = gamma5 Y on even, B = gamma5 (M_oo^-1)^dag H_oe Y on odd.
// Only the two hops through the link U_mu(x) depend on it, so
//     L^dag dDhop R = s [ tr(dU M1) + tr(dU^dag M2) ],
//     M1 = sum_spin [(1 - gamma_mu) R(x+mu)] L(x)^dag,
//     M2 = sum_spin [(1 + gamma_mu) R(x)]    L(x+mu)^dag,
// s the boundary sign of the hop x -> x+mu.  Since (1 -+ gamma_mu)/2 are
// projectors, each sum is two colour outer products of half-spinors:
// M1 = sum_b h_b k_b^dag with h, k the upper pairs of the (1 - gamma_mu)
// projections of R(x+mu) and L(x); M2 likewise with (1 + gamma_mu) of R(x)
// and L(x+mu).  Hence
//     dS/dU (the gradient w.r.t. the complex entries, dS = Re tr(G^dag dU))
//         G = 2 kappa^2 s (M1^dag + M2),
//     force for U -> exp(eps T) U, T in su(3), <T_a, F> = dS/deps_a with
//     <A,B> = -2 tr(AB):  F = -kappa^2 s TA(U M1 - M2 U^dag),
// TA(W) = (W - W^dag)/2 - tr((W - W^dag)/2)/3 the traceless anti-Hermitian part.
#pragma once

#include "tm_device.cuh"

namespace twm {

template <typename R> using Mat = cpx<R>[3][3];

// m = sum_b a_b k_b^dag (colour outer products of two half-spinors)
template <typename R> TM_HD void outer(const Half<R> &h, const Half<R> &k, Mat<R> &m)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cpx<R> acc = {R(0), R(0)};
#pragma unroll
            for (int b = 0; b < 2; ++b) acc = cmadd(h[b][a], conj(k[b][c]), acc);
            m[a][c] = acc;
        }
}

// out = gamma5 in (spins 2, 3 negated)
template <typename R> TM_HD void apply_g5(Spinor<R> &s)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[2][c] = -s[2][c];
        s[3][c] = -s[3][c];
    }
}

enum { FORCE_SU3 = 0, FORCE_GRAD = 1 };

// The anti-Hermitian part A = W - W^dag of a 3x3 matrix W, kept as its three
// upper off-diagonal entries and the imaginary parts of W's diagonal
// (A_aa = 2 i Im W_aa; A_ca = -conj(A_ac)).  The force needs only this part,
// so W itself is never formed.
template <typename R> struct AntiH {
    cpx<R> off[3];  // A_01, A_02, A_12
    R dg[3];        // Im W_00, Im W_11, Im W_22
};

template <typename R> TM_HD void antih_zero(AntiH<R> &A)
{
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        A.off[q] = {R(0), R(0)};
        A.dg[q] = R(0);
    }
}

// A += SGN * AH(sum_b x_b y_b^dag) for two colour vectors per argument:
// (x y^dag)_ac - conj((x y^dag)_ca) = x_a conj(y_c) - conj(x_c) y_a.
template <int SGN, typename R> TM_HD void antih_outer(const Half<R> &x, const Half<R> &y, AntiH<R> &A)
{
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int a = q == 2 ? 1 : 0, c = q == 0 ? 1 : 2;
        cpx<R> acc = A.off[q];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const cpx<R> xa = x[b][a], xc = x[b][c];
            if (SGN > 0) {
                acc = cjmadd(y[b][c], xa, acc);
                acc = cjmadd(cpx<R>{-xc.re, -xc.im}, y[b][a], acc);
            } else {
                acc = cjmadd(y[b][c], cpx<R>{-xa.re, -xa.im}, acc);
                acc = cjmadd(xc, y[b][a], acc);
            }
        }
        A.off[q] = acc;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R d = A.dg[a];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const cpx<R> xa = x[b][a], ya = y[b][a];
            if (SGN > 0) d = d + xa.im * ya.re - xa.re * ya.im;  // Im(x_a conj(y_a))
            else d = d - xa.im * ya.re + xa.re * ya.im;
        }
        A.dg[a] = d;
    }
}

// out = c TA(W), TA(W) = (W - W^dag)/2 - tr((W - W^dag)/2)/3, from A = AH(W).
// The result is anti-Hermitian exactly (the lower half is the negated
// conjugate of the upper half, the diagonal real parts are zero).
template <typename R> TM_HD void antih_store(const AntiH<R> &A, R c, Mat<R> &out)
{
    const R h = R(0.5) * c;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int a = q == 2 ? 1 : 0, b = q == 0 ? 1 : 2;
        const cpx<R> v = {h * A.off[q].re, h * A.off[q].im};
        out[a][b] = v;
        out[b][a] = {-v.re, v.im};
    }
    const R t = (A.dg[0] + A.dg[1] + A.dg[2]) / R(3);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a][a] = {R(0), c * (A.dg[a] - t)};
}

// Force (mode FORCE_SU3) or complex gradient (FORCE_GRAD) of the link U_mu(x)
// from the fields at its two ends; sgn is the boundary sign of the link.
// SU3: W = U M1 - M2 U^dag = sum_b (U h_b) k_b^dag - h'_b (U k'_b)^dag with
// h, k the (1 - gamma_mu) halves of R(x+mu), L(x) and h', k' the
// (1 + gamma_mu) halves of R(x), L(x+mu): two link-times-half-spinor
// products instead of two 3x3 matrix products.
template <int MU, typename R>
TM_HD void force_link(const Link<R> &u, const Spinor<R> &Rx, const Spinor<R> &Lx, const Spinor<R> &Rxp,
                      const Spinor<R> &Lxp, R kappa2, R sgn, int mode, Mat<R> &out)
{
    Half<R> h, k;
    if (mode == FORCE_GRAD) {
        Mat<R> M1, M2;
        project<MU, -1>(Rxp, h);
        project<MU, -1>(Lx, k);
        outer(h, k, M1);
        project<MU, +1>(Rx, h);
        project<MU, +1>(Lxp, k);
        outer(h, k, M2);
        const R c = R(2) * kappa2 * sgn;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) out[a][b] = c * (conj(M1[b][a]) + M2[a][b]);
        return;
    }
    AntiH<R> A;
    antih_zero(A);
    Half<R> uv;
    project<MU, -1>(Rxp, h);
    link_mul<false>(u, h, uv);
    project<MU, -1>(Lx, k);
    antih_outer<+1>(uv, k, A);
    project<MU, +1>(Lxp, k);
    link_mul<false>(u, k, uv);
    project<MU, +1>(Rx, h);
    antih_outer<-1>(h, uv, A);
    antih_store(A, -kappa2 * sgn, out);  // F = -kappa^2 s TA(W)
}

// The two halves of the link force for the push schemes: the forward part
// (from the hop x -> x+mu, computed at the link's base x from R(x+mu), L(x))
// and the backward part (from the hop x+mu -> x, computed at its tip x+mu
// from R(x), L(x+mu)).  F = fwd + bwd; TA is linear, so
//   FORCE_SU3:  fwd = -kappa^2 s TA(U M1),  bwd = +kappa^2 s TA(M2 U^dag)
//   FORCE_GRAD: fwd = 2 kappa^2 s M1^dag,   bwd = 2 kappa^2 s M2.
template <int MU, typename R>
TM_HD void force_part_fwd(const Link<R> &u, const Spinor<R> &Rxp, const Spinor<R> &Lx, R kappa2, R sgn, int mode,
                          Mat<R> &out)
{
    Half<R> h, k;
    project<MU, -1>(Rxp, h);
    project<MU, -1>(Lx, k);
    if (mode == FORCE_GRAD) {
        Mat<R> M1;
        outer(h, k, M1);
        const R c = R(2) * kappa2 * sgn;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) out[a][b] = c * conj(M1[b][a]);
        return;
    }
    AntiH<R> A;
    antih_zero(A);
    Half<R> uv;
    link_mul<false>(u, h, uv);
    antih_outer<+1>(uv, k, A);
    antih_store(A, -kappa2 * sgn, out);
}

template <int MU, typename R>
TM_HD void force_part_bwd(const Link<R> &u, const Spinor<R> &Rx, const Spinor<R> &Lxp, R kappa2, R sgn, int mode,
                          Mat<R> &out)
{
    Half<R> h, k;
    project<MU, +1>(Rx, h);
    project<MU, +1>(Lxp, k);
    if (mode == FORCE_GRAD) {
        Mat<R> M2;
        outer(h, k, M2);
        const R c = R(2) * kappa2 * sgn;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) out[a][b] = c * M2[a][b];
        return;
    }
    AntiH<R> A;
    antih_zero(A);
    Half<R> uv;
    link_mul<false>(u, k, uv);
    antih_outer<+1>(h, uv, A);
    antih_store(A, kappa2 * sgn, out);
}

// One 3x3 complex matrix to its 144-byte slot of an FP64 force field, one
// 16-byte (re, im) store per entry, evict-first (the field is written once).
template <typename R> TM_HD void store_mat(double *o, const Mat<R> &m)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double2 v = make_double2(double(m[a][b].re), double(m[a][b].im));
            st_stream(reinterpret_cast<double2 *>(o) + 3 * a + b, v);
        }
}

// Lexicographic index of the site with even-odd index i and parity p.
TM_HD unsigned lex_of(const Geom &g, int p, unsigned i)
{
    unsigned r = i / g.hx;
    unsigned y = r % g.ly;
    r /= g.ly;
    unsigned z = r % g.lz, t = r / g.lz;
    return 2 * i + ((y + z + t + p) & 1);
}

// The force of link (mu, x) for x = (p, i).  Even sites hold X and Y (L =
// gamma5 Y), odd sites Z and B.  Writes the 3x3 result to F[mu][lex(x)].
template <int P, int RECON, int MU>
TM_HD void force_site(const Geom &g, int p, unsigned i, const typename LinkIO<P, RECON>::V *links, const void *Xe,
                      const void *Ye, const void *Zo, const void *Bo, double kappa2, int mode, double *F)
{
    using R = typename SpinorIO<P>::R;
    using L = LinkIO<P, RECON>;
    Nbrs n;
    neighbours(g, p, i, n);
    const unsigned j = n.fwd[MU];
    const R sgn = (n.wf[MU] && g.anti[MU]) ? R(-1) : R(1);
    Spinor<R> Rx, Lx, Rxp, Lxp;
    if (p == 0) {
        SpinorIO<P>::load(Xe, g.vh, i, Rx);
        SpinorIO<P>::load(Ye, g.vh, i, Lx);
        apply_g5(Lx);
        SpinorIO<P>::load(Zo, g.vh, j, Rxp);
        SpinorIO<P>::load(Bo, g.vh, j, Lxp);
    } else {
        SpinorIO<P>::load(Zo, g.vh, i, Rx);
        SpinorIO<P>::load(Bo, g.vh, i, Lx);
        SpinorIO<P>::load(Xe, g.vh, j, Rxp);
        SpinorIO<P>::load(Ye, g.vh, j, Lxp);
        apply_g5(Lxp);
    }
    Link<R> u;
    L::load(links + size_t(4 * p + MU) * L::NCHUNK * g.vh, g.vh, i, u);
    Mat<R> m;
    force_link<MU>(u, Rx, Lx, Rxp, Lxp, to_R<R>(kappa2), sgn, mode, m);
    store_mat(F + (size_t(MU) * 2 * g.vh + lex_of(g, p, i)) * 18, m);
}

}  // namespace twm
