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

// Force (mode FORCE_SU3) or complex gradient (FORCE_GRAD) of the link U_mu(x)
// from the fields at its two ends; sgn is the boundary sign of the link.
template <int MU, typename R>
TM_HD void force_link(const Link<R> &u, const Spinor<R> &Rx, const Spinor<R> &Lx, const Spinor<R> &Rxp,
                      const Spinor<R> &Lxp, R kappa2, R sgn, int mode, Mat<R> &out)
{
    Half<R> h, k;
    Mat<R> M1, M2;
    project<MU, -1>(Rxp, h);
    project<MU, -1>(Lx, k);
    outer(h, k, M1);
    project<MU, +1>(Rx, h);
    project<MU, +1>(Lxp, k);
    outer(h, k, M2);
    if (mode == FORCE_GRAD) {
        const R c = R(2) * kappa2 * sgn;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) out[a][b] = c * (conj(M1[b][a]) + M2[a][b]);
        return;
    }
    // W = U M1 - M2 U^dag
    Mat<R> W;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<R> acc = {R(0), R(0)};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc = cmadd(u[a][c], M1[c][b], acc);
                acc = acc - M2[a][c] * conj(u[b][c]);
            }
            W[a][b] = acc;
        }
    // F = -kappa^2 s TA(W)
    const R c = -kappa2 * sgn;
    cpx<R> tr = {R(0), R(0)};
#pragma unroll
    for (int a = 0; a < 3; ++a) tr = tr + R(0.5) * (W[a][a] - conj(W[a][a]));
    const cpx<R> tr3 = {R(0), tr.im / R(3)};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<R> v = R(0.5) * (W[a][b] - conj(W[b][a]));
            if (a == b) v = v - tr3;
            out[a][b] = c * v;
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
    double *o = F + (size_t(MU) * 2 * g.vh + lex_of(g, p, i)) * 18;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            o[6 * a + 2 * b] = double(m[a][b].re);
            o[6 * a + 2 * b + 1] = double(m[a][b].im);
        }
}

}  // namespace twm
