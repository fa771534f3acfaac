/*
 * tm_oracle.c -- plain FP64 CPU oracle for the even-odd preconditioned
 * Wilson twisted-mass operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code with the CUDA library.
 *
 * The paper (arXiv:1311.4521, Sec. 1-2) names the hopping matrix of the
 * tmLQCD suite ("Dirac matrix inversion for ... Wilson fermions with
 * twisted mass term", with the Frezzotti-Rossi reference) but prints no
 * formula.  This file writes out the textbook operator it refers to, in
 * the hopping-parameter normalisation:
 *
 *   M psi(x)     = psi(x) - kappa * Dhop psi(x) + i mut gamma5 psi(x),
 *                  mut = 2 kappa mu
 *   Dhop psi(x)  = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *   H_eo / H_oe  = Dhop restricted to even <- odd / odd <- even sites
 *   M_ee = M_oo  = 1 + i mut gamma5,  M_eo = -kappa H_eo, M_oe = -kappa H_oe
 *   Q_tm         = gamma5 (M_ee - M_eo M_oo^-1 M_oe)
 *
 * Conventions: direction mu = 0 is time (extent Lt), 1,2,3 are x,y,z.
 * Sites are numbered lex = x + Lx*(y + Ly*(z + Lz*t)).  A hop that wraps
 * around the lattice in direction mu is multiplied by bc[mu] (+1 periodic,
 * -1 antiperiodic).  Even-odd packed fields hold the sites of one parity
 * p = (x+y+z+t) mod 2 at index lex/2.  Gamma matrices are the chiral
 * Euclidean basis gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]
 * (2x2 blocks, s_k Pauli), gamma5 = gamma0 gamma1 gamma2 gamma3.
 *
 * Layouts (double complex, C order):
 *   gauge   U[mu][lex][a][b]
 *   spinor  psi[lex][spin][colour]     (full lattice)
 *           psi[i_eo][spin][colour]    (one parity, i_eo = lex/2)
 *
 * Pinning (tests/test_oracle_pins.py): Clifford relations; a dense matrix
 * assembled entry by entry on a 2^4 lattice and its dense Schur complement;
 * the free-field plane-wave closed form; gauge covariance; gamma5
 * hermiticity; the literal adjoint against the dense conjugate transpose;
 * CG against a dense solve; the force against finite differences of the
 * action; the non-degenerate doublet against its dense Schur complement and
 * its flavour-diagonal (mu_delta = 0) limit; the clover operator against
 * its dense Schur complement with an independently computed field strength,
 * its c_sw = 0 limit, gauge covariance and Q_sw(mu)^dag = Q_sw(-mu).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NSPIN 4
#define NCOL 3
#define SPINOR (NSPIN * NCOL)

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

/* Extent of direction mu for dims = {Lx, Ly, Lz, Lt}. */
static int extent(const int dims[4], int mu) { return mu == 0 ? dims[3] : dims[mu - 1]; }

static long volume(const int dims[4]) { return (long)dims[0] * dims[1] * dims[2] * dims[3]; }

/* Coordinates c[mu] (c[0]=t, c[1]=x, c[2]=y, c[3]=z) of a lexicographic site. */
static void coords(const int dims[4], long lex, int c[4])
{
    c[1] = (int)(lex % dims[0]); lex /= dims[0];
    c[2] = (int)(lex % dims[1]); lex /= dims[1];
    c[3] = (int)(lex % dims[2]); lex /= dims[2];
    c[0] = (int)lex;
}

static long lexindex(const int dims[4], const int c[4])
{
    return c[1] + (long)dims[0] * (c[2] + (long)dims[1] * (c[3] + (long)dims[2] * c[0]));
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* Neighbour x + step*mu (step = +1 or -1); *wrapped says whether it crossed the edge. */
static long neighbour(const int dims[4], long lex, int mu, int step, int *wrapped)
{
    int c[4];
    coords(dims, lex, c);
    int L = extent(dims, mu);
    int v = c[mu] + step;
    *wrapped = (v < 0 || v >= L);
    c[mu] = (v + L) % L;
    return lexindex(dims, c);
}

int oracle_check_dims(const int dims[4])
{
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 2 || (dims[i] & 1)) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Gamma matrices                                                      */
/* ------------------------------------------------------------------ */

static void pauli(int k, cplx s[2][2])
{
    memset(s, 0, sizeof(cplx) * 4);
    if (k == 1) { s[0][1] = 1; s[1][0] = 1; }
    if (k == 2) { s[0][1] = -I; s[1][0] = I; }
    if (k == 3) { s[0][0] = 1; s[1][1] = -1; }
}

/* g[0..3] = gamma_mu, g[4] = gamma5 = gamma0 gamma1 gamma2 gamma3. */
void oracle_gammas(double complex g[5][4][4])
{
    memset(g, 0, sizeof(cplx) * 5 * 16);
    for (int a = 0; a < 2; ++a) {
        g[0][a][a + 2] = -1;
        g[0][a + 2][a] = -1;
    }
    for (int k = 1; k <= 3; ++k) {
        cplx s[2][2];
        pauli(k, s);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                g[k][a][b + 2] = -I * s[a][b];
                g[k][a + 2][b] = I * s[a][b];
            }
    }
    cplx t[4][4], u[4][4];
    memcpy(t, g[0], sizeof t);
    for (int k = 1; k <= 3; ++k) {
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx acc = 0;
                for (int c = 0; c < 4; ++c) acc += t[a][c] * g[k][c][b];
                u[a][b] = acc;
            }
        memcpy(t, u, sizeof t);
    }
    memcpy(g[4], t, sizeof t);
}

static cplx G[5][4][4];
static int gammas_ready = 0;

static void ensure_gammas(void)
{
    if (!gammas_ready) {
        oracle_gammas(G);
        gammas_ready = 1;
    }
}

/* out = (1 + sgn*gamma_mu) in, on one spinor (colour index untouched). */
static void one_pm_gamma(int mu, int sgn, const cplx *in, cplx *out)
{
    for (int a = 0; a < NSPIN; ++a)
        for (int c = 0; c < NCOL; ++c) {
            cplx acc = in[a * NCOL + c];
            for (int b = 0; b < NSPIN; ++b) acc += sgn * G[mu][a][b] * in[b * NCOL + c];
            out[a * NCOL + c] = acc;
        }
}

/* out = W in (colour matrix times every spin component); dag: use W^dagger. */
static void colour_mul(const cplx *W, int dag, const cplx *in, cplx *out)
{
    for (int s = 0; s < NSPIN; ++s)
        for (int a = 0; a < NCOL; ++a) {
            cplx acc = 0;
            for (int b = 0; b < NCOL; ++b) {
                cplx w = dag ? conj(W[b * NCOL + a]) : W[a * NCOL + b];
                acc += w * in[s * NCOL + b];
            }
            out[s * NCOL + a] = acc;
        }
}

/* ------------------------------------------------------------------ */
/* Hopping term on the full lattice                                    */
/* ------------------------------------------------------------------ */

/* Dhop psi at one site, written to out[12]. */
static void dhop_site(const int dims[4], const int bc[4], const cplx *U, const cplx *psi,
                      long x, cplx *out)
{
    long V = volume(dims);
    for (int k = 0; k < SPINOR; ++k) out[k] = 0;
    cplx t1[SPINOR], t2[SPINOR];
    for (int mu = 0; mu < 4; ++mu) {
        int wrap;
        /* forward: (1 - gamma_mu) U_mu(x) psi(x+mu) */
        long xp = neighbour(dims, x, mu, +1, &wrap);
        double s = wrap ? bc[mu] : 1.0;
        colour_mul(U + ((long)mu * V + x) * 9, 0, psi + xp * SPINOR, t1);
        one_pm_gamma(mu, -1, t1, t2);
        for (int k = 0; k < SPINOR; ++k) out[k] += s * t2[k];
        /* backward: (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) */
        long xm = neighbour(dims, x, mu, -1, &wrap);
        s = wrap ? bc[mu] : 1.0;
        colour_mul(U + ((long)mu * V + xm) * 9, 1, psi + xm * SPINOR, t1);
        one_pm_gamma(mu, +1, t1, t2);
        for (int k = 0; k < SPINOR; ++k) out[k] += s * t2[k];
    }
}

/*
 * out = Dhop psi at every site of parity out_parity (0 even, 1 odd, -1 all);
 * other sites of out are set to zero.  Pull form: each output site gathers
 * its eight neighbours, so sites are independent.
 */
void oracle_dhop(const int dims[4], const int bc[4], const double complex *U,
                 const double complex *psi, double complex *out, int out_parity)
{
    ensure_gammas();
    long V = volume(dims);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(dims, x, c);
        if (out_parity >= 0 && parity_of(c) != out_parity) {
            for (int k = 0; k < SPINOR; ++k) out[x * SPINOR + k] = 0;
            continue;
        }
        dhop_site(dims, bc, U, psi, x, out + x * SPINOR);
    }
}

/*
 * out = Dhop^dagger psi, the conjugate transpose of oracle_dhop written out
 * literally: every term block(x <- y) of Dhop is applied transposed and
 * conjugated, block(x <- y)^dagger psi(x), and scattered into out(y).
 * out_parity restricts which output sites are kept (-1: all).  Serial.
 */
void oracle_dhop_dagger(const int dims[4], const int bc[4], const double complex *U,
                        const double complex *psi, double complex *out, int out_parity)
{
    ensure_gammas();
    long V = volume(dims);
    memset(out, 0, sizeof(cplx) * V * SPINOR);
    cplx gd[4][2][4][4];               /* (1 -+ gamma_mu)^dagger */
    for (int mu = 0; mu < 4; ++mu)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx id = a == b ? 1 : 0;
                gd[mu][0][a][b] = conj(id - G[mu][b][a]);
                gd[mu][1][a][b] = conj(id + G[mu][b][a]);
            }
    cplx t1[SPINOR], t2[SPINOR];
    for (long x = 0; x < V; ++x) {
        for (int mu = 0; mu < 4; ++mu) {
            for (int dirn = 0; dirn < 2; ++dirn) {
                int wrap;
                long y = neighbour(dims, x, mu, dirn == 0 ? +1 : -1, &wrap);
                double s = wrap ? bc[mu] : 1.0;
                /* block(x <- y) = s (1 -+ gamma_mu) (x) W with W = U_mu(x) or U_mu(y)^dag */
                for (int a = 0; a < NSPIN; ++a)
                    for (int c = 0; c < NCOL; ++c) {
                        cplx acc = 0;
                        for (int b = 0; b < NSPIN; ++b)
                            acc += gd[mu][dirn][a][b] * psi[x * SPINOR + b * NCOL + c];
                        t1[a * NCOL + c] = acc;
                    }
                if (dirn == 0)
                    colour_mul(U + ((long)mu * V + x) * 9, 1, t1, t2);  /* (U)^dag */
                else
                    colour_mul(U + ((long)mu * V + y) * 9, 0, t1, t2);  /* (U^dag)^dag */
                for (int k = 0; k < SPINOR; ++k) out[y * SPINOR + k] += s * t2[k];
            }
        }
    }
    if (out_parity >= 0)
        for (long y = 0; y < V; ++y) {
            int c[4];
            coords(dims, y, c);
            if (parity_of(c) != out_parity)
                for (int k = 0; k < SPINOR; ++k) out[y * SPINOR + k] = 0;
        }
}

/* ------------------------------------------------------------------ */
/* Even-odd packing                                                    */
/* ------------------------------------------------------------------ */

void oracle_pack_eo(const int dims[4], int parity, const double complex *full, double complex *eo)
{
    long V = volume(dims);
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(dims, x, c);
        if (parity_of(c) == parity) memcpy(eo + (x / 2) * SPINOR, full + x * SPINOR, sizeof(cplx) * SPINOR);
    }
}

/* Writes the parity sites of full from eo and zeroes the other parity. */
void oracle_unpack_eo(const int dims[4], int parity, const double complex *eo, double complex *full)
{
    long V = volume(dims);
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(dims, x, c);
        if (parity_of(c) == parity) memcpy(full + x * SPINOR, eo + (x / 2) * SPINOR, sizeof(cplx) * SPINOR);
        else memset(full + x * SPINOR, 0, sizeof(cplx) * SPINOR);
    }
}

/*
 * H_eo (out_parity 0) or H_oe (out_parity 1) on packed fields: the input
 * field lives on the other parity.  dagger != 0 applies the literal adjoint
 * (Dhop^dagger restricted the same way).
 */
void oracle_hopping(const int dims[4], const int bc[4], const double complex *U, int out_parity,
                    const double complex *in_eo, double complex *out_eo, int dagger)
{
    long V = volume(dims);
    cplx *a = malloc(sizeof(cplx) * V * SPINOR);
    cplx *b = malloc(sizeof(cplx) * V * SPINOR);
    oracle_unpack_eo(dims, 1 - out_parity, in_eo, a);
    if (dagger) oracle_dhop_dagger(dims, bc, U, a, b, out_parity);
    else oracle_dhop(dims, bc, U, a, b, out_parity);
    oracle_pack_eo(dims, out_parity, b, out_eo);
    free(a);
    free(b);
}

/* ------------------------------------------------------------------ */
/* Site-local twisted-mass terms                                        */
/* ------------------------------------------------------------------ */

/* out = gamma5 in for n spinors. */
void oracle_gamma5(long n, const double complex *in, double complex *out)
{
    ensure_gammas();
    for (long i = 0; i < n; ++i)
        for (int a = 0; a < NSPIN; ++a)
            for (int c = 0; c < NCOL; ++c) {
                cplx acc = 0;
                for (int b = 0; b < NSPIN; ++b) acc += G[4][a][b] * in[i * SPINOR + b * NCOL + c];
                out[i * SPINOR + a * NCOL + c] = acc;
            }
}

/* out = (1 + i mut gamma5) in  (M_ee = M_oo). */
void oracle_twist(long n, double mut, const double complex *in, double complex *out)
{
    cplx *g = malloc(sizeof(cplx) * n * SPINOR);
    oracle_gamma5(n, in, g);
    for (long k = 0; k < n * SPINOR; ++k) out[k] = in[k] + I * mut * g[k];
    free(g);
}

/* out = (1 + i mut gamma5)^-1 in = (1 - i mut gamma5) in / (1 + mut^2), since gamma5^2 = 1. */
void oracle_twist_inv(long n, double mut, const double complex *in, double complex *out)
{
    cplx *g = malloc(sizeof(cplx) * n * SPINOR);
    oracle_gamma5(n, in, g);
    for (long k = 0; k < n * SPINOR; ++k) out[k] = (in[k] - I * mut * g[k]) / (1.0 + mut * mut);
    free(g);
}

/* ------------------------------------------------------------------ */
/* Q_tm and its adjoint                                                */
/* ------------------------------------------------------------------ */

/* out_e = Q_tm in_e = gamma5 (M_ee - M_eo M_oo^-1 M_oe) in_e. */
void oracle_Qtm(const int dims[4], const int bc[4], const double complex *U, double kappa, double mu,
                const double complex *in_e, double complex *out_e)
{
    long Vh = volume(dims) / 2;
    double mut = 2.0 * kappa * mu;
    cplx *t_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *u_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *v_e = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *w_e = malloc(sizeof(cplx) * Vh * SPINOR);
    oracle_hopping(dims, bc, U, 1, in_e, t_o, 0);                 /* H_oe in */
    for (long k = 0; k < Vh * SPINOR; ++k) t_o[k] *= -kappa;       /* M_oe in */
    oracle_twist_inv(Vh, mut, t_o, u_o);                           /* M_oo^-1 M_oe in */
    oracle_hopping(dims, bc, U, 0, u_o, v_e, 0);                   /* H_eo ... */
    for (long k = 0; k < Vh * SPINOR; ++k) v_e[k] *= -kappa;       /* M_eo M_oo^-1 M_oe in */
    oracle_twist(Vh, mut, in_e, w_e);                              /* M_ee in */
    for (long k = 0; k < Vh * SPINOR; ++k) w_e[k] -= v_e[k];
    oracle_gamma5(Vh, w_e, out_e);
    free(t_o); free(u_o); free(v_e); free(w_e);
}

/*
 * out_e = Q_tm^dagger in_e written out as the adjoint of the product:
 * Q^dag = (M_ee - M_eo M_oo^-1 M_oe)^dag gamma5
 *       = (M_ee^dag - M_oe^dag (M_oo^-1)^dag M_eo^dag) gamma5,
 * with M_ee^dag = 1 - i mut gamma5, (M_oo^-1)^dag = (1 + i mut gamma5)/(1+mut^2)
 * and H^dag from the literal conjugate transpose of Dhop.
 */
void oracle_Qtm_dagger(const int dims[4], const int bc[4], const double complex *U, double kappa,
                       double mu, const double complex *in_e, double complex *out_e)
{
    long Vh = volume(dims) / 2;
    double mut = 2.0 * kappa * mu;
    cplx *g_e = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *t_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *u_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *v_e = malloc(sizeof(cplx) * Vh * SPINOR);
    oracle_gamma5(Vh, in_e, g_e);
    oracle_hopping(dims, bc, U, 1, g_e, t_o, 1);                   /* (H_eo)^dag maps even -> odd */
    for (long k = 0; k < Vh * SPINOR; ++k) t_o[k] *= -kappa;       /* M_eo^dag */
    oracle_twist_inv(Vh, -mut, t_o, u_o);                          /* (M_oo^-1)^dag */
    oracle_hopping(dims, bc, U, 0, u_o, v_e, 1);                   /* (H_oe)^dag maps odd -> even */
    for (long k = 0; k < Vh * SPINOR; ++k) v_e[k] *= -kappa;       /* M_oe^dag */
    oracle_twist(Vh, -mut, g_e, out_e);                            /* M_ee^dag */
    for (long k = 0; k < Vh * SPINOR; ++k) out_e[k] -= v_e[k];
    free(g_e); free(t_o); free(u_o); free(v_e);
}

/* ------------------------------------------------------------------ */
/* Non-degenerate twisted-mass doublet                                  */
/* ------------------------------------------------------------------ */

/*
 * The mass-non-degenerate twisted doublet (Frezzotti and Rossi's
 * strange-charm doublet, one of the operators of the tmLQCD suite the
 * paper's introduction lists) acts on two flavours (psi_s, psi_c):
 *
 *   M_nd = (1 - kappa Dhop) x 1_f + i mubar gamma5 x tau3 - epsbar 1 x tau1,
 *   mubar = 2 kappa mu_sigma, epsbar = 2 kappa mu_delta,
 *
 * with Dhop acting on each flavour alone.  Even-odd: A = M_ee = M_oo =
 * 1 + i mubar gamma5 tau3 - epsbar tau1 (site-local, spin x flavour),
 * M_eo = -kappa H_eo, M_oe = -kappa H_oe, and
 *
 *   Q_nd = gamma5 (M_ee - M_eo M_oo^-1 M_oe)     on even doublets.
 *
 * Here A is built as an explicit 8x8 matrix (spin x flavour, colour is
 * untouched) and M_oo^-1 is its numerical inverse (Gauss-Jordan with
 * partial pivoting), not a closed form.  Layout of a doublet field: flavour
 * s in one array, c in another, each [i_eo][spin][colour].
 */

/* A = 1 + i mubar gamma5 tau3 - epsbar tau1, index f*4 + spin. */
static void nd_site_matrix(double mubar, double epsbar, cplx A[8][8])
{
    ensure_gammas();
    const double tau1[2][2] = {{0, 1}, {1, 0}}, tau3[2][2] = {{1, 0}, {0, -1}};
    for (int f = 0; f < 2; ++f)
        for (int a = 0; a < 4; ++a)
            for (int g = 0; g < 2; ++g)
                for (int b = 0; b < 4; ++b)
                    A[f * 4 + a][g * 4 + b] = (f == g && a == b ? 1.0 : 0.0) + I * mubar * G[4][a][b] * tau3[f][g] -
                                              epsbar * (a == b ? 1.0 : 0.0) * tau1[f][g];
}

/* B = A^-1 by Gauss-Jordan elimination with partial pivoting; returns 0 if singular. */
static int invert8(cplx A[8][8], cplx B[8][8])
{
    cplx M[8][16];
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 16; ++c) M[r][c] = c < 8 ? A[r][c] : (c - 8 == r ? 1.0 : 0.0);
    for (int c = 0; c < 8; ++c) {
        int piv = c;
        for (int r = c + 1; r < 8; ++r)
            if (cabs(M[r][c]) > cabs(M[piv][c])) piv = r;
        if (cabs(M[piv][c]) < 1e-300) return 0;
        for (int k = 0; k < 16; ++k) {
            cplx t = M[c][k];
            M[c][k] = M[piv][k];
            M[piv][k] = t;
        }
        cplx d = M[c][c];
        for (int k = 0; k < 16; ++k) M[c][k] /= d;
        for (int r = 0; r < 8; ++r) {
            if (r == c) continue;
            cplx f = M[r][c];
            for (int k = 0; k < 16; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) B[r][c] = M[r][c + 8];
    return 1;
}

/* (out_s, out_c) = W (in_s, in_c) at every site for a site-local 8x8 W. */
static void nd_apply(long n, cplx W[8][8], const cplx *in_s, const cplx *in_c, cplx *out_s, cplx *out_c)
{
    for (long i = 0; i < n; ++i)
        for (int col = 0; col < NCOL; ++col)
            for (int fa = 0; fa < 8; ++fa) {
                cplx acc = 0;
                for (int gb = 0; gb < 8; ++gb) {
                    const cplx *src = gb < 4 ? in_s : in_c;
                    acc += W[fa][gb] * src[i * SPINOR + (gb % 4) * NCOL + col];
                }
                cplx *dst = fa < 4 ? out_s : out_c;
                dst[i * SPINOR + (fa % 4) * NCOL + col] = acc;
            }
}

/* (out_s, out_c) = Q_nd (in_s, in_c) on even sites; returns 0 if M_oo is singular. */
int oracle_Qnd(const int dims[4], const int bc[4], const double complex *U, double kappa, double mu_sigma,
               double mu_delta, const double complex *in_s, const double complex *in_c, double complex *out_s,
               double complex *out_c)
{
    long Vh = volume(dims) / 2;
    cplx A[8][8], Ainv[8][8];
    nd_site_matrix(2.0 * kappa * mu_sigma, 2.0 * kappa * mu_delta, A);
    if (!invert8(A, Ainv)) return 0;
    long n = Vh * SPINOR;
    cplx *t[2], *u[2], *v[2], *w[2];
    for (int f = 0; f < 2; ++f) {
        t[f] = malloc(sizeof(cplx) * n);
        u[f] = malloc(sizeof(cplx) * n);
        v[f] = malloc(sizeof(cplx) * n);
        w[f] = malloc(sizeof(cplx) * n);
    }
    const cplx *in[2] = {in_s, in_c};
    for (int f = 0; f < 2; ++f) {
        oracle_hopping(dims, bc, U, 1, in[f], t[f], 0);             /* H_oe in */
        for (long k = 0; k < n; ++k) t[f][k] *= -kappa;              /* M_oe in */
    }
    nd_apply(Vh, Ainv, t[0], t[1], u[0], u[1]);                      /* M_oo^-1 M_oe in */
    for (int f = 0; f < 2; ++f) {
        oracle_hopping(dims, bc, U, 0, u[f], v[f], 0);              /* H_eo ... */
        for (long k = 0; k < n; ++k) v[f][k] *= -kappa;              /* M_eo M_oo^-1 M_oe in */
    }
    nd_apply(Vh, A, in_s, in_c, w[0], w[1]);                         /* M_ee in */
    for (int f = 0; f < 2; ++f)
        for (long k = 0; k < n; ++k) w[f][k] -= v[f][k];
    oracle_gamma5(Vh, w[0], out_s);
    oracle_gamma5(Vh, w[1], out_c);
    for (int f = 0; f < 2; ++f) {
        free(t[f]);
        free(u[f]);
        free(v[f]);
        free(w[f]);
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* Clover (Sheikholeslami-Wohlert) twisted-mass operator                */
/* ------------------------------------------------------------------ */

/*
 * The clover-improved twisted-mass operator of the tmLQCD suite (the
 * paper's introduction lists it among the suite's operators), in the
 * hopping-parameter normalisation:
 *
 *   M_sw  = 1 - kappa Dhop + T + i mut gamma5,
 *   T(x)  = c_sw kappa (i/2) sum_{mu,nu} sigma_munu F_munu(x)
 *         = c_sw kappa i sum_{mu<nu} sigma_munu F_munu(x),
 *   sigma_munu = (i/2) [gamma_mu, gamma_nu],
 *   F_munu(x) = (Q_munu(x) - Q_munu(x)^dag) / 8,
 *   Q_munu(x) = the four plaquettes in the (mu, nu) plane that start and
 *               end at x, each oriented mu before nu (the clover leaf),
 *
 * and Q_sw = gamma5 (A_ee - kappa^2 H_eo A_oo^-1 H_oe) with the site-local
 * A = 1 + T + i mut gamma5 on each parity.  The links enter F periodically
 * (the boundary sign belongs to the fermion hops only).  A_oo^-1 is the
 * numerical inverse of each odd site's 12x12 matrix (Gauss-Jordan).
 */

/* C = op(A) op(B) for 3x3 colour matrices, op = dagger if the flag is set. */
static void m3mul(const cplx *A, int da, const cplx *B, int db, cplx *C)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) {
                cplx x = da ? conj(A[k * 3 + a]) : A[a * 3 + k];
                cplx y = db ? conj(B[b * 3 + k]) : B[k * 3 + b];
                acc += x * y;
            }
            C[a * 3 + b] = acc;
        }
}

/* link U_mu(x) */
static const cplx *link_at(const cplx *U, long V, int mu, long x) { return U + ((long)mu * V + x) * 9; }

/* one plaquette product W = A^a B^b C^c D^d (each flag: dagger) */
static void prod4(const cplx *A, int da, const cplx *B, int db, const cplx *C, int dc, const cplx *D, int dd, cplx *W)
{
    cplx t1[9], t2[9];
    m3mul(A, da, B, db, t1);
    m3mul(t1, 0, C, dc, t2);
    m3mul(t2, 0, D, dd, W);
}

/* Q_munu(x): the clover leaf, sum of the four plaquettes around x. */
static void clover_leaf(const int dims[4], const cplx *U, long x, int mu, int nu, cplx Q[9])
{
    long V = volume(dims);
    int w;
    long xpm = neighbour(dims, x, mu, +1, &w), xmm = neighbour(dims, x, mu, -1, &w);
    long xpn = neighbour(dims, x, nu, +1, &w), xmn = neighbour(dims, x, nu, -1, &w);
    long xmm_pn = neighbour(dims, xmm, nu, +1, &w), xmm_mn = neighbour(dims, xmm, nu, -1, &w);
    long xmn_pm = neighbour(dims, xmn, mu, +1, &w);
    cplx P[9];
    for (int k = 0; k < 9; ++k) Q[k] = 0;
    /* U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    prod4(link_at(U, V, mu, x), 0, link_at(U, V, nu, xpm), 0, link_at(U, V, mu, xpn), 1, link_at(U, V, nu, x), 1, P);
    for (int k = 0; k < 9; ++k) Q[k] += P[k];
    /* U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu) */
    prod4(link_at(U, V, nu, x), 0, link_at(U, V, mu, xmm_pn), 1, link_at(U, V, nu, xmm), 1, link_at(U, V, mu, xmm), 0, P);
    for (int k = 0; k < 9; ++k) Q[k] += P[k];
    /* U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu) */
    prod4(link_at(U, V, mu, xmm), 1, link_at(U, V, nu, xmm_mn), 1, link_at(U, V, mu, xmm_mn), 0, link_at(U, V, nu, xmn), 0, P);
    for (int k = 0; k < 9; ++k) Q[k] += P[k];
    /* U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag */
    prod4(link_at(U, V, nu, xmn), 1, link_at(U, V, mu, xmn), 0, link_at(U, V, nu, xmn_pm), 0, link_at(U, V, mu, x), 1, P);
    for (int k = 0; k < 9; ++k) Q[k] += P[k];
}

/* T(x) = csw kappa i sum_{mu<nu} sigma_munu x F_munu(x) as a 12x12 matrix, index spin*3 + colour. */
void oracle_clover_site(const int dims[4], const double complex *U, double csw, double kappa, long x,
                        double complex *T)
{
    ensure_gammas();
    for (int k = 0; k < 144; ++k) T[k] = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            cplx Q[9], F[9], sig[4][4];
            clover_leaf(dims, U, x, mu, nu, Q);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) F[a * 3 + b] = (Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0;
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) {
                    cplx c = 0;
                    for (int k = 0; k < 4; ++k) c += G[mu][a][k] * G[nu][k][b] - G[nu][a][k] * G[mu][k][b];
                    sig[a][b] = 0.5 * I * c;
                }
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b)
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) T[(a * 3 + i) * 12 + b * 3 + j] += csw * kappa * I * sig[a][b] * F[i * 3 + j];
        }
}

/* B = A^-1 for an n x n matrix (n <= 12), Gauss-Jordan with partial pivoting; 0 if singular. */
static int invert_n(int n, const cplx *A, cplx *B)
{
    cplx M[12][24];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) M[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(M[r][c]) > cabs(M[piv][c])) piv = r;
        if (cabs(M[piv][c]) < 1e-300) return 0;
        for (int k = 0; k < 2 * n; ++k) {
            cplx t = M[c][k];
            M[c][k] = M[piv][k];
            M[piv][k] = t;
        }
        cplx d = M[c][c];
        for (int k = 0; k < 2 * n; ++k) M[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            cplx f = M[r][c];
            for (int k = 0; k < 2 * n; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) B[r * n + c] = M[r][c + n];
    return 1;
}

/* A(x) = 1 + T(x) + i mut gamma5 at every site of parity p, or its inverse (inv);
 * out[i] is the 12x12 matrix of the site with even-odd index i.  Returns 0 if singular. */
static int sw_site_matrices(const int dims[4], const cplx *U, double kappa, double mu, double csw, int p, int inv,
                            cplx *out)
{
    ensure_gammas();
    long V = volume(dims);
    double mut = 2.0 * kappa * mu;
    cplx T[144], A[144];
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(dims, x, c);
        if (parity_of(c) != p) continue;
        oracle_clover_site(dims, U, csw, kappa, x, T);
        for (int r = 0; r < 12; ++r)
            for (int q = 0; q < 12; ++q)
                A[r * 12 + q] = T[r * 12 + q] + (r == q ? 1.0 : 0.0) +
                                ((r % 3) == (q % 3) ? I * mut * G[4][r / 3][q / 3] : 0.0);
        cplx *dst = out + (x / 2) * 144;
        if (inv) {
            if (!invert_n(12, A, dst)) return 0;
        } else {
            for (int k = 0; k < 144; ++k) dst[k] = A[k];
        }
    }
    return 1;
}

static void site_matvec(long n, const cplx *M, const cplx *in, cplx *out)
{
    for (long i = 0; i < n; ++i)
        for (int r = 0; r < 12; ++r) {
            cplx acc = 0;
            for (int q = 0; q < 12; ++q) acc += M[i * 144 + r * 12 + q] * in[i * SPINOR + q];
            out[i * SPINOR + r] = acc;
        }
}

/* out_e = Q_sw in_e = gamma5 (A_ee - kappa^2 H_eo A_oo^-1 H_oe) in_e; returns 0 if A_oo is singular. */
int oracle_Qsw(const int dims[4], const int bc[4], const double complex *U, double kappa, double mu, double csw,
               const double complex *in_e, double complex *out_e)
{
    long Vh = volume(dims) / 2, n = Vh * SPINOR;
    cplx *Ae = malloc(sizeof(cplx) * Vh * 144), *Aoi = malloc(sizeof(cplx) * Vh * 144);
    cplx *t = malloc(sizeof(cplx) * n), *u = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n),
         *w = malloc(sizeof(cplx) * n);
    int ok = sw_site_matrices(dims, U, kappa, mu, csw, 0, 0, Ae) && sw_site_matrices(dims, U, kappa, mu, csw, 1, 1, Aoi);
    if (ok) {
        oracle_hopping(dims, bc, U, 1, in_e, t, 0);              /* H_oe in */
        for (long k = 0; k < n; ++k) t[k] *= -kappa;              /* M_oe in */
        site_matvec(Vh, Aoi, t, u);                               /* A_oo^-1 M_oe in */
        oracle_hopping(dims, bc, U, 0, u, v, 0);                  /* H_eo ... */
        for (long k = 0; k < n; ++k) v[k] *= -kappa;              /* M_eo A_oo^-1 M_oe in */
        site_matvec(Vh, Ae, in_e, w);                             /* A_ee in */
        for (long k = 0; k < n; ++k) w[k] -= v[k];
        oracle_gamma5(Vh, w, out_e);
    }
    free(Ae); free(Aoi); free(t); free(u); free(v); free(w);
    return ok;
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient on Q^dagger Q                                    */
/* ------------------------------------------------------------------ */

static double re_dot(long n, const cplx *a, const cplx *b)
{
    double s = 0;
    for (long k = 0; k < n; ++k) s += creal(conj(a[k]) * b[k]);
    return s;
}

static void QdagQ(const int dims[4], const int bc[4], const cplx *U, double kappa, double mu,
                  const cplx *in, cplx *tmp, cplx *out)
{
    oracle_Qtm(dims, bc, U, kappa, mu, in, tmp);
    oracle_Qtm_dagger(dims, bc, U, kappa, mu, tmp, out);
}

/*
 * Solves Q^dag Q x = b on even sites by textbook conjugate gradients
 * (Hestenes-Stiefel), starting from the x passed in.  Stops when the
 * recursive residual reaches tol*|b|, then recomputes the true residual
 * |b - Q^dag Q x| / |b| in FP64 and continues if that is still above tol.
 * Returns 0 on convergence, 1 if maxiter was reached.
 */
int oracle_cg_QdagQ(const int dims[4], const int bc[4], const double complex *U, double kappa,
                    double mu, const double complex *b, double complex *x, double tol, int maxiter,
                    int *iters, double *true_relres)
{
    long n = volume(dims) / 2 * SPINOR;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *Ap = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
    double bb = re_dot(n, b, b);
    int it = 0, status = 1;
    for (;;) {
        QdagQ(dims, bc, U, kappa, mu, x, tmp, Ap);
        for (long k = 0; k < n; ++k) r[k] = b[k] - Ap[k];
        double rr = re_dot(n, r, r);
        if (sqrt(rr / bb) <= tol) { status = 0; break; }
        if (it >= maxiter) break;
        memcpy(p, r, sizeof(cplx) * n);
        while (it < maxiter) {
            QdagQ(dims, bc, U, kappa, mu, p, tmp, Ap);
            double alpha = rr / re_dot(n, p, Ap);
            for (long k = 0; k < n; ++k) {
                x[k] += alpha * p[k];
                r[k] -= alpha * Ap[k];
            }
            double rr_new = re_dot(n, r, r);
            ++it;
            if (sqrt(rr_new / bb) <= tol) break;
            double beta = rr_new / rr;
            rr = rr_new;
            for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        }
    }
    QdagQ(dims, bc, U, kappa, mu, x, tmp, Ap);
    for (long k = 0; k < n; ++k) r[k] = b[k] - Ap[k];
    *true_relres = sqrt(re_dot(n, r, r) / bb);
    *iters = it;
    free(r); free(p); free(Ap); free(tmp);
    return status;
}

/* ------------------------------------------------------------------ */
/* Fermion force                                                        */
/* ------------------------------------------------------------------ */

/* Gell-Mann matrices lambda_1..lambda_8. */
static void gellmann(int a, cplx l[3][3])
{
    memset(l, 0, sizeof(cplx) * 9);
    switch (a) {
    case 0: l[0][1] = 1; l[1][0] = 1; break;
    case 1: l[0][1] = -I; l[1][0] = I; break;
    case 2: l[0][0] = 1; l[1][1] = -1; break;
    case 3: l[0][2] = 1; l[2][0] = 1; break;
    case 4: l[0][2] = -I; l[2][0] = I; break;
    case 5: l[1][2] = 1; l[2][1] = 1; break;
    case 6: l[1][2] = -I; l[2][1] = I; break;
    case 7: l[0][0] = 1 / sqrt(3.0); l[1][1] = 1 / sqrt(3.0); l[2][2] = -2 / sqrt(3.0); break;
    }
}

/*
 * Derivative of Dhop R along the link direction dU = T U_mu(x): only the
 * two terms that contain U_mu(x) change,
 *   (dDhop R)(x)    = s (1 - gamma_mu) dU       R(x+mu)
 *   (dDhop R)(x+mu) = s (1 + gamma_mu) dU^dag   R(x)
 * The two output spinors are written to at_x and at_xp.
 */
static void ddhop_link(const int dims[4], const int bc[4], const cplx *dU, int mu, long x,
                       const cplx *R, cplx *at_x, cplx *at_xp, long *xp_out)
{
    int wrap;
    long xp = neighbour(dims, x, mu, +1, &wrap);
    double s = wrap ? bc[mu] : 1.0;
    cplx t1[SPINOR];
    colour_mul(dU, 0, R + xp * SPINOR, t1);
    one_pm_gamma(mu, -1, t1, at_x);
    colour_mul(dU, 1, R + x * SPINOR, t1);
    one_pm_gamma(mu, +1, t1, at_xp);
    for (int k = 0; k < SPINOR; ++k) { at_x[k] *= s; at_xp[k] *= s; }
    *xp_out = xp;
}

static cplx sdot(const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (int k = 0; k < SPINOR; ++k) s += conj(a[k]) * b[k];
    return s;
}

/*
 * Force of S = phi^dag (Q^dag Q)^-1 phi on the links listed, given the
 * solution X = (Q^dag Q)^-1 phi (even sites).  For the link U_mu(x) and a
 * generator T_a = i lambda_a / 2 the perturbation U -> exp(eps T_a) U gives
 *   dS/deps = -X^dag d(Q^dag Q) X = -2 Re( Y^dag dQ X ),   Y = Q X,
 *   dQ = -kappa^2 gamma5 ( dH_eo M_oo^-1 H_oe + H_eo M_oo^-1 dH_oe ),
 * evaluated here term by term with dH from the local derivative of Dhop
 * and H_eo applied at the handful of sites where M_oo^-1 dH_oe X is not
 * zero.  The force is F = sum_a (dS/deps_a) T_a, which is the su(3)
 * element with <T_a, F> = dS/deps_a for <A,B> = -2 tr(AB).
 *
 * links: nlinks pairs (mu, lex); F: nlinks x 3 x 3 complex.
 */
void oracle_force(const int dims[4], const int bc[4], const double complex *U, double kappa, double mu,
                  const double complex *X_e, int nlinks, const int *links, double complex *F)
{
    ensure_gammas();
    long V = volume(dims), Vh = V / 2;
    double mut = 2.0 * kappa * mu;
    cplx *Y_e = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *t_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *Z_o = malloc(sizeof(cplx) * Vh * SPINOR);
    cplx *X = malloc(sizeof(cplx) * V * SPINOR);    /* X on even sites, full lattice */
    cplx *Z = malloc(sizeof(cplx) * V * SPINOR);    /* M_oo^-1 H_oe X on odd sites, full lattice */
    cplx *g5Y = malloc(sizeof(cplx) * V * SPINOR);  /* gamma5 Y on even sites, full lattice */
    cplx *w = calloc(V * SPINOR, sizeof(cplx));     /* sparse scratch field */
    oracle_Qtm(dims, bc, U, kappa, mu, X_e, Y_e);
    oracle_hopping(dims, bc, U, 1, X_e, t_o, 0);
    oracle_twist_inv(Vh, mut, t_o, Z_o);
    oracle_unpack_eo(dims, 0, X_e, X);
    oracle_unpack_eo(dims, 1, Z_o, Z);
    oracle_gamma5(Vh, Y_e, t_o);  /* reuse t_o as gamma5 Y (even) */
    oracle_unpack_eo(dims, 0, t_o, g5Y);

    for (int l = 0; l < nlinks; ++l) {
        int mu_l = links[2 * l];
        long x = links[2 * l + 1];
        const cplx *Ul = U + ((long)mu_l * V + x) * 9;
        int cx[4];
        coords(dims, x, cx);
        int x_even = parity_of(cx) == 0;
        cplx Fl[9] = {0};
        for (int a = 0; a < 8; ++a) {
            cplx lam[3][3], dU[9];
            gellmann(a, lam);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx acc = 0;
                    for (int k = 0; k < 3; ++k) acc += 0.5 * I * lam[i][k] * Ul[k * 3 + j];
                    dU[i * 3 + j] = acc;
                }
            cplx at_x[SPINOR], at_xp[SPINOR];
            long xp;
            /* term 1: (gamma5 Y)^dag dH_eo Z -- the even end of the link gets the odd neighbour's Z */
            ddhop_link(dims, bc, dU, mu_l, x, Z, at_x, at_xp, &xp);
            cplx term1 = x_even ? sdot(g5Y + x * SPINOR, at_x) : sdot(g5Y + xp * SPINOR, at_xp);
            /* term 2: (gamma5 Y)^dag H_eo M_oo^-1 dH_oe X -- dH_oe X lives on the odd end */
            ddhop_link(dims, bc, dU, mu_l, x, X, at_x, at_xp, &xp);
            long yodd = x_even ? xp : x;
            cplx *dv = x_even ? at_xp : at_x;
            oracle_twist_inv(1, mut, dv, w + yodd * SPINOR);
            /* H_eo w is non-zero only at the distinct even neighbours of yodd
             * (on an extent-2 direction x+nu and x-nu coincide: count it once) */
            long nb[8];
            int nnb = 0;
            for (int nu = 0; nu < 4; ++nu)
                for (int step = -1; step <= 1; step += 2) {
                    int wrap, seen = 0;
                    long ze = neighbour(dims, yodd, nu, step, &wrap);
                    for (int q = 0; q < nnb; ++q) seen |= nb[q] == ze;
                    if (!seen) nb[nnb++] = ze;
                }
            cplx term2 = 0;
            for (int q = 0; q < nnb; ++q) {
                cplx h[SPINOR];
                dhop_site(dims, bc, U, w, nb[q], h);
                term2 += sdot(g5Y + nb[q] * SPINOR, h);
            }
            memset(w + yodd * SPINOR, 0, sizeof(cplx) * SPINOR);
            double dS = 2.0 * kappa * kappa * creal(term1 + term2);  /* -2 Re(-kappa^2 (...)) */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Fl[i * 3 + j] += dS * 0.5 * I * lam[i][j];
        }
        memcpy(F + (long)l * 9, Fl, sizeof Fl);
    }
    free(Y_e); free(t_o); free(Z_o); free(X); free(Z); free(g5Y); free(w);
}
