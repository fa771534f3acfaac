"""Pins of the FP64 CPU oracle against things other than itself (no GPU).

Every check here comes from mathematics the operator must satisfy, not
from re-running the oracle's own code:

* the Clifford algebra and chirality of the gamma basis;
* a dense matrix of Dhop assembled entry by entry (block Kronecker
  products, a different computation from the oracle's site stencil) on
  lattices with an extent-2 direction, where x+mu and x-mu coincide;
* the dense Schur complement M_ee - M_eo M_oo^-1 M_oe with an explicit
  matrix inverse;
* the free-field plane-wave closed form Dhop = sum_mu (2 cos p_mu - 2 i
  gamma_mu sin p_mu) with antiperiodic time momenta;
* gauge covariance under random SU(3) transforms;
* gamma5 hermiticity and Q(mu)^dag = Q(-mu);
* CG against a dense solve, and the force against finite differences of
  the action computed with dense linear algebra.

The operator definitions are those in the header of oracle/tm_oracle.c
(Wilson twisted mass in hopping-parameter form, chiral gamma basis).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

HERE = os.path.dirname(os.path.abspath(__file__))
BC = (-1, 1, 1, 1)  # antiperiodic in time (direction 0), periodic in space

# ---- the chiral Euclidean basis, typed from its definition -------------------
I2 = np.eye(2)
Z2 = np.zeros((2, 2))
SIGMA = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], complex)]
GAMMA = [np.block([[Z2, -I2], [-I2, Z2]]).astype(complex)] + \
        [np.block([[Z2, -1j * s], [1j * s, Z2]]) for s in SIGMA]
GAMMA5 = np.diag([1, 1, -1, -1]).astype(complex)
I4 = np.eye(4)


# ---- geometry written independently of the oracle ---------------------------
def extent(dims, mu):
    return dims[3] if mu == 0 else dims[mu - 1]


def site_coords(dims):
    """(V, 4) array of (t, x, y, z) for lexicographic sites x-fastest."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return np.stack([t.ravel(), x.ravel(), y.ravel(), z.ravel()], axis=1)


def lex_of(dims, c):
    Lx, Ly, Lz, _ = dims
    return c[1] + Lx * (c[2] + Ly * (c[3] + Lz * c[0]))


def dense_dhop(dims, U, bc=BC):
    """Dhop as a dense (12V x 12V) matrix, block by block."""
    C = site_coords(dims)
    V = C.shape[0]
    D = np.zeros((12 * V, 12 * V), dtype=complex)
    for x in range(V):
        for mu in range(4):
            L = extent(dims, mu)
            for step in (+1, -1):
                c = C[x].copy()
                c[mu] += step
                s = 1.0
                if c[mu] < 0 or c[mu] >= L:
                    s = bc[mu]
                    c[mu] %= L
                y = lex_of(dims, c)
                if step == +1:
                    blk = np.kron(I4 - GAMMA[mu], U[mu, x])
                else:
                    blk = np.kron(I4 + GAMMA[mu], U[mu, y].conj().T)
                D[12 * x:12 * x + 12, 12 * y:12 * y + 12] += s * blk
    return D


def parity_sites(dims):
    C = site_coords(dims)
    par = C.sum(axis=1) % 2
    return np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]


def spin_index(sites):
    return (12 * sites[:, None] + np.arange(12)[None, :]).ravel()


def dense_Qtm(dims, U, kappa, mu, bc=BC):
    """gamma5 (M_ee - M_eo M_oo^-1 M_oe) from the dense full M, rows ordered by lex/2."""
    V = int(np.prod(dims))
    mut = 2 * kappa * mu
    M = np.eye(12 * V) - kappa * dense_dhop(dims, U, bc) + 1j * mut * np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    ev, od = parity_sites(dims)
    # order sites of each parity by their packed index lex//2 (= position in ev/od)
    ie, io = spin_index(ev), spin_index(od)
    Mee, Meo, Moe, Moo = M[np.ix_(ie, ie)], M[np.ix_(ie, io)], M[np.ix_(io, ie)], M[np.ix_(io, io)]
    S = Mee - Meo @ np.linalg.inv(Moo) @ Moe
    G5 = np.kron(np.eye(V // 2), np.kron(GAMMA5, np.eye(3)))
    return G5 @ S


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


# ---- tests -------------------------------------------------------------------
def test_splitmix64_published_outputs():
    lines = [l for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) if not l.startswith("#")]
    want = [int(l, 16) for l in lines if l.strip()]
    got = [int(v) for v in F.splitmix64(0, 0, len(want))]
    assert got == want


def test_generators_are_su3_and_deterministic():
    U = F.random_su3(1000, 5, 1)
    assert np.abs(np.einsum("nab,ncb->nac", U, U.conj()) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    W = F.near_identity_su3(1000, 5, 1, 0.3)
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-14
    # exp(i eps A) with A Hermitian traceless: close to the identity for small eps
    assert 0.8 < np.mean(np.trace(W, axis1=1, axis2=2).real) / 3 < 1.0
    np.testing.assert_array_equal(F.gaussian_spinor(10, 3, 4), F.gaussian_spinor(10, 3, 4))
    # draws do not depend on how the stream is chunked
    a = F.normal(F.stream_seed(1, 2), 0, 100)
    b = np.concatenate([F.normal(F.stream_seed(1, 2), 0, 40), F.normal(F.stream_seed(1, 2), 20, 60)])
    np.testing.assert_array_equal(a, b)


def test_generator_exponential_matches_library_expm():
    """The Cayley-Hamilton series of the link generator against scipy's expm."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    w = F.normal(F.stream_seed(9, 9), 0, 8 * 50).reshape(50, 8)
    X = 1j * 0.3 * np.einsum("na,aij->nij", w, F._LAMBDA) * 0.5
    X[0] *= 4.0   # a large-norm case
    E = F._expm_traceless(X)
    want = np.stack([scipy_linalg.expm(x) for x in X])
    assert np.abs(E - want).max() < 1e-13


def test_gamma_basis_clifford_and_chirality():
    g = O.gammas()
    for m in range(4):
        np.testing.assert_allclose(g[m], GAMMA[m], atol=0)
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            np.testing.assert_allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * I4, atol=1e-15)
    np.testing.assert_allclose(g[0] @ g[1] @ g[2] @ g[3], g[4], atol=1e-15)
    np.testing.assert_allclose(g[4], GAMMA5, atol=1e-15)


def test_dims_validation():
    assert O.check_dims((2, 2, 2, 2))
    assert not O.check_dims((3, 2, 2, 2))
    assert not O.check_dims((2, 2, 2, 0))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 6), (2, 4, 6, 2)])
def test_dhop_matches_dense_matrix(dims):
    V = int(np.prod(dims))
    U = F.gauge_field(dims, 11, "random")
    psi = F.gaussian_spinor(V, 11, 1)
    D = dense_dhop(dims, U)
    want = (D @ psi.reshape(-1)).reshape(V, 4, 3)
    got = O.dhop(dims, U, psi)
    assert rel(got, want) < 1e-14
    # the literal adjoint against the dense conjugate transpose
    got_dag = O.dhop(dims, U, psi, dagger=True)
    want_dag = (D.conj().T @ psi.reshape(-1)).reshape(V, 4, 3)
    assert rel(got_dag, want_dag) < 1e-14
    # D_hop only connects opposite parities
    ev, od = parity_sites(dims)
    ie, io = spin_index(ev), spin_index(od)
    assert np.abs(D[np.ix_(ie, ie)]).max() == 0 and np.abs(D[np.ix_(io, io)]).max() == 0


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 6)])
def test_hopping_eo_and_Qtm_match_dense_schur_complement(dims):
    V = int(np.prod(dims))
    Vh = V // 2
    kappa, mu = 0.16, 0.01
    U = F.gauge_field(dims, 12, "random")
    D = dense_dhop(dims, U)
    ev, od = parity_sites(dims)
    ie, io = spin_index(ev), spin_index(od)
    psi_o = F.gaussian_spinor(Vh, 12, 2)
    psi_e = F.gaussian_spinor(Vh, 12, 3)
    Heo = D[np.ix_(ie, io)]
    Hoe = D[np.ix_(io, ie)]
    assert rel(O.hopping(dims, U, psi_o, 0), (Heo @ psi_o.reshape(-1)).reshape(Vh, 4, 3)) < 1e-14
    assert rel(O.hopping(dims, U, psi_e, 1), (Hoe @ psi_e.reshape(-1)).reshape(Vh, 4, 3)) < 1e-14
    Q = dense_Qtm(dims, U, kappa, mu)
    assert rel(O.Qtm(dims, U, psi_e, kappa, mu), (Q @ psi_e.reshape(-1)).reshape(Vh, 4, 3)) < 1e-13
    assert rel(O.Qtm(dims, U, psi_e, kappa, mu, dagger=True),
               (Q.conj().T @ psi_e.reshape(-1)).reshape(Vh, 4, 3)) < 1e-13


def test_twisted_mass_inverse_is_dense_inverse():
    mut = 2 * 0.1394 * 0.0015
    psi = F.gaussian_spinor(5, 1, 1)
    A = np.kron(I4 + 1j * mut * GAMMA5, np.eye(3))
    want = (np.linalg.inv(A) @ psi.reshape(5, 12).T).T.reshape(5, 4, 3)
    assert rel(O.twist_inv(psi, mut), want) < 1e-15
    assert rel(O.twist(psi, mut), (A @ psi.reshape(5, 12).T).T.reshape(5, 4, 3)) < 1e-15


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 4), (1, 0, 3, 2)), ((8, 6, 4, 8), (3, 1, 2, 5))])
def test_free_field_plane_wave(dims, n):
    """U = 1: Dhop u e^{ipx} = sum_mu (2 cos p_mu - 2i gamma_mu sin p_mu) u e^{ipx}."""
    V = int(np.prod(dims))
    U = F.gauge_field(dims, 0, "unit")
    C = site_coords(dims)
    # n = (n_t, n_x, n_y, n_z); time momentum antiperiodic
    p = np.array([(2 * n[0] + 1) * np.pi / extent(dims, 0)] +
                 [2 * np.pi * n[m] / extent(dims, m) for m in (1, 2, 3)])
    u = F.gaussian_spinor(1, 3, 3)[0]
    phase = np.exp(1j * (C @ p))
    psi = phase[:, None, None] * u[None]
    K = sum(2 * np.cos(p[m]) * I4 - 2j * np.sin(p[m]) * GAMMA[m] for m in range(4))
    Ku = np.einsum("ab,bc->ac", K, u)
    assert rel(O.dhop(dims, U, psi), phase[:, None, None] * Ku[None]) < 1e-13
    # Q_tm on the even-site restriction of the wave, in closed form
    kappa, mu = 0.1394, 0.0015
    mut = 2 * kappa * mu
    ev, _ = parity_sites(dims)
    Tw = I4 + 1j * mut * GAMMA5
    Qp = GAMMA5 @ (Tw - kappa ** 2 * K @ np.linalg.inv(Tw) @ K)
    want = phase[ev][:, None, None] * np.einsum("ab,bc->ac", Qp, u)[None]
    got = O.Qtm(dims, U, O.pack_eo(dims, psi, 0), kappa, mu)
    assert rel(got, want) < 1e-13


def test_gauge_covariance():
    dims = (4, 2, 4, 6)
    V = int(np.prod(dims))
    U = F.gauge_field(dims, 21, "random")
    Om = F.random_su3(V, 21, 99)
    C = site_coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        c = C.copy()
        c[:, mu] = (c[:, mu] + 1) % extent(dims, mu)
        xp = lex_of(dims, c.T)
        Up[mu] = np.einsum("vab,vbc,vdc->vad", Om, U[mu], Om[xp].conj())
    psi = F.gaussian_spinor(V, 21, 5)
    rot = lambda f: np.einsum("vab,vsb->vsa", Om, f)
    assert rel(O.dhop(dims, Up, rot(psi)), rot(O.dhop(dims, U, psi))) < 1e-13
    ev, _ = parity_sites(dims)
    kappa, mu = 0.16, 0.01
    psi_e = O.pack_eo(dims, psi, 0)
    Om_e = Om[ev]
    rot_e = lambda f: np.einsum("vab,vsb->vsa", Om_e, f)
    assert rel(O.Qtm(dims, Up, rot_e(psi_e), kappa, mu), rot_e(O.Qtm(dims, U, psi_e, kappa, mu))) < 1e-13


def test_gamma5_hermiticity_and_Q_dagger_is_Q_minus_mu():
    dims = (4, 4, 2, 6)
    Vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 31, "random")
    chi_e = F.gaussian_spinor(Vh, 31, 1)
    psi_o = F.gaussian_spinor(Vh, 31, 2)
    lhs = np.vdot(chi_e, O.hopping(dims, U, psi_o, 0))
    rhs = np.vdot(O.gamma5(O.hopping(dims, U, O.gamma5(chi_e), 1)), psi_o)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    kappa, mu = 0.1394, 0.0015
    psi_e = F.gaussian_spinor(Vh, 31, 3)
    lhs = np.vdot(chi_e, O.Qtm(dims, U, psi_e, kappa, mu))
    rhs = np.vdot(O.Qtm(dims, U, chi_e, kappa, -mu), psi_e)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    assert rel(O.Qtm(dims, U, chi_e, kappa, mu, dagger=True), O.Qtm(dims, U, chi_e, kappa, -mu)) < 1e-13


def test_special_cases_reduce():
    dims = (4, 2, 2, 4)
    Vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 41, "random")
    psi_e = F.gaussian_spinor(Vh, 41, 1)
    # kappa = 0: Q = gamma5
    assert rel(O.Qtm(dims, U, psi_e, 0.0, 0.3), O.gamma5(psi_e)) < 1e-15
    # mu = 0: plain Wilson Schur complement gamma5 (1 - kappa^2 H_eo H_oe)
    k = 0.12
    want = O.gamma5(psi_e - k * k * O.hopping(dims, U, O.hopping(dims, U, psi_e, 1), 0))
    assert rel(O.Qtm(dims, U, psi_e, k, 0.0), want) < 1e-14
    # linearity
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    chi_e = F.gaussian_spinor(Vh, 41, 2)
    lin = O.Qtm(dims, U, a * psi_e + b * chi_e, 0.15, 0.02)
    assert rel(lin, a * O.Qtm(dims, U, psi_e, 0.15, 0.02) + b * O.Qtm(dims, U, chi_e, 0.15, 0.02)) < 1e-14


def test_cg_matches_dense_solve():
    dims = (2, 2, 2, 4)
    Vh = int(np.prod(dims)) // 2
    kappa, mu = 0.16, 0.01
    U = F.gauge_field(dims, 51, "random")
    b = F.gaussian_spinor(Vh, 51, 1)
    Q = dense_Qtm(dims, U, kappa, mu)
    want = np.linalg.solve(Q.conj().T @ Q, b.reshape(-1)).reshape(Vh, 4, 3)
    x, it, relres, ok = O.cg_QdagQ(dims, U, b, kappa, mu, tol=1e-12, maxiter=1000)
    assert ok and relres <= 1e-12 and it > 0
    assert rel(x, want) < 1e-9


def _dense_action(dims, U, phi, kappa, mu):
    Q = dense_Qtm(dims, U, kappa, mu)
    v = phi.reshape(-1)
    return float(np.real(np.vdot(v, np.linalg.solve(Q.conj().T @ Q, v))))


def _lambda():
    lam = np.zeros((8, 3, 3), complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def _expm3(X):
    w, v = np.linalg.eig(X)
    return v @ np.diag(np.exp(w)) @ np.linalg.inv(v)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_force_matches_finite_differences_of_dense_action(dims):
    V = int(np.prod(dims))
    Vh = V // 2
    kappa, mu = 0.16, 0.05
    U = F.gauge_field(dims, 61, "random")
    phi = F.gaussian_spinor(Vh, 61, 1)
    X, _, _, ok = O.cg_QdagQ(dims, U, phi, kappa, mu, tol=1e-14, maxiter=5000)
    assert ok
    rng = np.random.default_rng(3)
    links = [(int(rng.integers(4)), int(rng.integers(V))) for _ in range(6)] + [(0, V - 1), (0, 0)]
    Fl = O.force(dims, U, X, kappa, mu, links=links)
    lam = _lambda()
    h = 1e-5
    for (m, x), Fx in zip(links, Fl):
        # traceless anti-Hermitian
        assert np.abs(Fx + Fx.conj().T).max() < 1e-12 and abs(np.trace(Fx)) < 1e-12
        for a in range(8):
            T = 0.5j * lam[a]
            Sp, Sm = U.copy(), U.copy()
            Sp[m, x] = _expm3(h * T) @ U[m, x]
            Sm[m, x] = _expm3(-h * T) @ U[m, x]
            fd = (_dense_action(dims, Sp, phi, kappa, mu) - _dense_action(dims, Sm, phi, kappa, mu)) / (2 * h)
            got = float(np.real(-2 * np.trace(T @ Fx)))
            assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (m, x, a, got, fd)


def test_force_gauge_covariance():
    dims = (2, 2, 4, 2)
    V = int(np.prod(dims))
    kappa, mu = 0.15, 0.05
    U = F.gauge_field(dims, 71, "random")
    Om = F.random_su3(V, 71, 98)
    C = site_coords(dims)
    Up = np.empty_like(U)
    for m in range(4):
        c = C.copy()
        c[:, m] = (c[:, m] + 1) % extent(dims, m)
        Up[m] = np.einsum("vab,vbc,vdc->vad", Om, U[m], Om[lex_of(dims, c.T)].conj())
    ev, _ = parity_sites(dims)
    X = F.gaussian_spinor(V // 2, 71, 2)
    Xp = np.einsum("vab,vsb->vsa", Om[ev], X)
    Fa = O.force(dims, U, X, kappa, mu)
    Fb = O.force(dims, Up, Xp, kappa, mu)
    want = np.einsum("vab,mvbc,vdc->mvad", Om, Fa, Om.conj())
    assert rel(Fb, want) < 1e-12
