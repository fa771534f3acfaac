"""Pins of the oracle's clover twisted-mass operator (no GPU), against
things other than its own code:

* the field strength recomputed here by walking the four plaquette paths
  of the clover leaf link by link (a path walker, not the oracle's index
  arithmetic), sigma_munu from the gamma matrices typed in the degenerate
  pins, and the clover term T = c_sw kappa i sum_{mu<nu} sigma_munu F_munu
  compared with the oracle's site matrices; T is Hermitian and traceless;
* the dense Schur complement of M_sw = 1 - kappa Dhop + T + i mut gamma5
  with an explicit matrix inverse, on lattices with extent-2 directions;
* c_sw = 0 and the free field (F = 0) reduce to Q_tm;
* gauge covariance and Q_sw(mu)^dag = Q_sw(-mu).
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F
from test_oracle_pins import BC, GAMMA, GAMMA5, dense_dhop, extent, lex_of, parity_sites, rel, site_coords, spin_index


def _step(dims, C, x, mu, s):
    c = C[x].copy()
    c[mu] = (c[mu] + s) % extent(dims, mu)
    return lex_of(dims, c)


def walk(dims, U, C, x, path):
    """Product of links along a closed path of unit steps (mu, +-1) starting at x."""
    W = np.eye(3, dtype=complex)
    y = x
    for mu, s in path:
        if s > 0:
            W = W @ U[mu, y]
            y = _step(dims, C, y, mu, +1)
        else:
            y = _step(dims, C, y, mu, -1)
            W = W @ U[mu, y].conj().T
    assert y == x
    return W


def clover_term(dims, U, csw, kappa, x):
    C = site_coords(dims)
    T = np.zeros((12, 12), dtype=complex)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            leaves = [[(mu, 1), (nu, 1), (mu, -1), (nu, -1)], [(nu, 1), (mu, -1), (nu, -1), (mu, 1)],
                      [(mu, -1), (nu, -1), (mu, 1), (nu, 1)], [(nu, -1), (mu, 1), (nu, 1), (mu, -1)]]
            Q = sum(walk(dims, U, C, x, p) for p in leaves)
            Fmn = (Q - Q.conj().T) / 8
            sig = 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
            T += csw * kappa * 1j * np.kron(sig, Fmn)
    return T


def dense_Qsw(dims, U, kappa, mu, csw, bc=BC):
    V = int(np.prod(dims))
    mut = 2 * kappa * mu
    M = np.eye(12 * V, dtype=complex) - kappa * dense_dhop(dims, U, bc) + \
        1j * mut * np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    for x in range(V):
        M[12 * x:12 * x + 12, 12 * x:12 * x + 12] += clover_term(dims, U, csw, kappa, x)
    ev, od = parity_sites(dims)
    ie, io = spin_index(ev), spin_index(od)
    S = M[np.ix_(ie, ie)] - M[np.ix_(ie, io)] @ np.linalg.inv(M[np.ix_(io, io)]) @ M[np.ix_(io, ie)]
    G5 = np.kron(np.eye(V // 2), np.kron(GAMMA5, np.eye(3)))
    return G5 @ S


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_clover_term_matches_path_walk(dims):
    U = F.gauge_field(dims, 31, "random")
    V = int(np.prod(dims))
    for x in (0, 1, V // 2 + 1, V - 1):
        T = O.clover_site(dims, U, 1.7, 0.15, x)
        assert rel(T, clover_term(dims, U, 1.7, 0.15, x)) < 1e-14
        assert np.abs(T - T.conj().T).max() < 1e-14 * np.abs(T).max()      # Hermitian
        assert abs(np.trace(T)) < 1e-13 * np.abs(T).max()                   # traceless


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_Qsw_matches_dense_schur_complement(dims):
    Vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 32, "random")
    psi = F.gaussian_spinor(Vh, 32, 1)
    Q = dense_Qsw(dims, U, 0.13, 0.02, 1.6)
    assert rel(O.Qsw(dims, U, psi, 0.13, 0.02, 1.6), (Q @ psi.reshape(-1)).reshape(Vh, 4, 3)) < 1e-13


def test_Qsw_reduces_to_Qtm():
    dims = (4, 4, 4, 4)
    U = F.gauge_field(dims, 33, "random")
    psi = F.gaussian_spinor(128, 33, 1)
    assert rel(O.Qsw(dims, U, psi, 0.16, 0.01, 0.0), O.Qtm(dims, U, psi, 0.16, 0.01)) < 1e-15
    one = np.zeros_like(U)
    one[..., 0, 0] = one[..., 1, 1] = one[..., 2, 2] = 1     # free field: F = 0
    assert rel(O.Qsw(dims, one, psi, 0.16, 0.01, 1.9), O.Qtm(dims, one, psi, 0.16, 0.01)) < 1e-15
    # and with a non-trivial field the clover term does act
    assert rel(O.Qsw(dims, U, psi, 0.16, 0.01, 1.9), O.Qtm(dims, U, psi, 0.16, 0.01)) > 1e-3


def test_Qsw_gauge_covariance():
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    U = F.gauge_field(dims, 34, "random")
    Om = F.gauge_field(dims, 35, "random")[0]            # one SU(3) matrix per site
    C = site_coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        for x in range(V):
            Up[mu, x] = Om[x] @ U[mu, x] @ Om[_step(dims, C, x, mu, 1)].conj().T
    ev, _ = parity_sites(dims)
    psi = F.gaussian_spinor(V // 2, 34, 1)
    rot = np.einsum("iab,isb->isa", Om[ev], psi)
    want = np.einsum("iab,isb->isa", Om[ev], O.Qsw(dims, U, psi, 0.14, 0.03, 1.5))
    assert rel(O.Qsw(dims, Up, rot, 0.14, 0.03, 1.5), want) < 1e-13


def test_Qsw_adjoint_is_Qsw_with_minus_mu():
    dims = (4, 4, 4, 4)
    U = F.gauge_field(dims, 36, "near", 0.3)
    chi, psi = F.gaussian_spinor(128, 36, 1), F.gaussian_spinor(128, 36, 2)
    lhs = np.vdot(chi, O.Qsw(dims, U, psi, 0.1394, 0.0015, 1.76))
    rhs = np.vdot(O.Qsw(dims, U, chi, 0.1394, -0.0015, 1.76), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
