"""Pins of the oracle's non-degenerate twisted doublet (no GPU), against
things other than its own code:

* the dense doublet matrix M_nd = 1_f x (1 - kappa Dhop) + i mubar tau3 x
  gamma5 - epsbar tau1 x 1, built from the dense Dhop of the degenerate
  pins by Kronecker products, and its dense Schur complement with an
  explicit matrix inverse, on lattices with an extent-2 direction;
* the flavour-diagonal limit mu_delta = 0, where the doublet is
  (Q(mu) psi_s, Q(-mu) psi_c) with the pinned degenerate operator;
* Q_nd(mu_sigma, mu_delta)^dag = Q_nd(-mu_sigma, mu_delta) (derived like
  Q(mu)^dag = Q(-mu): gamma5 commutes with the flavour matrices and the
  hops are flavour-diagonal);
* a singular site-local matrix (epsbar^2 = 1 + mubar^2) is refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F
from test_oracle_pins import BC, GAMMA5, dense_dhop, parity_sites, rel, spin_index

TAU1 = np.array([[0, 1], [1, 0]], complex)
TAU3 = np.array([[1, 0], [0, -1]], complex)


def dense_Qnd(dims, U, kappa, mu_sigma, mu_delta, bc=BC):
    """gamma5 (M_ee - M_eo M_oo^-1 M_oe) of the dense doublet matrix, flavour-major rows."""
    V = int(np.prod(dims))
    mubar, epsbar = 2 * kappa * mu_sigma, 2 * kappa * mu_delta
    one = np.eye(12 * V)
    g5 = np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    M = np.kron(np.eye(2), one - kappa * dense_dhop(dims, U, bc)) + 1j * mubar * np.kron(TAU3, g5) - \
        epsbar * np.kron(TAU1, one)
    ev, od = parity_sites(dims)
    ie, io = spin_index(ev), spin_index(od)
    ie2 = np.concatenate([ie, 12 * V + ie])
    io2 = np.concatenate([io, 12 * V + io])
    Mee, Meo, Moe, Moo = M[np.ix_(ie2, ie2)], M[np.ix_(ie2, io2)], M[np.ix_(io2, ie2)], M[np.ix_(io2, io2)]
    S = Mee - Meo @ np.linalg.inv(Moo) @ Moe
    G5 = np.kron(np.eye(2), np.kron(np.eye(V // 2), np.kron(GAMMA5, np.eye(3))))
    return G5 @ S


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 6)])
def test_Qnd_matches_dense_schur_complement(dims):
    Vh = int(np.prod(dims)) // 2
    kappa, ms, md = 0.16, 0.013, 0.21
    U = F.gauge_field(dims, 21, "random")
    ps, pc = F.gaussian_spinor(Vh, 21, 1), F.gaussian_spinor(Vh, 21, 2)
    Q = dense_Qnd(dims, U, kappa, ms, md)
    want = Q @ np.concatenate([ps.reshape(-1), pc.reshape(-1)])
    os_, oc = O.Qnd(dims, U, ps, pc, kappa, ms, md)
    assert rel(np.concatenate([os_.reshape(-1), oc.reshape(-1)]), want) < 1e-13


def test_Qnd_without_splitting_is_two_degenerate_operators():
    dims = (4, 4, 4, 4)
    Vh = 128
    U = F.gauge_field(dims, 22, "random")
    ps, pc = F.gaussian_spinor(Vh, 22, 1), F.gaussian_spinor(Vh, 22, 2)
    os_, oc = O.Qnd(dims, U, ps, pc, 0.16, 0.01, 0.0)
    assert rel(os_, O.Qtm(dims, U, ps, 0.16, 0.01)) < 1e-14
    assert rel(oc, O.Qtm(dims, U, pc, 0.16, -0.01)) < 1e-14


def test_Qnd_adjoint_is_Qnd_with_minus_mu_sigma():
    dims = (4, 4, 4, 4)
    Vh = 128
    k, ms, md = 0.1394, 0.0015, 0.19
    U = F.gauge_field(dims, 23, "near", 0.3)
    ps, pc, cs, cc = (F.gaussian_spinor(Vh, 23, j) for j in range(1, 5))
    qs, qc = O.Qnd(dims, U, ps, pc, k, ms, md)
    rs, rc = O.Qnd(dims, U, cs, cc, k, -ms, md)
    lhs = np.vdot(cs, qs) + np.vdot(cc, qc)
    rhs = np.vdot(rs, ps) + np.vdot(rc, pc)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # and not with +mu_sigma: the pin would catch a wrong sign of the twist
    ws, wc = O.Qnd(dims, U, cs, cc, k, ms, md)
    assert abs(np.vdot(ws, ps) + np.vdot(wc, pc) - lhs) > 1e-6 * abs(lhs)


def test_Qnd_refuses_a_singular_site_matrix():
    dims = (2, 2, 2, 2)
    U = F.gauge_field(dims, 24, "random")
    psi = F.gaussian_spinor(8, 24, 1)
    with pytest.raises(ValueError):
        O.Qnd(dims, U, psi, psi, 0.5, 0.0, 1.0)     # epsbar = 1 = 1 + mubar^2
