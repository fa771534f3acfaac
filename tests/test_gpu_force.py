"""Adjoint path: the fermion force kernel and the autograd Functions.

* tm_force against the oracle's force (which evaluates dS/deps_a link by
  link from the definition, with no outer-product formula): every link on
  8^4, 20 sampled links on 24^3x48; FP64 and FP32 storage.
* Finite differences of S = phi^dag (Q^dag Q)^-1 phi, S evaluated with the
  GPU solver and the second-order accurate estimate 2 Re(phi^dag X) -
  X^dag Q^dag Q X: central steps of 1e-6 on 20 random (link, generator)
  pairs of an 8^4 lattice, and along one random su(3) direction of every
  link at once on 24^3x48.
* the two push schemes of tm_force_ex (FP64 atomic adds, and private
  forward/backward buffers summed by a second pass) against the oracle on
  8^4 and on shapes with extent-2 directions and a ragged tail, bit-equal to
  each other and, run twice, to themselves.
* autograd: dS/dphi = 2X against finite differences (exact for a quadratic
  form), dS/dU against the oracle force, and the backward passes of the
  linear operators against the oracle's literal adjoints.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F
from su3_util import su3_force

pytestmark = pytest.mark.gpu

TOLF = {"f64": 1e-12, "f64x": 1e-12, "f32": 1e-5, "f16": 5e-3}
RECON = {"f64": 18, "f64x": 18, "f32": 12, "f16": 12}
LAM = F._LAMBDA


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import autograd
    return autograd.context(0)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def small():
    dims = (8, 8, 8, 8)
    U = F.gauge_field(dims, F.SEED_SMALL_8, "random")
    X = F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_SMALL_8, 7)
    return dims, U, X


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16"])
def test_force_all_links_match_oracle(ctx, small, prec):
    from paper_1311_4521_gb300 import tmhop
    dims, U, X = small
    k, mu = 0.16, 0.01
    g = ctx.gauge(dims, U, prec, RECON[prec])
    Fg = ctx.force(g, ctx.pack(X, prec), k, mu, tmhop.TM_FORCE_SU3).cpu().numpy()
    g.close()
    want = O.force(dims, U, X, k, mu)
    assert rel(Fg, want) < TOLF[prec]
    # anti-Hermitian exactly (by construction), traceless to rounding of the storage precision
    assert np.abs(Fg + np.conj(np.swapaxes(Fg, -1, -2))).max() == 0.0
    assert np.abs(np.trace(Fg, axis1=-2, axis2=-1)).max() < TOLF[prec] * np.abs(Fg).max()


def test_gradient_mode_gives_the_force(ctx, small):
    from paper_1311_4521_gb300 import autograd, tmhop
    dims, U, X = small
    g = ctx.gauge(dims, U, "f64", 18)
    xp = ctx.pack(X, "f64")
    G = ctx.force(g, xp, 0.16, 0.01, tmhop.TM_FORCE_GRAD)
    Fs = ctx.force(g, xp, 0.16, 0.01, tmhop.TM_FORCE_SU3)
    g.close()
    assert rel(su3_force(U, G.cpu().numpy()), Fs.cpu().numpy()) < 1e-13


SCHEMES = ("atomic", "halo")


def force_scheme(ctx, dims, U, X, prec, scheme, mode=0, bc=(-1, 1, 1, 1), k=0.16, mu=0.01):
    from paper_1311_4521_gb300 import tmhop
    g = ctx.gauge(dims, U, prec, RECON[prec], bc)
    sch = {"owner": tmhop.TM_FORCE_OWNER, "atomic": tmhop.TM_FORCE_ATOMIC, "halo": tmhop.TM_FORCE_HALO}[scheme]
    out = ctx.force(g, ctx.pack(X, prec), k, mu, mode, sch).cpu().numpy()
    g.close()
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_push_schemes_match_oracle(ctx, small, prec, mode):
    dims, U, X = small
    want = O.force(dims, U, X, 0.16, 0.01)
    owner = force_scheme(ctx, dims, U, X, prec, "owner", mode)
    got = {s: force_scheme(ctx, dims, U, X, prec, s, mode) for s in SCHEMES}
    # two addends per entry onto zero: the order of the atomics cannot matter
    assert np.array_equal(got["atomic"], got["halo"])
    assert np.array_equal(got["atomic"], force_scheme(ctx, dims, U, X, prec, "atomic", mode))
    assert rel(got["halo"], owner) < TOLF[prec]
    if mode == 0:
        assert rel(got["halo"], want) < TOLF[prec]
    else:
        Fs = su3_force(U, got["halo"])
        assert rel(Fs, want) < TOLF[prec]


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), (-1, 1, 1, 1)), ((6, 4, 2, 10), (-1, 1, -1, 1)),
                                     ((10, 6, 4, 2), (1, -1, 1, -1))])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_push_schemes_ragged(ctx, dims, bc, scheme):
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 11, "random")
    X = F.gaussian_spinor(vh, 11, 5)
    want = O.force(dims, U, X, 0.1394, 0.0015, bc=bc)
    got = force_scheme(ctx, dims, U, X, "f64", scheme, bc=bc, k=0.1394, mu=0.0015)
    assert rel(got, want) < 1e-12


def test_push_scheme_errors(ctx, small):
    from paper_1311_4521_gb300 import tmhop
    dims, U, X = small
    g = ctx.gauge(dims, U, "f16", 12)
    with pytest.raises(tmhop.TmError) as e:
        ctx.force(g, ctx.pack(X, "f16"), 0.16, 0.01, 0, tmhop.TM_FORCE_ATOMIC)
    assert e.value.status == tmhop.TM_ERR_UNSUPPORTED
    g.close()
    g = ctx.gauge(dims, U, "f64", 18)
    with pytest.raises(tmhop.TmError) as e:
        ctx.force(g, ctx.pack(X, "f64"), 0.16, 0.01, 0, 7)
    assert e.value.status == tmhop.TM_ERR_ARG
    g.close()


def solve(ctx, dims, U, phi, kappa, mu, tol, prec="f64", with_ax=False):
    from paper_1311_4521_gb300 import tmhop
    vh = phi.shape[0]
    gh = ctx.gauge(dims, U, "f64", 18)
    gl = None if prec == "f64" else ctx.gauge(dims, U, prec, 12)
    x = ctx.empty(vh, "f64").zero_()
    st, info = ctx.cg(gh, x, ctx.pack(phi, "f64"), kappa, mu, tol, 100000, gl)
    assert st == tmhop.TM_OK, info
    # second-order accurate action: 2 Re phi^dag X - X^dag Q^dag Q X
    q = ctx.empty(vh, "f64")
    aq = ctx.empty(vh, "f64")
    ctx.Qtm(gh, q, x, kappa, mu, 1)
    ctx.Qtm(gh, aq, q, kappa, mu, -1)
    X = ctx.unpack(x, vh, "f64").cpu().numpy()
    AX = ctx.unpack(aq, vh, "f64").cpu().numpy()
    gh.close()
    if gl is not None:
        gl.close()
    S = 2 * np.real(np.vdot(phi, X)) - np.real(np.vdot(X, AX))
    return (S, X, AX) if with_ax else (S, X)


def action_difference(phi, a, b):
    """S~(a) - S~(b) for S~(X) = 2 Re phi^dag X - X^dag A X, from solver results a = (S, X, AX)
    and b, summed over elementwise differences so that rounding scales with the (small)
    difference and not with S."""
    _, Xa, AXa = a
    _, Xb, AXb = b
    dX = Xa - Xb
    d1 = 2 * np.real(np.vdot(phi, dX))
    d2 = np.real(np.vdot(dX, AXa)) + np.real(np.vdot(Xb, AXa - AXb))
    return d1 - d2


def _expm(X):
    return F._expm_traceless(X)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_force_production_size_sampled_links(ctx, prec):
    """24^3x48, kappa = 0.1394, mu = 0.0015: X from the GPU solver, force on
    every link on the GPU, 20 random links recomputed by the oracle."""
    from paper_1311_4521_gb300 import tmhop
    dims = (24, 24, 24, 48)
    k, mu = 0.1394, 0.0015
    U = F.gauge_field(dims, F.SEED_GRAD_24, "near", 0.3)
    V = int(np.prod(dims))
    phi = F.gaussian_spinor(V // 2, F.SEED_GRAD_24, 1)
    _, X = solve(ctx, dims, U, phi, k, mu, 1e-10, prec)
    g = ctx.gauge(dims, U, prec, RECON[prec])
    Fg = ctx.force(g, ctx.pack(X, prec), k, mu, tmhop.TM_FORCE_SU3).cpu().numpy()
    g.close()
    rng = np.random.default_rng(24)
    links = np.stack([rng.integers(0, 4, 20), rng.integers(0, V, 20)], axis=1)
    want = O.force(dims, U, X, k, mu, links=links)
    got = Fg[links[:, 0], links[:, 1]]
    assert rel(got, want) < TOLF[prec]


def test_force_finite_differences_single_links(ctx):
    """Central differences (step 1e-6) of S on 20 random (link, generator) pairs, 8^4."""
    from paper_1311_4521_gb300 import tmhop
    dims = (8, 8, 8, 8)
    k, mu = 0.16, 0.05
    U = F.gauge_field(dims, 81, "near", 0.3)
    V = int(np.prod(dims))
    phi = F.gaussian_spinor(V // 2, 81, 1)
    S0, X = solve(ctx, dims, U, phi, k, mu, 1e-14)
    g = ctx.gauge(dims, U, "f64", 18)
    Fg = ctx.force(g, ctx.pack(X, "f64"), k, mu, tmhop.TM_FORCE_SU3).cpu().numpy()
    g.close()
    rng = np.random.default_rng(8)
    h = 1e-6
    errs = []
    for _ in range(20):
        m, x, a = int(rng.integers(4)), int(rng.integers(V)), int(rng.integers(8))
        T = 0.5j * LAM[a]
        want = float(np.real(-2 * np.trace(T @ Fg[m, x])))
        res = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[m, x] = _expm((sgn * h * T)[None])[0] @ U[m, x]
            res.append(solve(ctx, dims, Up, phi, k, mu, 1e-14, with_ax=True))
        fd = action_difference(phi, res[0], res[1]) / (2 * h)
        errs.append(abs(fd - want) / abs(want))
    assert max(errs) < 1e-5, errs


def test_force_finite_differences_all_links_production_size(ctx):
    """24^3x48: every link moved along its own random su(3) direction; the
    derivative of S is sum over links of <T, F>."""
    from paper_1311_4521_gb300 import tmhop
    dims = (24, 24, 24, 48)
    k, mu = 0.1394, 0.0015
    U = F.gauge_field(dims, F.SEED_GRAD_24, "near", 0.3)
    V = int(np.prod(dims))
    phi = F.gaussian_spinor(V // 2, F.SEED_GRAD_24, 1)
    S0, X = solve(ctx, dims, U, phi, k, mu, 1e-13)
    g = ctx.gauge(dims, U, "f64", 18)
    Fg = ctx.force(g, ctx.pack(X, "f64"), k, mu, tmhop.TM_FORCE_SU3).cpu().numpy()
    g.close()
    w = F.normal(F.stream_seed(24, 48), 0, 4 * V * 8).reshape(4 * V, 8)
    T = 0.5j * np.einsum("na,aij->nij", w, LAM)
    want = float(np.real(-2 * np.einsum("nij,nji->", T, Fg.reshape(4 * V, 3, 3))))
    h = 1e-6
    res = []
    for sgn in (+1, -1):
        Up = (_expm(sgn * h * T) @ U.reshape(4 * V, 3, 3)).reshape(U.shape)
        res.append(solve(ctx, dims, Up, phi, k, mu, 1e-13, with_ax=True))
    fd = action_difference(phi, res[0], res[1]) / (2 * h)
    assert abs(fd - want) <= 1e-6 * abs(want), (fd, want)


def test_autograd_action_gradients(ctx):
    from paper_1311_4521_gb300 import autograd
    dims = (8, 8, 8, 8)
    k, mu = 0.16, 0.01
    U = F.gauge_field(dims, 91, "random")
    V = int(np.prod(dims))
    phi = F.gaussian_spinor(V // 2, 91, 1)
    dev = torch.device("cuda", 0)
    Ut = torch.from_numpy(U).to(dev).requires_grad_(True)
    pt = torch.from_numpy(phi).to(dev).requires_grad_(True)
    S = autograd.action(pt, Ut, dims, k, mu, tol=1e-13)
    gphi, gU = torch.autograd.grad(S, (pt, Ut))
    gphi = gphi.cpu().numpy()
    # dS/dphi against central differences on 20 components (exact for a quadratic form)
    rng = np.random.default_rng(1)
    for _ in range(20):
        s, sp, c = int(rng.integers(V // 2)), int(rng.integers(4)), int(rng.integers(3))
        for unit, part in ((1.0, "re"), (1j, "im")):
            dp = np.zeros_like(phi)
            dp[s, sp, c] = unit * 1e-3
            Sp = autograd.action(torch.from_numpy(phi + dp).to(dev), Ut.detach(), dims, k, mu, tol=1e-13).item()
            Sm = autograd.action(torch.from_numpy(phi - dp).to(dev), Ut.detach(), dims, k, mu, tol=1e-13).item()
            fd = (Sp - Sm) / 2e-3
            got = gphi[s, sp, c].real if part == "re" else gphi[s, sp, c].imag
            assert abs(fd - got) < 1e-7 * max(1.0, abs(got)), (fd, got)
    # dS/dU -> su(3) force against the oracle force for the solver's X
    X, _, _, ok = O.cg_QdagQ(dims, U, phi, k, mu, tol=1e-13, maxiter=10000)
    Fo = O.force(dims, U, X, k, mu)
    Fa = su3_force(U, gU.cpu().numpy())
    assert rel(Fa, Fo) < 1e-9


def test_autograd_linear_operators_backward(ctx):
    from paper_1311_4521_gb300 import autograd, tmhop
    dims = (6, 4, 8, 10)
    k, mu = 0.1394, 0.0015
    U = F.gauge_field(dims, 93, "near", 0.3)
    vh = int(np.prod(dims)) // 2
    psi = F.gaussian_spinor(vh, 93, 1)
    gout = F.gaussian_spinor(vh, 93, 2)
    dev = torch.device("cuda", 0)
    Ut = torch.from_numpy(U).to(dev)
    # Q: vjp = Q^dag g
    pt = torch.from_numpy(psi).to(dev).requires_grad_(True)
    out = autograd.qtm(pt, Ut, dims, k, mu)
    assert rel(out.detach().cpu().numpy(), O.Qtm(dims, U, psi, k, mu)) < 1e-13
    (g,) = torch.autograd.grad(out, pt, torch.from_numpy(gout).to(dev))
    assert rel(g.cpu().numpy(), O.Qtm(dims, U, gout, k, mu, dagger=True)) < 1e-13
    # hops: vjp = literal adjoint
    for direction, par in ((tmhop.TM_EO, 0), (tmhop.TM_OE, 1)):
        pt = torch.from_numpy(psi).to(dev).requires_grad_(True)
        out = autograd.hopping_eo(pt, Ut, dims, direction)
        assert rel(out.detach().cpu().numpy(), O.hopping(dims, U, psi, par)) < 1e-13
        (g,) = torch.autograd.grad(out, pt, torch.from_numpy(gout).to(dev))
        assert rel(g.cpu().numpy(), O.hopping(dims, U, gout, 1 - par, dagger=True)) < 1e-13
