"""Link gradients of the linear operators (tm_link_grad) and the autograd
Functions built on them.

For f(U) = Re <Y, Op(U) X> the gradient G w.r.t. the complex link entries
satisfies df = Re sum conj(G) dU.  H_eo and H_oe are linear in U and Q_tm
quadratic, so the oracle's central difference (f(U + e D) - f(U - e D)) / 2e
along any complex direction D is the exact directional derivative up to
rounding.  D runs over dense random directions (every link at once) and
directions supported on one link (so a misplaced or transposed link entry
cannot cancel out), with the boundary links of the antiperiodic time
direction among them.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 8)
VH = int(np.prod(DIMS)) // 2
KAPPA, MU = 0.16, 0.013


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def _f(op, U, X, Y, sign=1):
    """Re <Y, Op(U) X> with the oracle."""
    from paper_1311_4521_gb300 import tmhop
    if op == tmhop.TM_GRAD_QTM:
        out = O.Qtm(DIMS, U, X, KAPPA, sign * MU)
    elif op == tmhop.TM_GRAD_HOP_EO:
        out = O.hopping(DIMS, U, X, 0)
    else:
        out = O.hopping(DIMS, U, X, 1)
    return np.vdot(Y.reshape(-1), out.reshape(-1)).real


def _directions(rng, U):
    """Dense random directions and ones supported on single links: a bulk link
    in each direction and the t links that wrap around the boundary."""
    V = U.shape[1]
    out = []
    for _ in range(2):
        out.append(rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    Lx, Ly, Lz, Lt = DIMS
    lex = lambda x, y, z, t: x + Lx * (y + Ly * (z + Lz * t))
    for mu, site in ((0, lex(1, 2, 3, 4)), (1, lex(3, 0, 1, 2)), (2, lex(0, 3, 2, 5)), (3, lex(2, 1, 0, 3)),
                     (3, lex(1, 1, 2, Lt - 1)), (3, lex(2, 3, 0, Lt - 1))):
        D = np.zeros(U.shape, dtype=np.complex128)
        D[mu, site] = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        out.append(D)
    assert V == np.prod(DIMS)
    return out


def _check(G, op, U, X, Y, sign, tol):
    rng = np.random.default_rng(7)
    eps = 1e-3
    for D in _directions(rng, U):
        fd = (_f(op, U + eps * D, X, Y, sign) - _f(op, U - eps * D, X, Y, sign)) / (2 * eps)
        got = np.sum(np.conj(G) * D).real
        scale = np.linalg.norm(G) * np.linalg.norm(D) + abs(fd)
        assert abs(got - fd) <= tol * scale, (abs(got - fd), fd, scale)


def _fields(seed):
    U = F.gauge_field(DIMS, seed, "random")
    X = F.gaussian_spinor(VH, seed, 1)
    Y = F.gaussian_spinor(VH, seed, 2)
    return U, X, Y


@pytest.mark.parametrize("opname", ["qtm", "hop_eo", "hop_oe"])
@pytest.mark.parametrize("sign", [1, -1])
def test_link_grad_fp64_matches_oracle_differences(ctx, opname, sign):
    from paper_1311_4521_gb300 import tmhop
    op = {"qtm": tmhop.TM_GRAD_QTM, "hop_eo": tmhop.TM_GRAD_HOP_EO, "hop_oe": tmhop.TM_GRAD_HOP_OE}[opname]
    if op != tmhop.TM_GRAD_QTM and sign == -1:
        pytest.skip("sign enters Q_tm only")
    U, X, Y = _fields(211)
    g = ctx.gauge(DIMS, U, "f64", 18)
    G = ctx.link_grad(g, ctx.pack(X, "f64"), ctx.pack(Y, "f64"), op, KAPPA, MU, sign).cpu().numpy()
    g.close()
    _check(G, op, U, X, Y, sign, 1e-11)


@pytest.mark.parametrize("prec,recon,tol", [("f64", 12, 1e-11), ("f64x", 18, 1e-11), ("f32", 18, 2e-6),
                                            ("f32", 12, 2e-6), ("f16", 12, 2e-2)])
def test_link_grad_every_storage_format(ctx, prec, recon, tol):
    """The same gradient from every link/spinor storage: compared with the FP64
    gradient (itself pinned above by the oracle's differences)."""
    from paper_1311_4521_gb300 import tmhop
    U, X, Y = _fields(212)
    g64 = ctx.gauge(DIMS, U, "f64", 18)
    want = ctx.link_grad(g64, ctx.pack(X, "f64"), ctx.pack(Y, "f64"), tmhop.TM_GRAD_QTM, KAPPA, MU).cpu().numpy()
    g64.close()
    for op in (tmhop.TM_GRAD_QTM, tmhop.TM_GRAD_HOP_EO, tmhop.TM_GRAD_HOP_OE):
        g = ctx.gauge(DIMS, U, prec, recon)
        got = ctx.link_grad(g, ctx.pack(X, prec), ctx.pack(Y, prec), op, KAPPA, MU).cpu().numpy()
        g.close()
        if op == tmhop.TM_GRAD_QTM:
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err < tol, (prec, recon, err)
        else:
            _check(got, op, U, X, Y, 1, tol)


def test_link_grad_rejects_bad_arguments(ctx):
    from paper_1311_4521_gb300 import tmhop
    U, X, Y = _fields(213)
    g = ctx.gauge(DIMS, U, "f64", 18)
    x, y = ctx.pack(X, "f64"), ctx.pack(Y, "f64")
    G = torch.empty((4, 2 * VH, 3, 3, 2), dtype=torch.float64, device=ctx.device)
    with pytest.raises(tmhop.TmError):
        tmhop.tm_link_grad(ctx.handle, g.handle, G, x, y, 3)
    with pytest.raises(tmhop.TmError):
        tmhop.tm_link_grad(ctx.handle, g.handle, G, x, y, tmhop.TM_GRAD_QTM, KAPPA, MU, 0)
    g.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-6)])
def test_autograd_qtm_link_gradient(ctx, prec, tol):
    """torch.autograd through autograd.qtm: for L = Re <Y, Q psi> the link
    gradient matches the oracle's differences and the spinor gradient is
    Q^dag Y."""
    from paper_1311_4521_gb300 import autograd, tmhop
    U, X, Y = _fields(214)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    psi = torch.from_numpy(X).cuda().requires_grad_(True)
    Yt = torch.from_numpy(Y).cuda()
    out = autograd.qtm(psi, Ut, DIMS, KAPPA, MU, prec=prec)
    L = (Yt.conj() * out).real.sum()
    gpsi, gU = torch.autograd.grad(L, (psi, Ut))
    _check(gU.cpu().numpy(), tmhop.TM_GRAD_QTM, U, X, Y, 1, tol)
    want = O.Qtm(DIMS, U, Y, KAPPA, -MU)
    err = np.linalg.norm(gpsi.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < tol


@pytest.mark.parametrize("direction", [0, 1])
def test_autograd_hopping_link_gradient(ctx, direction):
    """torch.autograd through autograd.hopping_eo with the loss |H psi|^2:
    the upstream gradient is 2 H psi, and the link gradient matches the
    oracle's differences of that loss."""
    from paper_1311_4521_gb300 import autograd, tmhop
    U, X, _ = _fields(215)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    out = autograd.hopping_eo(torch.from_numpy(X).cuda(), Ut, DIMS, direction)
    (gU,) = torch.autograd.grad(out.abs().pow(2).sum(), Ut)
    G = gU.cpu().numpy()
    rng = np.random.default_rng(8)
    loss = lambda W: np.sum(np.abs(O.hopping(DIMS, W, X, direction)) ** 2)
    eps = 1e-3
    for D in _directions(rng, U):
        fd = (loss(U + eps * D) - loss(U - eps * D)) / (2 * eps)   # exact: the loss is quadratic in U
        got = np.sum(np.conj(G) * D).real
        assert abs(got - fd) <= 1e-11 * (np.linalg.norm(G) * np.linalg.norm(D) + abs(fd))


def test_link_grad_qtm_full_size(ctx):
    """The configuration the bench times (24^3x48, FP64-18, U = exp(0.3 i A)):
    the gradient along single links (bulk, and across the antiperiodic time
    boundary) and along one dense direction against the oracle's central
    differences, which are exact for Q_tm (quadratic in U)."""
    from paper_1311_4521_gb300 import tmhop
    dims = (24, 24, 24, 48)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_GRAD_24, "near", 0.3)
    X = F.gaussian_spinor(vh, F.SEED_GRAD_24, 1)
    Y = F.gaussian_spinor(vh, F.SEED_GRAD_24, 2)
    g = ctx.gauge(dims, U, "f64", 18)
    G = ctx.link_grad(g, ctx.pack(X, "f64"), ctx.pack(Y, "f64"), tmhop.TM_GRAD_QTM, KAPPA, MU).cpu().numpy()
    g.close()
    f = lambda W: np.vdot(Y.reshape(-1), O.Qtm(dims, W, X, KAPPA, MU).reshape(-1)).real
    rng = np.random.default_rng(17)
    Lx, Ly, Lz, Lt = dims
    lex = lambda x, y, z, t: x + Lx * (y + Ly * (z + Lz * t))
    dirs = []
    for mu, site in ((0, lex(3, 5, 7, Lt - 1)), (0, lex(10, 2, 19, 20)), (1, lex(Lx - 1, 4, 4, 4)), (3, lex(1, 2, 3, 0))):
        D = np.zeros(U.shape, dtype=np.complex128)
        D[mu, site] = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        dirs.append(D)
    dirs.append(rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    eps = 1e-3
    for D in dirs:
        fd = (f(U + eps * D) - f(U - eps * D)) / (2 * eps)
        got = np.sum(np.conj(G) * D).real
        assert abs(got - fd) <= 1e-10 * (np.linalg.norm(G) * np.linalg.norm(D) + abs(fd)), (got, fd)
