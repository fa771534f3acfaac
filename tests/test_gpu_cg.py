"""GPU conjugate gradients on Q^dag Q against the FP64 oracle.

CG solutions are unique only up to the tolerance, so the solution is
checked by its true residual |b - Q^dag Q x| / |b|, recomputed by the
oracle in FP64 on the host, and, where the system is well conditioned,
against the oracle's own CG solution.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def oracle_relres(dims, U, x, b, kappa, mu):
    Ax = O.Qtm(dims, U, O.Qtm(dims, U, x, kappa, mu), kappa, -mu)
    return float(np.linalg.norm(b - Ax) / np.linalg.norm(b))


def solve(ctx, dims, U, b, kappa, mu, inner, tol=1e-10, maxiter=20000, reliable_every=50, use_graph=True, x0=None):
    vh = b.shape[0]
    gh = ctx.gauge(dims, U, "f64", 18)
    gl = None if inner == "f64" else ctx.gauge(dims, U, inner, 12)
    x = ctx.pack(np.zeros_like(b) if x0 is None else x0, "f64")
    bd = ctx.pack(b, "f64")
    st, info = ctx.cg(gh, x, bd, kappa, mu, tol, maxiter, gl, reliable_every, use_graph)
    out = ctx.unpack(x, vh, "f64").cpu().numpy()
    gh.close()
    if gl is not None:
        gl.close()
    return st, info, out


@pytest.fixture(scope="module")
def small():
    dims = (8, 8, 8, 8)
    U = F.gauge_field(dims, F.SEED_SMALL_8, "random")
    b = F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_SMALL_8, 5)
    xo, it, rr, ok = O.cg_QdagQ(dims, U, b, 0.16, 0.01, tol=1e-12, maxiter=5000)
    assert ok
    return dims, U, b, xo


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_cg_small_true_residual_and_solution(ctx, small, inner):
    from paper_1311_4521_gb300 import tmhop
    dims, U, b, xo = small
    st, info, x = solve(ctx, dims, U, b, 0.16, 0.01, inner)
    assert st == tmhop.TM_OK, info
    assert info["true_relres"] <= 1e-10
    assert oracle_relres(dims, U, x, b, 0.16, 0.01) <= 1.05e-10
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8
    assert info["iters"] > 0


def test_cg_graph_and_direct_launch_agree_bitwise(ctx, small):
    dims, U, b, _ = small
    a = solve(ctx, dims, U, b, 0.16, 0.01, "f32", use_graph=True)
    c = solve(ctx, dims, U, b, 0.16, 0.01, "f32", use_graph=False)
    d = solve(ctx, dims, U, b, 0.16, 0.01, "f32", use_graph=True)
    assert np.array_equal(a[2], c[2]) and np.array_equal(a[2], d[2])
    assert a[1]["iters"] == c[1]["iters"] == d[1]["iters"]


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_cg_near_thermalised_ragged(ctx, inner):
    """kappa = 0.1394, mu = 0.0015 on an odd-shaped lattice with exp(0.3 i A) links."""
    from paper_1311_4521_gb300 import tmhop
    dims = (6, 4, 8, 10)
    U = F.gauge_field(dims, F.SEED_CG_48, "near", 0.3)
    b = F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_CG_48, 1)
    st, info, x = solve(ctx, dims, U, b, 0.1394, 0.0015, inner, maxiter=30000)
    assert st == tmhop.TM_OK, info
    assert oracle_relres(dims, U, x, b, 0.1394, 0.0015) <= 1.05e-10


def test_cg_maxiter_reports_not_converged(ctx, small):
    from paper_1311_4521_gb300 import tmhop
    dims, U, b, _ = small
    for inner in ("f64", "f32"):
        st, info, x = solve(ctx, dims, U, b, 0.16, 0.01, inner, maxiter=7, reliable_every=5)
        assert st == tmhop.TM_ERR_NOT_CONVERGED
        assert info["true_relres"] > 1e-10
        assert abs(oracle_relres(dims, U, x, b, 0.16, 0.01) - info["true_relres"]) < 1e-6


def test_cg_starting_from_the_solution_takes_no_iterations(ctx, small):
    from paper_1311_4521_gb300 import tmhop
    dims, U, b, xo = small
    st, info, x = solve(ctx, dims, U, b, 0.16, 0.01, "f64", x0=xo)
    assert st == tmhop.TM_OK and info["iters"] == 0


def test_cg_nonfinite_source(ctx, small):
    from paper_1311_4521_gb300 import tmhop
    dims, U, b, _ = small
    bad = b.copy()
    bad[3, 1, 2] = np.nan
    for inner in ("f64", "f32"):
        st, info, _ = solve(ctx, dims, U, bad, 0.16, 0.01, inner)
        assert st == tmhop.TM_ERR_NONFINITE


def test_cg_argument_errors(ctx, small):
    from paper_1311_4521_gb300 import tmhop
    dims, U, b, _ = small
    g32 = ctx.gauge(dims, U, "f32", 12)
    x = ctx.pack(np.zeros_like(b), "f64")
    bd = ctx.pack(b, "f64")
    with pytest.raises(tmhop.TmError) as e:
        ctx.cg(g32, x, bd, 0.16, 0.01)            # U_hi must be FP64
    assert e.value.status == tmhop.TM_ERR_ARG
    gh = ctx.gauge(dims, U, "f64", 18)
    with pytest.raises(tmhop.TmError):
        ctx.cg(gh, x, bd, 0.16, 0.01, tol=0.0)
    other = ctx.gauge((4, 4, 4, 4), F.gauge_field((4, 4, 4, 4), 1, "random"), "f32", 12)
    with pytest.raises(tmhop.TmError):
        ctx.cg(gh, x, bd, 0.16, 0.01, U_lo=other)


def test_cg_production_size_oracle_residual(ctx):
    """48^3x96, kappa = 0.1394, mu = 0.0015: the mixed FP16 and FP32 solutions,
    checked by the oracle's FP64 residual |b - Q(-mu) Q(mu) x| / |b|."""
    from paper_1311_4521_gb300 import tmhop
    dims = (48, 48, 48, 96)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_CG_48, "near", 0.3)
    b = F.gaussian_spinor(vh, F.SEED_CG_48, 1)
    gh = ctx.gauge(dims, U, "f64", 18)
    bd = ctx.pack(b, "f64")
    for inner in ("f16", "f32"):
        gl = ctx.gauge(dims, U, inner, 12)
        x = ctx.empty(vh, "f64").zero_()
        st, info = ctx.cg(gh, x, bd, 0.1394, 0.0015, 1e-10, 30000, gl)
        gl.close()
        assert st == tmhop.TM_OK, info
        xs = ctx.unpack(x, vh, "f64").cpu().numpy()
        assert oracle_relres(dims, U, xs, b, 0.1394, 0.0015) <= 1.05e-10
    gh.close()


@pytest.mark.parametrize("inner", ["f64x", "f32", "f16"])
def test_cg_double_float_outer_solver(ctx, inner):
    """U_hi in double-float storage (TM_F64X): x and b packed as F64X; plain
    F64X CG or mixed precision with F64X reliable updates."""
    from paper_1311_4521_gb300 import tmhop
    dims = (6, 4, 8, 10)
    U = F.gauge_field(dims, F.SEED_CG_48, "near", 0.3)
    vh = int(np.prod(dims)) // 2
    b = F.gaussian_spinor(vh, F.SEED_CG_48, 1)
    gh = ctx.gauge(dims, U, "f64x", 18)
    gl = None if inner == "f64x" else ctx.gauge(dims, U, inner, 12)
    x = ctx.empty(vh, "f64x").zero_()
    st, info = ctx.cg(gh, x, ctx.pack(b, "f64x"), 0.1394, 0.0015, 1e-10, 30000, gl)
    assert st == tmhop.TM_OK, info
    xs = ctx.unpack(x, vh, "f64x").cpu().numpy()
    assert oracle_relres(dims, U, xs, b, 0.1394, 0.0015) <= 1.05e-10
