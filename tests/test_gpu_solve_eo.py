"""Full-lattice solve M x = b by even-odd preconditioning (source
preparation, CG on the even sites, odd-site reconstruction), checked on the
full lattice with the oracle's pinned pieces: M x = x - kappa Dhop x +
i mut gamma5 x, and against a dense solve on a small lattice."""
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


def apply_M(dims, U, x, kappa, mu):
    mut = 2 * kappa * mu
    return x - kappa * O.dhop(dims, U, x) + 1j * mut * O.gamma5(x)


def gpu_solve(ctx, dims, U, b_full, kappa, mu, inner, tol):
    from paper_1311_4521_gb300 import tmhop
    vh = int(np.prod(dims)) // 2
    gh = ctx.gauge(dims, U, "f64", 18)
    gl = None if inner == "f64" else ctx.gauge(dims, U, inner, 12)
    be, bo = ctx.pack(O.pack_eo(dims, b_full, 0), "f64"), ctx.pack(O.pack_eo(dims, b_full, 1), "f64")
    xe, xo = ctx.empty(vh, "f64").zero_(), ctx.empty(vh, "f64")
    st, info = ctx.solve_eo(gh, xe, xo, be, bo, kappa, mu, tol, 30000, gl)
    assert st == tmhop.TM_OK, info
    x = O.unpack_eo(dims, ctx.unpack(xe, vh, "f64").cpu().numpy(), 0) + \
        O.unpack_eo(dims, ctx.unpack(xo, vh, "f64").cpu().numpy(), 1)
    gh.close()
    if gl is not None:
        gl.close()
    return x, info


def test_solve_eo_matches_dense_solve(ctx):
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    kappa, mu = 0.16, 0.05
    U = F.gauge_field(dims, 17, "random")
    b = F.gaussian_spinor(V, 17, 1)
    # dense M from the oracle's pinned operator, column by column
    M = np.zeros((12 * V, 12 * V), complex)
    for j in range(12 * V):
        e = np.zeros(12 * V, complex)
        e[j] = 1
        M[:, j] = apply_M(dims, U, e.reshape(V, 4, 3), kappa, mu).reshape(-1)
    want = np.linalg.solve(M, b.reshape(-1)).reshape(V, 4, 3)
    x, _ = gpu_solve(ctx, dims, U, b, kappa, mu, "f64", 1e-13)
    assert np.linalg.norm(x - want) / np.linalg.norm(want) < 1e-10


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_solve_eo_full_residual(ctx, inner):
    dims = (8, 8, 8, 16)
    kappa, mu = 0.1394, 0.0015
    U = F.gauge_field(dims, F.SEED_CG_48, "near", 0.3)
    b = F.gaussian_spinor(int(np.prod(dims)), F.SEED_CG_48, 3)
    x, info = gpu_solve(ctx, dims, U, b, kappa, mu, inner, 1e-12)
    r = b - apply_M(dims, U, x, kappa, mu)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10, info
