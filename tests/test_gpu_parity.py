"""GPU parity of the hopping matrix and Q_tm against the FP64 CPU oracle.

Inputs are seeded and synthetic (paper_1311_4521_gb300.fields); both sides
get the same host arrays.  Tolerances are relative L2 errors over the whole
output field: 1e-13 for FP64 storage, 1e-6 for FP32 and 5e-3 for FP16
(FP32 arithmetic in both reduced-precision paths).
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16": 5e-3}
STORAGE = [("f64", 18), ("f64", 12), ("f64x", 18), ("f64x", 12), ("f32", 18), ("f32", 12), ("f16", 12)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    return tmhop.Context(0)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu_apply(ctx, dims, U, psi, prec, recon, op, **kw):
    from paper_1311_4521_gb300 import tmhop
    g = ctx.gauge(dims, U, prec, recon, kw.get("bc", (-1, 1, 1, 1)))
    vh = psi.shape[0]
    src = ctx.pack(psi, prec)
    dst = ctx.empty(vh, prec)
    if op == "qtm":
        ctx.Qtm(g, dst, src, kw["kappa"], kw["mu"], kw.get("sign", 1))
    else:
        ctx.hopping_eo(g, dst, src, tmhop.TM_EO if op == "eo" else tmhop.TM_OE, kw.get("dagger", False))
    out = ctx.unpack(dst, vh, prec).cpu().numpy()
    g.close()
    return out


# 8^4 random SU(3), antiperiodic time, kappa = 0.16, mu = 0.01 (the small plain case)
@pytest.fixture(scope="module")
def small():
    dims = (8, 8, 8, 8)
    U = F.gauge_field(dims, F.SEED_SMALL_8, "random")
    psi = F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_SMALL_8, 1)
    return dims, U, psi


@pytest.mark.parametrize("prec,recon", STORAGE)
@pytest.mark.parametrize("op", ["eo", "oe"])
@pytest.mark.parametrize("dagger", [False, True])
def test_hopping_small(ctx, small, prec, recon, op, dagger):
    dims, U, psi = small
    want = O.hopping(dims, U, psi, 0 if op == "eo" else 1, dagger=dagger)
    got = gpu_apply(ctx, dims, U, psi, prec, recon, op, dagger=dagger)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec,recon", STORAGE)
@pytest.mark.parametrize("sign", [1, -1])
def test_Qtm_small(ctx, small, prec, recon, sign):
    dims, U, psi = small
    kappa, mu = 0.16, 0.01
    want = O.Qtm(dims, U, psi, kappa, sign * mu)
    got = gpu_apply(ctx, dims, U, psi, prec, recon, "qtm", kappa=kappa, mu=mu, sign=sign)
    assert rel(got, want) < TOL[prec]


# ragged shapes: Vh not a multiple of the block size, extent-2 directions,
# periodic and antiperiodic boundaries in several directions
@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), (-1, 1, 1, 1)), ((6, 4, 2, 10), (-1, 1, 1, 1)),
                                     ((10, 6, 4, 2), (1, -1, 1, -1)), ((4, 14, 6, 6), (-1, -1, -1, -1))])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64x", 18), ("f32", 12), ("f16", 12)])
def test_ragged_lattices(ctx, dims, bc, prec, recon):
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 7, "random")
    psi = F.gaussian_spinor(vh, 7, 2)
    for op, par in (("eo", 0), ("oe", 1)):
        want = O.hopping(dims, U, psi, par, bc=bc)
        assert rel(gpu_apply(ctx, dims, U, psi, prec, recon, op, bc=bc), want) < TOL[prec]
    want = O.Qtm(dims, U, psi, 0.1394, 0.0015, bc=bc)
    got = gpu_apply(ctx, dims, U, psi, prec, recon, "qtm", kappa=0.1394, mu=0.0015, bc=bc)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16"])
def test_pack_roundtrip(ctx, prec):
    psi = F.gaussian_spinor(1000, 3, 3)
    back = ctx.unpack(ctx.pack(psi, prec), 1000, prec).cpu().numpy()
    assert rel(back, psi) < {"f64": 0, "f64x": 1e-14, "f32": 1e-7, "f16": 1e-3}[prec] + 1e-300
    # an all-zero site survives the half-precision norm
    z = np.zeros((3, 4, 3), complex)
    assert np.all(ctx.unpack(ctx.pack(z, prec), 3, prec).cpu().numpy() == 0)


def test_bitwise_reproducible(ctx, small):
    dims, U, psi = small
    a = gpu_apply(ctx, dims, U, psi, "f64", 18, "qtm", kappa=0.16, mu=0.01)
    b = gpu_apply(ctx, dims, U, psi, "f64", 18, "qtm", kappa=0.16, mu=0.01)
    assert np.array_equal(a, b)


def test_argument_errors(ctx):
    import torch
    from paper_1311_4521_gb300 import tmhop
    U = torch.zeros((4, 3 * 2 * 2 * 2, 3, 3), dtype=torch.complex128)
    with pytest.raises(tmhop.TmError) as e:
        ctx.gauge((3, 2, 2, 2), U)
    assert e.value.status == tmhop.TM_ERR_ARG
    U = torch.zeros((4, 16, 3, 3), dtype=torch.complex128)
    with pytest.raises(tmhop.TmError) as e:
        ctx.gauge((2, 2, 2, 2), U, "f16", 18)
    assert e.value.status == tmhop.TM_ERR_UNSUPPORTED
    with pytest.raises(tmhop.TmError) as e:
        ctx.gauge((2, 2, 2, 2), U, "f64", 18, bc=(0, 1, 1, 1))
    assert e.value.status == tmhop.TM_ERR_ARG
    g = ctx.gauge((2, 2, 2, 2), U)
    buf = ctx.empty(8, "f64")
    with pytest.raises(tmhop.TmError) as e:
        ctx.Qtm(g, buf, buf, 0.1, 0.1)   # aliasing is rejected
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError):
        ctx.hopping_eo(g, buf, ctx.empty(8, "f64"), 5)
    # a field pointer 8 bytes off a 16-byte boundary is rejected before any launch
    flat = ctx.empty(9, "f64")
    with pytest.raises(tmhop.TmError) as e:
        ctx.Qtm(g, flat[8:], buf, 0.1, 0.1)
    assert e.value.status == tmhop.TM_ERR_ARG


# 32^3x64, near-thermalised links exp(0.3 i A), kappa = 0.1394, mu = 0.0015:
# the production size the benchmark times, compared over the whole field.
@pytest.fixture(scope="module")
def prod():
    dims = (32, 32, 32, 64)
    U = F.gauge_field(dims, F.SEED_PROD_32, "near", 0.3)
    psi = F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_PROD_32, 1)
    want = O.Qtm(dims, U, psi, 0.1394, 0.0015)
    return dims, U, psi, want


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64x", 18), ("f32", 12), ("f16", 12)])
def test_Qtm_production_size(ctx, prod, prec, recon):
    dims, U, psi, want = prod
    got = gpu_apply(ctx, dims, U, psi, prec, recon, "qtm", kappa=0.1394, mu=0.0015)
    assert rel(got, want) < TOL[prec]


# degenerate parameters of the method: kappa = 0 (Q = gamma5 (1 + i mut gamma5)
# acting alone), mu = 0 (plain Wilson), both, the free field (U = 1), an
# all-zero input, and all-periodic boundaries
@pytest.mark.parametrize("kappa,mu", [(0.0, 0.01), (0.16, 0.0), (0.0, 0.0)])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64x", 12), ("f32", 12), ("f16", 12)])
def test_Qtm_degenerate_parameters(ctx, small, kappa, mu, prec, recon):
    dims, U, psi = small
    want = O.Qtm(dims, U, psi, kappa, mu)
    got = gpu_apply(ctx, dims, U, psi, prec, recon, "qtm", kappa=kappa, mu=mu)
    assert rel(got, want) < TOL[prec]
    if kappa == 0.0 and mu == 0.0:   # Q = gamma5: exact in every storage format up to its rounding
        g5 = psi.copy()
        g5[:, 2:] *= -1
        assert rel(got, g5) < TOL[prec]


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 12)])
def test_free_field_zero_input_periodic(ctx, prec, recon):
    dims = (4, 6, 4, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 0, "unit")
    psi = F.gaussian_spinor(vh, 9, 4)
    for bc in ((1, 1, 1, 1), (-1, 1, 1, 1)):
        want = O.Qtm(dims, U, psi, 0.125, 0.05, bc=bc)
        assert rel(gpu_apply(ctx, dims, U, psi, prec, recon, "qtm", kappa=0.125, mu=0.05, bc=bc), want) < TOL[prec]
    zero = np.zeros_like(psi)
    out = gpu_apply(ctx, dims, U, zero, prec, recon, "qtm", kappa=0.125, mu=0.05)
    assert np.all(out == 0)
