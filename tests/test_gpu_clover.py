"""The clover twisted-mass operator Q_sw on the GPU (clover blocks built
from the links once per gauge field in FP64, applied in the epilogues of
the two hop launches) against the FP64 oracle's literal operator, whose
pins are in tests/test_oracle_sw_pins.py."""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6}
RECON = {"f64": 18, "f32": 12}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def run(ctx, dims, U, psi, prec, kappa, mu, csw, sign=1, recon=None, bc=(-1, 1, 1, 1)):
    from paper_1311_4521_gb300 import tmhop
    vh = psi.shape[0]
    g = ctx.gauge(dims, U, prec, recon or RECON[prec], bc)
    C = ctx.clover(g, U, csw, kappa, mu)
    out = ctx.empty(vh, prec)
    out.fill_(0xFF)
    ctx.Qsw(g, C, out, ctx.pack(psi, prec), sign)
    got = ctx.unpack(out, vh, prec).cpu().numpy()
    tmhop.tm_clover_destroy(C)
    g.close()
    return got


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 2, 10), (2, 2, 2, 2), (4, 6, 4, 8)])
def test_Qsw_matches_oracle(ctx, prec, dims):
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 701, "random")
    psi = F.gaussian_spinor(vh, 701, 1)
    for sign in (1, -1):
        got = run(ctx, dims, U, psi, prec, 0.13, 0.02, 1.6, sign)
        assert np.all(np.isfinite(got))
        assert rel(got, O.Qsw(dims, U, psi, 0.13, sign * 0.02, 1.6)) < TOL[prec], sign


def test_Qsw_boundary_signs_and_reconstruction(ctx):
    dims = (4, 4, 6, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 702, "near", 0.3)
    psi = F.gaussian_spinor(vh, 702, 1)
    for bc in ((1, 1, 1, 1), (-1, -1, 1, -1)):
        got = run(ctx, dims, U, psi, "f64", 0.1394, 0.0015, 1.76, 1, recon=12, bc=bc)
        assert rel(got, O.Qsw(dims, U, psi, 0.1394, 0.0015, 1.76, bc=bc)) < 1e-13


def test_Qsw_without_clover_is_Qtm(ctx):
    dims = (8, 8, 8, 16)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 703, "near", 0.3)
    psi = F.gaussian_spinor(vh, 703, 1)
    got = run(ctx, dims, U, psi, "f64", 0.1394, 0.0015, 0.0)
    assert rel(got, O.Qtm(dims, U, psi, 0.1394, 0.0015)) < 1e-13


def test_Qsw_production_size(ctx):
    """24^3 x 48 (the differentiation workload's lattice), FP64 and FP32, c_sw = 1.76."""
    dims = (24, 24, 24, 48)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_GRAD_24, "near", 0.3)
    psi = F.gaussian_spinor(vh, F.SEED_GRAD_24, 1)
    want = O.Qsw(dims, U, psi, 0.1394, 0.0015, 1.76)
    for prec in ("f64", "f32"):
        assert rel(run(ctx, dims, U, psi, prec, 0.1394, 0.0015, 1.76), want) < TOL[prec], prec


def test_Qsw_argument_errors(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (4, 4, 4, 4)
    U = F.gauge_field(dims, 704, "random")
    g16 = ctx.gauge(dims, U, "f16", 12)
    with pytest.raises(tmhop.TmError) as e:
        ctx.clover(g16, U, 1.0, 0.13, 0.01)
    assert e.value.status == tmhop.TM_ERR_UNSUPPORTED
    g16.close()
    g = ctx.gauge(dims, U, "f64", 18)
    g8 = ctx.gauge((4, 4, 4, 8), F.gauge_field((4, 4, 4, 8), 705, "random"), "f64", 18)
    C = ctx.clover(g, U, 1.0, 0.13, 0.01)
    assert tmhop.tm_clover_bytes(C) == 4 * 36 * 16 * 256
    a, b = ctx.empty(128, "f64"), ctx.empty(128, "f64")
    with pytest.raises(tmhop.TmError):   # a clover handle of another lattice
        tmhop.tm_Qsw(ctx.handle, g8.handle, C, ctx.empty(256, "f64"), ctx.empty(256, "f64"))
    with pytest.raises(tmhop.TmError):
        tmhop.tm_Qsw(ctx.handle, g.handle, C, a, a)
    tmhop.tm_clover_destroy(C)
    g.close()
    g8.close()
