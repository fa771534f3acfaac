"""The non-degenerate twisted doublet Q_nd on the GPU (one thread hops both
flavours of a site with one load of each link; the site-local flavour
mixing is fused into the two launches) against the FP64 oracle's literal
doublet, whose pins are in tests/test_oracle_nd_pins.py."""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}
RECON = {"f64": 18, "f32": 12, "f16": 12}


def rel2(a, b):
    """Relative L2 error of a doublet."""
    num = np.linalg.norm(a[0] - b[0]) ** 2 + np.linalg.norm(a[1] - b[1]) ** 2
    return float(np.sqrt(num / (np.linalg.norm(b[0]) ** 2 + np.linalg.norm(b[1]) ** 2)))


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def run(ctx, dims, U, ps, pc, prec, kappa, ms, md, sign=1, recon=None, bc=(-1, 1, 1, 1)):
    vh = ps.shape[0]
    g = ctx.gauge(dims, U, prec, recon or RECON[prec], bc)
    outs = [ctx.empty(vh, prec), ctx.empty(vh, prec)]
    for o in outs:
        o.fill_(0xFF)
    ctx.Qnd(g, outs, [ctx.pack(ps, prec), ctx.pack(pc, prec)], kappa, ms, md, sign)
    g.close()
    return [ctx.unpack(o, vh, prec).cpu().numpy() for o in outs]


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 2, 10), (2, 2, 2, 2)])
def test_Qnd_matches_oracle(ctx, prec, dims):
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 601, "random")
    ps, pc = F.gaussian_spinor(vh, 601, 1), F.gaussian_spinor(vh, 601, 2)
    for sign in (1, -1):
        got = run(ctx, dims, U, ps, pc, prec, 0.1394, 0.0015, 0.19, sign)
        assert all(np.all(np.isfinite(x)) for x in got)
        want = O.Qnd(dims, U, ps, pc, 0.1394, sign * 0.0015, 0.19)
        assert rel2(got, want) < TOL[prec], (sign, rel2(got, want))


def test_Qnd_reconstruct_and_boundary_signs(ctx):
    dims = (4, 6, 4, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 602, "near", 0.3)
    ps, pc = F.gaussian_spinor(vh, 602, 1), F.gaussian_spinor(vh, 602, 2)
    for bc in ((1, 1, 1, 1), (-1, -1, 1, -1)):
        got = run(ctx, dims, U, ps, pc, "f64", 0.16, 0.02, 0.3, 1, recon=12, bc=bc)
        assert rel2(got, O.Qnd(dims, U, ps, pc, 0.16, 0.02, 0.3, bc=bc)) < 1e-13


def test_Qnd_without_splitting_equals_Qtm(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (8, 8, 8, 16)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 603, "near", 0.3)
    ps, pc = F.gaussian_spinor(vh, 603, 1), F.gaussian_spinor(vh, 603, 2)
    got = run(ctx, dims, U, ps, pc, "f64", 0.1394, 0.0015, 0.0)
    g = ctx.gauge(dims, U, "f64", 18)
    a, b = ctx.empty(vh, "f64"), ctx.empty(vh, "f64")
    ctx.Qtm(g, a, ctx.pack(ps, "f64"), 0.1394, 0.0015, 1)
    ctx.Qtm(g, b, ctx.pack(pc, "f64"), 0.1394, 0.0015, -1)
    g.close()
    want = [ctx.unpack(a, vh, "f64").cpu().numpy(), ctx.unpack(b, vh, "f64").cpu().numpy()]
    assert rel2(got, want) < 1e-14


def test_Qnd_production_size(ctx):
    """32^3 x 64, the production lattice, FP64 and FP32 against the oracle."""
    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_PROD_32, "near", 0.3)
    ps, pc = F.gaussian_spinor(vh, F.SEED_PROD_32, 1), F.gaussian_spinor(vh, F.SEED_PROD_32, 2)
    want = O.Qnd(dims, U, ps, pc, 0.1394, 0.0015, 0.0018)
    for prec in ("f64", "f32"):
        got = run(ctx, dims, U, ps, pc, prec, 0.1394, 0.0015, 0.0018)
        assert rel2(got, want) < TOL[prec], prec


def test_Qnd_argument_errors(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (4, 4, 4, 4)
    U = F.gauge_field(dims, 604, "random")
    g = ctx.gauge(dims, U, "f64", 18)
    a, b, c, d = (ctx.empty(128, "f64") for _ in range(4))
    with pytest.raises(tmhop.TmError) as e:   # epsbar^2 = 1 + mubar^2
        tmhop.tm_Qnd(ctx.handle, g.handle, a, b, c, d, 0.5, 0.0, 1.0)
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError):        # an output that is an input
        tmhop.tm_Qnd(ctx.handle, g.handle, a, b, a, d, 0.16, 0.01, 0.1)
    with pytest.raises(tmhop.TmError):        # one output for both flavours
        tmhop.tm_Qnd(ctx.handle, g.handle, a, a, c, d, 0.16, 0.01, 0.1)
    g.close()
    gx = ctx.gauge(dims, U, "f64x", 18)
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_Qnd(ctx.handle, gx.handle, a, b, c, d, 0.16, 0.01, 0.1)
    assert e.value.status == tmhop.TM_ERR_UNSUPPORTED
    gx.close()
