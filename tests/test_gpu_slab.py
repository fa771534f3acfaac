"""The lattice cut along time into slabs (the surface/body split with face
exchange of the paper's Sec. 2.5): every slab of a lattice on one GPU, the
faces moved by device-to-device copies on a separate stream while the
interior launches run.  The assembled result must equal the operator on the
whole lattice, i.e. the FP64 oracle, for any number of slabs: one slab (its
faces are its own: the periodic wrap with the boundary sign), two, four, and
slabs of extent 2 (every site on a face)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}
RECON = {"f64": 18, "f32": 12, "f16": 12}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("nslab", [1, 2, 4, 8])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_slab_Qtm_matches_oracle(ctx, nslab, prec):
    from paper_1311_4521_gb300.slab import LocalSlabs
    dims = (4, 6, 4, 16)
    kappa, mu = 0.1394, 0.0015
    U = F.gauge_field(dims, 301, "near", 0.3)
    psi = F.gaussian_spinor(int(np.prod(dims)) // 2, 301, 1)
    sl = LocalSlabs(ctx, dims, U, nslab, prec, RECON[prec])
    ins = sl.pack_fields(torch.from_numpy(psi))
    outs = sl.empty()
    for o in outs:
        o.fill_(0xFF)            # every site must be written by one of the two launches
    for sign in (1, -1):
        sl.Qtm(outs, ins, kappa, mu, sign)
        got = sl.gather(outs).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, O.Qtm(dims, U, psi, kappa, sign * mu)) < TOL[prec]
    sl.close()


@pytest.mark.parametrize("nslab", [1, 2, 3])
@pytest.mark.parametrize("bc", [(-1, 1, 1, 1), (1, 1, 1, 1), (-1, -1, 1, -1)])
def test_slab_hops_and_adjoint_match_oracle(ctx, nslab, bc):
    """H_eo, H_oe and their adjoints on slabs, for several boundary signs
    (the time sign lives on the faces, the spatial ones in the slabs)."""
    from paper_1311_4521_gb300 import tmhop
    from paper_1311_4521_gb300.slab import LocalSlabs
    dims = (6, 4, 2, 12)
    U = F.gauge_field(dims, 302, "random")
    vh = int(np.prod(dims)) // 2
    psi = F.gaussian_spinor(vh, 302, 1)
    sl = LocalSlabs(ctx, dims, U, nslab, "f64", 18, bc)
    ins = sl.pack_fields(torch.from_numpy(psi))
    for direction, out_par in ((tmhop.TM_EO, 0), (tmhop.TM_OE, 1)):
        for dagger in (False, True):
            outs = sl.empty()
            sl.hopping_eo(outs, ins, direction, dagger)
            got = sl.gather(outs).cpu().numpy()
            # the adjoint between the same parities: H_oe^dag (even out) for TM_EO, H_eo^dag for TM_OE
            want = O.hopping(dims, U, psi, out_par, bc=bc, dagger=dagger)
            assert rel(got, want) < 1e-13, (direction, dagger)
    sl.close()


def test_slab_production_shape(ctx):
    """32^3 x 64 cut into 4 slabs of 16 time slices, FP64 and FP32, against
    the oracle's Q_tm on the whole lattice."""
    from paper_1311_4521_gb300.slab import LocalSlabs
    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_PROD_32, "near", 0.3)
    psi = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    want = O.Qtm(dims, U, psi, 0.1394, 0.0015)
    for prec in ("f64", "f32"):
        sl = LocalSlabs(ctx, dims, U, 4, prec, RECON[prec])
        outs = sl.Qtm(sl.empty(), sl.pack_fields(torch.from_numpy(psi)), 0.1394, 0.0015)
        got = sl.gather(outs).cpu().numpy()
        assert rel(got, want) < TOL[prec], prec
        sl.close()
        del outs, got


def test_slab_rejects_bad_arguments(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (4, 4, 4, 8)
    U = F.gauge_field(dims, 303, "random")
    vh = int(np.prod(dims)) // 2
    g = ctx.gauge(dims, U, "f64x", 18)
    assert tmhop.tm_slab_face_bytes(g.handle) == 0
    a, b = ctx.empty(vh, "f64x"), ctx.empty(vh, "f64x")
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_slab_pack(ctx.handle, g.handle, a, tmhop.TM_OE, 0, b, b)
    assert e.value.status in (tmhop.TM_ERR_ARG, tmhop.TM_ERR_UNSUPPORTED)
    g.close()
    g = ctx.gauge(dims, U, "f64", 18)
    a, b = ctx.empty(vh, "f64"), ctx.empty(vh, "f64")
    face = torch.empty(tmhop.tm_slab_face_bytes(g.handle), dtype=torch.uint8, device="cuda")
    with pytest.raises(tmhop.TmError):   # stage B needs the even input x
        tmhop.tm_slab_hop(ctx.handle, g.handle, a, b, face, face, tmhop.TM_EO, 0, tmhop.TM_SLAB_ALL,
                          tmhop.TM_SLAB_QTM_B, 0.1, 0.01, 1, None, 1, 1)
    with pytest.raises(tmhop.TmError):   # the face sites need the received faces
        tmhop.tm_slab_hop(ctx.handle, g.handle, a, b, None, None, tmhop.TM_EO, 0, tmhop.TM_SLAB_BOUNDARY,
                          tmhop.TM_SLAB_HOP)
    with pytest.raises(tmhop.TmError):   # stage A writes odd sites
        tmhop.tm_slab_hop(ctx.handle, g.handle, a, b, face, face, tmhop.TM_EO, 0, tmhop.TM_SLAB_ALL,
                          tmhop.TM_SLAB_QTM_A, 0.1, 0.01, 1)
    g.close()
