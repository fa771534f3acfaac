"""tm_Qtm_host: Q_tm on fields in host memory, pipelined through two device
staging slots.  Every output against the FP64 oracle (tolerances of the
storage precision as in the parity tests), bit-equal to the device-resident
tm_Qtm on the same input, pinned and pageable buffers, one field and several,
and the argument checks."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16": 5e-3}


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    return tmhop.Context(0)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 2, 10)])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f64x", 18), ("f32", 12), ("f16", 12)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_fields_match_oracle(ctx, dims, prec, recon, pinned):
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 21, "random")
    psis = [F.gaussian_spinor(vh, 21, 10 + k) for k in range(5)]
    g = ctx.gauge(dims, U, prec, recon)
    ins = [torch.from_numpy(p.copy()) for p in psis]
    outs = [torch.empty_like(t) for t in ins]
    if pinned:
        ins = [t.pin_memory() for t in ins]
        outs = [t.pin_memory() for t in outs]
    ctx.Qtm_host(g, outs, ins, 0.1394, 0.0015, -1)
    for p, o in zip(psis, outs):
        assert rel(o.numpy(), O.Qtm(dims, U, p, 0.1394, -0.0015)) < TOL[prec]
    # same kernels as the device-resident call: identical results
    dev = ctx.empty(vh, prec)
    ctx.Qtm(g, dev, ctx.pack(psis[3], prec), 0.1394, 0.0015, -1)
    assert np.array_equal(ctx.unpack(dev, vh, prec).cpu().numpy(), outs[3].numpy())
    g.close()


@pytest.mark.parametrize("map_name", ["box4x2x2x2", "linear64"])
def test_host_fields_with_a_site_map(ctx, map_name):
    """FP64 host fields go through the hops' canonical-layout launches with the
    handle's site map: the same bits as tm_Qtm on packed fields with that map."""
    from paper_1311_4521_gb300 import tmhop
    dims = (8, 8, 8, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 23, "near", 0.3)
    psis = [F.gaussian_spinor(vh, 23, k) for k in range(3)]
    g = ctx.gauge(dims, U, "f64", 18)
    tmhop.tm_gauge_set_map(ctx.handle, g.handle, map_name)
    ins = [torch.from_numpy(p.copy()).pin_memory() for p in psis]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    ctx.Qtm_host(g, outs, ins, 0.1394, 0.0015)
    for p, o in zip(psis, outs):
        dev = ctx.empty(vh, "f64")
        ctx.Qtm(g, dev, ctx.pack(p, "f64"), 0.1394, 0.0015)
        assert np.array_equal(ctx.unpack(dev, vh, "f64").cpu().numpy(), o.numpy())
        assert rel(o.numpy(), O.Qtm(dims, U, p, 0.1394, 0.0015)) < 1e-13
    g.close()


def test_single_field_and_repeated_input(ctx):
    dims = (4, 4, 4, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 5, "near", 0.3)
    psi = torch.from_numpy(F.gaussian_spinor(vh, 5, 1)).pin_memory()
    g = ctx.gauge(dims, U, "f64", 18)
    want = O.Qtm(dims, U, psi.numpy(), 0.16, 0.01)
    one = [torch.empty_like(psi).pin_memory()]
    ctx.Qtm_host(g, one, [psi], 0.16, 0.01)
    assert rel(one[0].numpy(), want) < 1e-13
    # the same input buffer several times, every output written
    outs = [torch.zeros_like(psi) for _ in range(4)]
    ctx.Qtm_host(g, outs, [psi] * 4, 0.16, 0.01)
    for o in outs:
        assert np.array_equal(o.numpy(), one[0].numpy())
    g.close()


def test_host_argument_errors(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (2, 2, 2, 2)
    U = F.gauge_field(dims, 1, "random")
    g = ctx.gauge(dims, U, "f64", 18)
    a = torch.zeros((8, 4, 3), dtype=torch.complex128)
    b = torch.zeros_like(a)
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_Qtm_host(ctx.handle, g.handle, [a, b], [b, a], 0.1, 0.1)   # an output is an input
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_Qtm_host(ctx.handle, g.handle, [], [], 0.1, 0.1)           # no fields
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_Qtm_host(ctx.handle, g.handle, [a], [b], 0.1, 0.1, sign=2)
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(ValueError):
        ctx.Qtm_host(g, [a], [torch.zeros((8, 4, 3), dtype=torch.complex64)], 0.1, 0.1)
    g.close()
