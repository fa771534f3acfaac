"""tm_Qtm_noalloc: the Q_tm entry point for callers that cannot let the
library allocate device memory (a framework that owns all device memory
through its own pool, a plugin with a fixed memory budget, a loop that
cannot take an allocation's device synchronisation).  Its odd temporary
lives in a static device array instead of the context's cudaMalloc'd
scratch buffer.

Checked through the C ABI against the FP64 oracle with the tolerances the
parity tests use, and against tm_Qtm, the existing entry point, on two
calls in a row with different inputs (so a stale temporary from the first
call would show up in the second).  A fresh context that only ever calls
tm_Qtm_noalloc must hold no device memory afterwards.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 12)])
def test_noalloc_matches_oracle_and_Qtm_on_two_calls(ctx, prec, recon):
    from paper_1311_4521_gb300 import tmhop
    dims = (8, 8, 8, 16)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 77, "near", 0.3)
    g = ctx.gauge(dims, U, prec, recon)
    calls = [(F.gaussian_spinor(vh, 77, 1), 0.1394, 0.0015, 1), (F.gaussian_spinor(vh, 77, 2), 0.16, 0.01, -1)]
    for psi, kappa, mu, sign in calls:
        want = O.Qtm(dims, U, psi, kappa, mu * sign)
        src = ctx.pack(psi, prec)
        ref = ctx.empty(vh, prec)
        tmhop.tm_Qtm(ctx.handle, g.handle, ref, src, kappa, mu, sign)
        out = ctx.empty(vh, prec)
        out.fill_(0xFF)   # NaN patterns: every site must be written
        tmhop.tm_Qtm_noalloc(ctx.handle, g.handle, out, src, kappa, mu, sign)
        a = ctx.unpack(out, vh, prec).cpu().numpy()
        b = ctx.unpack(ref, vh, prec).cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel(a, want) < TOL[prec]
        assert rel(a, b) < TOL[prec]
    g.close()


def test_noalloc_on_a_fresh_context_allocates_nothing():
    """A context that has only ever run tm_Qtm_noalloc holds no device memory,
    and once the library's code is loaded on the device the calls leave the
    device's free memory unchanged."""
    import torch
    from paper_1311_4521_gb300 import tmhop
    dims = (16, 16, 16, 16)          # FP64 odd temporary 6.3 MB: a cudaMalloc of it would show
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 78, "near", 0.3)
    psi = F.gaussian_spinor(vh, 78, 1)
    c = tmhop.Context(0)
    try:
        g = c.gauge(dims, U, "f64", 18)
        src = c.pack(psi, "f64")
        outs = [c.empty(vh, "f64") for _ in range(3)]
        tmhop.tm_Qtm_noalloc(c.handle, g.handle, outs[0], src, 0.1394, 0.0015, 1)   # loads the code if needed
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for o in outs[1:]:
            tmhop.tm_Qtm_noalloc(c.handle, g.handle, o, src, 0.1394, 0.0015, 1)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert tmhop.tm_ctx_device_bytes(c.handle) == 0
        assert free1 == free0
        want = O.Qtm(dims, U, psi, 0.1394, 0.0015)
        for o in outs:
            assert rel(c.unpack(o, vh, "f64").cpu().numpy(), want) < TOL["f64"]
        g.close()
    finally:
        c.close()


def test_noalloc_rejects_lattices_beyond_the_static_array(ctx):
    import torch
    from paper_1311_4521_gb300 import tmhop
    dims = (24, 24, 24, 48)   # FP64 odd temporary: 331,776 x 192 B > 32 MiB
    vh = int(np.prod(dims)) // 2
    assert tmhop.tm_spinor_bytes(vh, tmhop.TM_F64) > tmhop.TM_QTM_NOALLOC_MAX_BYTES
    U = torch.zeros((4, 2 * vh, 3, 3), dtype=torch.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    g = ctx.gauge(dims, U, "f64", 18)
    buf_in, buf_out = ctx.empty(vh, "f64"), ctx.empty(vh, "f64")
    with pytest.raises(tmhop.TmError) as e:
        tmhop.tm_Qtm_noalloc(ctx.handle, g.handle, buf_out, buf_in, 0.1, 0.01, 1)
    assert e.value.status == tmhop.TM_ERR_ARG and "static scratch" in str(e.value)
    g.close()
