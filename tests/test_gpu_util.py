"""The measurement and field utilities of the C ABI: the FMA throughput
probe (the measured arithmetic peak of the FP64 roofline), the FP64 inner
product of packed fields (the global reduction of the paper's Sec. 3 on one
GPU) and the scaling of complex arrays by a device scalar, plus the
autograd layer that is built on them."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def test_fma_probe_is_plausible(ctx):
    """FP64 FMA throughput of a GB300 is of order 1 TFLOP/s (2 FMA lanes per
    SM and clock: 1.26 at 2.07 GHz), FP32 tens of TFLOP/s; the probe must
    land near those and FP32 must beat FP64 many times over."""
    from paper_1311_4521_gb300 import tmhop
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f64 = tmhop.tm_probe_fma(ctx.handle, tmhop.TM_F64)
    f32 = tmhop.tm_probe_fma(ctx.handle, tmhop.TM_F32)
    nominal64 = sms * 2 * 2 * 2.07e9 / 1e12
    assert 0.3 * nominal64 < f64 < 1.2 * nominal64, (f64, nominal64)
    assert f32 > 16 * f64, (f32, f64)
    with pytest.raises(tmhop.TmError):
        tmhop.tm_probe_fma(ctx.handle, tmhop.TM_F16)


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16"])
def test_spinor_dot_matches_definition(ctx, prec):
    """<a, b> = sum conj(a) b over every site and component, compared with
    numpy's vdot of the same (unpacked) values; bit-identical on repeat."""
    from paper_1311_4521_gb300 import tmhop
    vh = 10007                       # not a multiple of the block size
    a = F.gaussian_spinor(vh, 5, 1)
    b = F.gaussian_spinor(vh, 5, 2)
    pa, pb = ctx.pack(a, prec), ctx.pack(b, prec)
    # the reference uses the values as stored (rounded to the storage precision)
    ua, ub = ctx.unpack(pa, vh, prec).cpu().numpy(), ctx.unpack(pb, vh, prec).cpu().numpy()
    want = np.vdot(ua.reshape(-1), ub.reshape(-1))
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    tmhop.tm_spinor_dot(ctx.handle, vh, pa, pb, tmhop.PREC[prec], out)
    got = complex(out[0].item(), out[1].item())
    assert abs(got - want) <= 1e-12 * abs(want) + 1e-12 * np.sqrt(vh * 12)
    again = torch.empty_like(out)
    tmhop.tm_spinor_dot(ctx.handle, vh, pa, pb, tmhop.PREC[prec], again)
    assert torch.equal(out, again)
    # <a, a> is |a|^2 (its imaginary part cancels to rounding)
    tmhop.tm_spinor_dot(ctx.handle, vh, pa, pa, tmhop.PREC[prec], out)
    nrm = np.vdot(ua, ua).real
    assert abs(out[1].item()) <= 1e-13 * nrm
    assert abs(out[0].item() - nrm) <= 1e-12 * nrm


def test_spinor_dot_empty_field(ctx):
    from paper_1311_4521_gb300 import tmhop
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    tmhop.tm_spinor_dot(ctx.handle, 0, None, None, tmhop.TM_F64, out)
    assert out.tolist() == [0.0, 0.0]


def test_scale_complex(ctx):
    from paper_1311_4521_gb300 import tmhop
    z = torch.randn(1001, dtype=torch.complex128, device="cuda")
    z0 = z.clone()
    alpha = torch.tensor(-0.75, dtype=torch.float64, device="cuda")
    tmhop.tm_scale_complex(ctx.handle, z.numel(), torch.view_as_real(z), alpha, 2.0)
    assert torch.equal(z, z0 * (-1.5))
    tmhop.tm_scale_complex(ctx.handle, z.numel(), torch.view_as_real(z), None, 0.5)
    assert torch.equal(z, z0 * (-0.75))


def test_action_value_matches_oracle(ctx):
    """S = Re <phi, X> with X the solver's solution, against the oracle CG."""
    from paper_1311_4521_gb300 import autograd
    dims = (4, 4, 4, 8)
    k, mu = 0.16, 0.01
    U = F.gauge_field(dims, 92, "random")
    phi = F.gaussian_spinor(int(np.prod(dims)) // 2, 92, 1)
    S = autograd.action(torch.from_numpy(phi).cuda(), torch.from_numpy(U).cuda(), dims, k, mu, tol=1e-13)
    X, _, _, ok = O.cg_QdagQ(dims, U, phi, k, mu, tol=1e-13, maxiter=10000)
    assert ok
    want = np.vdot(phi.reshape(-1), X.reshape(-1)).real
    assert abs(S.item() - want) <= 1e-11 * abs(want)
