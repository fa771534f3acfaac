"""The seeded input generators (paper_1311_4521_gb300.fields) against the
properties the input recipe states: SU(3) links to rounding, the mean of
Re tr U / 3 over the near-thermalised ensemble against its series in eps,
Gaussian spinor moments, counter-based values that do not depend on how
the work is chunked, and distinct streams per field.
CPU only."""
import numpy as np
import pytest

from paper_1311_4521_gb300 import fields as F


def unitarity_error(U):
    I = np.eye(3)
    UU = np.einsum("...ab,...cb->...ac", U, np.conj(U))
    return float(np.abs(UU - I).max())


@pytest.mark.parametrize("kind", ["random", "near"])
def test_links_are_su3(kind):
    U = F.gauge_field((4, 4, 4, 8), 3, kind)
    assert U.shape == (4, 512, 3, 3)
    assert unitarity_error(U) < 1e-14
    assert float(np.abs(np.linalg.det(U) - 1).max()) < 1e-14
    # the third row is conj(row0 x row1): what 12-real reconstruction assumes
    r2 = np.conj(np.cross(U[..., 0, :], U[..., 1, :]))
    assert float(np.abs(r2 - U[..., 2, :]).max()) < 1e-14


def test_unit_gauge_is_identity():
    U = F.gauge_field((2, 2, 2, 2), 0, "unit")
    assert np.array_equal(U, np.broadcast_to(np.eye(3), U.shape))


def test_near_ensemble_mean_trace():
    # U = exp(i eps A), A = sum_a w_a lambda_a / 2, w_a ~ N(0,1):
    # <Re tr U>/3 = 1 - eps^2 <tr A^2>/6 + eps^4 <tr A^4>/72 - ...,
    # <tr A^2> = sum_a <w_a^2> tr(lambda_a^2)/4 = 8 * 2 / 4 = 4, so to second
    # order 1 - 0.09 * 4 / 6 = 0.94 at eps = 0.3 (the quartic term adds ~+1e-3)
    U = F.near_identity_su3(400000, 11, 1, 0.3)
    m = float(np.mean(np.real(np.trace(U, axis1=-2, axis2=-1))) / 3)
    assert abs(m - 0.94) < 4e-3
    U0 = F.near_identity_su3(1000, 11, 1, 0.0)
    assert np.allclose(U0, np.eye(3), atol=1e-15)


def test_spinor_moments():
    psi = F.gaussian_spinor(200000, 5, 1)
    assert psi.shape == (200000, 4, 3)
    re, im = psi.real.ravel(), psi.imag.ravel()
    for v in (re, im):
        assert abs(v.mean()) < 5e-3
        assert abs(v.var() - 1.0) < 5e-3
        assert abs(np.mean(v ** 4) - 3.0) < 3e-2   # Gaussian kurtosis
    assert abs(np.corrcoef(re, im)[0, 1]) < 5e-3


def test_values_do_not_depend_on_chunking(monkeypatch):
    a = F.gauge_field((4, 4, 8, 8), 9, "near")
    b = F.gaussian_spinor(3000, 9, 2)
    monkeypatch.setattr(F, "_CHUNK", 37)
    assert np.array_equal(F.gauge_field((4, 4, 8, 8), 9, "near"), a)
    assert np.array_equal(F.gaussian_spinor(3000, 9, 2), b)


def test_streams_are_distinct_and_prefix_stable():
    a = F.gaussian_spinor(100, 1, 1)
    assert not np.allclose(a, F.gaussian_spinor(100, 1, 2))   # another field
    assert not np.allclose(a, F.gaussian_spinor(100, 2, 1))   # another seed
    # a longer draw starts with the shorter one (values are indexed by counter)
    assert np.array_equal(F.gaussian_spinor(250, 1, 1)[:100], a)
