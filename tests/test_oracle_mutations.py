"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle's C source (a flipped projector sign, U where U^dag belongs,
the backward link taken at the wrong site, the boundary sign dropped, the
sign of M_oo^-1 or of kappa flipped, one force term with the wrong sign,
the doublet's flavour splitting or twist or M_oo^-1 wrong, the clover
field strength's normalisation, a leaf's orientation or sigma's factor i),
builds it into a scratch library, points the oracle at it and requires at
least one of the oracle pins to fail.  The unmodified oracle passes the same
pins.  CPU only; the planted mistakes live in temporary files only."""
import ctypes
import os
import subprocess

import pytest

import oracle as O

import test_oracle_nd_pins as nd_pins
import test_oracle_pins as pins
import test_oracle_sw_pins as sw_pins

SRC = os.path.join(os.path.dirname(O.__file__), "tm_oracle.c")

# (name, text in tm_oracle.c, replacement); the first occurrence is replaced
MUTANTS = [
    ("forward projector sign", "one_pm_gamma(mu, -1, t1, t2);", "one_pm_gamma(mu, +1, t1, t2);"),
    ("U^dag for U on the forward hop", "colour_mul(U + ((long)mu * V + x) * 9, 0, psi + xp * SPINOR, t1);",
     "colour_mul(U + ((long)mu * V + x) * 9, 1, psi + xp * SPINOR, t1);"),
    ("backward link read at x instead of x - mu", "colour_mul(U + ((long)mu * V + xm) * 9, 1, psi + xm * SPINOR, t1);",
     "colour_mul(U + ((long)mu * V + x) * 9, 1, psi + xm * SPINOR, t1);"),
    ("boundary sign dropped", "double s = wrap ? bc[mu] : 1.0;", "double s = 1.0;"),
    ("M_oo^-1 with the wrong twist sign", "oracle_twist_inv(Vh, mut, t_o, u_o);", "oracle_twist_inv(Vh, -mut, t_o, u_o);"),
    ("minus sign of M_oe = -kappa H_oe dropped", "t_o[k] *= -kappa;", "t_o[k] *= kappa;"),
    ("force: second term with the wrong sign", "creal(term1 + term2)", "creal(term1 - term2)"),
    ("doublet: sign of the flavour splitting", "epsbar * (a == b ? 1.0 : 0.0) * tau1[f][g]",
     "-epsbar * (a == b ? 1.0 : 0.0) * tau1[f][g]"),
    ("doublet: twist without tau3", "I * mubar * G[4][a][b] * tau3[f][g]", "I * mubar * G[4][a][b] * (f == g ? 1.0 : 0.0)"),
    ("doublet: M_oo instead of M_oo^-1", "nd_apply(Vh, Ainv, t[0], t[1], u[0], u[1]);",
     "nd_apply(Vh, A, t[0], t[1], u[0], u[1]);"),
    ("clover: field strength normalisation", "(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0",
     "(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 4.0"),
    ("clover: one leaf with a link not daggered", "link_at(U, V, mu, xpn), 1, link_at(U, V, nu, x), 1, P);",
     "link_at(U, V, mu, xpn), 0, link_at(U, V, nu, x), 1, P);"),
    ("clover: sigma without its factor i", "sig[a][b] = 0.5 * I * c;", "sig[a][b] = 0.5 * c;"),
]


def run_pins():
    """The oracle pins that do not depend on the generators; returns the failures."""
    cases = [
        (pins.test_dhop_matches_dense_matrix, ((2, 2, 2, 2),)),
        (pins.test_dhop_matches_dense_matrix, ((4, 2, 2, 6),)),
        (pins.test_hopping_eo_and_Qtm_match_dense_schur_complement, ((2, 2, 2, 2),)),
        (pins.test_free_field_plane_wave, ((4, 4, 4, 4), (1, 0, 3, 2))),
        (pins.test_gauge_covariance, ()),
        (pins.test_gamma5_hermiticity_and_Q_dagger_is_Q_minus_mu, ()),
        (pins.test_special_cases_reduce, ()),
        (pins.test_force_matches_finite_differences_of_dense_action, ((2, 2, 2, 2),)),
        (pins.test_force_gauge_covariance, ()),
        (nd_pins.test_Qnd_matches_dense_schur_complement, ((2, 2, 2, 2),)),
        (nd_pins.test_Qnd_without_splitting_is_two_degenerate_operators, ()),
        (nd_pins.test_Qnd_adjoint_is_Qnd_with_minus_mu_sigma, ()),
        (sw_pins.test_clover_term_matches_path_walk, ((2, 2, 2, 2),)),
        (sw_pins.test_Qsw_matches_dense_schur_complement, ((2, 2, 2, 2),)),
        (sw_pins.test_Qsw_adjoint_is_Qsw_with_minus_mu, ()),
    ]
    failed = []
    for fn, args in cases:
        try:
            fn(*args)
        except Exception as e:   # an assertion or a numerical breakdown
            failed.append(f"{fn.__name__}{args}: {type(e).__name__}")
    return failed


def load_mutant(tmp_path, old, new):
    text = open(SRC).read()
    assert text.count(old) >= 1, old
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new, 1))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(src), "-lm"])
    return O._bind(ctypes.CDLL(str(lib)))


def test_unmodified_oracle_passes_the_pins():
    assert run_pins() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new):
    monkeypatch.setattr(O, "_lib", load_mutant(tmp_path, old, new))
    failed = run_pins()
    assert failed, f"no pin caught: {name}"
