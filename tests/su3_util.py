"""Test-side su(3) algebra: the force F from the complex link gradient G.

The library returns either the su(3) force (TM_FORCE_SU3) or the gradient
with respect to the complex link entries (TM_FORCE_GRAD).  The tests check
that the two agree through the relation below, so it lives here, beside
the tests, and not in the package (whose arithmetic runs in the kernels).

For U -> exp(eps T) U with T in su(3), dS = Re tr(G^dag dU) = Re tr(G^dag T U)
= Re tr(T (U G^dag)), so with <A, B> = -2 tr(AB) and the orthonormal basis
T_a = i lambda_a / 2 the force is F = -TA(U G^dag) / 2, TA the traceless
anti-Hermitian part.
"""
import numpy as np


def su3_force(U: np.ndarray, G: np.ndarray) -> np.ndarray:
    """F = -TA(U G^dag)/2 per link; U and G complex arrays of shape (..., 3, 3)."""
    W = U @ np.conj(np.swapaxes(G, -1, -2))
    A = 0.5 * (W - np.conj(np.swapaxes(W, -1, -2)))
    tr = np.trace(A, axis1=-2, axis2=-1) / 3
    return -0.5 * (A - tr[..., None, None] * np.eye(3))
