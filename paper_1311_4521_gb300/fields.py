"""Seeded synthetic inputs for the twisted-mass operator: gauge links and spinors.

This module only draws random numbers and builds SU(3) matrices from them.
It holds none of the operator's arithmetic (no gamma matrices, no hopping
term, no even-odd geometry), so that the CPU oracle and the CUDA path can
both take their inputs from here without sharing any of the method.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: the k-th draw of stream ``s`` is ``mix(s + k*G)``
with G = 0x9E3779B97F4A7C15, exactly the k-th output of a SplitMix64
generator seeded with ``s``.  Draws therefore do not depend on chunking or
thread order.  Normal deviates use the Box-Muller transform on consecutive
pairs of draws.

Layouts produced (all complex128, C-contiguous):

* gauge field ``U[mu, site, a, b]`` with ``mu`` 0 = t, 1 = x, 2 = y, 3 = z
  and ``site = x + Lx*(y + Ly*(z + Lz*t))``;
* spinor field ``psi[site, spin, colour]`` of shape ``(n, 4, 3)``; a field on
  one parity is simply ``n = V/2`` independent Gaussian spinors.

Workload recipes (near-thermalised links ``exp(i*eps*A)`` with
``A = sum_a w_a lambda_a / 2``, ``w_a ~ N(0,1)``; random SU(3) by
Gram-Schmidt of complex Gaussian rows) follow the lattice QCD convention of
generating test gauge fields close to the identity for production-like
spectra and fully random ones for small correctness cases.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 18
_THREADS = max(1, min(32, os.cpu_count() or 1))


def _chunked(n: int, fill) -> None:
    """Calls fill(lo, m) for consecutive chunks of [0, n) on a thread pool.

    Every draw is addressed by its counter, so the result does not depend
    on the chunking or on the order in which chunks run; numpy releases the
    GIL inside its array operations, so chunks run in parallel.
    """
    spans = [(lo, min(_CHUNK, n - lo)) for lo in range(0, n, _CHUNK)]
    if len(spans) <= 1 or _THREADS == 1:
        for lo, m in spans:
            fill(lo, m)
        return
    with ThreadPoolExecutor(_THREADS) as ex:
        list(ex.map(lambda a: fill(*a), spans))


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to a uint64 array."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(stream: int, first: int, count: int) -> np.ndarray:
    """Draws ``first+1 .. first+count`` of a SplitMix64 stream seeded ``stream``."""
    with np.errstate(over="ignore"):
        k = np.arange(first + 1, first + count + 1, dtype=np.uint64)
        return _mix(np.uint64(stream & 0xFFFFFFFFFFFFFFFF) + k * _G)


def stream_seed(seed: int, field: int) -> int:
    """Seed of the independent stream for (workload seed, field id)."""
    with np.errstate(over="ignore"):
        key = np.array([((seed & 0xFFFFFFFFFFFF) << 16) | (field & 0xFFFF)], dtype=np.uint64)
        return int(_mix(key + _G)[0])


def uniform(stream: int, first: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(stream, first, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(stream: int, first_pair: int, count: int) -> np.ndarray:
    """``count`` N(0,1) deviates; pair ``j`` of the stream uses draws 2j, 2j+1."""
    npairs = (count + 1) // 2
    u = uniform(stream, 2 * first_pair, 2 * npairs).reshape(npairs, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    th = 2.0 * np.pi * u[:, 1]
    out = np.empty((npairs, 2))
    out[:, 0] = r * np.cos(th)
    out[:, 1] = r * np.sin(th)
    return out.reshape(-1)[:count]


def _complex_normals(stream: int, first: int, count: int) -> np.ndarray:
    """``count`` complex numbers with independent N(0,1) real and imaginary parts."""
    x = normal(stream, first, 2 * count).reshape(count, 2)
    return x[:, 0] + 1j * x[:, 1]


def _orthonormal_rows(v1: np.ndarray, v2: np.ndarray) -> np.ndarray:
    """SU(3) from two complex 3-vectors per matrix: Gram-Schmidt, third row conj(r1 x r2)."""
    r1 = v1 / np.linalg.norm(v1, axis=1, keepdims=True)
    proj = np.sum(np.conj(r1) * v2, axis=1, keepdims=True)
    r2 = v2 - proj * r1
    r2 = r2 / np.linalg.norm(r2, axis=1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=1)


def random_su3(n: int, seed: int, field: int) -> np.ndarray:
    """``n`` Haar-like random SU(3) matrices, shape (n, 3, 3)."""
    s = stream_seed(seed, field)
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def fill(lo, m):
        z = _complex_normals(s, 6 * lo, 6 * m).reshape(m, 2, 3)
        out[lo:lo + m] = _orthonormal_rows(z[:, 0], z[:, 1])

    _chunked(n, fill)
    return out


# Gell-Mann matrices lambda_1..lambda_8 (standard normalisation tr(l_a l_b) = 2 delta_ab).
_LAMBDA = np.zeros((8, 3, 3), dtype=np.complex128)
_LAMBDA[0][0, 1] = _LAMBDA[0][1, 0] = 1
_LAMBDA[1][0, 1], _LAMBDA[1][1, 0] = -1j, 1j
_LAMBDA[2][0, 0], _LAMBDA[2][1, 1] = 1, -1
_LAMBDA[3][0, 2] = _LAMBDA[3][2, 0] = 1
_LAMBDA[4][0, 2], _LAMBDA[4][2, 0] = -1j, 1j
_LAMBDA[5][1, 2] = _LAMBDA[5][2, 1] = 1
_LAMBDA[6][1, 2], _LAMBDA[6][2, 1] = -1j, 1j
_LAMBDA[7][0, 0] = _LAMBDA[7][1, 1] = 1 / np.sqrt(3)
_LAMBDA[7][2, 2] = -2 / np.sqrt(3)


def _expm_traceless(X: np.ndarray, terms: int = 24) -> np.ndarray:
    """exp(X) for a batch of traceless 3x3 matrices, shape (n, 3, 3).

    By Cayley-Hamilton a traceless 3x3 matrix obeys X^3 = -c X + d 1 with
    c = -tr(X^2)/2 and d = det X, so every power X^k/k! is a_k 1 + b_k X +
    c_k X^2 and the Taylor series reduces to a scalar recurrence on
    (a_k, b_k, c_k).  For ||X|| <= 1.5 the remainder after 24 terms is
    below 1e-20.
    """
    X2 = np.matmul(X, X)
    c = -0.5 * (X2[:, 0, 0] + X2[:, 1, 1] + X2[:, 2, 2])
    d = (X[:, 0, 0] * (X[:, 1, 1] * X[:, 2, 2] - X[:, 1, 2] * X[:, 2, 1])
         - X[:, 0, 1] * (X[:, 1, 0] * X[:, 2, 2] - X[:, 1, 2] * X[:, 2, 0])
         + X[:, 0, 2] * (X[:, 1, 0] * X[:, 2, 1] - X[:, 1, 1] * X[:, 2, 0]))
    a = np.ones_like(c)
    b = np.zeros_like(c)
    q = np.zeros_like(c)
    fa, fb, fq = a.copy(), b.copy(), q.copy()
    for k in range(1, terms + 1):
        a, b, q = q * d / k, (a - q * c) / k, b / k
        fa += a
        fb += b
        fq += q
    E = fb[:, None, None] * X + fq[:, None, None] * X2
    for i in range(3):
        E[:, i, i] += fa
    return E


def near_identity_su3(n: int, seed: int, field: int, eps: float = 0.3) -> np.ndarray:
    """``n`` matrices exp(i*eps*A), A = sum_a w_a lambda_a/2, re-unitarised to SU(3)."""
    s = stream_seed(seed, field)
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def fill(lo, m):
        w = normal(s, 4 * lo, 8 * m).reshape(m, 8)
        A = np.einsum("na,aij->nij", w, _LAMBDA) * 0.5
        U = _expm_traceless(1j * eps * A)
        out[lo:lo + m] = _orthonormal_rows(U[:, 0], U[:, 1])

    _chunked(n, fill)
    return out


def gauge_field(dims, seed: int, kind: str = "random", eps: float = 0.3) -> np.ndarray:
    """Gauge field for a lattice ``dims = (Lx, Ly, Lz, Lt)``, shape (4, V, 3, 3).

    ``kind`` is "random" (random SU(3) per link), "near" (exp(i*eps*A)) or
    "unit" (every link the identity, the free field).
    """
    V = int(np.prod(dims))
    if kind == "unit":
        U = np.zeros((4, V, 3, 3), dtype=np.complex128)
        U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
        return U
    U = np.empty((4, V, 3, 3), dtype=np.complex128)
    for mu in range(4):
        if kind == "random":
            U[mu] = random_su3(V, seed, 16 + mu)
        elif kind == "near":
            U[mu] = near_identity_su3(V, seed, 16 + mu, eps)
        else:
            raise ValueError(f"unknown gauge kind {kind!r}")
    return U


def gaussian_spinor(n: int, seed: int, field: int) -> np.ndarray:
    """``n`` spinors with i.i.d. complex Gaussian components, shape (n, 4, 3)."""
    s = stream_seed(seed, field)
    out = np.empty(n * 12, dtype=np.complex128)

    def fill(lo, m):
        out[lo:lo + m] = _complex_normals(s, lo, m)

    _chunked(n * 12, fill)
    return out.reshape(n, 4, 3)


# Workload seeds: one per lattice configuration, as used by tests and benchmarks.
SEED_SMALL_8 = 1311          # 8^4, random SU(3)
SEED_PROD_32 = 4521          # 32^3x64, near-thermalised
SEED_CG_48 = 2013            # 48^3x96, near-thermalised
SEED_GRAD_24 = 31            # 24^3x48, near-thermalised
SEED_BATCH_LATTICE = 100     # + lattice index k
SEED_BATCH_RHS = 200         # + right-hand side index j
