"""Plain FP64 CPU oracle for the Wilson twisted-mass operator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the library under
``paper_1311_4521_gb300`` never does.  The arithmetic lives in
``tm_oracle.c`` (plain C99, double complex), compiled here with gcc; it shares
no code with the CUDA path.  See the header of ``tm_oracle.c`` for the
operator definitions and conventions, and for what pins each function.

All arrays are numpy complex128, C-contiguous, in the canonical layouts:
gauge ``U[4, V, 3, 3]`` (mu 0 = t), spinors ``[V, 4, 3]`` (full lattice) or
``[V/2, 4, 3]`` (one parity, index lex/2).  ``dims = (Lx, Ly, Lz, Lt)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ANTIPERIODIC_T = (-1, 1, 1, 1)


def build(force: bool = False) -> str:
    """Compiles ``liboracle.so`` next to its source (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declares the argument and result types of the library's functions."""
    P = ctypes.c_void_p
    I4 = ctypes.POINTER(ctypes.c_int)
    D = ctypes.c_double
    L = ctypes.c_long
    lib.oracle_check_dims.argtypes = [I4]
    lib.oracle_check_dims.restype = ctypes.c_int
    lib.oracle_gammas.argtypes = [P]
    lib.oracle_dhop.argtypes = [I4, I4, P, P, P, ctypes.c_int]
    lib.oracle_dhop_dagger.argtypes = [I4, I4, P, P, P, ctypes.c_int]
    lib.oracle_pack_eo.argtypes = [I4, ctypes.c_int, P, P]
    lib.oracle_unpack_eo.argtypes = [I4, ctypes.c_int, P, P]
    lib.oracle_hopping.argtypes = [I4, I4, P, ctypes.c_int, P, P, ctypes.c_int]
    lib.oracle_gamma5.argtypes = [L, P, P]
    lib.oracle_twist.argtypes = [L, D, P, P]
    lib.oracle_twist_inv.argtypes = [L, D, P, P]
    lib.oracle_Qtm.argtypes = [I4, I4, P, D, D, P, P]
    lib.oracle_Qtm_dagger.argtypes = [I4, I4, P, D, D, P, P]
    lib.oracle_Qnd.argtypes = [I4, I4, P, D, D, D, P, P, P, P]
    lib.oracle_Qnd.restype = ctypes.c_int
    lib.oracle_clover_site.argtypes = [I4, P, D, D, L, P]
    lib.oracle_Qsw.argtypes = [I4, I4, P, D, D, D, P, P]
    lib.oracle_Qsw.restype = ctypes.c_int
    lib.oracle_cg_QdagQ.argtypes = [I4, I4, P, D, D, P, P, D, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(D)]
    lib.oracle_cg_QdagQ.restype = ctypes.c_int
    lib.oracle_force.argtypes = [I4, I4, P, D, D, P, ctypes.c_int, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _i4(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _c(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def check_dims(dims) -> bool:
    return bool(_load().oracle_check_dims(_i4(dims)))


def gammas() -> np.ndarray:
    """gamma_0..gamma_3 and gamma_5 as a (5, 4, 4) complex array."""
    g = np.zeros((5, 4, 4), dtype=np.complex128)
    _load().oracle_gammas(_p(g))
    return g


def dhop(dims, U, psi, out_parity=-1, bc=ANTIPERIODIC_T, dagger=False):
    """Dhop psi (or Dhop^dagger psi) on the full lattice, kept at out_parity sites."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    f = _load().oracle_dhop_dagger if dagger else _load().oracle_dhop
    f(_i4(dims), _i4(bc), _p(U), _p(psi), _p(out), int(out_parity))
    return out


def pack_eo(dims, full, parity):
    full = _c(full)
    eo = np.empty((full.shape[0] // 2, 4, 3), dtype=np.complex128)
    _load().oracle_pack_eo(_i4(dims), int(parity), _p(full), _p(eo))
    return eo


def unpack_eo(dims, eo, parity):
    eo = _c(eo)
    full = np.empty((eo.shape[0] * 2, 4, 3), dtype=np.complex128)
    _load().oracle_unpack_eo(_i4(dims), int(parity), _p(eo), _p(full))
    return full


def hopping(dims, U, in_eo, out_parity, bc=ANTIPERIODIC_T, dagger=False):
    """H_eo (out_parity 0) or H_oe (out_parity 1) on even-odd packed fields."""
    U, in_eo = _c(U), _c(in_eo)
    out = np.empty_like(in_eo)
    _load().oracle_hopping(_i4(dims), _i4(bc), _p(U), int(out_parity), _p(in_eo), _p(out), int(bool(dagger)))
    return out


def gamma5(psi):
    psi = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_gamma5(psi.shape[0], _p(psi), _p(out))
    return out


def twist(psi, mut):
    """(1 + i mut gamma5) psi."""
    psi = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_twist(psi.shape[0], float(mut), _p(psi), _p(out))
    return out


def twist_inv(psi, mut):
    """(1 + i mut gamma5)^-1 psi."""
    psi = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_twist_inv(psi.shape[0], float(mut), _p(psi), _p(out))
    return out


def Qtm(dims, U, psi_e, kappa, mu, bc=ANTIPERIODIC_T, dagger=False):
    """Q_tm psi_e (or its literal adjoint) on even-site packed fields."""
    U, psi_e = _c(U), _c(psi_e)
    out = np.empty_like(psi_e)
    f = _load().oracle_Qtm_dagger if dagger else _load().oracle_Qtm
    f(_i4(dims), _i4(bc), _p(U), float(kappa), float(mu), _p(psi_e), _p(out))
    return out


def Qnd(dims, U, psi_s, psi_c, kappa, mu_sigma, mu_delta, bc=ANTIPERIODIC_T):
    """The non-degenerate twisted doublet Q_nd on an even-site doublet (psi_s, psi_c);
    returns (out_s, out_c).  Raises ValueError if M_oo is singular."""
    U, psi_s, psi_c = _c(U), _c(psi_s), _c(psi_c)
    out_s, out_c = np.empty_like(psi_s), np.empty_like(psi_c)
    ok = _load().oracle_Qnd(_i4(dims), _i4(bc), _p(U), float(kappa), float(mu_sigma), float(mu_delta),
                            _p(psi_s), _p(psi_c), _p(out_s), _p(out_c))
    if not ok:
        raise ValueError("Qnd: the site-local matrix M_oo is singular")
    return out_s, out_c


def clover_site(dims, U, csw, kappa, lex):
    """The clover term T(x) = csw kappa i sum_{mu<nu} sigma_munu F_munu(x) at site lex, 12x12 (spin*3+colour)."""
    U = _c(U)
    T = np.empty((12, 12), dtype=np.complex128)
    _load().oracle_clover_site(_i4(dims), _p(U), float(csw), float(kappa), int(lex), _p(T))
    return T


def Qsw(dims, U, psi_e, kappa, mu, csw, bc=ANTIPERIODIC_T):
    """The clover twisted-mass operator Q_sw on an even-site field.  Raises ValueError if A_oo is singular."""
    U, psi_e = _c(U), _c(psi_e)
    out = np.empty_like(psi_e)
    if not _load().oracle_Qsw(_i4(dims), _i4(bc), _p(U), float(kappa), float(mu), float(csw), _p(psi_e), _p(out)):
        raise ValueError("Qsw: a site matrix A_oo is singular")
    return out


def cg_QdagQ(dims, U, b_e, kappa, mu, tol=1e-10, maxiter=10000, x0=None, bc=ANTIPERIODIC_T):
    """FP64 CG for Q^dag Q x = b.  Returns (x, iterations, true relative residual, converged)."""
    U, b_e = _c(U), _c(b_e)
    x = np.zeros_like(b_e) if x0 is None else _c(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = _load().oracle_cg_QdagQ(_i4(dims), _i4(bc), _p(U), float(kappa), float(mu), _p(b_e), _p(x),
                                 float(tol), int(maxiter), ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value, st == 0


def force(dims, U, X_e, kappa, mu, links=None, bc=ANTIPERIODIC_T):
    """su(3) force of S = phi^dag (Q^dag Q)^-1 phi for the links (mu, lex) given X = (Q^dag Q)^-1 phi.

    ``links=None`` evaluates every link; the result is then shaped (4, V, 3, 3),
    otherwise (len(links), 3, 3).
    """
    U, X_e = _c(U), _c(X_e)
    V = U.shape[1]
    if links is None:
        mus, sites = np.meshgrid(np.arange(4), np.arange(V), indexing="ij")
        lk = np.stack([mus.ravel(), sites.ravel()], axis=1).astype(np.int32)
    else:
        lk = np.ascontiguousarray(np.asarray(links, dtype=np.int32).reshape(-1, 2))
    F = np.zeros((lk.shape[0], 3, 3), dtype=np.complex128)
    _load().oracle_force(_i4(dims), _i4(bc), _p(U), float(kappa), float(mu), _p(X_e), lk.shape[0], _p(lk), _p(F))
    return F.reshape(4, V, 3, 3) if links is None else F


def action(dims, U, phi_e, kappa, mu, tol=1e-13, maxiter=100000, bc=ANTIPERIODIC_T):
    """S = phi^dag (Q^dag Q)^-1 phi by the oracle CG, and the solution X."""
    X, _, _, ok = cg_QdagQ(dims, U, phi_e, kappa, mu, tol=tol, maxiter=maxiter, bc=bc)
    return float(np.real(np.vdot(phi_e, X))), X
