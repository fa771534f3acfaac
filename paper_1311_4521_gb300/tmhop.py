"""Thin ctypes binding of ``libtmhop.so`` (the C ABI declared in include/tmhop.h).

Functions keep the C names and argument order; they only marshal pointers
and sizes and turn a non-zero ``tm_status`` into :class:`TmError`.  Every
step of the computation runs in the library's CUDA kernels.  PyTorch is
used for device memory and the current stream only.

If the shared library has not been built the import fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtmhop.so")

TM_OK, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_NOT_CONVERGED, TM_ERR_NONFINITE, TM_ERR_TIMEOUT, TM_ERR_UNSUPPORTED = range(7)
TM_F64, TM_F32, TM_F16, TM_F64X = 0, 1, 2, 3
TM_EO, TM_OE = 0, 1
TM_FORCE_SU3, TM_FORCE_GRAD = 0, 1
TM_FORCE_OWNER, TM_FORCE_ATOMIC, TM_FORCE_HALO = 0, 1, 2
TM_SLAB_INTERIOR, TM_SLAB_BOUNDARY, TM_SLAB_ALL = 1, 2, 3
TM_GRAD_QTM, TM_GRAD_HOP_EO, TM_GRAD_HOP_OE = 0, 1, 2
TM_SLAB_HOP, TM_SLAB_QTM_A, TM_SLAB_QTM_B = 0, 1, 2
PREC = {"f64": TM_F64, "f32": TM_F32, "f16": TM_F16, "f64x": TM_F64X}


class CgParams(ctypes.Structure):
    """tm_cg_params."""
    _fields_ = [("kappa", ctypes.c_double), ("mu", ctypes.c_double), ("tol", ctypes.c_double),
                ("maxiter", ctypes.c_int), ("reliable_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("reliable_delta", ctypes.c_double)]


class CgInfo(ctypes.Structure):
    """tm_cg_info."""
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_relres", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class TmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1311_4521_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, L, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_size_t
    I4 = ctypes.POINTER(ctypes.c_int)
    sig = {
        "tm_ctx_create": ([ctypes.POINTER(P), I], I),
        "tm_ctx_destroy": ([P], None),
        "tm_last_error": ([P], ctypes.c_char_p),
        "tm_status_string": ([I], ctypes.c_char_p),
        "tm_ctx_trace": ([P, P, I], I),
        "tm_spinor_bytes": ([L, I], S),
        "tm_spinor_pack": ([P, L, P, P, I, P], I),
        "tm_spinor_unpack": ([P, L, P, P, I, P], I),
        "tm_gauge_create": ([P, I4, P, I, I, I4, P, ctypes.POINTER(P)], I),
        "tm_gauge_destroy": ([P], None),
        "tm_gauge_bytes": ([P], S),
        "tm_hopping_eo": ([P, P, P, P, I, I, P], I),
        "tm_Qtm": ([P, P, P, P, D, D, I, P], I),
        "tm_Qtm_noalloc": ([P, P, P, P, D, D, I, P], I),
        "tm_cg_QdagQ": ([P, P, P, P, P, ctypes.POINTER(CgParams), ctypes.POINTER(CgInfo), P], I),
        "tm_ctx_set_autotune": ([P, I], I),
        "tm_ctx_tune_report": ([P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_size_t),
        "tm_force": ([P, P, P, P, D, D, I, P], I),
        "tm_force_ex": ([P, P, P, P, D, D, I, I, P], I),
        "tm_solve_eo": ([P, P, P, P, P, P, P, ctypes.POINTER(CgParams), ctypes.POINTER(CgInfo), P], I),
        "tm_Qtm_batch": ([P, I, P, P, P, D, D, I, P], I),
        "tm_Qtm_host": ([P, P, I, P, P, D, D, I, P], I),
        "tm_cg_QdagQ_batch": ([P, I, P, P, P, P, ctypes.POINTER(CgParams), P, P], I),
        "tm_probe_fma": ([P, I, ctypes.POINTER(D), P], I),
        "tm_spinor_dot": ([P, L, P, P, I, P, P], I),
        "tm_scale_complex": ([P, S, P, P, D, P], I),
        "tm_ctx_device_bytes": ([P], S),
        "tm_slab_face_bytes": ([P], S),
        "tm_ctx_set_tune_cache": ([P, ctypes.c_char_p], I),
        "tm_Qnd": ([P, P, P, P, P, P, D, D, D, I, P], I),
        "tm_link_grad": ([P, P, P, P, P, I, D, D, I, P], I),
        "tm_ctx_check": ([P], I),
        "tm_ctx_selftest_wait": ([P, P], I),
        "tm_clover_create": ([P, P, P, D, D, D, P, ctypes.POINTER(P)], I),
        "tm_clover_destroy": ([P], None),
        "tm_clover_bytes": ([P], S),
        "tm_Qsw": ([P, P, P, P, P, I, P], I),
        "tm_ctx_set_batch_config": ([P, I, ctypes.c_uint], I),
        "tm_gauge_tune": ([P, P, P], I),
        "tm_gauge_set_map": ([P, P, ctypes.c_char_p], I),
        "tm_gauge_map": ([P, ctypes.c_char_p, S], S),
        "tm_slab_pack": ([P, P, P, I, I, P, P, P], I),
        "tm_slab_hop": ([P, P, P, P, P, P, I, I, I, I, D, D, I, P, I, I, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _i4(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t) -> ctypes.c_void_p:
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t) if t is not None else 0)


def _check(ctx_handle, status: int):
    if status != TM_OK:
        msg = lib.tm_last_error(ctx_handle).decode() if ctx_handle else ""
        raise TmError(status, msg or lib.tm_status_string(status).decode())


# ---- C-named functions -------------------------------------------------------
def tm_ctx_create(device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    st = lib.tm_ctx_create(ctypes.byref(h), int(device))
    if st != TM_OK:
        raise TmError(st, f"tm_ctx_create(device={device}): {lib.tm_status_string(st).decode()}")
    return h


def tm_ctx_destroy(ctx) -> None:
    lib.tm_ctx_destroy(ctx)


def tm_last_error(ctx) -> str:
    return lib.tm_last_error(ctx).decode()


def tm_status_string(status: int) -> str:
    return lib.tm_status_string(int(status)).decode()


def tm_ctx_trace(ctx, events) -> None:
    """Records the given torch.cuda.Event objects at kernel boundaries (None stops)."""
    if events is None:
        _check(ctx, lib.tm_ctx_trace(ctx, None, 0))
        return
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    _check(ctx, lib.tm_ctx_trace(ctx, arr, len(events)))


def tm_spinor_bytes(vh: int, prec: int) -> int:
    return int(lib.tm_spinor_bytes(int(vh), int(prec)))


def tm_spinor_pack(ctx, vh, in_dev, out_dev, prec, stream=None):
    _check(ctx, lib.tm_spinor_pack(ctx, int(vh), _ptr(in_dev), _ptr(out_dev), int(prec), _stream(stream)))


def tm_spinor_unpack(ctx, vh, in_dev, out_dev, prec, stream=None):
    _check(ctx, lib.tm_spinor_unpack(ctx, int(vh), _ptr(in_dev), _ptr(out_dev), int(prec), _stream(stream)))


def tm_gauge_create(ctx, dims, U_dev, prec, reconstruct, bc, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(ctx, lib.tm_gauge_create(ctx, _i4(dims), _ptr(U_dev), int(prec), int(reconstruct), _i4(bc),
                                    _stream(stream), ctypes.byref(h)))
    return h


def tm_gauge_destroy(g) -> None:
    lib.tm_gauge_destroy(g)


def tm_gauge_bytes(g) -> int:
    return int(lib.tm_gauge_bytes(g))


def tm_hopping_eo(ctx, U, out_dev, in_dev, dir, dagger=0, stream=None):
    _check(ctx, lib.tm_hopping_eo(ctx, U, _ptr(out_dev), _ptr(in_dev), int(dir), int(dagger), _stream(stream)))


def tm_Qtm(ctx, U, out_e_dev, in_e_dev, kappa, mu, sign=1, stream=None):
    _check(ctx, lib.tm_Qtm(ctx, U, _ptr(out_e_dev), _ptr(in_e_dev), float(kappa), float(mu), int(sign),
                           _stream(stream)))


def tm_cg_QdagQ(ctx, U_hi, U_lo, x_dev, b_dev, params: CgParams, stream=None):
    """Runs the solver; returns (status, CgInfo).  Raises TmError for argument and CUDA errors only:
    TM_ERR_NOT_CONVERGED and TM_ERR_NONFINITE come back as the status."""
    info = CgInfo()
    st = lib.tm_cg_QdagQ(ctx, U_hi, U_lo, _ptr(x_dev), _ptr(b_dev), ctypes.byref(params), ctypes.byref(info),
                         _stream(stream))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED, TM_ERR_NONFINITE):
        _check(ctx, st)
    return st, info


def tm_solve_eo(ctx, U_hi, U_lo, x_e, x_o, b_e, b_o, params: CgParams, stream=None):
    """Full-lattice solve M x = b; returns (status, CgInfo of the even-site solve)."""
    info = CgInfo()
    st = lib.tm_solve_eo(ctx, U_hi, U_lo, _ptr(x_e), _ptr(x_o), _ptr(b_e), _ptr(b_o), ctypes.byref(params),
                         ctypes.byref(info), _stream(stream))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED, TM_ERR_NONFINITE):
        _check(ctx, st)
    return st, info


def tm_force(ctx, U, F_dev, X_e_dev, kappa, mu, mode=TM_FORCE_SU3, stream=None):
    _check(ctx, lib.tm_force(ctx, U, _ptr(F_dev), _ptr(X_e_dev), float(kappa), float(mu), int(mode), _stream(stream)))


def tm_force_ex(ctx, U, F_dev, X_e_dev, kappa, mu, mode=TM_FORCE_SU3, scheme=TM_FORCE_OWNER, stream=None):
    _check(ctx, lib.tm_force_ex(ctx, U, _ptr(F_dev), _ptr(X_e_dev), float(kappa), float(mu), int(mode), int(scheme),
                                _stream(stream)))


def tm_ctx_set_autotune(ctx, on: bool) -> None:
    _check(ctx, lib.tm_ctx_set_autotune(ctx, int(bool(on))))


def tm_ctx_tune_report(ctx) -> str:
    """The launch configurations the context's autotuner has chosen, one line per batch shape."""
    n = lib.tm_ctx_tune_report(ctx, None, 0)
    buf = ctypes.create_string_buffer(n)
    lib.tm_ctx_tune_report(ctx, buf, n)
    return buf.value.decode()


def _parr(items):
    return (ctypes.c_void_p * len(items))(*[(_ptr(t).value or 0) if not isinstance(t, ctypes.c_void_p) else t.value
                                            for t in items])


def tm_Qtm_batch(ctx, gauges, outs, ins, kappa, mu, sign=1, stream=None):
    """gauges: list of gauge handles (ctypes pointers), outs/ins: lists of device buffers."""
    n = len(gauges)
    _check(ctx, lib.tm_Qtm_batch(ctx, n, _parr(gauges), _parr(outs), _parr(ins), float(kappa), float(mu), int(sign),
                                 _stream(stream)))


def tm_Qtm_host(ctx, U, outs_host, ins_host, kappa, mu, sign=1, stream=None):
    """Q_tm on host-resident fields: outs_host[k] = Q ins_host[k] (host buffers of complex double
    [Vh][4][3]; pinned for overlapped copies).  Synchronous."""
    n = len(ins_host)
    if len(outs_host) != n:
        raise ValueError("tm_Qtm_host: as many outputs as inputs")
    _check(ctx, lib.tm_Qtm_host(ctx, U, n, _parr(outs_host), _parr(ins_host), float(kappa), float(mu), int(sign),
                                _stream(stream)))


def tm_cg_QdagQ_batch(ctx, U_hi, U_lo, xs, bs, params: CgParams, stream=None):
    """Returns (status, [CgInfo per system]); raises only for argument and CUDA errors."""
    n = len(U_hi)
    infos = (CgInfo * n)()
    lo = _parr(U_lo) if U_lo is not None else None
    st = lib.tm_cg_QdagQ_batch(ctx, n, _parr(U_hi), lo, _parr(xs), _parr(bs), ctypes.byref(params), infos,
                               _stream(stream))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED, TM_ERR_NONFINITE):
        _check(ctx, st)
    return st, list(infos)


def tm_Qtm_noalloc(ctx, U, out_e_dev, in_e_dev, kappa, mu, sign=1, stream=None):
    """tm_Qtm with its temporary in the library's static device array: no device allocation."""
    _check(ctx, lib.tm_Qtm_noalloc(ctx, U, _ptr(out_e_dev), _ptr(in_e_dev), float(kappa), float(mu), int(sign),
                                   _stream(stream)))


TM_QTM_NOALLOC_MAX_BYTES = 32 << 20


def tm_probe_fma(ctx, prec=TM_F64, stream=None) -> float:
    """Measured FMA throughput of the device in TFLOP/s (prec TM_F64 or TM_F32).  Synchronous."""
    out = ctypes.c_double()
    _check(ctx, lib.tm_probe_fma(ctx, int(prec), ctypes.byref(out), _stream(stream)))
    return out.value


def tm_spinor_dot(ctx, vh, a_dev, b_dev, prec, out_dev, stream=None):
    """out_dev (two device doubles) = <a, b> of two packed fields, FP64, fixed summation order."""
    _check(ctx, lib.tm_spinor_dot(ctx, int(vh), _ptr(a_dev), _ptr(b_dev), int(prec), _ptr(out_dev),
                                  _stream(stream)))


def tm_scale_complex(ctx, n, z_dev, alpha_dev, c, stream=None):
    """z <- c * alpha * z for n complex doubles in device memory (alpha_dev: device double or None)."""
    _check(ctx, lib.tm_scale_complex(ctx, int(n), _ptr(z_dev), _ptr(alpha_dev), float(c), _stream(stream)))


def tm_Qnd(ctx, U, out_s, out_c, in_s, in_c, kappa, mu_sigma, mu_delta, sign=1, stream=None):
    """The non-degenerate twisted doublet on packed even fields (see include/tmhop.h)."""
    _check(ctx, lib.tm_Qnd(ctx, U, _ptr(out_s), _ptr(out_c), _ptr(in_s), _ptr(in_c), float(kappa), float(mu_sigma),
                           float(mu_delta), int(sign), _stream(stream)))


def tm_ctx_check(ctx):
    """Raises TmError if a bounded device wait of the context ran out since the last check."""
    _check(ctx, lib.tm_ctx_check(ctx))


def tm_ctx_selftest_wait(ctx, stream=None):
    """Enqueues the bounded-wait test kernel (a wait that runs out after about a second)."""
    _check(ctx, lib.tm_ctx_selftest_wait(ctx, _stream(stream)))


def tm_link_grad(ctx, U, G_dev, X_dev, Y_dev, op, kappa=0.0, mu=0.0, sign=1, stream=None):
    """G_dev <- gradient w.r.t. the complex links of Re <Y, Op X> (op: TM_GRAD_QTM / _HOP_EO / _HOP_OE)."""
    _check(ctx, lib.tm_link_grad(ctx, U, _ptr(G_dev), _ptr(X_dev), _ptr(Y_dev), int(op), float(kappa), float(mu),
                                 int(sign), _stream(stream)))


def tm_clover_create(ctx, U, U_dev, csw, kappa, mu, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(ctx, lib.tm_clover_create(ctx, U, _ptr(U_dev), float(csw), float(kappa), float(mu), _stream(stream),
                                     ctypes.byref(h)))
    return h


def tm_clover_destroy(C) -> None:
    lib.tm_clover_destroy(C)


def tm_clover_bytes(C) -> int:
    return int(lib.tm_clover_bytes(C))


def tm_Qsw(ctx, U, C, out_e_dev, in_e_dev, sign=1, stream=None):
    _check(ctx, lib.tm_Qsw(ctx, U, C, _ptr(out_e_dev), _ptr(in_e_dev), int(sign), _stream(stream)))


def tm_ctx_set_tune_cache(ctx, path) -> None:
    """Autotune cache file of the context (None: no file)."""
    _check(ctx, lib.tm_ctx_set_tune_cache(ctx, None if path is None else str(path).encode()))


def tm_ctx_set_batch_config(ctx, code: int, cap: int = 0) -> None:
    """Fixes the batched hop's configuration (code -1: back to the autotuner)."""
    _check(ctx, lib.tm_ctx_set_batch_config(ctx, int(code), int(cap)))


def tm_gauge_tune(ctx, U, stream=None) -> None:
    """Chooses the hop's site-to-thread map for the handle's lattice (cache, else timing)."""
    _check(ctx, lib.tm_gauge_tune(ctx, U, _stream(stream)))


def tm_gauge_set_map(ctx, U, name: str) -> None:
    _check(ctx, lib.tm_gauge_set_map(ctx, U, name.encode()))


def tm_gauge_map(U) -> str:
    """Name of the handle's current site-to-thread map."""
    n = lib.tm_gauge_map(U, None, 0)
    buf = ctypes.create_string_buffer(n)
    lib.tm_gauge_map(U, buf, n)
    return buf.value.decode()


def tm_slab_face_bytes(U) -> int:
    """Bytes of one face of the slab whose gauge handle is U."""
    return int(lib.tm_slab_face_bytes(U))


def tm_slab_pack(ctx, U, in_dev, dir, dagger, send_lower_dev, send_upper_dev, stream=None):
    _check(ctx, lib.tm_slab_pack(ctx, U, _ptr(in_dev), int(dir), int(dagger), _ptr(send_lower_dev),
                                 _ptr(send_upper_dev), _stream(stream)))


def tm_slab_hop(ctx, U, out_dev, in_dev, recv_lower_dev, recv_upper_dev, dir, dagger, region, op, kappa=0.0,
                mu=0.0, sign=1, x_dev=None, sign_lower=1, sign_upper=1, stream=None):
    _check(ctx, lib.tm_slab_hop(ctx, U, _ptr(out_dev), _ptr(in_dev), _ptr(recv_lower_dev), _ptr(recv_upper_dev),
                                int(dir), int(dagger), int(region), int(op), float(kappa), float(mu), int(sign),
                                _ptr(x_dev), int(sign_lower), int(sign_upper), _stream(stream)))


def tm_ctx_device_bytes(ctx) -> int:
    """Bytes of device memory the context holds (not counting gauge handles)."""
    return int(lib.tm_ctx_device_bytes(ctx))


# ---- convenience layer over torch tensors -----------------------------------------
class Gauge:
    """A gauge handle: the library's packed copy of U in one precision."""

    def __init__(self, ctx: "Context", dims, U: torch.Tensor, prec="f64", reconstruct=18, bc=(-1, 1, 1, 1)):
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        self.reconstruct = int(reconstruct)
        self.bc = tuple(bc)
        self.vh = int(np.prod(self.dims)) // 2
        Ur = _as_real_dev(U, ctx.device)
        self.handle = tm_gauge_create(ctx.handle, self.dims, Ur, self.prec, self.reconstruct, self.bc)

    @property
    def nbytes(self) -> int:
        return tm_gauge_bytes(self.handle)

    def close(self):
        if self.handle:
            tm_gauge_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_real_dev(t: torch.Tensor, device) -> torch.Tensor:
    """complex128 tensor -> contiguous float64 view on the device (re, im interleaved)."""
    if not isinstance(t, torch.Tensor):
        t = torch.from_numpy(np.ascontiguousarray(t))
    t = t.to(device=device, dtype=torch.complex128).contiguous()
    return torch.view_as_real(t).contiguous()


class Context:
    """Owns a ``tm_ctx`` on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.handle = tm_ctx_create(device)

    def close(self):
        if self.handle:
            tm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # fields
    def gauge(self, dims, U, prec="f64", reconstruct=18, bc=(-1, 1, 1, 1)) -> Gauge:
        return Gauge(self, dims, U, prec, reconstruct, bc)

    def empty(self, vh: int, prec) -> torch.Tensor:
        prec = PREC[prec] if isinstance(prec, str) else int(prec)
        return torch.empty(tm_spinor_bytes(vh, prec), dtype=torch.uint8, device=self.device)

    def pack(self, psi, prec) -> torch.Tensor:
        """(Vh, 4, 3) complex spinors -> packed field of precision ``prec``."""
        prec = PREC[prec] if isinstance(prec, str) else int(prec)
        src = _as_real_dev(psi, self.device)
        vh = src.shape[0]
        out = self.empty(vh, prec)
        tm_spinor_pack(self.handle, vh, src, out, prec)
        return out

    def unpack(self, buf: torch.Tensor, vh: int, prec) -> torch.Tensor:
        prec = PREC[prec] if isinstance(prec, str) else int(prec)
        out = torch.empty((vh, 4, 3, 2), dtype=torch.float64, device=self.device)
        tm_spinor_unpack(self.handle, vh, buf, out, prec)
        return torch.view_as_complex(out)

    # operator
    def hopping_eo(self, U: Gauge, out, inp, dir, dagger=False):
        tm_hopping_eo(self.handle, U.handle, out, inp, dir, int(bool(dagger)))
        return out

    def Qtm(self, U: Gauge, out, inp, kappa, mu, sign=1):
        tm_Qtm(self.handle, U.handle, out, inp, kappa, mu, sign)
        return out

    def solve_eo(self, U_hi: Gauge, x_e, x_o, b_e, b_o, kappa, mu, tol=1e-10, maxiter=30000,
                 U_lo: Gauge | None = None, reliable_every=50, use_graph=True, reliable_delta=-1.0):
        prm = CgParams(float(kappa), float(mu), float(tol), int(maxiter), int(reliable_every), int(bool(use_graph)),
                       float(reliable_delta))
        st, info = tm_solve_eo(self.handle, U_hi.handle, U_lo.handle if U_lo is not None else None,
                               x_e, x_o, b_e, b_o, prm)
        return st, info.as_dict()

    def force(self, U: Gauge, X_e, kappa, mu, mode=TM_FORCE_SU3, scheme=TM_FORCE_OWNER) -> torch.Tensor:
        """Force (or complex gradient) of S = phi^dag (Q^dag Q)^-1 phi given packed X; (4, V, 3, 3) complex128."""
        V = 2 * U.vh
        F = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=self.device)
        tm_force_ex(self.handle, U.handle, F, X_e, kappa, mu, mode, scheme)
        return torch.view_as_complex(F)

    def Qnd(self, U: Gauge, outs, ins, kappa, mu_sigma, mu_delta, sign=1):
        """(out_s, out_c) = Q_nd (in_s, in_c) on packed even fields."""
        tm_Qnd(self.handle, U.handle, outs[0], outs[1], ins[0], ins[1], kappa, mu_sigma, mu_delta, sign)
        return outs

    def link_grad(self, U: Gauge, X, Y, op, kappa=0.0, mu=0.0, sign=1) -> torch.Tensor:
        """Gradient w.r.t. the complex links of Re <Y, Op X> for packed X, Y; (4, V, 3, 3) complex128."""
        G = torch.empty((4, 2 * U.vh, 3, 3, 2), dtype=torch.float64, device=self.device)
        tm_link_grad(self.handle, U.handle, G, X, Y, op, kappa, mu, sign)
        return torch.view_as_complex(G)

    def clover(self, U: Gauge, U_field, csw, kappa, mu) -> ctypes.c_void_p:
        """Clover blocks for gauge handle U (U_field: the same links, complex128 (4, V, 3, 3))."""
        return tm_clover_create(self.handle, U.handle, _as_real_dev(U_field, self.device), csw, kappa, mu)

    def Qsw(self, U: Gauge, C, out, inp, sign=1):
        tm_Qsw(self.handle, U.handle, C, out, inp, sign)
        return out

    def Qtm_host(self, U: Gauge, outs, ins, kappa, mu, sign=1):
        """Q_tm on host tensors (complex128 [Vh, 4, 3], contiguous, on the CPU; pin them for overlap)."""
        for t in list(outs) + list(ins):
            if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.complex128
                    and t.is_contiguous() and t.numel() == 12 * U.vh):
                raise ValueError("Qtm_host: fields must be contiguous complex128 CPU tensors of Vh x 4 x 3")
        tm_Qtm_host(self.handle, U.handle, outs, ins, kappa, mu, sign)
        return outs

    def Qtm_batch(self, gauges, outs, ins, kappa, mu, sign=1):
        tm_Qtm_batch(self.handle, [g.handle for g in gauges], outs, ins, kappa, mu, sign)
        return outs

    def cg_batch(self, U_hi, xs, bs, kappa, mu, tol=1e-10, maxiter=30000, U_lo=None, reliable_every=50,
                 use_graph=True, reliable_delta=-1.0):
        """Solves Q^dag Q x[k] = b[k] for all k at once.  Returns (status, [info dict per system])."""
        prm = CgParams(float(kappa), float(mu), float(tol), int(maxiter), int(reliable_every), int(bool(use_graph)),
                       float(reliable_delta))
        st, infos = tm_cg_QdagQ_batch(self.handle, [g.handle for g in U_hi],
                                      [g.handle for g in U_lo] if U_lo is not None else None, xs, bs, prm)
        return st, [i.as_dict() for i in infos]

    def cg(self, U_hi: Gauge, x, b, kappa, mu, tol=1e-10, maxiter=30000, U_lo: Gauge | None = None,
           reliable_every=50, use_graph=True, reliable_delta=-1.0):
        """Solves Q^dag Q x = b (x: packed FP64 even field, in/out).  Returns (status, info dict)."""
        prm = CgParams(float(kappa), float(mu), float(tol), int(maxiter), int(reliable_every), int(bool(use_graph)),
                       float(reliable_delta))
        st, info = tm_cg_QdagQ(self.handle, U_hi.handle, U_lo.handle if U_lo is not None else None, x, b, prm)
        return st, info.as_dict()
