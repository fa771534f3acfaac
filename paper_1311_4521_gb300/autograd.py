"""torch.autograd Functions over the C ABI: the hopping matrix, Q_tm and the
action S = phi^dag (Q^dag Q)^-1 phi with its gauge-link gradient.

Spinor tensors are complex128 of shape (V/2, 4, 3) (one parity, index
lex/2) and gauge tensors complex128 of shape (4, V, 3, 3) on the CUDA
device.  Every computation runs in the library's kernels: forward through
tm_hopping_eo / tm_Qtm / tm_cg_QdagQ, backward through the adjoint
operators (the daggered hop, Q(-mu) = Q^dag), tm_link_grad and tm_force.

Gradients follow PyTorch's convention for a real loss of complex inputs,
grad = dL/dRe z + i dL/dIm z: for S, dS/dphi = 2 X with X = (Q^dag Q)^-1 phi,
and dS/dU = 2 kappa^2 s (M1^dag + M2) per link (see tm_force).  The action
value, the scaling of the spinor gradient and of the link gradient by the
upstream gradient are library calls too (tm_spinor_dot, tm_scale_complex):
this module only moves buffers between torch and the library.

HoppingEO and Qtm are differentiable in the spinor and in the links: the
link gradient of an operator output with upstream gradient g is the
gradient of Re <g, Op(U) psi>, computed by tm_link_grad with the force
kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tmhop

_contexts: dict = {}


def context(device: int | None = None) -> tmhop.Context:
    """The library context of a CUDA device (created on first use)."""
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = tmhop.Context(d)
    return _contexts[d]


RECON = {"f64": 18, "f32": 12, "f16": 12}


class _Packed:
    """Packs (V/2, 4, 3) complex tensors into the library layout and back."""

    def __init__(self, ctx: tmhop.Context, prec: str):
        self.ctx, self.prec = ctx, prec

    def pack(self, psi: torch.Tensor) -> torch.Tensor:
        return self.ctx.pack(psi.detach(), self.prec)

    def unpack(self, buf: torch.Tensor, vh: int) -> torch.Tensor:
        return self.ctx.unpack(buf, vh, self.prec)


def _gauge(ctx, dims, U, prec, bc):
    return ctx.gauge(dims, U.detach(), prec, RECON[prec], bc)


class HoppingEO(torch.autograd.Function):
    """out = H psi with H = H_eo (direction TM_EO) or H_oe (TM_OE); backward applies H^dag."""

    @staticmethod
    def forward(fctx, psi, U, dims, direction, prec="f64", bc=(-1, 1, 1, 1)):
        ctx = context(psi.device.index)
        pk = _Packed(ctx, prec)
        g = _gauge(ctx, dims, U, prec, bc)
        vh = psi.shape[0]
        out = ctx.empty(vh, prec)
        ctx.hopping_eo(g, out, pk.pack(psi), direction)
        res = pk.unpack(out, vh)
        fctx.save_for_backward(U, psi)
        fctx.cfg = (dims, direction, prec, bc)
        g.close()
        return res

    @staticmethod
    def backward(fctx, grad):
        U, psi = fctx.saved_tensors
        dims, direction, prec, bc = fctx.cfg
        ctx = context(grad.device.index)
        pk = _Packed(ctx, prec)
        g = _gauge(ctx, dims, U, prec, bc)
        vh = grad.shape[0]
        gp = pk.pack(grad.contiguous())
        res = grad_U = None
        if fctx.needs_input_grad[0]:
            out = ctx.empty(vh, prec)
            # (H_eo)^dag maps even -> odd: the daggered hop with odd output, and vice versa
            ctx.hopping_eo(g, out, gp, 1 - direction, dagger=True)
            res = pk.unpack(out, vh)
        if fctx.needs_input_grad[1]:
            op = tmhop.TM_GRAD_HOP_EO if direction == tmhop.TM_EO else tmhop.TM_GRAD_HOP_OE
            grad_U = ctx.link_grad(g, pk.pack(psi), gp, op)
        g.close()
        return res, grad_U, None, None, None, None


class Qtm(torch.autograd.Function):
    """out = Q_tm(mu) psi on even sites; backward applies Q^dag = Q(-mu)."""

    @staticmethod
    def forward(fctx, psi, U, dims, kappa, mu, prec="f64", bc=(-1, 1, 1, 1)):
        ctx = context(psi.device.index)
        pk = _Packed(ctx, prec)
        g = _gauge(ctx, dims, U, prec, bc)
        vh = psi.shape[0]
        out = ctx.empty(vh, prec)
        ctx.Qtm(g, out, pk.pack(psi), kappa, mu, 1)
        res = pk.unpack(out, vh)
        fctx.save_for_backward(U, psi)
        fctx.cfg = (dims, kappa, mu, prec, bc)
        g.close()
        return res

    @staticmethod
    def backward(fctx, grad):
        U, psi = fctx.saved_tensors
        dims, kappa, mu, prec, bc = fctx.cfg
        ctx = context(grad.device.index)
        pk = _Packed(ctx, prec)
        g = _gauge(ctx, dims, U, prec, bc)
        vh = grad.shape[0]
        gp = pk.pack(grad.contiguous())
        res = grad_U = None
        if fctx.needs_input_grad[0]:
            out = ctx.empty(vh, prec)
            ctx.Qtm(g, out, gp, kappa, mu, -1)
            res = pk.unpack(out, vh)
        if fctx.needs_input_grad[1]:
            grad_U = ctx.link_grad(g, pk.pack(psi), gp, tmhop.TM_GRAD_QTM, kappa, mu, 1)
        g.close()
        return res, grad_U, None, None, None, None, None


class Action(torch.autograd.Function):
    """S = phi^dag (Q^dag Q)^-1 phi (a real scalar).

    Forward solves Q^dag Q X = phi with tm_cg_QdagQ (FP64 outer solver; inner
    precision ``inner``: "f64" plain, "f32"/"f16" mixed).  Backward returns
    dS/dphi = 2 X and dS/dU from tm_force in gradient mode, evaluated with
    links and X stored in precision ``force_prec``.
    """

    @staticmethod
    def forward(fctx, phi, U, dims, kappa, mu, tol=1e-10, inner="f64", force_prec="f64", bc=(-1, 1, 1, 1)):
        ctx = context(phi.device.index)
        vh = phi.shape[0]
        gh = _gauge(ctx, dims, U, "f64", bc)
        gl = None if inner == "f64" else _gauge(ctx, dims, U, inner, bc)
        b = ctx.pack(phi.detach(), "f64")
        x = ctx.empty(vh, "f64").zero_()
        st, info = ctx.cg(gh, x, b, kappa, mu, tol, 100000, gl)
        gh.close()
        if gl is not None:
            gl.close()
        if st != tmhop.TM_OK:
            raise tmhop.TmError(st, f"Action: solver failed: {info}")
        X = ctx.unpack(x, vh, "f64")
        dot = torch.empty(2, dtype=torch.float64, device=x.device)
        tmhop.tm_spinor_dot(ctx.handle, vh, b, x, tmhop.TM_F64, dot)   # <phi, X>, real up to rounding
        S = dot[0].clone()
        fctx.save_for_backward(U, X)
        fctx.cfg = (dims, kappa, mu, force_prec, bc)
        return S

    @staticmethod
    def backward(fctx, gS):
        U, X = fctx.saved_tensors
        dims, kappa, mu, force_prec, bc = fctx.cfg
        grad_phi = grad_U = None
        ctx = context(X.device.index)
        gS = gS.detach().to(device=X.device, dtype=torch.float64).contiguous()
        if fctx.needs_input_grad[0]:
            grad_phi = X.clone()      # dS/dphi = 2 X, times the upstream gradient
            tmhop.tm_scale_complex(ctx.handle, grad_phi.numel(), torch.view_as_real(grad_phi), gS, 2.0)
        if fctx.needs_input_grad[1]:
            g = _gauge(ctx, dims, U, force_prec, bc)
            grad_U = ctx.force(g, ctx.pack(X, force_prec), kappa, mu, tmhop.TM_FORCE_GRAD)
            g.close()
            tmhop.tm_scale_complex(ctx.handle, grad_U.numel(), torch.view_as_real(grad_U), gS, 1.0)
        return grad_phi, grad_U, None, None, None, None, None, None, None


def hopping_eo(psi, U, dims, direction, prec="f64", bc=(-1, 1, 1, 1)):
    return HoppingEO.apply(psi, U, tuple(dims), int(direction), prec, tuple(bc))


def qtm(psi, U, dims, kappa, mu, prec="f64", bc=(-1, 1, 1, 1)):
    return Qtm.apply(psi, U, tuple(dims), float(kappa), float(mu), prec, tuple(bc))


def action(phi, U, dims, kappa, mu, tol=1e-10, inner="f64", force_prec="f64", bc=(-1, 1, 1, 1)):
    return Action.apply(phi, U, tuple(dims), float(kappa), float(mu), float(tol), inner, force_prec, tuple(bc))
