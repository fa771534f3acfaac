"""A lattice cut along time into slabs, one per GPU: geometry, face
exchange and the Q_tm / hop schedule over the slab entry points of the C
ABI (tm_slab_pack, tm_slab_hop).

This is the GPU form of the paper's Sec. 2.5: the hopping matrix of a
distributed lattice splits into the surface (here the two time faces of a
slab) and the body; the projected half-spinors of the surface are
exchanged while the body (the slab's interior time slices) is computed.
The schedule of one hop on every slab is

    pack faces of the input (stream s)  ->  exchange (comm stream, after s)
    interior hop (stream s, overlaps the exchange)
    face-site hop (stream s, after the exchange)

and Q_tm is two such hops (stage A into an odd temporary, stage B with the
even input re-read).  Two transports move the faces: ``LocalSlabs`` keeps
every slab of a lattice on one device in one process (the faces move by
device-to-device copies on a separate stream: the one-GPU form, used by
the tests), ``DistributedSlabs`` has one slab per process and moves faces
with torch.distributed point-to-point messages (NCCL between GPUs).  Only
bookkeeping lives here: every arithmetic step runs in the library.

The geometry and the collective steps are in slab_geometry.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tmhop
from .slab_geometry import SlabGeometry, exchange_faces, split


class _SlabState:
    """Device buffers of one slab: gauge handle, odd temporary, four faces."""

    def __init__(self, ctx: tmhop.Context, geo: SlabGeometry, U, prec: str, recon: int, bc):
        self.geo = geo
        self.prec = prec
        lbc = (1,) + tuple(bc[1:])          # the slab's own t wrap is never used across a face
        self.gauge = ctx.gauge(geo.local_dims, geo.links(U), prec, recon, lbc)
        nb = tmhop.tm_slab_face_bytes(self.gauge.handle)
        if nb == 0:
            raise tmhop.TmError(tmhop.TM_ERR_UNSUPPORTED, f"slabs do not support {prec} storage")
        dev = ctx.device
        self.send_lower, self.send_upper, self.recv_lower, self.recv_upper = (
            torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(4))
        self.tmp = ctx.empty(geo.vh, prec)

    def close(self):
        self.gauge.close()


class _Schedule:
    """The hop and Q_tm schedule shared by the transports; a subclass
    provides ``_exchange(states, stream)`` which fills every recv face from
    the matching send faces and orders it after `stream`'s work so far and
    before what `stream` does after the returned event."""

    def _hops(self, states, outs, ins, direction, dagger, op, kappa=0.0, mu=0.0, sign=1, xs=None):
        ctx = self.ctx
        s = torch.cuda.current_stream(ctx.device)
        for st, inp in zip(states, ins):
            tmhop.tm_slab_pack(ctx.handle, st.gauge.handle, inp, direction, dagger, st.send_lower, st.send_upper, s)
        done = self._exchange(states, s)
        for k, (st, out, inp) in enumerate(zip(states, outs, ins)):
            tmhop.tm_slab_hop(ctx.handle, st.gauge.handle, out, inp, None, None, direction, dagger,
                              tmhop.TM_SLAB_INTERIOR, op, kappa, mu, sign, xs[k] if xs else None, 1, 1, s)
        s.wait_event(done)
        for k, (st, out, inp) in enumerate(zip(states, outs, ins)):
            tmhop.tm_slab_hop(ctx.handle, st.gauge.handle, out, inp, st.recv_lower, st.recv_upper, direction, dagger,
                              tmhop.TM_SLAB_BOUNDARY, op, kappa, mu, sign, xs[k] if xs else None,
                              st.geo.sign_lower, st.geo.sign_upper, s)

    def _qtm(self, states, outs, ins, kappa, mu, sign=1):
        tmps = [st.tmp for st in states]
        self._hops(states, tmps, ins, tmhop.TM_OE, 0, tmhop.TM_SLAB_QTM_A, kappa, mu, sign)
        self._hops(states, outs, tmps, tmhop.TM_EO, 0, tmhop.TM_SLAB_QTM_B, kappa, mu, sign, xs=ins)


class LocalSlabs(_Schedule):
    """Every slab of one lattice on one device, in one process.  The faces
    move by device-to-device copies on a communication stream while the
    compute stream runs the interior hops."""

    def __init__(self, ctx: tmhop.Context, dims, U, n: int, prec="f64", recon=18, bc=(-1, 1, 1, 1)):
        self.ctx = ctx
        self.geos = split(dims, n, bc[0])
        Ut = U if isinstance(U, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(U))
        self.states = [_SlabState(ctx, g, Ut, prec, recon, bc) for g in self.geos]
        self.comm = torch.cuda.Stream(ctx.device)

    def _exchange(self, states, s):
        ready = torch.cuda.Event()
        ready.record(s)
        self.comm.wait_event(ready)
        with torch.cuda.stream(self.comm):
            for st in states:
                st.recv_upper.copy_(states[st.geo.next].send_lower, non_blocking=True)
                st.recv_lower.copy_(states[st.geo.prev].send_upper, non_blocking=True)
        done = torch.cuda.Event()
        done.record(self.comm)
        return done

    def pack_fields(self, psi, prec=None):
        """Packed slab fields of a global canonical one-parity field."""
        return [self.ctx.pack(g.field(psi), prec or st.prec) for g, st in zip(self.geos, self.states)]

    def empty(self):
        return [self.ctx.empty(g.vh, st.prec) for g, st in zip(self.geos, self.states)]

    def gather(self, fields) -> torch.Tensor:
        """The global canonical field from packed slab fields (slab order = time order)."""
        return torch.cat([self.ctx.unpack(f, g.vh, st.prec) for f, g, st in zip(fields, self.geos, self.states)])

    def Qtm(self, outs, ins, kappa, mu, sign=1):
        self._qtm(self.states, outs, ins, kappa, mu, sign)
        return outs

    def hopping_eo(self, outs, ins, direction, dagger=False):
        self._hops(self.states, outs, ins, direction, int(bool(dagger)), tmhop.TM_SLAB_HOP)
        return outs

    def close(self):
        for st in self.states:
            st.close()


class DistributedSlabs(_Schedule):
    """One slab per process (rank r of torch.distributed holds slab r); the
    faces move by point-to-point messages on a communication stream."""

    def __init__(self, ctx: tmhop.Context, dist, dims, U_slab, prec="f64", recon=18, bc=(-1, 1, 1, 1)):
        self.ctx, self.dist = ctx, dist
        self.geo = SlabGeometry(tuple(int(d) for d in dims), dist.get_world_size(), dist.get_rank(), bc[0])
        Us = U_slab if isinstance(U_slab, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(U_slab))
        self.state = _SlabState(ctx, _Local(self.geo), Us, prec, recon, bc)
        self.comm = torch.cuda.Stream(ctx.device)

    def _exchange(self, states, s):
        st = states[0]
        ready = torch.cuda.Event()
        ready.record(s)
        self.comm.wait_event(ready)
        with torch.cuda.stream(self.comm):
            exchange_faces(self.dist, self.geo, st.send_lower, st.send_upper, st.recv_lower, st.recv_upper)
        done = torch.cuda.Event()
        done.record(self.comm)
        return done

    def Qtm(self, out, inp, kappa, mu, sign=1):
        self._qtm([self.state], [out], [inp], kappa, mu, sign)
        return out

    def hopping_eo(self, out, inp, direction, dagger=False):
        self._hops([self.state], [out], [inp], direction, int(bool(dagger)), tmhop.TM_SLAB_HOP)
        return out

    def close(self):
        self.state.close()


class _Local:
    """Adapter: a slab geometry whose links() takes the slab's own links."""

    def __init__(self, geo: SlabGeometry):
        self._g = geo

    def __getattr__(self, name):
        return getattr(self._g, name)

    def links(self, U):
        return U
