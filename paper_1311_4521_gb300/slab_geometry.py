"""Host-side bookkeeping of a lattice cut along time into slabs, one per
GPU (the surface/body decomposition of the paper's Sec. 2.5): the slab
geometry, which rank each face goes to, the sign each face carries, and
the collective steps (face exchange by point-to-point messages, the
all-reduce of per-rank inner products).  Pure host logic: it needs no GPU
and no compiled library, so it is tested on CPU ranks (gloo).

Global fields in canonical layout (one parity, index lex/2 with
lex = x + Lx (y + Ly (z + Lz t))) split into slabs as contiguous index
ranges, because the index is t-major.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


@dataclass(frozen=True)
class SlabGeometry:
    """Slab r of a lattice dims = (Lx, Ly, Lz, Lt) cut into n slabs along t.

    Every slab has extent lt = Lt / n (even, >= 2) and starts at t0 = r lt
    (even), so a site's parity is the same locally and globally.  bc_t is
    the boundary sign of the global time direction: it multiplies the hops
    through the lower face of slab 0 and the upper face of slab n-1."""

    dims: tuple
    n: int
    r: int
    bc_t: int = -1

    def __post_init__(self):
        lx, ly, lz, lt = self.dims
        if self.n < 1 or not 0 <= self.r < self.n:
            raise ValueError(f"slab {self.r} of {self.n}")
        if lt % self.n or (lt // self.n) % 2 or lt // self.n < 2:
            raise ValueError(f"Lt = {lt} does not split into {self.n} slabs of even extent >= 2")
        if any(d % 2 or d < 2 for d in self.dims):
            raise ValueError(f"extents must be even and >= 2: {self.dims}")
        if self.bc_t not in (1, -1):
            raise ValueError("bc_t must be +1 or -1")

    @property
    def lt(self) -> int:
        return self.dims[3] // self.n

    @property
    def t0(self) -> int:
        return self.r * self.lt

    @property
    def local_dims(self) -> tuple:
        return (self.dims[0], self.dims[1], self.dims[2], self.lt)

    @property
    def v3(self) -> int:
        """Sites of one time slice (both parities)."""
        return self.dims[0] * self.dims[1] * self.dims[2]

    @property
    def st(self) -> int:
        """Sites of one time slice and parity: the length of a face."""
        return self.v3 // 2

    @property
    def vh(self) -> int:
        """Sites of the slab per parity."""
        return self.st * self.lt

    @property
    def prev(self) -> int:
        return (self.r - 1) % self.n

    @property
    def next(self) -> int:
        return (self.r + 1) % self.n

    @property
    def sign_lower(self) -> int:
        return self.bc_t if self.r == 0 else 1

    @property
    def sign_upper(self) -> int:
        return self.bc_t if self.r == self.n - 1 else 1

    def eo_range(self) -> slice:
        """Index range of the slab's sites in a global one-parity field."""
        return slice(self.t0 * self.st, (self.t0 + self.lt) * self.st)

    def lex_range(self) -> slice:
        """Range of the slab's sites in the global lexicographic order."""
        return slice(self.t0 * self.v3, (self.t0 + self.lt) * self.v3)

    def links(self, U):
        """The slab's links U[4][Vs][3][3] from the global U[4][V][3][3] (a view)."""
        return U[:, self.lex_range()]

    def field(self, psi):
        """The slab's part of a global one-parity field (a view)."""
        return psi[self.eo_range()]

    def global_lex(self, parity: int) -> np.ndarray:
        """Global lexicographic index of every local site of the given parity, by local index."""
        lx, ly, lz, _ = self.dims
        i = np.arange(self.vh)
        xh, rest = i % (lx // 2), i // (lx // 2)
        y, rest = rest % ly, rest // ly
        z, t = rest % lz, rest // lz
        x = 2 * xh + ((y + z + t + parity) & 1)
        return x + lx * (y + ly * (z + lz * (t + self.t0)))

    def face_sites(self, parity: int, which: str) -> np.ndarray:
        """Global lexicographic index of the sites a face of a parity-`parity`
        field describes, by face index: "lower" = local t = 0, "upper" = t = lt-1."""
        g = self.global_lex(parity)
        return g[: self.st] if which == "lower" else g[(self.lt - 1) * self.st:]


def split(dims, n, bc_t=-1):
    """The n slab geometries of a lattice."""
    return [SlabGeometry(tuple(int(d) for d in dims), n, r, bc_t) for r in range(n)]


def exchange_faces(dist, geo: SlabGeometry, send_lower, send_upper, recv_lower, recv_upper) -> None:
    """Moves one slab's faces between ranks with point-to-point messages:
    send_lower goes to the previous rank (its recv_upper), send_upper to the
    next rank (its recv_lower).  Tags keep the two directions apart when the
    previous and next rank are the same process (two ranks).  Blocking."""
    if geo.n == 1:
        recv_upper.copy_(send_lower)
        recv_lower.copy_(send_upper)
        return
    reqs = [dist.irecv(recv_upper, src=geo.next, tag=1), dist.irecv(recv_lower, src=geo.prev, tag=2),
            dist.isend(send_lower, dst=geo.prev, tag=1), dist.isend(send_upper, dst=geo.next, tag=2)]
    for q in reqs:
        q.wait()


def allreduce_dot(dist, partial: torch.Tensor) -> torch.Tensor:
    """Global inner product from each rank's partial <a, b> (two FP64 values
    from tm_spinor_dot on its slab): an FP64 sum over ranks by the
    transport's all-reduce (NCCL between GPUs), the paper's scalar_prod_r
    (Sec. 3).  In place; returns `partial`, now the global value."""
    dist.all_reduce(partial)
    return partial
