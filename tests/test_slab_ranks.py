"""The host-side bookkeeping of the time-slab decomposition on two and four
CPU ranks (gloo): slab geometry, the routing of the faces between ranks
(send_lower to the previous rank, send_upper to the next one, the ends of
the global time direction joined), the sign carried by each face, and the
all-reduce of per-rank inner products.  Every face is filled with the
global site numbers it describes; each rank checks that, for every site on
its own faces, the entry it reads from the received face is its global
time neighbour."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1311_4521_gb300.slab_geometry import SlabGeometry, allreduce_dot, exchange_faces, split

DIMS = (4, 6, 2, 12)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _neighbour_t(dims, lex, step):
    lx, ly, lz, lt = dims
    v3 = lx * ly * lz
    t, r = lex // v3, lex % v3
    return r + v3 * ((t + step) % lt), ((t + step) % lt) != t + step


def _check_rank(rank, world, dims):
    geo = SlabGeometry(dims, world, rank, -1)
    errors = []
    for q in (0, 1):                      # parity of the input field
        p = 1 - q                          # parity of the output sites
        lower = torch.from_numpy(geo.face_sites(q, "lower").astype(np.float64))
        upper = torch.from_numpy(geo.face_sites(q, "upper").astype(np.float64))
        recv_lower, recv_upper = torch.empty_like(lower), torch.empty_like(upper)
        exchange_faces(dist, geo, lower, upper, recv_lower, recv_upper)
        out = geo.global_lex(p)
        top = (geo.lt - 1) * geo.st
        for i in range(geo.st):
            # a t = 0 output site: its backward neighbour is entry i of the received lower face
            nb, crosses = _neighbour_t(dims, out[i], -1)
            if recv_lower[i].item() != nb:
                errors.append(("lower", q, i))
            if crosses != (geo.sign_lower == -1):
                errors.append(("sign_lower", q, i))
            # a t = lt-1 output site: its forward neighbour is entry i of the received upper face
            nb, crosses = _neighbour_t(dims, out[top + i], +1)
            if recv_upper[i].item() != nb:
                errors.append(("upper", q, i))
            if crosses != (geo.sign_upper == -1):
                errors.append(("sign_upper", q, i))
    part = torch.tensor([float(rank + 1), -0.5 * rank], dtype=torch.float64)
    total = allreduce_dot(dist, part)
    want = [sum(r + 1 for r in range(world)), -0.5 * sum(range(world))]
    if total.tolist() != want:
        errors.append(("allreduce", total.tolist(), want))
    return errors


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _check_rank(rank, world, DIMS)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_face_routing_on_cpu_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        for p in procs:
            p.join(timeout=120)
    finally:
        for p in procs:
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    for p in procs:
        assert p.exitcode == 0
    results = dict(q.get(timeout=10) for _ in range(world))
    for r in range(world):
        assert results[r] == [], (r, results[r][:5])


def test_geometry_of_the_split():
    geos = split(DIMS, 3, -1)
    assert [g.t0 for g in geos] == [0, 4, 8]
    assert [(g.sign_lower, g.sign_upper) for g in geos] == [(-1, 1), (1, 1), (1, -1)]
    assert [(g.prev, g.next) for g in geos] == [(2, 1), (0, 2), (1, 0)]
    # the slabs' parity-p sites tile the global parity-p field in order
    for p in (0, 1):
        lex = np.concatenate([g.global_lex(p) for g in geos])
        assert np.array_equal(lex // 2, np.arange(int(np.prod(DIMS)) // 2))
        assert np.all((lex % DIMS[0] + lex // DIMS[0] % DIMS[1] + lex // (DIMS[0] * DIMS[1]) % DIMS[2]
                       + lex // (DIMS[0] * DIMS[1] * DIMS[2])) % 2 == p)
    one = split(DIMS, 1, -1)[0]
    assert (one.sign_lower, one.sign_upper, one.prev, one.next) == (-1, -1, 0, 0)
    with pytest.raises(ValueError):
        SlabGeometry(DIMS, 4, 0)          # 12 / 4 = 3: odd slab extent
    with pytest.raises(ValueError):
        SlabGeometry(DIMS, 12, 0)         # extent 1
