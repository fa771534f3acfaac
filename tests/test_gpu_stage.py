"""The staged batched hop (configuration code 100 of tm_Qtm_batch): boxes of
8 x 2 x 2 x 2 half-sites whose neighbour spinors and links are copied into
shared memory by TMA tensor copies.  Checked system by system against the
FP64 oracle on lattices whose faces wrap onto the box itself (an extent of
2), onto the neighbouring box, and across the antiperiodic time boundary,
with fewer persistent CTAs than boxes (several boxes per CTA, so both link
buffers and every stage buffer are reused), and with more."""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "f16": 5e-3}


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _batch(spec, seed0):
    lats, systems = [], []
    for li, (dims, nrhs) in enumerate(spec):
        U = F.gauge_field(dims, seed0 + li, "random" if li % 2 else "near", 0.3)
        lats.append((dims, U))
        for j in range(nrhs):
            systems.append((li, F.gaussian_spinor(int(np.prod(dims)) // 2, seed0 + 10 * li + j, 3)))
    return lats, systems


def _run(ctx, prec, recon, spec, code, cap, seed0, signs=(1, -1), bc=(-1, 1, 1, 1)):
    from paper_1311_4521_gb300 import tmhop
    lats, systems = _batch(spec, seed0)
    gauges = [ctx.gauge(d, U, prec, recon, bc) for d, U in lats]
    ins = [ctx.pack(psi, prec) for _, psi in systems]
    try:
        tmhop.tm_ctx_set_batch_config(ctx.handle, code, cap)
        for sign in signs:
            outs = [ctx.empty(psi.shape[0], prec) for _, psi in systems]
            for o in outs:
                o.fill_(0xFF)   # NaN in every format: a site left unwritten fails
            ctx.Qtm_batch([gauges[li] for li, _ in systems], outs, ins, 0.1394, 0.0015, sign)
            tmhop.tm_ctx_check(ctx.handle)
            for (li, psi), out in zip(systems, outs):
                dims, U = lats[li]
                got = ctx.unpack(out, psi.shape[0], prec).cpu().numpy()
                want = O.Qtm(dims, U, psi, 0.1394, sign * 0.0015, bc=bc)
                assert np.all(np.isfinite(got)), (prec, recon, dims, sign)
                assert rel(got, want) < TOL[prec], (prec, recon, dims, sign, rel(got, want))
    finally:
        tmhop.tm_ctx_set_batch_config(ctx.handle, -1, 0)
        for g in gauges:
            g.close()


@pytest.mark.parametrize("prec,recon", [("f32", 12), ("f32", 18), ("f16", 12)])
@pytest.mark.parametrize("cap", [0, 3])
def test_staged_hop_matches_oracle(ctx, prec, recon, cap):
    # (16, 2, 2, 4): every y and z face is the box itself; (32, 4, 6, 8): two
    # boxes per row in x, faces on other boxes, the t faces across the boundary
    spec = [((32, 4, 6, 8), 3), ((16, 2, 2, 4), 2)]
    _run(ctx, prec, recon, spec, 100, cap, 700)


def test_staged_hop_single_rhs_groups(ctx):
    """Groups of one right-hand side next to a group of several: the box
    loop, the link buffers and the stage ring stay in step."""
    spec = [((16, 4, 4, 4), 1), ((16, 2, 4, 6), 4), ((32, 2, 2, 2), 1)]
    _run(ctx, "f32", 12, spec, 100, 2, 800, signs=(1,))


def test_staged_hop_tuned_larger_lattice(ctx):
    """The autotuner (staged hop among its candidates) on 16^3x32 with 6
    right-hand sides: whatever it picks, the result matches the oracle."""
    spec = [((16, 16, 16, 32), 6)]
    _run(ctx, "f32", 12, spec, -1, 0, 900, signs=(1,))


def test_staged_code_ignored_where_unavailable(ctx):
    """Lx not a multiple of 16: code 100 is ignored there and the tuner
    configures the launch; the result is still right."""
    spec = [((8, 8, 8, 8), 3)]
    _run(ctx, "f32", 12, spec, 100, 0, 950, signs=(1,))


@pytest.mark.parametrize("bc", [(1, -1, -1, 1), (-1, 1, -1, -1), (1, 1, 1, 1)])
def test_staged_hop_boundary_signs(ctx, bc):
    """Antiperiodic boundaries in x, y or z (bc is (t, x, y, z)): the wrap
    signs of the staged hop come from the lattice's boundary flags, not from
    the position in the box."""
    spec = [((32, 4, 4, 6), 2)]
    _run(ctx, "f32", 12, spec, 100, 2, 990, signs=(1,), bc=bc)


def test_bounded_wait_runs_out_and_reports(ctx):
    """A shared-memory barrier wait that nothing completes gives up after its
    limit, the status reaches the host through tm_ctx_check (once: the check
    clears it), and the context goes on working."""
    import time

    from paper_1311_4521_gb300 import tmhop
    tmhop.tm_ctx_check(ctx.handle)   # nothing pending
    t0 = time.perf_counter()
    tmhop.tm_ctx_selftest_wait(ctx.handle)
    with pytest.raises(tmhop.TmError):
        tmhop.tm_ctx_check(ctx.handle)
    assert time.perf_counter() - t0 < 30.0
    tmhop.tm_ctx_check(ctx.handle)   # cleared
    _run(ctx, "f32", 12, [((16, 2, 2, 4), 2)], 100, 0, 995, signs=(1,))


@pytest.mark.parametrize("code", [-1, 100])
def test_batched_qtm_12rhs_full_size(ctx, code):
    """The benchmark's batching workload, 12 right-hand sides on 32^3x64 in
    FP32-12 storage, in the configuration the bench times (the tuned one)
    and with the TMA-staged hop forced: every right-hand side against the
    oracle's FP64 Q_tm."""
    from paper_1311_4521_gb300 import tmhop
    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_PROD_32, "near", 0.3)
    g = ctx.gauge(dims, U, "f32", 12)
    rhs = [F.gaussian_spinor(vh, F.SEED_BATCH_RHS + j, 0) for j in range(12)]
    ins = [ctx.pack(r, "f32") for r in rhs]
    outs = [ctx.empty(vh, "f32") for _ in rhs]
    try:
        tmhop.tm_ctx_set_batch_config(ctx.handle, code, 0)
        ctx.Qtm_batch([g] * 12, outs, ins, 0.1394, 0.0015)
        tmhop.tm_ctx_check(ctx.handle)
        for r, o in zip(rhs, outs):
            want = O.Qtm(dims, U, r, 0.1394, 0.0015)
            assert rel(ctx.unpack(o, vh, "f32").cpu().numpy(), want) < TOL["f32"]
    finally:
        tmhop.tm_ctx_set_batch_config(ctx.handle, -1, 0)
        g.close()
