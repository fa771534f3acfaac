"""Batched operator and solver: several right-hand sides on one lattice and
several lattices of uneven volume in one launch per step, against the FP64
oracle system by system."""
import numpy as np
import pytest

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}
RECON = {"f64": 18, "f32": 12, "f16": 12}
# the uneven lattices of the batching workload, (Lx, Ly, Lz, Lt)
UNEVEN = [(16, 16, 16, 32), (20, 20, 20, 40), (24, 24, 24, 48), (28, 28, 28, 56), (32, 32, 32, 64),
          (16, 16, 16, 64), (24, 24, 24, 32), (12, 12, 12, 24)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_batch(spec, seed0=100):
    """spec: list of (dims, nrhs) -> lattices [(dims, U)], systems [(lattice index, psi)]."""
    lats, systems = [], []
    for li, (dims, nrhs) in enumerate(spec):
        U = F.gauge_field(dims, seed0 + li, "near" if li % 2 else "random", 0.3)
        lats.append((dims, U))
        for j in range(nrhs):
            systems.append((li, F.gaussian_spinor(int(np.prod(dims)) // 2, F.SEED_BATCH_RHS + j, li)))
    return lats, systems


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("spec", [
    [((8, 8, 8, 8), 5)],                                   # multi-RHS on one lattice
    [((6, 4, 2, 10), 1), ((8, 8, 8, 8), 1), ((4, 4, 6, 6), 1)],   # uneven lattices
    [((8, 8, 8, 8), 3), ((6, 4, 2, 10), 1), ((10, 6, 4, 2), 2)],  # both
])
@pytest.mark.parametrize("autotune", [True, False])
def test_Qtm_batch_matches_oracle(ctx, prec, spec, autotune):
    from paper_1311_4521_gb300 import tmhop
    tmhop.tm_ctx_set_autotune(ctx.handle, autotune)
    lats, systems = make_batch(spec)
    gauges = [ctx.gauge(d, U, prec, RECON[prec]) for d, U in lats]
    ins = [ctx.pack(psi, prec) for _, psi in systems]
    outs = [ctx.empty(psi.shape[0], prec) for _, psi in systems]
    for sign in (1, -1):
        ctx.Qtm_batch([gauges[li] for li, _ in systems], outs, ins, 0.1394, 0.0015, sign)
        for (li, psi), out in zip(systems, outs):
            dims, U = lats[li]
            want = O.Qtm(dims, U, psi, 0.1394, sign * 0.0015)
            assert rel(ctx.unpack(out, psi.shape[0], prec).cpu().numpy(), want) < TOL[prec]
    for g in gauges:
        g.close()
    if autotune:   # the autotuner's choice for this shape is on the context's report
        rep = tmhop.tm_ctx_tune_report(ctx.handle)
        key = "bhop/%d/%d/" % (tmhop.PREC[prec], RECON[prec])
        assert any(line.startswith(key) and " nrb=" in line and " ms3=" in line for line in rep.splitlines()), rep
    tmhop.tm_ctx_set_autotune(ctx.handle, True)


def test_Qtm_batch_repeated_and_rebuilt(ctx):
    """A repeated batch reuses its device tables (new field contents, same
    buffers); a different batch on another stream rebuilds them."""
    import torch
    dims = (8, 8, 8, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 77, "random")
    g = ctx.gauge(dims, U, "f32", 12)
    ins = [ctx.pack(F.gaussian_spinor(vh, 77, 10 + j), "f32") for j in range(3)]
    outs = [ctx.empty(vh, "f32") for _ in range(3)]
    ctx.Qtm_batch([g] * 3, outs, ins, 0.1394, 0.0015)
    psis = [F.gaussian_spinor(vh, 78, 10 + j) for j in range(3)]
    for buf, psi in zip(ins, psis):
        buf.copy_(ctx.pack(psi, "f32"))
    ctx.Qtm_batch([g] * 3, outs, ins, 0.1394, 0.0015)
    for out, psi in zip(outs, psis):
        assert rel(ctx.unpack(out, vh, "f32").cpu().numpy(), O.Qtm(dims, U, psi, 0.1394, 0.0015)) < TOL["f32"]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ctx.Qtm_batch([g] * 2, outs[:2], ins[1:], 0.1394, 0.0015, -1)
    torch.cuda.synchronize()
    for out, psi in zip(outs[:2], psis[1:]):
        assert rel(ctx.unpack(out, vh, "f32").cpu().numpy(), O.Qtm(dims, U, psi, 0.1394, -0.0015)) < TOL["f32"]
    g.close()


def test_Qtm_batch_argument_errors(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, F.gauge_field(dims, 5, "random"), "f32", 12)
    a, b, c = (ctx.empty(128, "f32") for _ in range(3))
    with pytest.raises(tmhop.TmError) as e:
        ctx.Qtm_batch([g, g], [a, a], [b, c], 0.1, 0.1)     # one output for two systems
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError) as e:
        ctx.Qtm_batch([g, g], [a, b], [b, c], 0.1, 0.1)     # an output read by another system
    assert e.value.status == tmhop.TM_ERR_ARG
    ctx.Qtm_batch([g, g], [a, b], [c, c], 0.1, 0.1)         # a repeated input is fine
    g.close()


def oracle_relres(dims, U, x, b, kappa, mu):
    Ax = O.Qtm(dims, U, O.Qtm(dims, U, x, kappa, mu), kappa, -mu)
    return float(np.linalg.norm(b - Ax) / np.linalg.norm(b))


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_cg_batch_small(ctx, inner):
    from paper_1311_4521_gb300 import tmhop
    spec = [((8, 8, 8, 8), 3), ((6, 4, 8, 10), 1), ((4, 4, 6, 6), 2)]
    lats, systems = make_batch(spec, seed0=300)
    gh = [ctx.gauge(d, U, "f64", 18) for d, U in lats]
    gl = None if inner == "f64" else [ctx.gauge(d, U, inner, 12) for d, U in lats]
    xs = [ctx.empty(psi.shape[0], "f64").zero_() for _, psi in systems]
    bs = [ctx.pack(psi, "f64") for _, psi in systems]
    st, infos = ctx.cg_batch([gh[li] for li, _ in systems], xs, bs, 0.1394, 0.0015, 1e-10, 20000,
                             None if gl is None else [gl[li] for li, _ in systems])
    assert st == tmhop.TM_OK, infos
    for (li, psi), x, inf in zip(systems, xs, infos):
        dims, U = lats[li]
        assert inf["status"] == tmhop.TM_OK and inf["true_relres"] <= 1e-10
        xs_ = ctx.unpack(x, psi.shape[0], "f64").cpu().numpy()
        assert oracle_relres(dims, U, xs_, psi, 0.1394, 0.0015) <= 1.05e-10
    # the batched solver follows the single-system algorithm: same iteration counts
    for (li, psi), inf in zip(systems, infos):
        dims, U = lats[li]
        x1 = ctx.empty(psi.shape[0], "f64").zero_()
        st1, inf1 = ctx.cg(gh[li], x1, ctx.pack(psi, "f64"), 0.1394, 0.0015, 1e-10, 20000,
                           None if gl is None else gl[li])
        assert st1 == tmhop.TM_OK
        assert abs(inf1["iters"] - inf["iters"]) <= 2
    for g in gh + (gl or []):
        g.close()


def test_cg_batch_argument_errors(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (4, 4, 4, 4)
    U = F.gauge_field(dims, 1, "random")
    g64, g32, g16 = ctx.gauge(dims, U, "f64", 18), ctx.gauge(dims, U, "f32", 12), ctx.gauge(dims, U, "f16", 12)
    b = ctx.pack(F.gaussian_spinor(128, 1, 1), "f64")
    x = ctx.empty(128, "f64").zero_()
    x2 = ctx.empty(128, "f64").zero_()
    with pytest.raises(tmhop.TmError):   # systems sharing U_hi with different U_lo
        ctx.cg_batch([g64, g64], [x, x2], [b, b], 0.1, 0.01, U_lo=[g32, g16])
    with pytest.raises(tmhop.TmError):   # inner handles of mixed precisions
        g64b = ctx.gauge(dims, U, "f64", 18)
        ctx.cg_batch([g64, g64b], [x, x2], [b, b], 0.1, 0.01, U_lo=[g32, g16])
    with pytest.raises(tmhop.TmError):   # FP32 as U_hi
        ctx.cg_batch([g32], [x], [b], 0.1, 0.01)
    with pytest.raises(tmhop.TmError) as e:   # one solution field for two systems
        ctx.cg_batch([g64, g64], [x, x], [b, b], 0.1, 0.01)
    assert e.value.status == tmhop.TM_ERR_ARG
    with pytest.raises(tmhop.TmError) as e:   # a solution that is another system's source
        ctx.cg_batch([g64, g64], [x, x2], [b, x], 0.1, 0.01)
    assert e.value.status == tmhop.TM_ERR_ARG


def test_batching_workload_full_size(ctx):
    """12 right-hand sides on 32^3x64 and the 8 uneven lattices, FP32 storage,
    solved in one batched call; every system checked by the oracle's FP64
    residual."""
    from paper_1311_4521_gb300 import tmhop
    big = (32, 32, 32, 64)
    Ub = F.gauge_field(big, F.SEED_PROD_32, "near", 0.3)
    lats = [(big, Ub)] + [(d, F.gauge_field(d, F.SEED_BATCH_LATTICE + k, "near", 0.3)) for k, d in enumerate(UNEVEN)]
    systems = [(0, F.gaussian_spinor(int(np.prod(big)) // 2, F.SEED_BATCH_RHS + j, 0)) for j in range(12)]
    systems += [(k + 1, F.gaussian_spinor(int(np.prod(d)) // 2, F.SEED_BATCH_LATTICE + k, 1)) for k, d in enumerate(UNEVEN)]
    gh = [ctx.gauge(d, U, "f64", 18) for d, U in lats]
    gl = [ctx.gauge(d, U, "f32", 12) for d, U in lats]
    xs = [ctx.empty(psi.shape[0], "f64").zero_() for _, psi in systems]
    bs = [ctx.pack(psi, "f64") for _, psi in systems]
    st, infos = ctx.cg_batch([gh[li] for li, _ in systems], xs, bs, 0.1394, 0.0015, 1e-10, 20000,
                             [gl[li] for li, _ in systems])
    assert st == tmhop.TM_OK, infos
    for (li, psi), x, inf in zip(systems, xs, infos):
        dims, U = lats[li]
        xs_ = ctx.unpack(x, psi.shape[0], "f64").cpu().numpy()
        assert oracle_relres(dims, U, xs_, psi, 0.1394, 0.0015) <= 1.05e-10, (dims, inf)
    for g in gh + gl:
        g.close()


CODES = {"f64": [0, 1, 4], "f32": [0, 1, 2, 4, 10, 12, 14], "f16": [0, 1, 2, 4, 10, 12, 14]}


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_every_batch_configuration(ctx, prec):
    """Every configuration of the batched hop (pass width, right-hand sides
    per thread, CTA cap), forced instead of tuned, against the oracle, with
    an odd number of right-hand sides (a thread pair with one member idle)
    and a second lattice; and the batched solver (the norm and update modes
    of the hop) in the reduced-precision formats."""
    from paper_1311_4521_gb300 import tmhop
    spec = [((8, 8, 8, 8), 5), ((6, 4, 2, 10), 1)]
    lats, systems = make_batch(spec, seed0=500)
    gauges = [ctx.gauge(d, U, prec, RECON[prec]) for d, U in lats]
    ins = [ctx.pack(psi, prec) for _, psi in systems]
    want = [O.Qtm(lats[li][0], lats[li][1], psi, 0.1394, 0.0015) for li, psi in systems]
    try:
        for code in CODES[prec]:
            for cap in (0, 7):
                tmhop.tm_ctx_set_batch_config(ctx.handle, code, cap)
                outs = [ctx.empty(psi.shape[0], prec) for _, psi in systems]
                for o in outs:
                    o.fill_(0xFF)
                ctx.Qtm_batch([gauges[li] for li, _ in systems], outs, ins, 0.1394, 0.0015)
                for (li, psi), out, w in zip(systems, outs, want):
                    got = ctx.unpack(out, psi.shape[0], prec).cpu().numpy()
                    assert np.all(np.isfinite(got)) and rel(got, w) < TOL[prec], (code, cap)
            if prec == "f64":
                continue
            gh = [ctx.gauge(d, U, "f64", 18) for d, U in lats]
            xs = [ctx.empty(psi.shape[0], "f64").zero_() for _, psi in systems]
            bs = [ctx.pack(psi, "f64") for _, psi in systems]
            st, infos = ctx.cg_batch([gh[li] for li, _ in systems], xs, bs, 0.1394, 0.0015, 1e-10, 20000,
                                     [gauges[li] for li, _ in systems])
            assert st == tmhop.TM_OK, (code, infos)
            for (li, psi), x in zip(systems, xs):
                dims, U = lats[li]
                assert oracle_relres(dims, U, ctx.unpack(x, psi.shape[0], "f64").cpu().numpy(), psi,
                                     0.1394, 0.0015) <= 1.05e-10, code
            for g in gh:
                g.close()
        with pytest.raises(tmhop.TmError):
            tmhop.tm_ctx_set_batch_config(ctx.handle, 3, 0)
    finally:
        tmhop.tm_ctx_set_batch_config(ctx.handle, -1, 0)
        for g in gauges:
            g.close()
