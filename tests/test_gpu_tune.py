"""The autotuner of the single-lattice hop: every site-to-thread map gives
bit-identical results (the per-site arithmetic does not depend on the map),
the tuned map matches the oracle like the default one, and the choice is
kept in the cache file and reused by a new context without timing."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1311_4521_gb300 import fields as F

pytestmark = pytest.mark.gpu

RECON = {"f64": 18, "f64x": 18, "f32": 12, "f16": 12}
TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16": 5e-3}


@pytest.fixture(scope="module")
def ctx():
    from paper_1311_4521_gb300 import tmhop
    c = tmhop.Context(0)
    yield c
    c.close()


def qtm_bytes(ctx, g, src, vh, prec):
    out = ctx.empty(vh, prec)
    out.fill_(0xFF)
    ctx.Qtm(g, out, src, 0.1394, 0.0015)
    return out


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16"])
@pytest.mark.parametrize("dims", [(16, 8, 8, 16), (24, 8, 4, 8)])
def test_every_map_gives_identical_bits(ctx, prec, dims):
    from paper_1311_4521_gb300 import tmhop
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 401, "near", 0.3)
    psi = F.gaussian_spinor(vh, 401, 1)
    g = ctx.gauge(dims, U, prec, RECON[prec])
    src = ctx.pack(psi, prec)
    assert tmhop.tm_gauge_map(g.handle) == "linear128"
    ref = qtm_bytes(ctx, g, src, vh, prec)
    got = ctx.unpack(ref, vh, prec).cpu().numpy()
    assert np.linalg.norm(got - O.Qtm(dims, U, psi, 0.1394, 0.0015)) / np.linalg.norm(got) < TOL[prec]
    names = ["linear64", "linear96", "box4x2x2x2", "box4x4x2x1", "box8x2x2x2", "box4x2x1x4", "box8x1x2x4",
             "box8x1x1x8"]
    tried = 0
    for name in names:
        try:
            tmhop.tm_gauge_set_map(ctx.handle, g.handle, name)
        except tmhop.TmError:
            continue                      # the box does not divide this lattice
        assert tmhop.tm_gauge_map(g.handle) == name
        assert torch.equal(qtm_bytes(ctx, g, src, vh, prec), ref), name
        tried += 1
    assert tried >= 4
    # the force's hops use the same map
    if prec in ("f64", "f32"):
        X = ctx.pack(psi, prec)
        tmhop.tm_gauge_set_map(ctx.handle, g.handle, "box4x2x2x2")
        Fa = ctx.force(g, X, 0.1394, 0.0015)
        tmhop.tm_gauge_set_map(ctx.handle, g.handle, "linear128")
        Fb = ctx.force(g, X, 0.1394, 0.0015)
        assert torch.equal(Fa, Fb)
    g.close()


def test_bad_maps_are_rejected(ctx):
    from paper_1311_4521_gb300 import tmhop
    dims = (12, 4, 4, 8)                  # Lx/2 = 6: no box of 4 along the half-row
    U = F.gauge_field(dims, 402, "random")
    g = ctx.gauge(dims, U, "f64", 18)
    for name in ("box4x2x2x2", "box2x2x2x2", "linear200", "linear33", "nonsense", "box3x4x4x2"):
        with pytest.raises(tmhop.TmError):
            tmhop.tm_gauge_set_map(ctx.handle, g.handle, name)
    assert tmhop.tm_gauge_map(g.handle) == "linear128"
    g.close()


def test_tune_persists_in_the_cache_file(tmp_path):
    from paper_1311_4521_gb300 import tmhop
    dims = (16, 16, 16, 16)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 403, "near", 0.3)
    psi = F.gaussian_spinor(vh, 403, 1)
    cache = tmp_path / "tune.txt"
    c1 = tmhop.Context(0)
    tmhop.tm_ctx_set_tune_cache(c1.handle, str(cache))
    g1 = c1.gauge(dims, U, "f32", 12)
    tmhop.tm_gauge_tune(c1.handle, g1.handle)
    chosen = tmhop.tm_gauge_map(g1.handle)
    rep = tmhop.tm_ctx_tune_report(c1.handle)
    assert "hop/" in rep and f"map={chosen}" in rep and "candidates=" in rep
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[1] == chosen and "|16x16x16x16|prec1|recon12|nrhs1" in lines[0]
    out1 = qtm_bytes(c1, g1, c1.pack(psi, "f32"), vh, "f32")
    # a new context with the same cache: the handle gets the map at creation, and tuning is a cache hit
    c2 = tmhop.Context(0)
    tmhop.tm_ctx_set_tune_cache(c2.handle, str(cache))
    g2 = c2.gauge(dims, U, "f32", 12)
    assert tmhop.tm_gauge_map(g2.handle) == chosen
    tmhop.tm_gauge_tune(c2.handle, g2.handle)
    assert "(cache)" in tmhop.tm_ctx_tune_report(c2.handle)
    assert len(cache.read_text().splitlines()) == 1
    out2 = qtm_bytes(c2, g2, c2.pack(psi, "f32"), vh, "f32")
    assert torch.equal(out1, out2)
    # without a cache and with autotuning off the default map stays
    c3 = tmhop.Context(0)
    tmhop.tm_ctx_set_autotune(c3.handle, False)
    g3 = c3.gauge(dims, U, "f32", 12)
    tmhop.tm_gauge_tune(c3.handle, g3.handle)
    assert tmhop.tm_gauge_map(g3.handle) == "linear128"
    for g, c in ((g1, c1), (g2, c2), (g3, c3)):
        g.close()
        c.close()


def test_batched_choice_persists_in_the_cache_file(tmp_path):
    """The batched hop's tuned configuration goes to the same cache file,
    keyed by GPU, storage and the batch's (Vh x nrhs) groups; a new context
    with that file takes it without timing (no second line) and computes the
    same result, which matches the oracle."""
    from paper_1311_4521_gb300 import tmhop
    dims = (16, 8, 8, 8)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, 404, "near", 0.3)
    psis = [F.gaussian_spinor(vh, 404, 1 + j) for j in range(4)]
    cache = tmp_path / "tune.txt"
    outs, reports = [], []
    for _ in range(2):
        c = tmhop.Context(0)
        tmhop.tm_ctx_set_tune_cache(c.handle, str(cache))
        g = c.gauge(dims, U, "f32", 12)
        ins = [c.pack(p, "f32") for p in psis]
        o = [c.empty(vh, "f32") for _ in psis]
        c.Qtm_batch([g] * 4, o, ins, 0.1394, 0.0015)
        outs.append([c.unpack(t, vh, "f32").cpu().numpy() for t in o])
        reports.append([ln for ln in tmhop.tm_ctx_tune_report(c.handle).splitlines() if ln.startswith("bhop/")])
        g.close()
        c.close()
    lines = [ln for ln in cache.read_text().splitlines() if "|bhop/" in ln]
    assert len(lines) == 1, lines
    assert f"{vh}x4" in lines[0] and lines[0].split()[1].startswith("code")
    nrb, cap = lines[0].split()[1][len("code"):].split("-cap")
    for rep in reports:
        assert any(f"nrb={nrb} cap={cap}" in ln for ln in rep), rep
    for a, b, p in zip(outs[0], outs[1], psis):
        assert np.array_equal(a, b)
        want = O.Qtm(dims, U, p, 0.1394, 0.0015)
        assert np.linalg.norm(a - want) / np.linalg.norm(want) < 1e-6
