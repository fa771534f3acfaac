#!/usr/bin/env python
"""Benchmark of the twisted-mass operator Q_tm on one GB300 per rank.

Workload: the production-size plain FP64 operator, a 32^3x64 lattice with
near-thermalised links U = exp(0.3 i A) (A Gaussian in su(3)), a Gaussian
spinor, kappa = 0.1394, mu = 0.0015, antiperiodic in time.  One step is one
application of Q_tm = gamma5 (M_ee - M_eo M_oo^-1 M_oe) (two fused hop
launches) with every input already resident in HBM.

Reported per step (one even site = one unit):
  bytes  algorithmic: each input spinor read once, the 8 links of every
         output site read, each output written once, plus the re-read of
         psi_e in the final update (see algo_bytes);
  flops  1320 per site per hop + 72 + 96 site-local = 2808 per even site.

The JSON line also carries the dominant kernel's roofline (live CUDA-event
timing of each launch), the FP32/FP16 storage variants, an end-to-end
number through the C ABI with host buffers, clocks sampled during the timed
region and the FP64 CPU oracle timed on this host's cores.  With
``--impl reference`` the oracle alone is timed as the reference arm.

Multi-GPU: replicas only -- every rank applies Q_tm to its own copy of the
lattice (the operator needs no exchange on one GPU), value = all ranks'
bytes / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hopping-matrix GB/s & Gflop/s vs HBM roofline; mixed vs FP64 CG time to 1e-10"
DIMS = (32, 32, 32, 64)
KAPPA, MU = 0.1394, 0.0015
HBM_NOMINAL_GBS = 7900.0     # nominal HBM3e bandwidth of a GB300, for context beside the measured copy peak
SAMPLE_DIMS = (16, 16, 16, 16)       # bounded sample for the CPU reference arm
L2_BYTES = 129 * 2 ** 20
REAL = {"f64": 8, "f64x": 8, "f32": 4, "f16": 2}
HOP_FLOPS = 1320
QTM_FLOPS = 2 * HOP_FLOPS + 72 + 96
FP64_FMA_PER_SM_CLK = 2     # nominal FP64 FMA lanes per SM and clock of a GB300 (context beside the probe)


def fp64_nominal_tflops(sm_count: int, sm_mhz: float) -> float:
    """Nominal FP64 FMA rate: SMs x FMA lanes x 2 flop x clock."""
    return sm_count * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes (read + write) per launch of Q_tm's launch B from ncu captures of
# the dominant kernel on the 32^3x64 workload lattice (per site, so that
# another lattice scales by its site count), valid only for the kernel
# sources they were taken from (hash of csrc/tm_device.cuh +
# csrc/tm_kernels.cu).
TRAFFIC = {"src": "4d1e82678e27f879",
           "per_site": {("f64", 18): 1790570752 / 1048576, ("f64x", 18): 1790290944 / 1048576,
                        ("f32", 12): 678930688 / 1048576, ("f16", 12): 341252096 / 1048576}}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("tm_device.cuh", "tm_kernels.cu"):
        with open(os.path.join(ROOT, "paper_1311_4521_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(prec: str, recon: int, vh: int):
    per = TRAFFIC["per_site"].get((prec, recon))
    if per is None or kernel_source_hash() != TRAFFIC["src"]:
        return None
    return round(per * vh)


def hop_bytes(prec: str, recon: int) -> int:
    """Algorithmic bytes of one hop per output site: in spinor, out spinor, 8 links."""
    b = (24 + 24 + 8 * recon) * REAL[prec]
    return b + (8 if prec == "f16" else 0)           # per-site norms of the f16 spinors


def workload_config(dims, prec: str, recon: int, world: int) -> dict:
    """The `config` of the JSON line: the workload one step processes."""
    vh = int(np.prod(dims)) // 2
    return {"workload": f"Q_tm, {'x'.join(str(d) for d in dims)}, {prec} storage, {recon}-real links, "
                        "U=exp(0.3iA), kappa=0.1394, mu=0.0015, antiperiodic t",
            "lattice": list(dims), "even_sites": vh, "storage": prec, "reconstruct": recon,
            "bytes_per_step": vh * algo_bytes(prec, recon)["qtm"], "flops_per_step": vh * QTM_FLOPS,
            "parallelism": f"replicas x{world}"}


def algo_bytes(prec: str, recon: int) -> dict:
    reread = 24 * REAL[prec] + (4 if prec == "f16" else 0)
    a = hop_bytes(prec, recon)
    b = hop_bytes(prec, recon) + reread
    return {"kernel_a": a, "kernel_b": b, "qtm": a + b}


class Ranks:
    """Rank bookkeeping of a replicas-only run (one process per GPU, no data
    exchange): a barrier around timed regions and the maximum of a time over
    ranks.  ``dist`` is torch.distributed (initialised) or None for one rank."""

    def __init__(self, dist=None, device="cuda"):
        self.dist = dist
        self.device = device

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def allmax(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def job_throughput(world: int, units_per_rank: int, bytes_per_unit: float, max_ms: float) -> float:
    """Whole-job GB/s: every rank's units over the slowest rank's time."""
    return world * units_per_rank * bytes_per_unit / (max_ms * 1e-3) / 1e9


def tune_gauge(tmhop, ctx, g) -> dict:
    """Runs the library's site-map autotuner for a gauge handle and returns
    its choice: the map, its time per launch, the default map's time and
    the gain (from the context's tune report)."""
    tmhop.tm_gauge_tune(ctx.handle, g.handle)
    out = {"map": tmhop.tm_gauge_map(g.handle)}
    tag = f"|{g.dims[0]}x{g.dims[1]}x{g.dims[2]}x{g.dims[3]}|prec{g.prec}|recon{g.reconstruct}|"
    for line in tmhop.tm_ctx_tune_report(ctx.handle).splitlines():
        if not line.startswith("hop/") or tag not in line.split()[0]:
            continue
        for tok in line.split()[1:]:
            k, _, v = tok.partition("=")
            if k in ("ms", "linear128_ms", "gain"):
                out[k] = float(v)
            elif k == "candidates":
                out[k] = int(v)
    return out


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(", ") for r in self.tmp.read().strip().splitlines() if r.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        if self.uuid:
            mine = [r for r in rows if len(r) > 1 and self.uuid in r[1]]
            rows = mine or rows
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 10:
                continue
            try:
                sm.append(float(r[2].split()[0]))
                smax.append(float(r[3].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, r[6:10]):
                if v.strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
def time_qtm(ctx, tmhop, torch, g, src, dst, steps: int, warmup: int, dist_barrier):
    """Times `steps` Q_tm applications; per-launch CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.Qtm(g, dst, src, KAPPA, MU)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for trio in ev:          # torch creates the CUDA event on first record
        for e in trio:
            e.record(stream)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist_barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(steps):
        tmhop.tm_ctx_trace(ctx.handle, ev[k])
        ctx.Qtm(g, dst, src, KAPPA, MU)
    tmhop.tm_ctx_trace(ctx.handle, None)
    t1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    total_ms = t0.elapsed_time(t1)
    ka = [e[0].elapsed_time(e[1]) for e in ev]
    kb = [e[1].elapsed_time(e[2]) for e in ev]
    return total_ms, float(np.mean(ka)), float(np.mean(kb))


def gpu_arm(args) -> None:
    import torch
    from paper_1311_4521_gb300 import fields as F
    from paper_1311_4521_gb300 import tmhop

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ranks = Ranks(dist, "cuda")
    barrier, allmax = ranks.barrier, ranks.allmax

    DIMS = args.lattice
    prec, recon = args.prec, args.recon
    vh = int(np.prod(DIMS)) // 2
    U = F.gauge_field(DIMS, F.SEED_PROD_32, "near", 0.3)
    psi = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    ctx = tmhop.Context(local)
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "") or "") or None
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid

    if args.only:
        out = only_section(args, ctx, tmhop, torch, F, U, psi, DIMS, vh, barrier, allmax)
        if rank == 0:
            print(json.dumps(out), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- the FP64 arithmetic peak, measured on this GPU in this process
    # (FMA throughput probe of the library) with the clocks it ran at
    sms = props.multi_processor_count
    pclk = ClockSampler(uuid).start()
    f64s, t_probe = [], time.perf_counter()
    while time.perf_counter() - t_probe < 1.0 or len(f64s) < 3:   # ~1 s, so that the clocks get sampled
        f64s.append(tmhop.tm_probe_fma(ctx.handle, tmhop.TM_F64))
    fp64_peak = max(f64s)
    fp32_peak = tmhop.tm_probe_fma(ctx.handle, tmhop.TM_F32)
    pck = pclk.stop()
    probe = {"fp64_tflops": round(fp64_peak, 4), "fp64_tflops_median": round(statistics.median(f64s), 4),
             "probe_calls": len(f64s), "fp32_tflops": round(fp32_peak, 2), "sm_count": sms,
             "sm_mhz": pck.get("sm_mhz"), "reasons": pck.get("reasons"),
             "fp64_nominal_tflops_at_max_clock": round(fp64_nominal_tflops(sms, pck.get("sm_max_mhz") or 2070.0), 4),
             "how": "tm_probe_fma: 8 CTAs x 256 threads per SM, 8 independent FMA chains per thread, "
                    "best of 3 timed launches of ~10 ms, 2 flop per FMA"}

    # ---- headline: FP64 storage, 18-real links (by default); the hop's
    # site-to-thread map is chosen by the library's autotuner first
    g = ctx.gauge(DIMS, U, prec, recon)
    site_map = tune_gauge(tmhop, ctx, g)
    src = ctx.pack(psi, prec)
    dst = ctx.empty(vh, prec)
    clocks = ClockSampler(uuid).start()
    total_ms, ka_ms, kb_ms = time_qtm(ctx, tmhop, torch, g, src, dst, args.steps, args.warmup, barrier)
    ck = clocks.stop()
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(ck["reasons"]):
        clocks = ClockSampler(uuid).start()
        total_ms, ka_ms, kb_ms = time_qtm(ctx, tmhop, torch, g, src, dst, args.steps, args.warmup, barrier)
        ck = clocks.stop()
        ck["remeasured"] = True
    max_ms = allmax(total_ms)
    ab = algo_bytes(prec, recon)
    ms_per_step = max_ms / args.steps
    value = job_throughput(world, vh, ab["qtm"], ms_per_step)
    gflops = world * vh * QTM_FLOPS / (ms_per_step * 1e-3) / 1e9
    kb_tflops = vh * (HOP_FLOPS + 96) / (kb_ms * 1e-3) / 1e12
    kb_gbs = vh * ab["kernel_b"] / (kb_ms * 1e-3) / 1e9
    traffic = args.traffic if args.traffic is not None else traffic_per_launch(prec, recon, vh)
    kname = f"k_hop<{prec.upper()},{recon},HASX> (Q_tm second launch: H_eo + gamma5 twisted update)"
    if prec == "f64":
        roofline = {"bound": "alu", "achieved": round(kb_tflops, 4), "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": round(kb_tflops / fp64_peak, 4), "traffic": traffic,
                    "kernel": kname,
                    "peak_source": "measured: FP64 FMA throughput probe (tm_probe_fma) in this process, "
                                   "see fp64_probe",
                    "peak_nominal": probe["fp64_nominal_tflops_at_max_clock"],
                    "hbm_achieved_gbs": round(kb_gbs, 1), "hbm_frac": round(kb_gbs / hbm_peak, 4)}
    else:
        roofline = {"bound": "hbm", "achieved": round(kb_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(kb_gbs / hbm_peak, 4), "traffic": traffic, "kernel": kname,
                    "peak_source": f"{hbm_src} HBM copy bandwidth"}
    roofline.update({"site_map": site_map, "kernel_a_ms": round(ka_ms, 4), "kernel_b_ms": round(kb_ms, 4),
                     "bytes_per_launch": vh * ab["kernel_b"], "flops_per_launch": vh * (HOP_FLOPS + 96)})

    # ---- FP64-accurate operator in double-float storage and arithmetic (not the headline)
    f64x = None
    if prec == "f64" and not args.no_table:
        gx = ctx.gauge(DIMS, U, "f64x", 18)
        tune_gauge(tmhop, ctx, gx)
        sx, dx = ctx.pack(psi, "f64x"), ctx.empty(vh, "f64x")
        n = max(1, min(args.steps, args.table_steps))
        tx, ax_ms, bx_ms = time_qtm(ctx, tmhop, torch, gx, sx, dx, n, args.warmup, barrier)
        sx_ms = allmax(tx) / n
        f64x = {"storage": "f64x-18", "dtype": "f32x2 double-float (~48-bit significand)",
                "ms_per_qtm": round(sx_ms, 4), "GBps": round(job_throughput(world, vh, ab["qtm"], sx_ms), 1),
                "gflops": round(world * vh * QTM_FLOPS / (sx_ms * 1e-3) / 1e9, 1),
                "speedup_vs_native_f64": round(ms_per_step / sx_ms, 2),
                "kernel_b_ms": round(bx_ms, 4), "traffic": traffic_per_launch("f64x", 18, vh),
                "parity": "relative L2 ~3e-15 against the FP64 oracle (FP64 bar 1e-13), tested",
                "note": "FP64 values stored as FP32 (hi, lo) pairs, error-free transformations on the FP32 "
                        "pipes; GB300 issues 64 FP32 FMAs per FP64 FMA"}
        gx.close()
        del sx, dx

    # ---- end to end through the C ABI with host buffers (pinned), copies in the timed region:
    # tm_Qtm_host over `ne` host-resident fields, each copied in, packed,
    # multiplied, unpacked and copied out (copies of neighbouring fields
    # overlap the kernels on two copy streams)
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(np.ascontiguousarray(psi)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        ne = max(1, min(args.steps, args.e2e_steps))
        stream = torch.cuda.current_stream()
        for _ in range(max(1, args.warmup // 4)):
            tmhop.tm_Qtm_host(ctx.handle, g.handle, [host_out] * 4, [host_in] * 4, KAPPA, MU, 1, stream.cuda_stream)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        s0.record(stream)
        tmhop.tm_Qtm_host(ctx.handle, g.handle, [host_out] * ne, [host_in] * ne, KAPPA, MU, 1, stream.cuda_stream)
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = allmax(s0.elapsed_time(s1)) / ne
        nbytes = host_in.numel() * 16
        e2e = {"value": round(world * vh * ab["qtm"] / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": round(e2e_ms, 4),
               "steps": ne,
               # FP64: the two hops read and write the canonical host layout themselves; other formats add
               # a pack and an unpack launch per field
               "gpu_launches_per_step": 2 if prec == "f64" else 4,
               "api": "tm_Qtm_host (pinned host fields, pipelined copies)"}
        del host_in, host_out
    links_gb = tmhop.tm_gauge_bytes(g.handle) / 1e9
    g.close()

    # ---- storage-precision table (HBM-bound variants)
    table = {}
    if not args.no_table:
        for tp, tr in (("f64", 12), ("f64x", 18), ("f64x", 12), ("f32", 18), ("f32", 12), ("f16", 12)):
            gp = ctx.gauge(DIMS, U, tp, tr)
            gmap = tune_gauge(tmhop, ctx, gp)
            sp = ctx.pack(psi, tp)
            dp = ctx.empty(vh, tp)
            n = max(1, min(args.steps, args.table_steps))
            t_ms, a_ms, b_ms = time_qtm(ctx, tmhop, torch, gp, sp, dp, n, args.warmup, barrier)
            abp = algo_bytes(tp, tr)
            step_ms = allmax(t_ms) / n
            bgbs = vh * abp["kernel_b"] / (b_ms * 1e-3) / 1e9
            table[f"{tp}-{tr}"] = {
                "ms_per_qtm": round(step_ms, 4), "GBps": round(vh * abp["qtm"] / (step_ms * 1e-3) / 1e9, 1),
                "gflops": round(vh * QTM_FLOPS / (step_ms * 1e-3) / 1e9, 1),
                "kernel_b_ms": round(b_ms, 4), "kernel_b_GBps": round(bgbs, 1),
                "kernel_b_hbm_frac": round(bgbs / hbm_peak, 4),
                "kernel_b_nominal_frac": round(bgbs / HBM_NOMINAL_GBS, 4), "kernel_a_ms": round(a_ms, 4),
                "site_map": gmap}
            gp.close()
            del sp, dp

    # ---- the non-degenerate twisted doublet (two flavours, links loaded once for both)
    nd = sw = slabs = None
    if not args.no_table:
        nd = nd_section(args, ctx, tmhop, torch, F, U, DIMS, vh, hbm_peak, allmax)
        sw = clover_section(args, ctx, tmhop, torch, F, U, DIMS, vh, hbm_peak, allmax)
        slabs = slab_section(args, ctx, tmhop, torch, F, U, DIMS, vh)

    # ---- CG on Q^dag Q to true relative residual 1e-10: FP64 vs mixed precision
    cg = None
    cg_host = None
    if not args.no_cg:
        cg, cg_host = cg_section(args, ctx, tmhop, torch, F, allmax, barrier, keep_host=(rank == 0 and not args.no_cpu))

    # ---- batching: 12 right-hand sides on 32^3x64 and 8 uneven lattices, FP32 storage
    batch = None
    if not args.no_batch:
        batch = batch_section(args, ctx, tmhop, torch, F, allmax, barrier, U if DIMS == (32, 32, 32, 64) else None)

    # ---- differentiation: S = phi^dag (Q^dag Q)^-1 phi and dS/dphi, dS/dU on 24^3x48
    grad = None
    if not args.no_grad:
        grad = grad_section(args, ctx, tmhop, torch, F)

    # ---- CPU baseline: the FP64 oracle on this host's cores, same lattice
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle as O
        O.build()
        t = time.perf_counter()
        n = 0
        while True:
            O.Qtm(DIMS, U, psi, KAPPA, MU)
            n += 1
            if time.perf_counter() - t > args.cpu_seconds or n >= 8:
                break
        dt = (time.perf_counter() - t) / n
        lat = "x".join(str(d) for d in DIMS)
        cpu = {"value": round(vh * ab["qtm"] / dt / 1e9, 3), "unit": "GB/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
               "kind": "oracle", "sample": f"{n} full Q_tm applications on {lat} (FP64, OpenMP over sites)",
               "s_per_qtm": round(dt, 3), "gflops": round(vh * QTM_FLOPS / dt / 1e9, 3)}
        if cg_host is not None:
            # the FP64 oracle CG on the CG lattice would take about an hour:
            # time what one of its iterations costs, one Q_tm and one literal
            # Q_tm^dag (its Q^dag Q; the vector updates are negligible beside
            # them), and scale by the GPU FP64 solver's iteration count
            cdims, cU, cb = cg_host
            t = time.perf_counter()
            O.Qtm(cdims, cU, O.Qtm(cdims, cU, cb, KAPPA, MU), KAPPA, MU, dagger=True)
            per_it = time.perf_counter() - t
            iters = cg["fp64"]["iters"]
            cpu["cg_estimate"] = {
                "lattice": list(cdims), "kind": "estimate", "s_per_iter": round(per_it, 3), "iters": iters,
                "seconds": round(per_it * iters, 1),
                "speedup_of_gpu_fp64": round(per_it * iters / cg["fp64"]["seconds"], 1),
                "speedup_of_gpu_best": round(per_it * iters / min(v["seconds"] for v in cg.values()
                                                                   if isinstance(v, dict) and "seconds" in v), 1),
                "how": "one oracle Q_tm plus one oracle Q_tm^dag (its CG's Q^dag Q) x the GPU FP64 iteration count"}
            del cg_host, cU, cb

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
            "config": dict(workload_config(DIMS, prec, recon, world),
                           l2=f"inputs larger than L2 ({links_gb:.2f} GB links "
                              f"+ {tmhop.tm_spinor_bytes(vh, tmhop.PREC[prec]) / 1e9:.3f} GB spinor read per step), no flush"),
            "gflops": round(gflops, 2), "roofline": roofline, "fp64_probe": probe, "hbm_peak_gbs": hbm_peak,
            "hbm_peak_source": hbm_src,
            "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": ck, "precisions": table, "nd_doublet": nd, "clover": sw, "slabs": slabs, "f64x_equivalent": f64x, "cg": cg, "batch": batch, "grad": grad,
            "cpu_baseline": cpu, "paper_context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# The paper's own figures on its hardware, as context (not targets, no
# ratio): it prints its hopping-matrix and inverter throughput only in plots
# that its text does not contain; these are the figures its prose states.
PAPER_CONTEXT = {
    "note": "figures stated in the text of arXiv:1311.4521 for its CPU machines; "
            "its throughput plots are not in the text",
    "items": [
        {"what": "loss of the hop's floating-point rate from OpenMP threading (1 process x 64 threads "
                 "against 64 processes per node, communication off)",
         "value": "about 11 GFlop/s per node", "hardware": "IBM BlueGene/Q (JuQueen), 32 nodes, 12^4 sites per node",
         "where": "Sec. 3"},
        {"what": "gain from overlapping the halo exchange with the hop's body",
         "value": "about 100 MFlop/s per core", "hardware": "Cray XC30 and SuperMUC", "where": "Sec. 2.5"},
        {"what": "full-spinor hop with a precomputed neighbour-index order (g_hi) against "
                 "two-dimensional neighbour tables",
         "value": "almost 20 % faster", "hardware": "multi-core Intel CPUs", "where": "Sec. 2.2"},
    ],
}


def nd_section(args, ctx, tmhop, torch, F, U, dims, vh, hbm_peak, allmax) -> dict:
    """The non-degenerate twisted doublet Q_nd (mu_sigma = 0.0015, mu_delta =
    0.0018) on the workload lattice in FP64-18, FP32-12 and FP16-12: ms per
    application and launch B's algorithmic GB/s.  Per even site, launch A
    reads two flavours' spinors and the 8 links once and writes two
    flavours; launch B also re-reads both even inputs."""
    psi_s = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    psi_c = F.gaussian_spinor(vh, F.SEED_PROD_32, 2)
    out = {"mu_sigma": 0.0015, "mu_delta": 0.0018}
    stream = torch.cuda.current_stream()
    for prec, recon in (("f64", 18), ("f32", 12), ("f16", 12)):
        g = ctx.gauge(dims, U, prec, recon)
        ins = [ctx.pack(psi_s, prec), ctx.pack(psi_c, prec)]
        outs = [ctx.empty(vh, prec), ctx.empty(vh, prec)]
        n = max(3, min(args.steps, args.table_steps))
        for _ in range(args.warmup):
            ctx.Qnd(g, outs, ins, KAPPA, 0.0015, 0.0018)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        for trio in ev:
            for e in trio:
                e.record(stream)
        torch.cuda.synchronize()
        for k in range(n):
            tmhop.tm_ctx_trace(ctx.handle, ev[k])
            ctx.Qnd(g, outs, ins, KAPPA, 0.0015, 0.0018)
        tmhop.tm_ctx_trace(ctx.handle, None)
        torch.cuda.synchronize()
        total = allmax(sum(e[0].elapsed_time(e[2]) for e in ev) / n)
        kb = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
        sp = 24 * REAL[prec] + (4 if prec == "f16" else 0)      # one spinor per site
        links = 8 * recon * REAL[prec]
        a_bytes, b_bytes = 2 * (sp + sp) + links, 2 * (sp + sp + sp) + links
        gbs = vh * b_bytes / (kb * 1e-3) / 1e9
        out[f"{prec}-{recon}"] = {"ms_per_qnd": round(total, 4), "kernel_b_ms": round(kb, 4),
                                  "GBps": round(vh * (a_bytes + b_bytes) / (total * 1e-3) / 1e9, 1),
                                  "kernel_b_GBps": round(gbs, 1), "kernel_b_hbm_frac": round(gbs / hbm_peak, 4),
                                  "gflops": round(vh * 2 * (2 * HOP_FLOPS) / (total * 1e-3) / 1e9, 1)}
        g.close()
        del ins, outs
    out["note"] = ("bytes per even site: launch A 2 x (in + out) + 8 links, launch B 2 x (in + out + x) + 8 links; "
                   "flops counted: the two flavours' hops (2 x 2 x 1320)")
    return out


def slab_section(args, ctx, tmhop, torch, F, U, dims, vh) -> dict:
    """Q_tm on the workload lattice cut into n = 1, 2, 4 time slabs on this
    one GPU (paper_1311_4521_gb300.slab.LocalSlabs: per hop, the faces are
    packed, copied on a second stream while the interior runs, and the face
    sites run last), FP64-18 and FP32-12, against the monolithic Q_tm: what
    the surface/body split costs in launches and face traffic.  All slabs
    run one after the other here, so `ms_per_slab` = ms / n is one slab's
    share; across GPUs the slabs would run at once (not measured: one GPU)."""
    from paper_1311_4521_gb300.slab import LocalSlabs
    psi = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    stream = torch.cuda.current_stream()
    out = {"note": "n slabs of one lattice on one GPU, run in turn; ms_per_slab = ms / n"}
    reps = max(3, min(args.steps, 50))

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for prec, recon in (("f64", 18), ("f32", 12)):
        g = ctx.gauge(dims, U, prec, recon)
        src, dst = ctx.pack(psi, prec), ctx.empty(vh, prec)
        mono = timed(lambda: ctx.Qtm(g, dst, src, KAPPA, MU))
        g.close()
        row = {"monolithic_ms": round(mono, 4)}
        for n in (1, 2, 4):
            sl = LocalSlabs(ctx, dims, U, n, prec, recon)
            ins, outs = sl.pack_fields(psi), sl.empty()
            ms = timed(lambda: sl.Qtm(outs, ins, KAPPA, MU))
            entry = {"ms": round(ms, 4), "ms_per_slab": round(ms / n, 4),
                     "overhead_vs_monolithic": round(ms / mono - 1.0, 4)}
            # the same schedule captured once in a CUDA graph: without the
            # per-call host submission of its 6n launches and 4n copies
            try:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    sl.Qtm(outs, ins, KAPPA, MU)
                gms = timed(graph.replay)
                entry.update({"graph_ms": round(gms, 4), "graph_overhead_vs_monolithic": round(gms / mono - 1.0, 4)})
                del graph
            except Exception as exc:   # capture is an extra measurement, not part of the schedule
                entry["graph_ms"] = None
                entry["graph_note"] = f"capture failed: {type(exc).__name__}"
            sl.close()
            row[f"{n}_slabs"] = entry
        out[f"{prec}-{recon}"] = row
    return out


def clover_section(args, ctx, tmhop, torch, F, U, dims, vh, hbm_peak, allmax) -> dict:
    """The clover twisted-mass operator Q_sw (c_sw = 1.76) on the workload
    lattice in FP64-18 and FP32-12: ms per application and launch B's
    algorithmic GB/s (per even site: the input, the output, 8 links and the
    site's two 6x6 complex blocks, plus the re-read input in launch B), and
    the one-time cost of building the blocks."""
    psi = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    out = {"csw": 1.76}
    stream = torch.cuda.current_stream()
    for prec, recon in (("f64", 18), ("f32", 12)):
        g = ctx.gauge(dims, U, prec, recon)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        C = ctx.clover(g, U, 1.76, KAPPA, MU)
        e1.record(stream)
        torch.cuda.synchronize()
        setup_ms = e0.elapsed_time(e1)
        src, dst = ctx.pack(psi, prec), ctx.empty(vh, prec)
        n = max(3, min(args.steps, args.table_steps))
        for _ in range(args.warmup):
            ctx.Qsw(g, C, dst, src)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        for trio in ev:
            for e in trio:
                e.record(stream)
        torch.cuda.synchronize()
        for k in range(n):
            tmhop.tm_ctx_trace(ctx.handle, ev[k])
            ctx.Qsw(g, C, dst, src)
        tmhop.tm_ctx_trace(ctx.handle, None)
        torch.cuda.synchronize()
        total = allmax(sum(e[0].elapsed_time(e[2]) for e in ev) / n)
        kb = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
        sp = 24 * REAL[prec]
        blocks = 72 * 2 * REAL[prec]
        b_bytes = 3 * sp + 8 * recon * REAL[prec] + blocks
        a_bytes = 2 * sp + 8 * recon * REAL[prec] + blocks
        gbs = vh * b_bytes / (kb * 1e-3) / 1e9
        out[f"{prec}-{recon}"] = {"ms_per_qsw": round(total, 4), "kernel_b_ms": round(kb, 4),
                                  "GBps": round(vh * (a_bytes + b_bytes) / (total * 1e-3) / 1e9, 1),
                                  "kernel_b_GBps": round(gbs, 1), "kernel_b_hbm_frac": round(gbs / hbm_peak, 4),
                                  "block_setup_ms": round(setup_ms, 2),
                                  "block_bytes": tmhop.tm_clover_bytes(C)}
        tmhop.tm_clover_destroy(C)
        g.close()
        del src, dst
    return out


def cg_section(args, ctx, tmhop, torch, F, allmax, barrier, keep_host=False):
    """Time to a true relative residual of 1e-10 for Q^dag Q x = b on the CG
    lattice (48^3x96 by default, U = exp(0.3 i A), Gaussian source): plain
    FP64 CG against mixed precision with FP32 and FP16 storage (FP32
    arithmetic, FP64 reliable updates).  Each solver runs once to warm up,
    then once timed with CUDA events around the (synchronous) call.
    Returns the results and, with keep_host, the host links and source (for
    the oracle's time estimate), else None."""
    dims = args.cg_lattice
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_CG_48, "near", 0.3)
    b = F.gaussian_spinor(vh, F.SEED_CG_48, 1)
    gh = ctx.gauge(dims, U, "f64", 18)
    gx = ctx.gauge(dims, U, "f64x", 18)
    lo = {"mixed_f32": ctx.gauge(dims, U, "f32", 12), "mixed_f16": ctx.gauge(dims, U, "f16", 12)}
    host = (dims, U, b) if keep_host else None
    del U
    bd = ctx.pack(b, "f64")
    bx = ctx.pack(b, "f64x")
    x = ctx.empty(vh, "f64")
    out = {"lattice": list(dims), "tol": 1e-10, "kappa": KAPPA, "mu": MU, "reliable_every": 50,
           "reliable_delta": args.cg_delta if args.cg_delta >= 0 else {"f32": 1e-3, "f16": 2 ** -5.5}, "source": "Gaussian, seed 2013", "time": "CUDA events around one warm solve"}
    stream = torch.cuda.current_stream()
    runs = (("fp64", gh, bd, None), ("mixed_f32", gh, bd, lo["mixed_f32"]), ("mixed_f16", gh, bd, lo["mixed_f16"]),
            ("fp64x", gx, bx, None), ("mixed_f32_fp64x", gx, bx, lo["mixed_f32"]),
            ("mixed_f16_fp64x", gx, bx, lo["mixed_f16"]))
    for name, ghi, bb, gl in runs:
        for rep in range(2):
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            st, info = ctx.cg(ghi, x, bb, KAPPA, MU, 1e-10, 30000, gl, 50, True, args.cg_delta)
            e1.record(stream)
            torch.cuda.synchronize()
        sec = allmax(e0.elapsed_time(e1) / 1e3)
        out[name] = {"seconds": round(sec, 4), "iters": info["iters"], "reliable_updates": info["reliable_updates"],
                     "true_relres": info["true_relres"], "converged": st == tmhop.TM_OK}
    for name in ("mixed_f32", "mixed_f16", "fp64x", "mixed_f32_fp64x", "mixed_f16_fp64x"):
        out[name]["speedup_vs_fp64"] = round(out["fp64"]["seconds"] / out[name]["seconds"], 2)
    out["fp64x_note"] = ("fp64x: x, b and the reliable updates in double-float storage/arithmetic (TM_F64X, "
                         "~48-bit significand); convergence still judged on the true residual")
    for g in [gh, gx] + list(lo.values()):
        g.close()
    return out, host


def only_section(args, ctx, tmhop, torch, F, U, psi, dims, vh, barrier, allmax) -> dict:
    """One part of the benchmark alone, for profiling captures:
    batch-qtm  Q_tm on 12 right-hand sides of --lattice, --steps batched calls;
    cg         the CG section on --cg-lattice;
    force      the force call (3 hops + assembly by --force-scheme) on
               --lattice, --steps calls;
    solve      the even-odd full-lattice solve on --lattice (FP32 inner);
    nd         the non-degenerate doublet Q_nd on --lattice, --steps calls;
    clover     the clover operator Q_sw (c_sw 1.76) on --lattice, --steps calls.
    --batch-code fixes the batched hop's configuration for batch-qtm (e.g.
    100, the TMA-staged hop); -1 leaves it to the autotuner."""
    res = {"only": args.only, "lattice": list(dims)}
    stream = torch.cuda.current_stream()
    def timed_calls(fn):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    if args.only == "nd":
        g = ctx.gauge(dims, U, args.prec, args.recon)
        ins = [ctx.pack(psi, args.prec), ctx.pack(F.gaussian_spinor(vh, F.SEED_PROD_32, 2), args.prec)]
        outs = [ctx.empty(vh, args.prec), ctx.empty(vh, args.prec)]
        res["ms_per_qnd"] = timed_calls(lambda: ctx.Qnd(g, outs, ins, KAPPA, 0.0015, 0.0018))
        g.close()
    elif args.only == "clover":
        g = ctx.gauge(dims, U, args.prec, args.recon)
        C = ctx.clover(g, U, 1.76, KAPPA, MU)
        src, dst = ctx.pack(psi, args.prec), ctx.empty(vh, args.prec)
        res["ms_per_qsw"] = timed_calls(lambda: ctx.Qsw(g, C, dst, src))
        tmhop.tm_clover_destroy(C)
        g.close()
    elif args.only == "batch-qtm":
        tmhop.tm_ctx_set_batch_config(ctx.handle, args.batch_code, args.batch_cap)
        res["batch_code"], res["batch_cap"] = args.batch_code, args.batch_cap
        g = ctx.gauge(dims, U, args.prec, args.recon)
        ins = [ctx.pack(F.gaussian_spinor(vh, F.SEED_BATCH_RHS + j, 0), args.prec) for j in range(12)]
        outs = [ctx.empty(vh, args.prec) for _ in range(12)]
        for _ in range(args.warmup):
            ctx.Qtm_batch([g] * 12, outs, ins, KAPPA, MU)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.Qtm_batch([g] * 12, outs, ins, KAPPA, MU)
        e1.record(stream)
        torch.cuda.synchronize()
        res["ms_per_batched_qtm"] = e0.elapsed_time(e1) / args.steps
        tmhop.tm_ctx_check(ctx.handle)
        tmhop.tm_ctx_set_batch_config(ctx.handle, -1, 0)
        g.close()
    elif args.only == "cg":
        args.cg_lattice = dims
        res.update(cg_section(args, ctx, tmhop, torch, F, allmax, barrier)[0])
    elif args.only == "force":
        g = ctx.gauge(dims, U, args.prec, args.recon)
        xp = ctx.pack(psi, args.prec)
        sch = {"owner": tmhop.TM_FORCE_OWNER, "atomic": tmhop.TM_FORCE_ATOMIC,
               "halo": tmhop.TM_FORCE_HALO}[args.force_scheme]
        res["scheme"] = args.force_scheme
        for _ in range(args.warmup):
            ctx.force(g, xp, KAPPA, MU, tmhop.TM_FORCE_SU3, sch)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.force(g, xp, KAPPA, MU, tmhop.TM_FORCE_SU3, sch)
        e1.record(stream)
        torch.cuda.synchronize()
        res["ms_per_force"] = e0.elapsed_time(e1) / args.steps
        g.close()
    elif args.only == "solve":
        gh, gl = ctx.gauge(dims, U, "f64", 18), ctx.gauge(dims, U, "f32", 12)
        be, bo = ctx.pack(psi, "f64"), ctx.pack(F.gaussian_spinor(vh, F.SEED_PROD_32, 2), "f64")
        xe, xo = ctx.empty(vh, "f64").zero_(), ctx.empty(vh, "f64")
        ctx.solve_eo(gh, xe, xo, be, bo, KAPPA, MU, 1e-10, 30000, gl)   # warm-up (workspace, graphs)
        xe.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st, info = ctx.solve_eo(gh, xe, xo, be, bo, KAPPA, MU, 1e-10, 30000, gl)
        e1.record(stream)
        torch.cuda.synchronize()
        res.update({"status": st, "info": info, "seconds_total": round(e0.elapsed_time(e1) / 1e3, 4),
                    "note": "seconds_total: the whole even-odd solve (source preparation, CG, reconstruction); "
                            "info.seconds: its CG"})
        gh.close()
        gl.close()
    return res


def grad_section(args, ctx, tmhop, torch, F) -> dict:
    """24^3x48, U = exp(0.3 i A): the action S = phi^dag (Q^dag Q)^-1 phi
    through autograd (forward solve + backward force), and the force call
    alone (its three hops plus the force assembly) for each way of
    assembling the per-link force (one owner thread per link, pushes with
    FP64 atomics, pushes into private buffers plus a summing pass), and the
    link gradient of Re <Y, Q_tm X> (tm_link_grad, the backward of the
    autograd Q_tm), FP64 and FP32 storage (for information: correctness is
    covered by the tests)."""
    from paper_1311_4521_gb300 import autograd
    dims = (24, 24, 24, 48)
    vh = int(np.prod(dims)) // 2
    U = F.gauge_field(dims, F.SEED_GRAD_24, "near", 0.3)
    phi = F.gaussian_spinor(vh, F.SEED_GRAD_24, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    Ut = torch.from_numpy(U).to(dev).requires_grad_(True)
    pt = torch.from_numpy(phi).to(dev).requires_grad_(True)
    out = {"lattice": list(dims), "kappa": KAPPA, "mu": MU}
    stream = torch.cuda.current_stream()
    for inner, fprec in (("f64", "f64"), ("f32", "f32")):
        for rep in range(2):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record(stream)
            S = autograd.action(pt, Ut, dims, KAPPA, MU, tol=1e-10, inner=inner, force_prec=fprec)
            e1.record(stream)
            gphi, gU = torch.autograd.grad(S, (pt, Ut))
            e2.record(stream)
            torch.cuda.synchronize()
        g = ctx.gauge(dims, U, fprec, 18 if fprec == "f64" else 12)
        xp = ctx.pack(gphi.detach() / 2, fprec)
        sch_ms = {}
        for name, sch in (("owner", tmhop.TM_FORCE_OWNER), ("atomic", tmhop.TM_FORCE_ATOMIC),
                          ("halo", tmhop.TM_FORCE_HALO)):
            fe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ctx.force(g, xp, KAPPA, MU, tmhop.TM_FORCE_SU3, sch)
            fe[0].record(stream)
            for _ in range(10):
                ctx.force(g, xp, KAPPA, MU, tmhop.TM_FORCE_SU3, sch)
            fe[1].record(stream)
            torch.cuda.synchronize()
            sch_ms[name] = round(fe[0].elapsed_time(fe[1]) / 10, 4)
        # the link gradient of Re <Y, Q_tm X> (the backward of autograd.qtm): two hops + the per-link kernel
        yp = ctx.pack(phi, fprec)
        lg = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ctx.link_grad(g, xp, yp, tmhop.TM_GRAD_QTM, KAPPA, MU)
        lg[0].record(stream)
        for _ in range(10):
            ctx.link_grad(g, xp, yp, tmhop.TM_GRAD_QTM, KAPPA, MU)
        lg[1].record(stream)
        torch.cuda.synchronize()
        g.close()
        out[f"{inner}_solve_{fprec}_force"] = {
            "forward_s": round(e0.elapsed_time(e1) / 1e3, 4), "backward_s": round(e1.elapsed_time(e2) / 1e3, 4),
            "force_ms": sch_ms["owner"], "force_ms_by_scheme": sch_ms, "S": float(S.item()),
            "link_grad_qtm_ms": round(lg[0].elapsed_time(lg[1]) / 10, 4)}
    return out


UNEVEN = [(16, 16, 16, 32), (20, 20, 20, 40), (24, 24, 24, 48), (28, 28, 28, 56), (32, 32, 32, 64),
          (16, 16, 16, 64), (24, 24, 24, 32), (12, 12, 12, 24)]


def batch_section(args, ctx, tmhop, torch, F, allmax, barrier, U32=None) -> dict:
    """Batching workload, FP32 storage (12-real links): (a) Q_tm on 12
    right-hand sides of one 32^3x64 lattice in one launch per hop, against 12
    single Q_tm calls; (b) CG to 1e-10 on the 12 right-hand sides and (c) on
    8 lattices of uneven volume (sum of V = 5,187,072 sites), each batch in
    one call against the same systems solved one after the other; (d) Q_tm
    on the 8 uneven lattices and (e) on 64 lattices of 8^4 in one call
    against one call per lattice."""
    big = (32, 32, 32, 64)
    vh = int(np.prod(big)) // 2
    if U32 is None:
        U32 = F.gauge_field(big, F.SEED_PROD_32, "near", 0.3)
    g32 = ctx.gauge(big, U32, "f32", 12)
    g64 = ctx.gauge(big, U32, "f64", 18)
    rhs = [F.gaussian_spinor(vh, F.SEED_BATCH_RHS + j, 0) for j in range(12)]
    ins = [ctx.pack(r, "f32") for r in rhs]
    outs = [ctx.empty(vh, "f32") for _ in rhs]
    stream = torch.cuda.current_stream()
    out = {"storage": "f32-12", "kappa": KAPPA, "mu": MU}

    def timed(fn, reps):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return allmax(e0.elapsed_time(e1) / reps)

    reps = max(3, min(50, args.steps // 20))
    ms_batch = timed(lambda: ctx.Qtm_batch([g32] * 12, outs, ins, KAPPA, MU), reps)
    ms_single = timed(lambda: [ctx.Qtm(g32, o, i, KAPPA, MU) for o, i in zip(outs, ins)], reps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for e in ev:
        e.record(stream)
    tmhop.tm_ctx_trace(ctx.handle, ev)
    ctx.Qtm_batch([g32] * 12, outs, ins, KAPPA, MU)
    tmhop.tm_ctx_trace(ctx.handle, None)
    torch.cuda.synchronize()
    kb_ms = ev[1].elapsed_time(ev[2])
    # the autotuner's choice for this batch, and the TMA-staged hop (code 100) forced, for comparison
    tuned = next(([w for w in ln.split()[1:] if not w.startswith("ms3=")] for ln in tmhop.tm_ctx_tune_report(ctx.handle).splitlines()
                  if ln.startswith("bhop/1/12/%dx12" % vh)), [])
    tmhop.tm_ctx_set_batch_config(ctx.handle, 100, 0)
    staged_b = []
    for _ in range(4):
        tmhop.tm_ctx_trace(ctx.handle, ev)
        ctx.Qtm_batch([g32] * 12, outs, ins, KAPPA, MU)
        tmhop.tm_ctx_trace(ctx.handle, None)
        torch.cuda.synchronize()
        staged_b.append(ev[1].elapsed_time(ev[2]))
    tmhop.tm_ctx_set_batch_config(ctx.handle, -1, 0)
    tmhop.tm_ctx_check(ctx.handle)
    staged_ms = float(np.median(staged_b[1:]))
    ctx.Qtm_batch([g32] * 12, outs, ins, KAPPA, MU)   # back to the tuned tables
    # bytes per even site and right-hand side: 2 hops of (spinor in + out + 8 links / 12) + psi_e re-read
    per = 2 * (96 + 96 + 384 / 12) + 96
    out["qtm_12rhs"] = {"ms_batched": round(ms_batch, 4), "ms_12_single_calls": round(ms_single, 4),
                        "speedup": round(ms_single / ms_batch, 2),
                        "GBps_algorithmic_amortised_links": round(12 * vh * per / (ms_batch * 1e-3) / 1e9, 1),
                        "kernel_b_ms": round(kb_ms, 4),
                        "kernel_b_GBps": round(12 * vh * (96 + 96 + 384 / 12 + 96) / (kb_ms * 1e-3) / 1e9, 1),
                        "tuned_config": " ".join(tuned),
                        "tma_staged_kernel_b_ms": round(staged_ms, 4),
                        "tma_staged_kernel_b_GBps": round(12 * vh * (96 + 96 + 384 / 12 + 96) / (staged_ms * 1e-3) / 1e9,
                                                          1)}
    del ins, outs

    def solve_batch(gh, gl, bs):
        xs = [ctx.empty(b.numel() // 192, "f64").zero_() for b in bs]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st, infos = ctx.cg_batch(gh, xs, bs, KAPPA, MU, 1e-10, 30000, gl)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, st, infos

    def solve_each(gh, gl, bs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        its = []
        for h, l, b in zip(gh, gl, bs):
            x = ctx.empty(b.numel() // 192, "f64").zero_()
            st, inf = ctx.cg(h, x, b, KAPPA, MU, 1e-10, 30000, l)
            its.append(inf["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, its

    bs = [ctx.pack(r, "f64") for r in rhs]
    solve_batch([g64] * 12, [g32] * 12, bs)   # warm-up (workspace, tuning)
    tb, st, infos = solve_batch([g64] * 12, [g32] * 12, bs)
    solve_each([g64] * 12, [g32] * 12, bs)
    te, its = solve_each([g64] * 12, [g32] * 12, bs)
    out["cg_12rhs_32x32x32x64"] = {"seconds_batched": round(allmax(tb), 4), "seconds_one_by_one": round(allmax(te), 4),
                                   "speedup": round(te / tb, 2), "converged": st == tmhop.TM_OK,
                                   "iters": [i["iters"] for i in infos],
                                   "max_true_relres": max(i["true_relres"] for i in infos)}
    del bs
    g32.close()
    g64.close()
    del U32
    lats = [(d, F.gauge_field(d, F.SEED_BATCH_LATTICE + k, "near", 0.3)) for k, d in enumerate(UNEVEN)]
    gh = [ctx.gauge(d, U, "f64", 18) for d, U in lats]
    gl = [ctx.gauge(d, U, "f32", 12) for d, U in lats]
    bs = [ctx.pack(F.gaussian_spinor(int(np.prod(d)) // 2, F.SEED_BATCH_LATTICE + k, 1), "f64")
          for k, (d, _) in enumerate(lats)]
    del lats
    solve_batch(gh, gl, bs)
    tb, st, infos = solve_batch(gh, gl, bs)
    solve_each(gh, gl, bs)
    te, its = solve_each(gh, gl, bs)
    out["cg_8_uneven_lattices"] = {"lattices": [list(d) for d in UNEVEN], "sites": int(sum(np.prod(d) for d in UNEVEN)),
                                   "seconds_batched": round(allmax(tb), 4), "seconds_one_by_one": round(allmax(te), 4),
                                   "speedup": round(te / tb, 2), "converged": st == tmhop.TM_OK,
                                   "iters": [i["iters"] for i in infos],
                                   "max_true_relres": max(i["true_relres"] for i in infos)}
    # (d) Q_tm on the 8 uneven lattices in one call vs 8 calls, and (e) on 64
    # small 8^4 lattices (an ensemble of small problems), FP32-12
    def many_lattices(dims_list, seed0):
        gs, ins_, outs_ = [], [], []
        for k, d in enumerate(dims_list):
            gs.append(ctx.gauge(d, F.gauge_field(d, seed0 + k, "near", 0.3), "f32", 12))
            v = int(np.prod(d)) // 2
            ins_.append(ctx.pack(F.gaussian_spinor(v, seed0 + k, 2), "f32"))
            outs_.append(ctx.empty(v, "f32"))
        r = max(3, min(50, args.steps // 20))
        mb = timed(lambda: ctx.Qtm_batch(gs, outs_, ins_, KAPPA, MU), r)
        ms = timed(lambda: [ctx.Qtm(g, o, i, KAPPA, MU) for g, o, i in zip(gs, outs_, ins_)], r)
        for g in gs:
            g.close()
        return {"lattices": len(dims_list), "sites": int(sum(np.prod(d) for d in dims_list)),
                "ms_batched": round(mb, 4), "ms_one_call_each": round(ms, 4), "speedup": round(ms / mb, 2)}

    out["qtm_8_uneven_lattices"] = many_lattices(UNEVEN, F.SEED_BATCH_LATTICE)
    out["qtm_8_uneven_lattices"]["note"] = (
        "every lattice but 12^3x24 has >= 65,536 even sites (>= 430 per SM) and fills the GPU alone: "
        "one persistent launch for all eight saves launches, not time")
    out["qtm_64_lattices_8x8x8x8"] = many_lattices([(8, 8, 8, 8)] * 64, F.SEED_BATCH_LATTICE + 1000)
    out["qtm_64_lattices_8x8x8x8"]["note"] = "1,024 even sites per lattice, less than one CTA per SM: batching pays"
    for g in gh + gl:
        g.close()
    return out


# ---------------------------------------------------------------- reference arm
def reference_arm(args) -> None:
    """The FP64 CPU oracle as the reference implementation: each step is one
    Q_tm on a 16^4 sample lattice of the same link distribution, on this
    host's cores."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    from paper_1311_4521_gb300 import fields as F
    O.build()
    vh = int(np.prod(SAMPLE_DIMS)) // 2
    U = F.gauge_field(SAMPLE_DIMS, F.SEED_PROD_32, "near", 0.3)
    psi = F.gaussian_spinor(vh, F.SEED_PROD_32, 1)
    for _ in range(args.warmup):
        O.Qtm(SAMPLE_DIMS, U, psi, KAPPA, MU)
    t = time.perf_counter()
    for _ in range(args.steps):
        O.Qtm(SAMPLE_DIMS, U, psi, KAPPA, MU)
    dt = (time.perf_counter() - t) / args.steps
    ab = algo_bytes("f64", 18)
    value = vh * ab["qtm"] / dt / 1e9
    cores = int(os.environ["OMP_NUM_THREADS"])
    sample = ("one Q_tm per step on a 16^4 sample lattice of the workload (same link distribution, kappa, "
              "mu; FP64), its GB/s scaled per site to the workload's bytes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args.lattice, "f64", 18, args.gpus), sample_lattice=list(SAMPLE_DIMS)),
        "gflops": round(vh * QTM_FLOPS / dt / 1e9, 3),
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--lattice", type=lambda v: tuple(int(a) for a in v.split(",")), default=DIMS,
                    help="Lx,Ly,Lz,Lt (default 32,32,32,64)")
    ap.add_argument("--prec", choices=["f64", "f64x", "f32", "f16"], default="f64")
    ap.add_argument("--recon", type=int, choices=[12, 18], default=18)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--table-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture of this build")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-table", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--only", choices=["batch-qtm", "cg", "force", "solve", "nd", "clover"], default=None,
                    help="run one section alone (for profiling captures)")
    ap.add_argument("--batch-code", type=int, default=-1,
                    help="batched-hop configuration for --only batch-qtm (-1: autotuned; 100: TMA-staged)")
    ap.add_argument("--batch-cap", type=int, default=0,
                    help="persistent CTA cap with --batch-code (0: one CTA per work item; code 100: one per SM)")
    ap.add_argument("--cg-delta", type=float, default=-1.0,
                    help="reliable-update threshold of the mixed-precision solvers (residual drop factor); "
                         "negative: the library's automatic choice (FP32 1e-3, FP16 0.022)")
    ap.add_argument("--force-scheme", choices=["owner", "atomic", "halo"], default="owner",
                    help="force assembly for --only force")
    ap.add_argument("--cg-lattice", type=lambda v: tuple(int(a) for a in v.split(",")), default=(48, 48, 48, 96))
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
