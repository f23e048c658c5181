#!/usr/bin/env python
"""Throughput of the patch-AMR wave-propagation hot path on GB300.

Workload (one rank): an adaptive single-tree swirl forest, levels 2-6,
32x32 patches with 2 ghost layers, walls, MC limiter with transverse
corrections, CFL 0.9, multirate subcycling (16 finest substeps per coarse
step), regrid every 4 coarse steps, FP32.  A "step" is one coarse step: for
each level substep the ghost fill (Alg. 1 phases) and the patch update, plus
the regrid when it falls due.  Metric: cell updates per second, the paper's
rate (mx^2 x patch advances / wall time).

Variants on the same line: the same forest in FP64; a batched ensemble of
256 independent swirl forests (maximum level drawn from {4,5,6}) advanced
together -- one launch per level substep covers every forest -- at 32^2 and
16^2 patches and in FP64; the cubed sphere (levels 1-7, capacity form); and
the adjoint (gradient of a final-time misfit over 25 coarse multirate steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode full|batched|sphere|sphere_deform|adjoint|sweep]

Multi-GPU (torchrun): each rank advances its own independent forest (seeded
by rank): weak scaling, no collective on the data path.  Prints one JSON line
on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "cell-updates/s"
L2_FLUSH_BYTES = 512 << 20
WORKLOAD = ("adaptive swirl forest, levels 2-6, 32x32 patches, mbc 2, walls, MC + transverse, "
            "CFL 0.9, multirate, regrid every 4 coarse steps")
SPHERE_WORKLOAD = ("cubed sphere (6 trees), levels 1-7, 32x32 patches, mbc 2, solid-body rotation "
                   "|omega| = 2 pi, two cosine bells + slotted cylinder, capacity form, CFL 0.9, "
                   "multirate, regrid every 4 coarse steps")
SPHERE_DEFORM_WORKLOAD = ("cubed sphere (6 trees), levels 2-6, 32x32 patches, mbc 2, the deformational "
                          "flow of Sec. 5.3 (kappa 2, T 0.5, T_f 5; fluxes refreshed per substep), two "
                          "slotted cylinders, dt 2.5e-3 at level 2, multirate, max - min tagging "
                          "(0.25 / 0.001), regrid every coarse step")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--no-variants", action="store_true", help="skip FP64, batched and CPU legs")
    ap.add_argument("--ensemble", type=int, default=256, help="forests in the batched variant")
    ap.add_argument("--variant", default="auto",
                    help="update kernel of the headline (and --mode batched) forest: auto "
                         "(autotuned per launch size), or NAME[:WARPS] with NAME staged, walk, "
                         "walk1 or band -- e.g. to profile the kernels a default run's tuning "
                         "chose (a profiler distorts the tuner's timings)")
    ap.add_argument("--mode", choices=["full", "batched", "sphere", "sphere_deform", "adjoint",
                                       "sweep"],
                    default="full",
                    help="batched: time only the ensemble (a case sized for profiling)")
    return ap.parse_args()


def cell_updates(leaves: np.ndarray, lmin: int, mx: int) -> int:
    """mx^2 x patch advances of one coarse multirate step."""
    lev = leaves[:, 2].astype(np.int64)
    return int(np.sum((1 << (lev - lmin)) * mx * mx))


def q0_fn(workloads):
    mx = workloads[0].mx

    def q0(leaves):
        out = np.empty((len(leaves), mx, mx))
        for f in np.unique(leaves[:, 0]):
            sel = leaves[:, 0] == f
            w = workloads[int(f)]
            if w.domain == "sphere":
                out[sel] = synth.evaluate_sphere(w, synth.sphere_cell_centres(leaves[sel], mx))
            else:
                x, y = synth.cell_centres(leaves[sel], mx)
                out[sel] = synth.evaluate(w, x, y)
        return out
    return q0


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # the sampler's start-up (driver queries) must not land in the timed
        # steps: wait, bounded, for its first sample before they begin
        t_end = time.time() + 3.0
        while (self.proc is not None and self.proc.poll() is None and time.time() < t_end
               and os.path.getsize(self.f.name) == 0):
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_workload(rank: int):
    """The independent forest a rank advances (weak scaling: one forest per GPU)."""
    return synth.swirl(seed=rank)


def aggregate(values, ops, dist=None, device="cpu"):
    """Combine per-rank scalars across ranks: ops[k] is "max" (times) or "sum"
    (work).  The only collective of the run; it sits outside the data path."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    out = []
    for v, op in zip(values, ops):
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        out.append(float(t.item()))
    return out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ ours

class Runner:
    """One forest (or ensemble) on this rank's GPU, stepped coarse step by coarse step."""

    def __init__(self, fc, torch, workloads, dtype, variant="auto"):
        self.fc, self.torch, self.ws = fc, torch, workloads
        w = workloads[0]
        self.w = w
        self.lmax = max(x.lmax for x in workloads)
        self.lmax_f = [x.lmax for x in workloads]
        _, self.dtc = synth.time_step(w, self.lmax)
        domain = {"walls": fc.WALLS, "periodic": fc.PERIODIC, "sphere": fc.SPHERE}[w.domain]
        desc = fc.make_desc(domain=domain, mx=w.mx, lmin=w.lmin, lmax=self.lmax, dtype=dtype,
                            velocity=w.velocity, nforests=len(workloads),
                            indicator={"gradient": 0, "maxmin": 1}[w.indicator],
                            smooth=int(w.smooth))
        self.F = fc.initial_forest(desc, q0_fn(workloads), lmax_f=self.lmax_f,
                                   tau_r=w.tau_refine, tau_c=w.tau_coarsen)
        names = ["staged", "walk", "walk1", "band"]
        if variant != "auto":  # one kernel for every launch
            name, _, warps = variant.partition(":")
            warps = int(warps or 4)
            self.F.set_advance_variant(names.index(name), warps)
            self.tuning = {"all": {"variant": name, "warps": warps, "fill": "fused"}}
        else:
            # pick the patch-update kernel per launch size on this layout (untimed setup)
            self.tuning = {int(b): {"variant": names[v], "warps": k,
                                    "fill": "fused" if fu else "separate", "ns": ns}
                           for b, (v, k, fu, ns) in self.F.autotune().items()}
        self.n = 0

    def updates(self) -> int:
        return cell_updates(self.F.leaves(), self.w.lmin, self.w.mx)

    def step(self):
        self.F.step_multirate(self.n * self.dtc, self.dtc)
        self.n += 1
        if self.n % self.w.regrid_every == 0:
            self.F.tag_regrid(self.w.tau_refine, self.w.tau_coarsen, self.lmax_f)


def measure(runner, steps, warmup, flush_buf, clock_index):
    """W untimed warm-up steps, then the K timed steps (CUDA events around
    each step on the launching stream, L2 flushed before each, outside the
    events), then K more steps with the library's per-launch phase timers on
    (an event pair around every kernel, graph nodes included) for the
    per-kernel rooflines -- kept out of the timed steps, whose value they
    would otherwise slow down."""
    torch, fc, F = runner.torch, runner.fc, runner.F
    for _ in range(warmup):
        runner.step()
    torch.cuda.synchronize()
    fc.launch_count(reset=True)
    events, updates = [], 0
    with Clocks(clock_index) as clk:
        torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed region
        for _ in range(steps):
            flush_buf.zero_()  # a write larger than L2 between timed steps (untimed)
            updates += runner.updates()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            runner.step()
            e1.record()
            events.append((e0, e1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    launches = fc.launch_count()
    step_ms = [a.elapsed_time(b) for a, b in events]
    ms = sum(step_ms)
    # per-kernel timing pass
    F.timers(True)
    for ph in range(4):
        F.read_timer(ph, reset=True)
    for _ in range(steps):
        flush_buf.zero_()
        runner.step()
    torch.cuda.synchronize()
    phases = {k: F.read_timer(ph) for ph, k in enumerate(["advance", "fill", "regrid"])}
    F.timers(False)
    return dict(ms=ms, updates=updates, phases=phases, launches=launches,
                clocks=clk.summary(), patches=len(F), tuning=runner.tuning,
                step_ms_median=statistics.median(step_ms) if step_ms else None,
                step_ms_max=max(step_ms) if step_ms else None)


# DRAM bytes per patch advance of an update kernel at (element size, mx),
# from one ncu capture of every update launch of two timed coarse steps of the
# swirl forest (band, FP32, 32^2: 62 launches, 9706 patch advances, 84.8 MB
# read and nothing written back -- the new interiors stay in the 129 MB L2 --
# so 8734 B per patch against 9280 B algorithmic).  Reported while the
# kernel's sources are the ones captured (their hash; taken again after
# edits of host-only declarations in the shared header, the kernel unchanged)
# and every timed launch runs that kernel, else null.
DRAM_PER_PATCH = {("band", 4, 32): 8734.0}
KERNEL_SOURCES = {"band": ('advance_band.cu', 'ghost_gather.cuh', 'device_util.cuh', 'walk_edge.cuh', 'fc_internal.hpp')}
KERNEL_SOURCES_SHA = {"band": "16d2b9fd61c0685d"}


def sources_sha(variant):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[variant]:
        with open(os.path.join(ROOT, "paper_1703_03116_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(phase, tuning, esize, mx):
    """DRAM bytes per advance launch from the captured per-patch figure (the
    launches' patch counts from their algorithmic bytes), or None."""
    ms, n, nbytes = phase
    variants = {t["variant"] for t in tuning.values()} if tuning else set()
    if n <= 0 or len(variants) != 1:
        return None
    v = variants.pop()
    per = DRAM_PER_PATCH.get((v, esize, mx))
    if per is None or sources_sha(v) != KERNEL_SOURCES_SHA[v]:
        return None
    patches_per_launch = nbytes / n / (((mx + 4) ** 2 + mx * mx) * esize)
    return per * patches_per_launch


def roofline_of(phase, peak_gbs, peak_src, traffic=None):
    ms, n, nbytes = phase
    achieved = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": achieved / peak_gbs if achieved else None, "traffic": traffic,
            "kernel": "advance_kernel", "peak_source": peak_src, "timed_launches": n,
            "avg_launch_us": 1e3 * ms / max(n, 1), "bytes_per_launch": nbytes / max(n, 1)}


# FP64 pipe operations (DADD, DMUL, DFMA, DMNMX, DSETP; one each) per cell
# update of the wave-propagation update as the kernels compute it: per edge
# 23 (speed split 2, jump and upwind jump 3, correction coefficient 3, MC
# limiter 8, limited correction 1, flux 2, fluctuations 4), two edges per
# cell; edge speeds 4; transverse increments of the two final fluxes 10;
# fluctuation sums 2; flux difference and update 4.
FP64_OPS_PER_CELL = 66
# GB300 FP64 pipe: 2 operations per clock per SM
FP64_OPS_PER_CLK_SM = 2
GB300_SMS = 152


def roofline_fp64_alu(phase, mx, sm_mhz):
    """The FP64 update against the FP64 pipe (the bound in FP64 on this GPU):
    achieved = FP64_OPS_PER_CELL x cells updated / advance-kernel time."""
    ms, n, nbytes = phase
    cells = nbytes * mx * mx / (((mx + 4) ** 2 + mx * mx) * 8.0)  # advance bytes -> cells
    peak = FP64_OPS_PER_CLK_SM * GB300_SMS * sm_mhz * 1e6 / 1e9
    achieved = FP64_OPS_PER_CELL * cells / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s (FP64 pipe)",
            "frac": achieved / peak if achieved else None, "ops_per_cell": FP64_OPS_PER_CELL,
            "peak_source": f"{FP64_OPS_PER_CLK_SM} FP64 ops/clk/SM x {GB300_SMS} SMs x "
                           f"{sm_mhz:.0f} MHz"}


def adjoint_cost(fc, torch, flush_buf, ncoarse: int = 25, variant: str = "auto"):
    """Forward vs gradient cost of the adjoint workload: the swirl forest
    frozen after its initial regrid, 25 coarse multirate steps (400
    finest-level substeps), FP32, every step recorded by the forward pass
    (and, for comparison, sqrt(N) checkpoints); L = 1/2 |q_N -
    q_target|^2 (target: the run from the shifted disc), gradients with
    respect to q0 and the velocity scale.  Also the adjoint of one coarse step
    alone against the forward coarse step."""
    from paper_1703_03116_gb300.autograd import advect
    w = synth.swirl(seed=0)
    tw = synth.adjoint_target(w)
    desc = fc.make_desc(domain=fc.WALLS, mx=w.mx, lmin=w.lmin, lmax=w.lmax, dtype=fc.F32,
                        velocity=w.velocity)
    F = fc.initial_forest(desc, q0_fn([w]), tau_r=w.tau_refine, tau_c=w.tau_coarsen)
    if variant == "auto":
        F.autotune()
    else:  # one update kernel for every launch (see --variant)
        name, _, warps = variant.partition(":")
        F.set_advance_variant(["staged", "walk", "walk1", "band"].index(name), int(warps or 4))
    leaves = F.leaves()
    dev = flush_buf.device
    q0 = torch.tensor(q0_fn([w])(leaves), dtype=torch.float32, device=dev)
    qt = torch.tensor(q0_fn([tw])(leaves), dtype=torch.float32, device=dev)
    _, dtc = synth.time_step(w)
    updates = ncoarse * cell_updates(leaves, w.lmin, w.mx)

    def timed(fn):
        flush_buf.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    times = {}
    for name, tape in (("warm-up", "forward"), ("warm-up", "recompute"), ("forward", "auto"),
                       ("forward+backward", "forward"), ("recompute", "recompute")):
        q = q0.clone().requires_grad_(name != "forward")
        s = torch.ones((), dtype=torch.float32, device=dev, requires_grad=name != "forward")

        def run():
            qN = advect(q, s, F, 0.0, dtc, ncoarse, multirate=True, tape=tape)
            loss = 0.5 * ((qN - qt) ** 2).sum()
            if name != "forward":
                loss.backward()
        times[name] = timed(run)
    fwd, both, rec = times["forward"], times["forward+backward"], times["recompute"]
    # one coarse step: forward vs its adjoint (which replays the forward once)
    F.set_q(q0)
    lam = (q0 - qt).contiguous()
    ds = torch.zeros(1, dtype=torch.float64, device=dev)
    F.adjoint_step_multirate(0.0, dtc, lam, ds)  # warm-up (state buffers)
    K = 5
    t_fwd = timed(lambda: [F.step_multirate(k * dtc, dtc) for k in range(K)]) / K
    F.set_q(q0)
    torch.cuda.nvtx.range_push("adjoint_steps")  # lets a profiler select these steps
    t_adj = timed(lambda: [F.adjoint_step_multirate(0.0, dtc, lam, ds) for _ in range(K)]) / K
    torch.cuda.nvtx.range_pop()
    # the same step recorded, then reversed from its tape
    F.set_q(q0)
    t_rec = timed(lambda: [F.step_multirate_record(k * dtc, dtc, k) for k in range(K)]) / K
    t_rev = timed(lambda: [F.adjoint_step_multirate_taped(k * dtc, dtc, k, lam, ds)
                           for k in range(K - 1, -1, -1)]) / K
    return {"workload": f"swirl forest frozen after the initial regrid ({len(leaves)} patches), "
                        f"{ncoarse} coarse multirate steps = {ncoarse * 16} finest substeps, FP32; "
                        "gradient: every step recorded by the forward pass, reversed from its "
                        "tape (gradient_recompute_ms: sqrt(N) checkpoints, each segment "
                        "recomputed and recorded in the backward)",
            "forward_ms": fwd, "gradient_ms": both - fwd,
            "gradient_over_forward": (both - fwd) / fwd,
            "gradient_recompute_ms": rec - fwd, "gradient_recompute_over_forward": (rec - fwd) / fwd,
            "coarse_step_forward_ms": t_fwd, "coarse_step_adjoint_ms": t_adj,
            "adjoint_step_over_forward_step": t_adj / t_fwd,
            "coarse_step_recorded_ms": t_rec, "coarse_step_reverse_from_tape_ms": t_rev,
            "reverse_from_tape_over_forward_step": t_rev / t_fwd,
            "forward_cell_updates_per_s": updates / (fwd * 1e-3)}


def granularity_sweep(fc, torch, hbm):
    """Efficiency of one level substep against patches per launch (the GPU
    counterpart of the paper's grids-per-process study, Sec. 5): uniform
    periodic forests of 4^l patches (l = 2..7) for mx = 8, 16, 32, FP32; each
    substep timed by the autotuner (candidates replayed from a CUDA graph),
    the fastest kept."""
    rows = []
    for mx in (8, 16, 32):
        for level in range(2, 8):
            w = synth.uniform_periodic(seed=0, level=level, mx=mx)
            desc = fc.make_desc(domain=fc.PERIODIC, mx=mx, lmin=level, lmax=level, dtype=fc.F32,
                                velocity=w.velocity)
            leaves = fc.uniform_leaves(level)
            F = fc.Forest(desc, leaves)
            F.set_q(q0_fn([w])(leaves))
            rep = F.autotune()
            n = len(leaves)
            b = max(k for k in rep if (1 << k) <= n)
            v, warps, fused, ns = rep[b]
            cells = n * mx * mx
            nbytes = n * ((mx + 4) ** 2 + mx * mx) * 4
            rows.append({"mx": mx, "patches": n, "variant": ["staged", "walk", "walk1", "band"][v],
                         "warps": warps, "us_per_substep": ns * 1e-3,
                         "cell_updates_per_s": cells / (ns * 1e-9),
                         "hbm_frac": nbytes / (ns * 1e-9) / 1e9 / hbm})
            F.close()
            torch.cuda.synchronize()
    return {"workload": "uniform periodic forests, levels 2-7 (16-16384 patches), mx 8/16/32, "
                        "FP32, constant velocity, one level substep (gather fused)",
            "rows": rows}


def run_ours(args):
    import torch

    import paper_1703_03116_gb300 as fc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def reduce(v, op):
        return aggregate([v], [op], dist, dev)[0]

    MAX, SUM = "max", "sum"
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0

    dtype = fc.F32 if args.dtype == "f32" else fc.F64
    if args.mode == "sweep":  # substep efficiency against launch size
        if rank == 0:
            print(json.dumps({"variants": {"granularity": granularity_sweep(fc, torch, hbm)}}),
                  flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.mode == "adjoint":  # the adjoint cost alone (a case sized for profiling)
        if rank == 0:
            print(json.dumps({"variants": {"adjoint": adjoint_cost(fc, torch, flush_buf, variant=args.variant)}}),
                  flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.mode in ("batched", "sphere", "sphere_deform"):
        if args.mode == "batched":
            ws = synth.ensemble(args.ensemble, seed=rank, mx=32)
            label = (f"{args.ensemble} independent swirl forests, levels 2 to 4/5/6, "
                     "32x32 patches")
        elif args.mode == "sphere_deform":
            ws = [synth.sphere_deform(seed=rank, lmin=2, lmax=6, mx=32)]
            label = SPHERE_DEFORM_WORKLOAD
        else:
            ws = [synth.sphere(seed=rank)]
            label = SPHERE_WORKLOAD
        b = measure(Runner(fc, torch, ws, dtype, args.variant), args.steps, args.warmup,
                    flush_buf, local)
        line = {"metric": METRIC, "value": reduce(float(b["updates"]), SUM) /
                (reduce(b["ms"], MAX) * 1e-3), "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": label, "patches": b["patches"]},
                "gpu_launches": b["launches"], "clocks": b["clocks"],
                "roofline": roofline_of(b["phases"]["advance"], hbm, peak_src),
                "phases_ms": {k: x[0] for k, x in b["phases"].items()}, "autotune": b["tuning"]}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    run = Runner(fc, torch, [rank_workload(rank)], dtype, args.variant)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    r = measure(run, args.steps, args.warmup, flush_buf, local)
    if dist is not None:
        dist.barrier()
    ms_max = reduce(r["ms"], MAX)
    updates_all = reduce(float(r["updates"]), SUM)
    value = updates_all / (ms_max * 1e-3)

    # end to end through the C ABI with host buffers: per step the H2D copy of
    # the step's input field from pinned memory, the step, the D2H of the
    # per-forest mass
    F = run.F
    pin_dtype = torch.float32 if dtype == fc.F32 else torch.float64

    def pinned_copy():
        h = torch.empty((len(F), run.w.mx, run.w.mx), dtype=pin_dtype, pin_memory=True).numpy()
        h[...] = F.get_q()
        return h

    host = pinned_copy()
    e2e_steps = max(4, args.steps // 2)
    e2e_s, e2e_up, h2d, d2h = 0.0, 0, 0, 0
    for _ in range(e2e_steps):
        if host.shape[0] != len(F):
            host = pinned_copy()
        flush_buf.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.set_q(host)
        e2e_up += run.updates()
        h2d += host.nbytes
        run.step()
        m = F.mass()
        d2h += m.nbytes
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    e2e_s = reduce(e2e_s, MAX)
    e2e_up = reduce(float(e2e_up), SUM)
    e2e = {"value": e2e_up / e2e_s, "unit": METRIC, "h2d_bytes_per_step": h2d // e2e_steps,
           "d2h_bytes_per_step": d2h // e2e_steps}

    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "step_ms_median": r["step_ms_median"], "step_ms_max": r["step_ms_max"],
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one coarse step (16 finest-level substeps)",
                   "patches": r["patches"], "l2": "flushed (512 MiB write) before every timed step",
                   "parallelism": f"independent forest per GPU x{world}"},
        "clocks": r["clocks"], "e2e": e2e, "gpu_launches": r["launches"],
        "roofline": roofline_of(r["phases"]["advance"], hbm, peak_src,
                                measured_traffic(r["phases"]["advance"], r["tuning"],
                                               4 if dtype == fc.F32 else 8, synth.swirl(seed=0).mx)),
        "phases_ms": {k: v[0] for k, v in r["phases"].items()} | {"step_total": r["ms"]},
        "autotune": r["tuning"],
    }
    if rank == 0 and not args.no_variants:
        variants = {}
        other = fc.F64 if dtype == fc.F32 else fc.F32
        vr = Runner(fc, torch, [synth.swirl(seed=0)], other)
        v = measure(vr, max(8, args.steps // 4), 2, flush_buf, local)
        variants["f64" if other == fc.F64 else "f32"] = {
            "value": v["updates"] / (v["ms"] * 1e-3), "ms_per_step": v["ms"] / max(8, args.steps // 4),
            "roofline": roofline_of(v["phases"]["advance"], hbm, peak_src),
            "phases_ms": {k: x[0] for k, x in v["phases"].items()}}
        if other == fc.F64:
            variants["f64"]["roofline_fp64_alu"] = roofline_fp64_alu(
                v["phases"]["advance"], 32, v["clocks"].get("sm_mhz") or 2070.0)
        del vr
        if args.ensemble > 0:
            # the ensemble at 32^2 in the line's dtype, at 16^2, and in the other dtype
            for key, mxb, dtb in (("batched", 32, dtype), ("batched_mx16", 16, dtype),
                                  ("batched_f64" if other == fc.F64 else "batched_f32", 32,
                                   other)):
                ws = synth.ensemble(args.ensemble, seed=0, mx=mxb)
                br = Runner(fc, torch, ws, dtb)
                nsteps = 8
                b = measure(br, nsteps, 2, flush_buf, local)
                variants[key] = {
                    "workload": f"{args.ensemble} independent swirl forests, levels 2 to 4/5/6 "
                                f"(seeded), {mxb}x{mxb} patches, one launch per level substep "
                                "for all",
                    "dtype": "f32" if dtb == fc.F32 else "f64",
                    "patches": b["patches"], "value": b["updates"] / (b["ms"] * 1e-3),
                    "ms_per_step": b["ms"] / nsteps, "steps": nsteps,
                    "roofline": roofline_of(b["phases"]["advance"], hbm, peak_src),
                    "phases_ms": {k: x[0] for k, x in b["phases"].items()},
                    "gpu_launches": b["launches"], "clocks": b["clocks"], "autotune": b["tuning"]}
                if dtb == fc.F64:
                    variants[key]["roofline_fp64_alu"] = roofline_fp64_alu(
                        b["phases"]["advance"], mxb, b["clocks"].get("sm_mhz") or 2070.0)
                del br
        sr = Runner(fc, torch, [synth.sphere(seed=0)], fc.F32)
        nsteps = 8
        sv = measure(sr, nsteps, 2, flush_buf, local)
        variants["sphere"] = {
            "workload": SPHERE_WORKLOAD, "dtype": "f32 field and update, f64 metrics and mass",
            "patches": sv["patches"], "value": sv["updates"] / (sv["ms"] * 1e-3),
            "ms_per_step": sv["ms"] / nsteps, "steps": nsteps,
            "roofline": roofline_of(sv["phases"]["advance"], hbm, peak_src),
            "phases_ms": {k: x[0] for k, x in sv["phases"].items()},
            "gpu_launches": sv["launches"], "clocks": sv["clocks"]}
        del sr
        variants["adjoint"] = adjoint_cost(fc, torch, flush_buf)
        out["variants"] = variants
        out["cpu_baseline"] = cpu_baseline(synth.swirl(seed=0))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ oracle (CPU)

def _oracle_rate(w, budget_s: float, openmp: bool):
    """(cell-updates/s, coarse steps, patches, setup s) of the oracle on a
    bounded prefix of the run: coarse multirate steps until budget_s of
    stepping has elapsed (at least one)."""
    import oracle
    oracle.use_openmp(openmp)
    try:
        t0 = time.perf_counter()
        ref = oracle.initial_forest(w)
        setup = time.perf_counter() - t0
        _, dtc = synth.time_step(w)
        done, up, el = 0, 0, 0.0
        while done < 1 or el < budget_s:
            up += cell_updates(ref.leaves(), w.lmin, w.mx)
            t0 = time.perf_counter()
            ref.step_multirate(done * dtc, dtc)
            el += time.perf_counter() - t0
            done += 1
        return up / el, done, len(ref), setup, oracle.threads()
    finally:
        oracle.use_openmp(False)


def cpu_baseline(w, budget_s: float = 10.0):
    """The FP64 oracle on a bounded prefix of the same run: the OpenMP build
    of its sources on all host threads (the line's value), and the plain
    build on one thread beside it."""
    v1, n1, npatch, setup, _ = _oracle_rate(w, budget_s, False)
    try:
        va, na, _, _, cores = _oracle_rate(w, budget_s, True)
    except Exception as e:  # no OpenMP compiler on this host: the plain build only
        return {"value": v1, "unit": METRIC, "cores": 1, "kind": "oracle",
                "sample": f"{n1} coarse multirate steps of the same swirl forest ({npatch} "
                          f"patches), FP64, single thread (OpenMP build unavailable: {e})"}
    return {"value": va, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{na} coarse multirate steps of the same swirl forest ({npatch} patches), "
                      f"FP64, the oracle's sources built with OpenMP (patch loops on {cores} host "
                      f"threads), setup {setup:.1f}s untimed",
            "single_thread": {"value": v1, "cores": 1,
                              "sample": f"{n1} coarse multirate steps, plain build"}}


def run_reference(args):
    """The reference arm: the paper has no code, so the FP64 oracle stands in,
    built with OpenMP over patches and run on all host threads."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    try:
        oracle.use_openmp(True)
    except Exception:
        oracle.use_openmp(False)
    cores = oracle.threads()
    w = synth.swirl(seed=0)
    ref = oracle.initial_forest(w)
    _, dtc = synth.time_step(w)
    n = 0

    def step():
        nonlocal n
        ref.step_multirate(n * dtc, dtc)
        n += 1
        if n % w.regrid_every == 0:
            ref.regrid(w.tau_refine, w.tau_coarsen)

    # each bench step is a bounded sample: one coarse step of the oracle
    for _ in range(args.warmup):
        step()
    el, up = 0.0, 0
    for _ in range(args.steps):
        up += cell_updates(ref.leaves(), w.lmin, w.mx)
        t0 = time.perf_counter()
        step()
        el += time.perf_counter() - t0
    value = up / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "step": "one coarse step (16 finest-level substeps)",
                      "patches": len(ref)},
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} coarse steps after {args.warmup} warm-up "
                                      "steps of the swirl forest, FP64 oracle, patch loops on "
                                      f"{cores} host threads"},
           "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
