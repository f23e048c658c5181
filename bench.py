#!/usr/bin/env python
"""Throughput of the patch-AMR wave-propagation hot path on GB300.

Workload (one rank): an adaptive single-tree swirl forest, levels 2-6,
32x32 patches with 2 ghost layers, walls, MC limiter with transverse
corrections, CFL 0.9, multirate subcycling (16 finest substeps per coarse
step), regrid every 4 coarse steps.  A "step" is one coarse step: for each
level substep the ghost fill (Alg. 1 phases) and the patch update, plus the
regrid when it falls due.  Metric: cell updates per second, the paper's rate
(mx^2 x patch advances / wall time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): each rank advances its own independent forest (seeded
by rank): weak scaling, no collective on the data path.  Prints one JSON line
on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "cell-updates/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64 and CPU legs")
    return ap.parse_args()


def workload(rank: int):
    return synth.swirl(seed=rank)


def cell_updates(leaves: np.ndarray, w) -> int:
    """mx^2 x patch advances of one coarse multirate step."""
    lev = leaves[:, 2].astype(np.int64)
    return int(np.sum((1 << (lev - w.lmin)) * w.mx * w.mx))


def q0_fn(w):
    def q0(leaves):
        x, y = synth.cell_centres(leaves, w.mx)
        return synth.evaluate(w, x, y)
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
                 "-lms", "200", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
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


# ------------------------------------------------------------------ ours

def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


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

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def reduce(v, op):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=op)
        return float(t.item())

    w = workload(rank)
    n_coarse, dtc = synth.time_step(w)

    def build(dtype):
        desc = fc.make_desc(domain=fc.WALLS, mx=w.mx, lmin=w.lmin, lmax=w.lmax, dtype=dtype,
                            velocity=w.velocity)
        return fc.initial_forest(desc, q0_fn(w), tau_r=w.tau_refine, tau_c=w.tau_coarsen)

    def measure(dtype, steps, warmup):
        F = build(dtype)
        step_no = [0]

        def one_step():
            n = step_no[0]
            F.step_multirate(n * dtc, dtc)
            step_no[0] += 1
            if step_no[0] % w.regrid_every == 0:
                F.tag_regrid(w.tau_refine, w.tau_coarsen)

        for _ in range(warmup):
            one_step()
        barrier()
        F.timers(True)
        for ph in range(4):
            F.read_timer(ph, reset=True)
        fc.launch_count(reset=True)
        events = []
        updates = 0
        with Clocks(local) as clk:
            for _ in range(steps):
                flush_buf.zero_()  # write > L2 between timed steps (untimed)
                updates += cell_updates(F.leaves(), w)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                one_step()
                e1.record()
                events.append((e0, e1))
            torch.cuda.synchronize()
        launches = fc.launch_count()
        ms = sum(a.elapsed_time(b) for a, b in events)
        adv = F.read_timer(0)
        fill = F.read_timer(1)
        regrid = F.read_timer(2)
        F.timers(False)
        barrier()
        ms_max = reduce(ms, dist.ReduceOp.MAX if dist else None)
        updates_all = reduce(float(updates), dist.ReduceOp.SUM if dist else None)
        return dict(F=F, ms=ms_max, updates=updates_all, adv=adv, fill=fill, regrid=regrid,
                    launches=launches, clocks=clk.summary(), patches=len(F), step_no=step_no,
                    one_step=one_step)

    dtype = fc.F32 if args.dtype == "f32" else fc.F64
    r = measure(dtype, args.steps, args.warmup)
    value = r["updates"] / (r["ms"] * 1e-3)
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    adv_ms, adv_n, adv_bytes = r["adv"]
    achieved = adv_bytes / (adv_ms * 1e-3) / 1e9 if adv_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": None,
                "kernel": "advance_kernel", "peak_source": peak_note,
                "launches": adv_n, "avg_launch_us": 1e3 * adv_ms / max(adv_n, 1),
                "bytes_per_launch": adv_bytes / max(adv_n, 1)}

    # end to end through the C ABI with host buffers: H2D of the step's input
    # field from pinned memory, the step, D2H of the per-forest mass
    F, one_step = r["F"], r["one_step"]
    esize = 4 if dtype == fc.F32 else 8
    host = torch.empty((len(F), w.mx, w.mx), dtype=torch.float32 if esize == 4 else torch.float64,
                       pin_memory=True).numpy()
    host[...] = F.get_q()
    e2e_steps = max(4, args.steps // 2)
    e2e_s, e2e_up, h2d, d2h = 0.0, 0, 0, 0
    for _ in range(e2e_steps):
        if host.shape[0] != len(F):
            host = torch.empty((len(F), w.mx, w.mx), dtype=torch.float32 if esize == 4
                               else torch.float64, pin_memory=True).numpy()
            host[...] = F.get_q()
        flush_buf.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.set_q(host)
        e2e_up += cell_updates(F.leaves(), w)
        h2d += host.nbytes
        one_step()
        m = F.mass()
        d2h += m.nbytes
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    e2e_s = reduce(e2e_s, dist.ReduceOp.MAX if dist else None)
    e2e_up = reduce(float(e2e_up), dist.ReduceOp.SUM if dist else None)
    e2e = {"value": e2e_up / e2e_s, "unit": METRIC, "h2d_bytes_per_step": h2d // e2e_steps,
           "d2h_bytes_per_step": d2h // e2e_steps}

    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": "adaptive swirl forest, levels 2-6, 32x32 patches, mbc 2, "
                               "multirate, regrid every 4 coarse steps",
                   "step": "one coarse step (16 finest substeps)", "patches": r["patches"],
                   "l2": "flushed (512 MiB write) before every timed step",
                   "parallelism": f"replicas x{world} (one forest per GPU)"},
        "clocks": r["clocks"], "e2e": e2e, "gpu_launches": r["launches"], "roofline": roofline,
        "phases_ms": {"advance": adv_ms, "fill": r["fill"][0], "regrid_kernels": r["regrid"][0],
                      "total": r["ms"]},
    }
    if rank == 0 and not args.no_variants:
        other = fc.F64 if dtype == fc.F32 else fc.F32
        v = measure(other, max(8, args.steps // 4), 2)
        a_ms, a_n, a_b = v["adv"]
        out["variants"] = {("f64" if other == fc.F64 else "f32"): {
            "value": v["updates"] / (v["ms"] * 1e-3), "ms_per_step": v["ms"] / max(8, args.steps // 4),
            "advance_GBps": a_b / (a_ms * 1e-3) / 1e9 if a_ms > 0 else None,
            "advance_avg_launch_us": 1e3 * a_ms / max(a_n, 1)}}
        out["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ oracle (CPU)

def cpu_baseline(w, budget_s: float = 15.0, min_steps: int = 1):
    """The FP64 oracle, single-threaded, on a bounded prefix of the same run."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.initial_forest(w)
    setup = time.perf_counter() - t0
    _, dtc = synth.time_step(w)
    done, up, el = 0, 0, 0.0
    while done < min_steps or el < budget_s:
        up += cell_updates(ref.leaves(), w)
        t0 = time.perf_counter()
        ref.step_multirate(done * dtc, dtc)
        el += time.perf_counter() - t0
        done += 1
        if el > budget_s:
            break
    return {"value": up / el, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{done} coarse multirate steps of the same swirl forest "
                      f"({len(ref)} patches), FP64, single thread, setup {setup:.1f}s untimed"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = workload(0)
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
        up += cell_updates(ref.leaves(), w)
        t0 = time.perf_counter()
        step()
        el += time.perf_counter() - t0
    value = up / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "adaptive swirl forest, levels 2-6, 32x32 patches, mbc 2, "
                                  "multirate, regrid every 4 coarse steps",
                      "step": "one coarse step (16 finest substeps)", "patches": len(ref)},
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} coarse steps after {args.warmup} warm-up "
                                      "steps, FP64 oracle, single thread"},
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
