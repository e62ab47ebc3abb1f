#!/usr/bin/env python
"""Throughput of the explicit energy-conserving PIC step on one GB300.

Workload: the 1D1V two-stream instability, 2^23 electron markers, 512 cells,
quadratic shapes, dt = 0.05, ESEC2 (Sec. 3.3), synthetic and seeded.  A "step"
is one full time step of the scheme (both particle passes, the field updates
and the per-step energy and fallback reduction).  The metric is particle-steps
per second (markers x steps / time); each form of the library is reported with
its energy error max_n |TE^n - TE^0| / TE^0 over the run.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
(independent seed): weak scaling, no data-path collective.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s on 1 GB300 (plain FP64 vs chosen form) at |dW/W| <= 1e-11"
UNIT = "particle-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20          # > 2x the 126.5 MB L2
# Algorithmic bytes per marker per launch: the state that must cross HBM once per
# barrier-separated pass.  FP64 form: pass C reads x, v and writes v*; pass E
# reads x, v, v* and writes x, v.  Mixed form: pass C reads X, vh, vl and writes
# the integer V*; pass E reads X, vh, vl, V* and writes X, vh, vl.
ALGO_BYTES = {  # (form, kernel kind) -> bytes per marker
    ("fp64", 0): 24, ("fp64", 1): 40,    # pass C also writes v*, pass E reads it
    ("mixed", 0): 16, ("mixed", 1): 28,
    ("mixed_g64", 0): 16, ("mixed_g64", 1): 28,   # the mixed form, Gamma in FP64 for every marker
    # ESEC1, mixed form: one fused launch per step reads and writes X, vh, vl, V*
    # (32 bytes per particle-step); two launches: 16 + 28 as ESEC2
    ("mixed_esec1", 0): 16, ("mixed_esec1", 5): 32,
    ("mixed_esec1_2l", 0): 16, ("mixed_esec1_2l", 1): 28,
    ("standard", 1): 32,     # the comparator's one pass reads and writes x, v
}
# The FP64 form is bound by the FP64 pipe (2 thread-instructions per SM and
# clock on this part), not by HBM: its roofline counts FP64-pipe thread
# instructions per marker, measured once with ncu
# (sm__thread_inst_executed_pipe_fp64_pred_on.sum / markers) on these kernels.
FP64_INST_PER_MARKER = {("fp64", 0): 32.56, ("fp64", 1): 56.78, ("standard", 1): 45.39}
FP64_LANES_PER_SM_CLK = 2
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# ncu capture of the current kernels on this workload (2^23 markers); None where
# the kernel changed since it was taken.
TRAFFIC = {("mixed", 0): 111384320, ("mixed", 1): 177644544, ("mixed_esec1", 5): 208671488,
           ("fp64", 0): 631477504, ("fp64", 1): 754875648, ("standard", 1): 207165440}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--markers", type=int, default=1 << 23)
    ap.add_argument("--forms", default="mixed,fp64,standard",
                    help="library forms to time; the first available is the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--full-run", action=argparse.BooleanOptionalAction, default=True,
                    help="also run the workload's whole length per form, untimed, for its "
                         "energy error and fallbacks")
    ap.add_argument("--sort-period", type=int, default=None,
                    help="sort of the mixed form's markers every this many steps (0 = never; "
                         "default: 0 on the 1D workloads, 2 on the 2D3V Weibel workload)")
    ap.add_argument("--weibel2d", action="store_true",
                    help="time the 2D3V Yee/leapfrog path on the 128 x 128 Weibel workload "
                         "instead (not the default line)")
    ap.add_argument("--weibel1d", action="store_true",
                    help="time the 1D2V electromagnetic path (Crank-Nicolson and PSATD field "
                         "solves) on the Weibel workload instead (not the default line)")
    ap.add_argument("--grad", action="store_true",
                    help="time the reverse mode on the bump-on-tail workload instead (not the "
                         "default line), with the finite-difference agreement vs horizon")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="time a batch of this many independent runs instead (not the default "
                         "line): batched launches vs the same runs stepped one by one")
    ap.add_argument("--ensemble-markers", default="1e4:1e6",
                    help="MIN:MAX of the log-uniform marker counts of the ensemble's runs")
    ap.add_argument("--ensemble-cells", default="32:512",
                    help="MIN:MAX of the uniform cell counts of the ensemble's runs")
    args = ap.parse_args()
    if args.sort_period is None:
        # the fastest setting measured per workload: unsorted markers on the 1D
        # grids (the tile copies sit in shared memory), a quarter-cell sort every
        # second step on the 2D3V grid (the deposit's runs need sorted markers)
        args.sort_period = 2 if args.weibel2d else 0
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a scalar over all ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload(markers: int, seed: int):
    from paper_2411_09605_gb300 import workloads as W
    return W.two_stream(n=markers, seed=seed)


def config_dict(prob, extra=None):
    d = {"workload": "two_stream_1d1v", "markers": prob.n_markers, "cells": prob.nc,
         "shape_order": prob.order, "dt": prob.dt, "L": round(prob.L, 6), "scheme": "ESEC2",
         "v0": 3.0, "vth": 0.1, "seed_amplitude": 1e-3,
         "l2": "flushed (512 MiB write) before every timed step"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool = True):
        self.index, self.enabled, self.proc = index, enabled, None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        if self.enabled:
            try:
                self.f = open(self.path, "w")
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                     "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                    stderr=subprocess.DEVNULL)
            except OSError:
                self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- our arm


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def roofline(form, kname, k, markers, hbm_peak, hbm_src, clocks, nsm):
    """Roofline of the form's dominant kernel: HBM bytes for the mixed form, FP64-
    pipe thread instructions for the FP64 form and the standard comparator
    (achieved = algorithmic work per launch / average event-timed launch
    duration)."""
    t = k["avg_us"] * 1e-6
    if form in ("fp64", "standard"):
        inst = FP64_INST_PER_MARKER[(form, k["kind"])] * markers
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = FP64_LANES_PER_SM_CLK * nsm * mhz * 1e6 / 1e9
        ach = inst / t / 1e9
        return {"bound": "alu", "kernel": kname, "achieved": round(ach, 1), "peak": round(peak, 1),
                "unit": "Ginst/s (FP64 pipe)", "frac": round(ach / peak, 4),
                "traffic": TRAFFIC.get((form, k["kind"])),
                "peak_source": f"{FP64_LANES_PER_SM_CLK} FP64 lanes/SM/clk x {nsm} SMs x {mhz:.0f} MHz",
                "algorithmic_fp64_inst_per_launch": inst}
    algo = ALGO_BYTES[(form, k["kind"])] * markers
    ach = algo / t / 1e9
    return {"bound": "hbm", "kernel": kname, "achieved": round(ach, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
            "traffic": TRAFFIC.get((form, k["kind"])), "peak_source": hbm_src,
            "algorithmic_bytes_per_launch": algo}


def time_form(prob, precision_name: str, steps: int, warmup: int, profile_steps: int, stream,
              flush_buf, sort_period: int = 0):
    """Device-timed throughput of one library form on the resident workload."""
    import torch
    from paper_2411_09605_gb300 import pic
    mixed = precision_name.startswith("mixed")
    prec = pic.PIC_PREC_MIXED if mixed else pic.PIC_PREC_FP64
    scheme = pic.PIC_SCHEME_ESEC1 if "esec1" in precision_name else pic.PIC_SCHEME_ESEC2
    s = prob.species[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    x_d = torch.from_numpy(s.x).to(dev)
    v_d = torch.from_numpy(s.v).to(dev)
    # "standard": the comparison scheme of Sec. 5 (leapfrog Vlasov-Poisson, one
    # binomial filter pass on the charge) on the same workload
    std = precision_name == "standard"
    cfg = pic.make_config(prob.nc, prob.L, prob.dt, prob.order, scheme, prec,
                          ptr_on_device=1, stream=stream.cuda_stream,
                          sort_period=sort_period if precision_name == "mixed" else 0,
                          solver=pic.PIC_SOLVER_STANDARD_LEAPFROG if std else
                          pic.PIC_SOLVER_AMPERE_ES, binomial_passes=1 if std else 0,
                          gamma_fp64=1 if precision_name == "mixed_g64" else 0,
                          separate_passes=1 if precision_name == "mixed_esec1_2l" else 0)
    torch.cuda.synchronize()
    h = pic.pic_init(cfg, [dict(q=s.q, m=s.m, x=x_d, v=v_d, w=None, w0=s.w0)])
    del x_d, v_d
    try:
        te_dev = torch.zeros(max(1, warmup), dtype=torch.float64, device=dev)
        fb_dev = torch.zeros(max(1, warmup), dtype=torch.int64, device=dev)
        if warmup:
            pic.pic_step(h, warmup, fb_dev, te_dev)
        _, _, _, te0 = pic.pic_energy(h, 1)
        torch.cuda.synchronize()
        launches0 = pic.pic_launch_count(h)
        evs = []
        fbs, tes = [], []
        for k in range(steps):
            flush_buf.zero_()                          # L2 flush, outside the timed region
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pic.pic_step_async(h, 1)
            b.record(stream)
            evs.append((a, b))
            if (k + 1) % 1000 == 0:
                fb, te = pic.pic_read_stats(h)
                fbs.append(fb)
                tes.append(te)
        fb, te = pic.pic_read_stats(h)
        fbs.append(fb)
        tes.append(te)
        torch.cuda.synchronize()
        launches = pic.pic_launch_count(h) - launches0
        step_ms = np.array([a.elapsed_time(b) for a, b in evs])
        fb = np.concatenate(fbs)
        te = np.concatenate(tes)
        # per-kernel durations for the roofline (separate, profiled steps)
        pic.pic_set_profiling(h, True)
        for k in range(profile_steps):
            flush_buf.zero_()
            pic.pic_step_async(h, 1)
        pic.pic_read_stats(h)
        kern = {}
        for kind, name in ((0, "pass_c"), (1, "pass_e"), (2, "finalize"), (3, "sort"),
                           (5, "pass_ec")):
            n, ms = pic.pic_profile(h, kind)
            if n:
                kern[name] = {"kind": kind, "launches": n, "avg_us": 1e3 * ms / n}
        pic.pic_set_profiling(h, False)
    finally:
        pic.pic_free(h)
    allte = np.concatenate([[te0], te])
    return {"step_ms": step_ms, "fallbacks": int(fb.sum()),
            "max_rel_dTE": float(np.max(np.abs(allte - allte[0])) / abs(allte[0])),
            "launches": int(launches), "kernels": kern}


def e2e_form(prob, precision_name: str, steps: int, warmup: int, sort_period: int = 0):
    """End to end through the C ABI with host buffers: every step uploads the
    marker state from pinned host memory, steps once and reads the state and the
    step's energy/fallback back to pinned host memory."""
    import torch
    from paper_2411_09605_gb300 import pic
    prec = pic.PIC_PREC_MIXED if precision_name == "mixed" else pic.PIC_PREC_FP64
    s = prob.species[0]
    n = len(s.x)
    xh = torch.from_numpy(s.x.copy()).pin_memory()
    vh = torch.from_numpy(s.v.copy()).pin_memory()
    fb = torch.zeros(1, dtype=torch.int64).pin_memory()
    te = torch.zeros(1, dtype=torch.float64).pin_memory()
    cfg = pic.make_config(prob.nc, prob.L, prob.dt, prob.order, pic.PIC_SCHEME_ESEC2, prec,
                          sort_period=sort_period if precision_name == "mixed" else 0)
    h = pic.pic_init(cfg, [dict(q=s.q, m=s.m, x=xh.numpy(), v=vh.numpy(), w=None, w0=s.w0)])
    try:
        times = []
        for k in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pic.pic_set_particles(h, 0, xh.numpy(), vh.numpy())
            pic.pic_step(h, 1, fb.numpy(), te.numpy())
            pic.pic_get_particles(h, 0, xh.numpy(), vh.numpy())
            t1 = time.perf_counter()
            if k >= warmup:
                times.append(t1 - t0)
    finally:
        pic.pic_free(h)
    return {"s_per_step": float(np.mean(times)), "h2d": 16 * n, "d2h": 16 * n + 16}


def host_cpu() -> dict:
    """The host's CPU model and core counts (lscpu, else /proc/cpuinfo)."""
    import platform
    import subprocess
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model or "unknown", "arch": platform.machine(),
            "nproc": os.cpu_count(), "usable_cores": usable}


def _time_oracle(prob, threaded: bool, budget_s: float, max_steps: int):
    from oracle import oracle as O
    s = prob.species[0]
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=2)
    sp = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None, s.w0)]
    E = O.poisson_e0_1d(cfg, sp)
    O.es1d_step(cfg, sp, E, threaded=threaded)      # warm-up (thread pool, pages)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps and (time.perf_counter() - t0) < budget_s:
        O.es1d_step(cfg, sp, E, threaded=threaded)
        k += 1
    return k, time.perf_counter() - t0


def cpu_baseline_oracle(markers: int, seed: int, budget_s: float = 10.0, max_steps: int = 200):
    """The FP64 C oracle on a bounded sample of the workload, timed twice on the
    host: the OpenMP build of the same source on every usable core (the headline
    value) and the single-threaded checker build."""
    from oracle import oracle as O
    prob = workload(markers, seed)
    threads = O.omp_threads()
    k, dt = _time_oracle(prob, True, budget_s, max_steps)
    k1, dt1 = _time_oracle(prob, False, budget_s, max_steps)
    return {"value": markers * k / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{markers} markers of the same two-stream workload x {k} steps "
                      f"({dt:.1f} s, FP64 C oracle built with OpenMP, {threads} threads)",
            "host": host_cpu(),
            "single_thread": {"value": markers * k1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{markers} markers x {k1} steps ({dt1:.1f} s, "
                                        "the single-threaded checker build)"}}


def full_run(prob, form: str, steps: int):
    """The workload's whole run: energy error over the run (max over the steps
    of |TE^n - TE^0| / TE^0), the largest change of one step without a
    fallback (relative to TE^0), the fallbacks (Sec. 5.1), and the run's own
    throughput (wall clock around all steps, the stats read every 1000 steps,
    no L2 flush: the saturated phase, where the correction's FP64 path is
    taken, is inside it)."""
    from paper_2411_09605_gb300 import pic
    mixed = form.startswith("mixed")
    sim = pic.Simulation(prob, scheme=1 if "esec1" in form else 2,
                         precision=pic.PIC_PREC_MIXED if mixed else pic.PIC_PREC_FP64,
                         gamma_fp64=form == "mixed_g64")
    try:
        te0 = sim.energy()[3]
        fbs, tes = [], []
        t0 = time.perf_counter()
        for k in range(0, steps, 1000):
            fb, te = sim.step(min(1000, steps - k))
            fbs.append(fb)
            tes.append(te)
        wall = time.perf_counter() - t0
    finally:
        sim.close()
    fb, te = np.concatenate(fbs), np.concatenate(tes)
    d = np.abs(np.diff(np.concatenate([[te0], te]))) / abs(te0)
    first = int(np.argmax(fb > 0)) if fb.any() else -1
    return {"steps": steps, "particle_steps_per_s": prob.n_markers * steps / wall,
            "max_rel_dTE": float(np.max(np.abs(te - te0)) / abs(te0)),
            "max_step_dTE_without_fallback": float(np.max(d[fb == 0], initial=0.0)),
            "fallbacks": int(fb.sum()), "first_fallback_step": first,
            "max_rel_dTE_before_first_fallback":
                float(np.max(np.abs(te[:first] - te0)) / abs(te0)) if first > 0 else None}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    from paper_2411_09605_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2411_09605_gb300 import pic
    pic.lib()

    prob = workload(args.markers, seed=rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    forms = {}
    sampler = ClockSampler(local, enabled=not args.no_clocks)
    wall0 = time.perf_counter()
    with sampler:
        for name in [f.strip() for f in args.forms.split(",") if f.strip()]:
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            try:
                forms[name] = time_form(prob, name, args.steps, args.warmup, args.profile_steps,
                                        stream, flush, args.sort_period)
            except pic.PicError as e:
                if e.code == -7:      # form not built in this library version
                    forms[name] = {"unavailable": str(e)}
                    continue
                raise
            torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.summary()
    avail = [k for k, v in forms.items() if "unavailable" not in v]
    head = avail[0]
    peak, peak_src = hbm_peak()

    out_forms = {}
    for name in avail:
        f = forms[name]
        t_local = float(f["step_ms"].sum()) / 1e3
        t_max = max_over_ranks(t_local, world, dev)
        units = sum_over_ranks(float(prob.n_markers * args.steps), world, dev)
        kern = f["kernels"]
        dom = max(kern.items(), key=lambda kv: kv[1]["avg_us"] * kv[1]["launches"])
        dname, d = dom
        out_forms[name] = {
            "value": units / t_max, "ms_per_step": 1e3 * t_max / args.steps,
            "max_rel_dTE": f["max_rel_dTE"], "fallbacks": f["fallbacks"],
            "gpu_launches": f["launches"],
            "kernels_us": {k: round(v["avg_us"], 2) for k, v in kern.items()},
            "roofline": roofline(name, dname, d, prob.n_markers, peak, peak_src, clocks,
                                 torch.cuda.get_device_properties(dev).multi_processor_count),
            "roofline_hbm_by_kernel": {
                k: round(ALGO_BYTES[(name, v["kind"])] * prob.n_markers / (v["avg_us"] * 1e-6)
                         / 1e9 / peak, 4)
                for k, v in kern.items() if (name, v["kind"]) in ALGO_BYTES},
        }
    hf = out_forms[head]
    line = {
        "metric": METRIC, "value": hf["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": hf["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32+i64 (energy in f64)" if head.startswith("mixed") else "f64",
        "data": "synthetic (seeded two-stream markers)",
        "config": config_dict(prob, {"form": head, "parallelism": f"replicas{world}",
                                     "sort_period": args.sort_period if head == "mixed" else 0}),
        "roofline": hf["roofline"], "gpu_launches": hf["gpu_launches"], "clocks": clocks,
        "energy": {"max_rel_dTE": hf["max_rel_dTE"], "fallbacks": hf["fallbacks"],
                   "steps": args.warmup + args.steps},
        "forms": {k: {kk: vv for kk, vv in v.items()} for k, v in out_forms.items()},
        "unavailable_forms": {k: v["unavailable"] for k, v in forms.items() if k not in avail},
    }
    if not args.no_e2e:
        e = e2e_form(prob, head, max(2, min(args.steps, 10)), 1, args.sort_period)
        t = max_over_ranks(e["s_per_step"], world, dev)
        line["e2e"] = {"value": sum_over_ranks(prob.n_markers, world, dev) / t, "unit": UNIT,
                       "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"]}
    if rank == 0 and world == 1 and args.full_run:
        # the configuration's whole run (2000 steps) per form, untimed
        line["full_run"] = {name: full_run(prob, name, prob.steps)
                            for name in avail if name != "standard"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(1 << 21, 0)
    line["wall_s_timed_forms"] = round(wall, 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_ensemble(args):
    """Aggregate throughput of a batch of independent mixed-form runs
    (workloads.ensemble: Landau and two-stream problems of random size), one
    launch per pass for all runs, against the same runs stepped one by one."""
    import torch
    from paper_2411_09605_gb300 import build as B, pic, workloads as W
    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()             # every run and every event on one stream
    n_min, n_max = (float(a) for a in args.ensemble_markers.split(":"))
    nc_min, nc_max = (int(a) for a in args.ensemble_cells.split(":"))
    probs = W.ensemble(args.ensemble, seed=0, n_min=n_min, n_max=n_max, nc_min=nc_min,
                       nc_max=nc_max)
    markers = sum(p.n_markers for p in probs)
    steps = max(2, min(args.steps, 100))

    def timed(fn, k):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn(k)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    out = {}
    for graphs in (False, True):
        bt = pic.Batch(probs, graphs=graphs, stream=stream.cuda_stream)
        try:
            trips = pic.pic_batch_autotune(bt.b, 2)
            bt.step(args.warmup)
            t = timed(lambda k: pic.pic_batch_step(bt.b, k), steps)
            fb, te = pic.pic_batch_read_stats(bt.b, len(probs))
            nruns, nblocks, _ = pic.pic_batch_info(bt.b)
            drift = float(np.max(np.abs(te - te[:, :1]) / np.abs(te[:, :1])))
        finally:
            bt.close()
        out["graphs" if graphs else "launches"] = {"value": markers * steps / t,
                                                   "ms_per_step": 1e3 * t / steps,
                                                   "max_rel_dTE": drift,
                                                   "fallbacks": int(fb.sum()),
                                                   "steps_in_stats": int(fb.shape[1])}
    # the same runs, each stepped alone (one pair of launches per run and step)
    t_single = 0.0
    for p in probs:
        sim = pic.Simulation(p, precision=pic.PIC_PREC_MIXED, stream=stream.cuda_stream)
        try:
            sim.step(args.warmup)
            t_single += timed(lambda k: pic.pic_step_async(sim.h, k), steps)
            pic.pic_read_stats(sim.h)
        finally:
            sim.close()
    head = out["graphs"]
    line = {
        "metric": f"aggregate particle-steps/s, {len(probs)} independent runs (batched)",
        "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32+i64 (energy in f64)",
        "data": "synthetic (seeded Landau and two-stream runs)",
        "config": {"workload": "ensemble_1d1v", "runs": len(probs), "markers": markers,
                   "cells": f"U{{{nc_min}..{nc_max}}}",
                   "markers_per_run": f"log-uniform [{n_min:g}, {n_max:g}]",
                   "blocks_per_pass": nblocks, "trips_per_block (autotuned)": trips,
                   "l2": "not flushed: the batch state (%.0f MB) is larger than L2"
                         % (16e-6 * markers)},
        "forms": out,
        "runs_one_by_one": {"value": markers * steps / t_single,
                            "ms_per_step": 1e3 * t_single / steps},
        "speedup_vs_one_by_one": head["value"] / (markers * steps / t_single),
    }
    print(json.dumps(line), flush=True)


# 2D3V Yee path, FP64 form: pass C reads x, y, vx, vy, vz and writes v*; pass
# E reads them and v*, and writes x, y, v.  Mixed form: X, Y (u32), three
# float pairs and V* (3 x i32): pass C reads 32 bytes and writes 12, pass E
# reads 44 and writes 32.
EM2D_ALGO_BYTES = {("fp64", 0): 64, ("fp64", 1): 104, ("mixed", 0): 44, ("mixed", 1): 76,
                   ("fp64_charge_conserving", 0): 64, ("fp64_charge_conserving", 1): 104}
# FP64-pipe thread instructions per marker of the FP64 form (ncu, 2^20
# markers): that form is bound by the FP64 pipe
EM2D_FP64_INST_PER_MARKER = {("fp64", 0): 128.15, ("fp64", 1): 163.74,
                             ("fp64_charge_conserving", 0): 174.77,
                             ("fp64_charge_conserving", 1): 224.81}
EM2D_TRAFFIC = {("fp64", 0): 192259840, ("fp64", 1): 226352640,   # dram read + write per launch
                ("mixed", 0): None, ("mixed", 1): None,
                ("fp64_charge_conserving", 0): 45156096, ("fp64_charge_conserving", 1): 68527360}


def time_weibel2d(prob, precision, args, stream, flush, charge_conserving=False,
                  sort_period=0):
    """Warm-up, timed steps (one event pair per step, L2 flushed before each)
    and a profiled run of one form of the 2D3V Yee step.  With sort_period P
    the timed steps include the sorts that fall in them."""
    import torch
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation2D(prob, precision=precision, charge_conserving=charge_conserving,
                           sort_period=sort_period)
    try:
        te0 = sim.energy()[3]
        pic.pic_step_async(sim.h, max(3, args.warmup))
        pic.pic_read_stats(sim.h)
        launches0 = pic.pic_launch_count(sim.h)
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pic.pic_step_async(sim.h, 1)
            b.record(stream)
            evs.append((a, b))
        fb, te = pic.pic_read_stats(sim.h)
        torch.cuda.synchronize()
        launches = pic.pic_launch_count(sim.h) - launches0
        step_ms = np.array([a.elapsed_time(b) for a, b in evs])
        pic.pic_set_profiling(sim.h, True)
        for _ in range(args.profile_steps):
            flush.zero_()
            pic.pic_step_async(sim.h, 1)
        pic.pic_read_stats(sim.h)
        kern = {}
        for kind, kname in ((0, "pass_c"), (1, "pass_e"), (2, "finalize"), (4, "field"),
                            (3, "sort")):
            n, tot = pic.pic_profile(sim.h, kind)
            if n:
                kern[kname] = {"launches": n, "avg_us": 1e3 * tot / n}
        pic.pic_set_profiling(sim.h, False)
    finally:
        sim.close()
    return {"step_ms": step_ms, "kernels": kern, "launches": int(launches),
            "max_rel_dTE": float(np.max(np.abs(te - te0)) / te0), "fallbacks": int(fb.sum())}


def run_weibel2d(args):
    """The 2D3V Weibel workload with the Yee/leapfrog field step (Sec. 4.1):
    128 x 128 periodic cells, 64 markers per cell (1,048,576), bi-Maxwellian
    with T_perp / T_par = 10, vth_par = 0.05 c, CFL 0.5, ESEC2 form; the FP64
    and the mixed form on the same markers, the mixed form the headline."""
    import torch
    from paper_2411_09605_gb300 import build as B, pic, workloads as W
    B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()          # the handle uses the default stream
    peak, peak_src = hbm_peak()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    prob = W.weibel()
    n = prob.n_markers
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fp64_peak = FP64_LANES_PER_SM_CLK * nsm * 2070.0e6 / 1e9
    forms = {}
    with ClockSampler(0, enabled=not args.no_clocks) as clk:
        for name, precision, cc, sp in (("mixed", 1, False, args.sort_period),
                                        ("mixed_unsorted", 1, False, 0),
                                        ("fp64", 0, False, 0),
                                        ("fp64_charge_conserving", 0, True, 0)):
            if name == "mixed_unsorted" and args.sort_period == 0:
                continue
            forms[name] = time_weibel2d(prob, precision, args, stream, flush, cc, sp)
    out = {}
    for name, f in forms.items():
        kern = f["kernels"]
        for kind, kname in ((0, "pass_c"), (1, "pass_e")):
            if kname in kern:
                t = kern[kname]["avg_us"] * 1e-6
                ach = EM2D_ALGO_BYTES[("mixed" if name.startswith("mixed") else name, kind)] * n / t / 1e9
                kern[kname]["achieved_GBs"] = round(ach, 1)
                kern[kname]["frac_hbm"] = round(ach / peak, 4)
                if not name.startswith("mixed"):  # the FP64 forms: FP64-pipe instructions per marker (ncu)
                    kern[kname]["fp64_ginst_s"] = round(EM2D_FP64_INST_PER_MARKER[(name, kind)] * n / t / 1e9, 1)
                    kern[kname]["frac_fp64"] = round(kern[kname]["fp64_ginst_s"] / fp64_peak, 4)
        dom = max(("pass_c", "pass_e"), key=lambda k: kern[k]["avg_us"]) if "pass_e" in kern else None
        dk = 1 if dom == "pass_e" else 0
        if dom is None:
            roof = None                       # no profiled steps
        elif not name.startswith("mixed"):
            roof = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["fp64_ginst_s"],
                    "peak": round(fp64_peak, 1), "unit": "Ginst/s (FP64 pipe)",
                    "frac": kern[dom]["frac_fp64"], "traffic": EM2D_TRAFFIC[(name, dk)],
                    "peak_source": f"{FP64_LANES_PER_SM_CLK} FP64 lanes/SM/clk x SMs x 2070 MHz",
                    "hbm_frac": kern[dom]["frac_hbm"], "hbm_peak": peak,
                    "hbm_peak_source": peak_src}
        else:
            # the HBM fraction of the algorithmic bytes, reported for reference:
            # these passes are bound by L2 requests (the integer current's
            # global atomics), see the note
            roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_GBs"],
                    "peak": peak, "unit": "GB/s", "frac": kern[dom]["frac_hbm"],
                    "traffic": EM2D_TRAFFIC.get((name, dk)), "peak_source": peak_src,
                    "note": "bound by L2 requests (64-bit global atomics of the integer "
                            "current; ncu: L2 tag lookups near 70% of peak), not by HBM"}
        out[name] = {"value": n * args.steps / (f["step_ms"].sum() / 1e3),
                     "ms_per_step": float(f["step_ms"].mean()),
                     "energy": {"max_rel_dTE": f["max_rel_dTE"], "fallbacks": f["fallbacks"]},
                     "gpu_launches": f["launches"], "kernels": kern, "roofline": roof}
    hf = out["mixed"]
    line = {
        "metric": "particle-steps/s, 2D3V Weibel with the Yee/leapfrog field step",
        "value": hf["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": hf["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32+i64 (fields and energy in f64)",
        "data": "synthetic (seeded bi-Maxwellian markers)",
        "config": {"workload": "weibel_2d3v_yee", "cells": [prob.nx, prob.ny],
                   "markers": n, "dt": prob.dt, "c": prob.c, "scheme": "ESEC2",
                   "shape_order": prob.order, "form": "mixed",
                   "sort_period": args.sort_period,
                   "l2": "flushed (512 MiB write) before every timed step"},
        "energy": hf["energy"], "gpu_launches": hf["gpu_launches"],
        "kernels": hf["kernels"], "clocks": clk.summary(), "roofline": hf["roofline"],
        "forms": out,
    }
    print(json.dumps(line), flush=True)


# pass C reads y, vx, vy and writes v*; pass E reads them and v*, writes y, vx, vy
EM1D_ALGO_BYTES = {0: 40, 1: 64}          # pass C also writes v*, pass E reads it
# FP64-pipe thread instructions per marker of the 1D2V passes (ncu,
# sm__thread_inst_executed_pipe_fp64_pred_on.sum / markers at 2^23 markers):
# like the FP64 1D form these passes are bound by the FP64 pipe, not by HBM
EM1D_FP64_INST_PER_MARKER = {0: 42.57, 1: 74.38}
# DRAM bytes per launch at 2^23 markers (dram__bytes_read.sum + dram__bytes_write.sum)
EM1D_TRAFFIC = {0: 627530240, 1: 822075136}
# the mixed form: y (u32) and two float pairs; pass C writes V* (2 x i32),
# pass E reads it and writes y and the pairs
EM1D_MIX_ALGO_BYTES = {0: 28, 1: 48}
EM1D_MIX_TRAFFIC = {0: 206697216, 1: 342160384}   # dram read + write per launch, 2^23 markers


def _weibel1d_form(W, pic, torch, solver, precision, args, stream, flush, peak, long_steps):
    """One solver in one form: the paper's size over a long run (energy) and
    2^23 markers with per-step events and an L2 flush before each (throughput)."""
    res = {}
    # the paper's size: state 2.5 MB, L2-resident; chunks of <= 1000 steps
    prob = W.weibel_1d2v(seed=0)
    sim = pic.Simulation1D2V(prob, solver=solver, stream=stream.cuda_stream, precision=precision)
    try:
        te0 = sim.energy()[3]
        fbs, tes, ms = [], [], 0.0
        left = long_steps
        while left:
            k = min(left, 1000)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            pic.pic_step_async(sim.h, k)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            fb, te = pic.pic_read_stats(sim.h)
            fbs.append(fb)
            tes.append(te)
            left -= k
        fb, te = np.concatenate(fbs), np.concatenate(tes)
        WE = sim.energy()
    finally:
        sim.close()
    res["paper_size"] = {
        "markers": prob.n_markers, "steps": long_steps, "t_end": long_steps * prob.dt,
        "value": prob.n_markers * long_steps / (ms / 1e3), "us_per_step": 1e3 * ms / long_steps,
        "max_rel_dTE": float(np.max(np.abs(te - te0)) / te0), "fallbacks": int(fb.sum()),
        "W_B_end": WE[2], "l2": "resident (2.5 MB state), not flushed"}
    big = W.weibel_1d2v(ppc=(1 << 23) // 32, seed=1)
    sim = pic.Simulation1D2V(big, solver=solver, stream=stream.cuda_stream, precision=precision)
    try:
        te0 = sim.energy()[3]
        pic.pic_step_async(sim.h, max(3, args.warmup))
        pic.pic_read_stats(sim.h)
        evs = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):   # the flush on the handle's stream, before the step
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pic.pic_step_async(sim.h, 1)
            b.record(stream)
            evs.append((a, b))
        fb, te = pic.pic_read_stats(sim.h)
        torch.cuda.synchronize()
        step_ms = np.array([a.elapsed_time(b) for a, b in evs])
        pic.pic_set_profiling(sim.h, True)
        for _ in range(args.profile_steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            pic.pic_step_async(sim.h, 1)
        pic.pic_read_stats(sim.h)
        kern = {}
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        fp64_peak = FP64_LANES_PER_SM_CLK * nsm * 2070.0e6 / 1e9   # Ginst/s
        for kind, kname in ((0, "pass_c"), (1, "pass_e")):
            n, tot = pic.pic_profile(sim.h, kind)
            if n:
                avg = 1e3 * tot / n
                algo = (EM1D_MIX_ALGO_BYTES if precision else EM1D_ALGO_BYTES)[kind]
                ach = algo * big.n_markers / (avg * 1e-6) / 1e9
                kern[kname] = {"avg_us": avg, "launches": n, "achieved_GBs": round(ach, 1),
                               "frac_hbm": round(ach / peak, 4)}
                if not precision:
                    inst = EM1D_FP64_INST_PER_MARKER[kind] * big.n_markers / (avg * 1e-6) / 1e9
                    kern[kname].update({"fp64_ginst_s": round(inst, 1),
                                        "fp64_peak": round(fp64_peak, 1),
                                        "frac_fp64": round(inst / fp64_peak, 4)})
        pic.pic_set_profiling(sim.h, False)
    finally:
        sim.close()
    res["2p23"] = {"markers": big.n_markers, "steps": args.steps,
                   "value": big.n_markers * args.steps / (step_ms.sum() / 1e3),
                   "us_per_step": 1e3 * float(step_ms.mean()),
                   "max_rel_dTE": float(np.max(np.abs(te - te0)) / te0),
                   "fallbacks": int(fb.sum()), "kernels": kern,
                   "l2": "flushed (512 MiB write) before every timed step"}
    return res


def run_weibel1d(args):
    """The 1D2V Weibel test of Sec. 5 (32 cells, beta 0.01, beams +-0.3, b 0.001,
    k0 0.2, dt 0.1, c 1) with both spectral field solves, each in the FP64 and
    the mixed form: the paper's size (3200 markers per cell, 102,400 markers)
    over a long run for the energy error, and 2^23 markers (262,144 per cell)
    for throughput and the roofline of the passes.  The headline is PSATD in
    the mixed form at 2^23 markers."""
    import torch
    from paper_2411_09605_gb300 import build as B, pic, workloads as W
    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", 0)
    peak, peak_src = hbm_peak()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    long_steps = max(10, min(args.steps * 10, 4000))
    out = {}
    with ClockSampler(0, enabled=not args.no_clocks) as clk:
        for name, solver in (("cn", pic.PIC_SOLVER_CN_SPECTRAL), ("psatd", pic.PIC_SOLVER_PSATD)):
            for form, precision in (("fp64", 0), ("mixed", 1)):
                out[f"{name}_{form}"] = _weibel1d_form(W, pic, torch, solver, precision, args,
                                                       stream, flush, peak, long_steps)
    head = out["psatd_mixed"]["2p23"]
    dom = max(head["kernels"].items(), key=lambda kv: kv[1]["avg_us"]) if head["kernels"] else None
    line = {
        "metric": "particle-steps/s, 1D2V Weibel with spectral EM field solves",
        "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": head["us_per_step"] / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32+i64 (fields, field solve and energy in f64)",
        "data": "synthetic (seeded Weibel markers, quiet start in y)",
        "config": {"workload": "weibel_1d2v", "cells": 32, "dt": 0.1, "c": 1.0, "shape_order": 1,
                   "scheme": "ESEC2", "value_from": "PSATD, mixed form, at 2^23 markers"},
        "roofline": None if dom is None else {     # None: no profiled steps
            "bound": "hbm", "kernel": dom[0], "achieved": dom[1]["achieved_GBs"], "peak": peak,
            "unit": "GB/s", "frac": dom[1]["frac_hbm"],
            "traffic": EM1D_MIX_TRAFFIC[0 if dom[0] == "pass_c" else 1], "peak_source": peak_src},
        "solvers": out, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)

def run_grad(args):
    """Reverse mode of the FP64 form on the bump-on-tail workload (2^20 weighted
    markers, 256 cells, dt 0.1, 500 steps, checkpoints every 50): throughput of
    the forward + reverse pass, and for several horizons the derivative of the
    final W_E by the seed amplitude alpha (through the weights, the initial field
    held at its alpha = 0.04 value) against central differences."""
    import torch
    from paper_2411_09605_gb300 import build as B, pic, workloads as W
    B.build()
    torch.cuda.set_device(0)
    n, nc, k, a0 = 1 << 20, 256, 0.3, 0.04
    nsteps, every = 500, 50
    base = W.bump_on_tail(n=n, nc=nc, k=k, alpha=a0, seed=0)
    sim0 = pic.Simulation(base)
    E0 = sim0.field()
    sim0.close()
    s = base.species[0]
    dw = (base.L / n) * np.cos(k * s.x)

    def objective_and_grad(steps, alpha, want_grad):
        sim = pic.Simulation(W.bump_on_tail(n=n, nc=nc, k=k, alpha=alpha, seed=0), E0=E0)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if want_grad:
                pic.pic_grad_forward(sim.h, steps, every)
                fb, _ = pic.pic_read_stats(sim.h)
            else:
                fb, _ = sim.step(steps)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            E = sim.field()
            h = base.L / nc
            L = 0.5 * h * float(np.sum(E * E))
            g = None
            if want_grad:
                wb = np.zeros(n)
                pic.pic_grad_backward(sim.h, h * E, None, None, None, None, None, wb)
                torch.cuda.synchronize()
                g = float(np.dot(wb, dw))
            t2 = time.perf_counter()
        finally:
            sim.close()
        return L, g, t1 - t0, t2 - t1, int(np.sum(fb))

    objective_and_grad(20, a0, True)                    # warm-up
    L, g, t_fwd, t_bwd, nfb = objective_and_grad(nsteps, a0, True)
    # central differences at two step sizes: where they disagree with each other
    # the objective is not smooth on that scale (a marker switching between Gamma
    # and its fallback makes W_E jump), and no derivative can match them
    horizons = []
    for H in (10, 20, 50, 100, 200, 500):
        _, gh, _, _, fb_h = objective_and_grad(H, a0, True)
        fd = {}
        for eps in (1e-6, 1e-7):
            lp = objective_and_grad(H, a0 + eps, False)[0]
            lm = objective_and_grad(H, a0 - eps, False)[0]
            fd[eps] = (lp - lm) / (2 * eps)
        horizons.append({"steps": H, "ad": gh, "fd_eps_1e-6": fd[1e-6], "fd_eps_1e-7": fd[1e-7],
                         "rel_diff_ad_fd": abs(fd[1e-6] - gh) / max(abs(fd[1e-6]), 1e-300),
                         "rel_diff_fd_fd": abs(fd[1e-6] - fd[1e-7]) / max(abs(fd[1e-6]), 1e-300),
                         "fallbacks": fb_h})
    line = {
        "metric": "particle-steps/s of forward + reverse (bump-on-tail, FP64 form)",
        "value": n * nsteps / (t_fwd + t_bwd), "unit": UNIT, "n_gpus": 1, "steps": nsteps,
        "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded bump-on-tail, weighted markers)",
        "config": {"workload": "bump_on_tail_1d1v", "markers": n, "cells": nc, "dt": 0.1,
                   "checkpoint_every": every, "objective": "W_E after the steps",
                   "timing": "wall clock around forward and reverse (host synchronised; the "
                             "reverse includes the download of the weight adjoints)"},
        "forward_s": t_fwd, "reverse_s": t_bwd, "fallbacks": nfb,
        "dWE_dalpha": g, "horizons": horizons,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- reference arm


def run_reference(args):
    """The oracle as the reference arm: each step is one oracle step of a bounded
    sample (2^18 markers) of the same workload, on all host cores (the OpenMP
    build of the oracle's source)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    threads = O.omp_threads()
    markers = 1 << 18
    prob = workload(markers, 0)
    s = prob.species[0]
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=2)
    sp = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None, s.w0)]
    E = O.poisson_e0_1d(cfg, sp)
    for _ in range(args.warmup):
        O.es1d_step(cfg, sp, E, threaded=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.es1d_step(cfg, sp, E, threaded=True)
    dt = time.perf_counter() - t0
    value = markers * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded two-stream markers)",
        "config": config_dict(prob, {"form": "oracle", "sample_of_markers": 1 << 23}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{markers} of the 2^23 markers per step, FP64 C oracle "
                                   f"built with OpenMP ({threads} threads)",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.ensemble:
        run_ensemble(args)
    elif args.grad:
        run_grad(args)
    elif args.weibel1d:
        run_weibel1d(args)
    elif args.weibel2d:
        run_weibel2d(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
