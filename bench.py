#!/usr/bin/env python
"""Throughput of the adjoint-descent step on GB300.

Metric: curve-point adjoint-gradient evaluations per second, i.e. interior
curve points (M = N_s - 2 per curve) x descent steps / time.  One bench step is
one full descent step of the workload curve: the row phase (f, residual,
spatial adjoint, FP64 cost reductions), the s-phase with the descent update and
|G|^2, and the s-phase D_t u of the new state (one kernel each, three each in
the three-launch four-step form; one launch for both s-phases in the clustered
form, the bench workload's).

Default workload: L = 22, N_x = 64, N_s = 1024 (the differentiation workload),
FP32 storage and transforms with FP64 reductions.  The curve is far smaller
than L2, so L2 is flushed (a 256 MiB write) before every timed step and each
step is timed on its own with CUDA events on the curve's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own curve (independent replicas,
weak scaling); rank 0 prints the JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "curve-point adjoint-gradient evals/s"
UNIT = "point-evals/s"
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) per launch of the dominant kernel, from one
# `ncu --set full` capture of `bench.py --steps 30 --warmup 3` (caches flushed by
# ncu between its passes), keyed by (form, F, N_x, precision, fused step); other
# configurations report null, and an entry is dropped when its kernel changes.
NCU_TRAFFIC = {("fft4c", 4096, 64, "fp32", True): 960512}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--s-transform", choices=["auto", "dense", "fft", "dense_tc", "fft4", "fft4c"], default="auto",
                    help="how D_t is applied along s in the headline curve")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["curve", "batch"], default="curve",
                    help="curve: one L=22, N_x=64, N_s=1024 curve (default); batch: the 256-curve batch")
    return ap.parse_args()


def workload_spec():
    from paper_2301_11704_gb300 import gen
    return gen.workload(1)[0]


def workload_config(spec, precision):
    return {"workload": "KSE curve L=%g N_x=%d N_s=%d (M=%d), S=%g, dtau=%g, %s storage, FP64 reductions"
                        % (spec.L, spec.N, spec.Ns, spec.M, spec.S, spec.dtau, precision),
            "L": spec.L, "N_x": spec.N, "N_s": spec.Ns, "S": spec.S, "dtau": spec.dtau,
            "adjoint": "paper", "curves_per_gpu": 1,
            "l2": "flushed before every timed step (256 MiB write); each step timed alone",
            "parallelism": "independent replicas (one curve per GPU)"}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for name, val in zip(names, row[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- oracle (CPU)
def oracle_steps(spec, budget_s, max_steps=None):
    """Times the FP64 oracle's descent on the same curve until the budget is used."""
    import oracle
    from paper_2301_11704_gb300 import gen
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    U = oracle.curve_init(spec.M, spec.S, up, um, s0=spec.s0, amps=amps, vp=vp)
    oracle.curve_descend(U, spec.L, spec.S, 1, dtau=spec.dtau)          # build + warm caches
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        U, _, _, _ = oracle.curve_descend(U, spec.L, spec.S, 1, dtau=spec.dtau)
        times.append(time.perf_counter() - t0)
        if max_steps is not None and len(times) >= max_steps:
            break
        if max_steps is None and time.perf_counter() - t_all >= budget_s:
            break
    return times, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    spec = workload_spec()
    import oracle
    oracle.build()
    # warm-up steps are untimed; each timed step is one full oracle descent step of the curve
    oracle_steps(spec, 0.0, max_steps=max(1, min(args.warmup, 3)))
    times, cores = oracle_steps(spec, 0.0, max_steps=args.steps)
    total = sum(times)
    value = spec.M * len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(spec, "FP64"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d full descent steps of the workload curve" % len(times)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- batch workload
def run_batch(args):
    """256 curves, L ~ U[20,60], N_x in {32,64,128}, N_s ~ U[256,2048], FP32 storage,
    FP64 reductions, autotuned s-phase tiles, steps replayed from a CUDA graph.  The
    batch's fields (~0.4 GB) exceed L2, so steps are timed back to back."""
    import numpy as np
    import torch
    from paper_2301_11704_gb300 import gen
    from paper_2301_11704_gb300.batch import KSBatch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    specs = gen.workload(3)
    ins = [(gen.end_points(s), gen.perturbation(s)) for s in specs]
    b = KSBatch(specs, [i[0][0] for i in ins], [i[0][1] for i in ins], precision="fp32", conv="jrel", device=dev)
    b.init_trial(np.array([i[1][0] for i in ins]), [i[1][1] for i in ins])
    chosen = b.autotune(8)
    b.descend_async(args.warmup)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.descend_async(args.steps)
    e1.record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    points = sum(s.M for s in specs)
    from paper_2301_11704_gb300.build import fft_length

    def sflops(s):   # both s-contractions of a step, in the form the curve runs
        F = fft_length(s.Ns, True)
        return 2 * (s.N // 2) * (2 * 5.0 * F * np.log2(F) + 6.0 * F) if F else 4.0 * s.Ns * s.Ns * s.N
    flops = sum(sflops(s) for s in specs)
    ach = flops / (ms / args.steps / 1e3) / 1e12
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    bytes_alg = sum(2.0 * s.M * s.N * 4 for s in specs)   # state read + write per step
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = float(json.load(f).get("hbm_gbs", 6800.0))
    except OSError:
        hbm_peak = 6800.0
    hbm_ach = bytes_alg / (ms / args.steps / 1e3) / 1e9
    sc = b.scalars()
    line = {"metric": METRIC, "value": points * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of 256 KSE curves, L~U[20,60], N_x in {32,64,128}, N_s~U[256,2048]",
                       "curves": len(specs), "points_per_step": points, "tile_width": chosen,
                       "l2": "working set ~0.4 GB > L2; steps back to back (CUDA-graph replay)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": None, "kernel": "whole step: flops of both s-contractions (FFT form "
                                                     "where N_s allows) / step time",
                         "algorithmic_flops_per_step": flops,
                         "hbm": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
                                 "algorithmic_bytes_per_step": bytes_alg,
                                 "note": "B_alg = state read + write (2 N_x b per point)"}},
            "gpu_launches": None, "clocks": clk,
            "median_J_rel": float(np.median([x["J"] / max(x["Dnorm"], 1e-300) for x in sc]))}
    print(json.dumps(line))
    b.close()
    return 0


# ---------------------------------------------------------------------------- GPU
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2301_11704_gb300 import gen
    from paper_2301_11704_gb300.curve import KSCurve

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    spec = workload_spec()
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)

    def make_curve(precision, s_transform="auto"):
        c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, s0=spec.s0, dtau=spec.dtau, precision=precision,
                    s_transform=s_transform, device=dev)
        c.init_trial(0.0, None, amps, vp)
        return c

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed_steps(c, K, W, profile=0):
        for _ in range(W):
            flush.fill_(1)
            c.descend_async(1)
        torch.cuda.synchronize(dev)
        if profile:
            c.profile(profile)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        torch.cuda.synchronize(dev)
        for i in range(K):
            flush.fill_(i & 255)
            ev[i][0].record()
            c.descend_async(1)
            ev[i][1].record()
        torch.cuda.synchronize(dev)
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = c.profile_read() if profile else None
        if profile:
            c.profile(0)
        return ms, prof

    curve = make_curve(args.precision, args.s_transform)
    K, W = args.steps, args.warmup
    clocks = ClockSampler(local)
    clocks.start()
    # per-kernel events on the first 1/20 of the timed steps only: events between
    # kernels serialise them, so the other steps run as a user's would
    step_ms, prof = timed_steps(curve, K, W, profile=max(1, K // 20))
    clk = clocks.stop()
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms_max = float(t.item())
    points = spec.M
    value = world * points * K / (total_ms_max / 1e3)
    sc = curve.scalars()

    # ---- roofline of the dominant kernel (per-launch event times from inside the library)
    b = 4 if args.precision == "fp32" else 8
    field = spec.Ns * spec.N * b
    avg = {k: v["ms"] / max(v["launches"], 1) for k, v in prof.items()}
    dom = max(avg, key=avg.get)
    from paper_2301_11704_gb300.build import fft_length
    F = curve.fft_length
    form_name = {"dense": "dense contraction", "dense_tc": "dense contraction on the tensor cores",
                 "fft": "FFT convolution, one CTA per mode", "fft4": "four-step FFT convolution, three launches",
                 "fft4c": "four-step FFT convolution, one clustered launch"}[curve.s_form]
    if F:   # FFT form: per mode two complex FFTs of length F and the spectral product
        flops_dt = (spec.N // 2) * (2 * 5.0 * F * np.log2(F) + 6.0 * F)
        dt_form = "%s, F=%d" % (form_name, F)
    else:
        flops_dt = 2.0 * spec.Ns * spec.Ns * spec.N
        dt_form = form_name
    # kernels per timed step (one descend call of one step, whose row phase arms
    # the step limit): the row phase and two s-contractions (three launches each
    # in the three-launch four-step form, both in one launch in the clustered form)
    n_x = spec.N
    fused = curve.s_form == "fft4c" and ((n_x <= 64 and F <= 16384) or (n_x <= 128 and F <= 8192) if b == 4
                                         else n_x <= 16 and F == 4096)
    launches_per_step = 2 if fused else (7 if curve.s_form == "fft4" else 3)
    if fused:   # the update launch applies both contractions
        flops_dt *= 2
        dt_form += "; update and D_t u in one launch"
    peak_alu = (N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12) if b == 4 else 1.25
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    if dom == "rows":
        bytes_alg = 4 * field + spec.Ns * 32
        ach = bytes_alg / (avg[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": None, "kernel": "k_rows", "algorithmic_bytes": bytes_alg}
    else:
        ach = flops_dt / (avg[dom] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s", "frac": ach / peak_alu,
                "traffic": None, "kernel": "s-contraction (%s, %s)" % (dom, dt_form), "algorithmic_flops": flops_dt,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz" if b == 4 else
                "nominal FP64 1.25 TFLOP/s"}
    roof["phase_ms_per_launch"] = avg
    if dom != "rows":
        roof["traffic"] = NCU_TRAFFIC.get((curve.s_form, F, spec.N, args.precision, fused))

    # ---- end to end through the public API with host buffers
    e2e = None
    if rank == 0 or world > 1:
        dt = curve.dtype
        host_in = torch.empty((spec.Ns, spec.N), dtype=dt).pin_memory()
        host_out = torch.empty((spec.Ns, spec.N), dtype=dt).pin_memory()
        host_in.copy_(curve.get_state().cpu())
        dev_in = torch.empty((spec.Ns, spec.N), dtype=dt, device=dev)
        n_e2e = max(1, min(args.e2e_steps, K))
        nb = spec.Ns * spec.N * b
        # every step: the curve from pinned host memory (set_state), one descent
        # step, and its result J read back to the host (ks_curve_descend copies the
        # device scalar record, 176 bytes, and synchronises)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            dev_in.copy_(host_in, non_blocking=True)
            curve.set_state(dev_in, 1.0, 0.0)
            curve.descend(1)
        e2e_s = time.perf_counter() - t0
        # the same with the whole state read back as well (context)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            dev_in.copy_(host_in, non_blocking=True)
            curve.set_state(dev_in, 1.0, 0.0)
            curve.descend(1)
            host_out.copy_(curve.get_state(), non_blocking=True)
            torch.cuda.synchronize(dev)
        e2e_state_s = time.perf_counter() - t0
        e2e = {"value": points * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": 176, "steps": n_e2e,
               "path": "pinned host curve -> set_state -> descend(1), J read back",
               "with_state_readback": {"value": points * n_e2e / e2e_state_s, "d2h_bytes_per_step": nb + 176,
                                       "path": "... -> get_state -> pinned host"}}

    # ---- steady state: K consecutive steps in one call (graph replay, L2 not flushed)
    steady = None
    if rank == 0:
        curve.descend_async(min(K, 64))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        curve.descend_async(K)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        steady = {"value": points * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K, "steps": K,
                  "note": "descend_async(K): CUDA-graph replay, curve L2-resident (not the headline)"}

    # ---- the other form of the s-contraction (context)
    other = None
    other_form = "dense" if F else "fft"
    if F or fft_length(spec.Ns, b == 4):
        cd = make_curve(args.precision, other_form)
        kd = max(3, min(200, K))
        msd, _ = timed_steps(cd, kd, 3)
        other = {"form": other_form, "value": points * kd / (sum(msd) / 1e3), "unit": UNIT,
                 "ms_per_step": sum(msd) / kd, "steps": kd}
        cd.close()

    # ---- FP64 GPU path (context)
    fp64 = None
    if args.precision == "fp32":
        c64 = make_curve("fp64")
        k64 = max(3, min(50, K))
        ms64, _ = timed_steps(c64, k64, 3)
        fp64 = {"value": points * k64 / (sum(ms64) / 1e3), "unit": UNIT, "ms_per_step": sum(ms64) / k64,
                "steps": k64}
        c64.close()

    # ---- the larger workloads (context): L=44, N_x=128, N_s=4096 and L=100, N_x=256,
    # N_s=16384, FP32 storage, the form auto picks, L2 flushed before each step
    large = []
    if rank == 0 and args.precision == "fp32":
        for cfg in (2, 4):
            sp = gen.workload(cfg)[0]
            upl, uml = gen.end_points(sp)
            ampl, vpl = gen.perturbation(sp)
            cl = KSCurve(sp.L, sp.N, sp.Ns, sp.S, upl, uml, s0=sp.s0, dtau=sp.dtau, precision="fp32", device=dev)
            cl.init_trial(0.0, None, ampl, vpl)
            kl = max(3, min(50, K))
            msl, _ = timed_steps(cl, kl, 3)
            entry = {"workload": "L=%g N_x=%d N_s=%d FP32" % (sp.L, sp.N, sp.Ns),
                     "value": sp.M * kl / (sum(msl) / 1e3), "unit": UNIT, "ms_per_step": sum(msl) / kl,
                     "steps": kl, "s_transform": "%s%s" % (cl.s_form, (", F=%d" % cl.fft_length) if cl.fft_length
                                                           else "")}
            cl.close()
            if cfg == 4:
                # the mixed-precision workload's error against the plain FP64 GPU path:
                # J and J_arc of the trial curve, J and the curve after ten steps
                res = {}
                for prec in ("fp64", "fp32"):
                    ce = KSCurve(sp.L, sp.N, sp.Ns, sp.S, upl, uml, s0=sp.s0, dtau=sp.dtau, precision=prec,
                                 device=dev)
                    ce.init_trial(0.0, None, ampl, vpl)
                    j2, ja = ce.cost()
                    o = ce.descend(10)
                    res[prec] = (j2, ja, o["J"], ce.get_state().double())
                    ce.close()
                (j2d, jad, jd, ud), (j2s, jas, js, us) = res["fp64"], res["fp32"]
                entry["vs_fp64_gpu_path"] = {"J2_rel": abs(j2s - j2d) / j2d, "J_arc_rel": abs(jas - jad) / jad,
                                             "J_after_10_steps_rel": abs(js - jd) / jd,
                                             "u_after_10_steps_rel_2": float(((us - ud).norm() / ud.norm()).item())}
            large.append(entry)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        times, cores = oracle_steps(spec, args.cpu_seconds)
        cpu = {"value": points * len(times) / sum(times), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d full FP64 descent steps of the same curve (%.1f s)" % (len(times), sum(times))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms_max / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": dict(workload_config(spec, args.precision.upper()), s_transform=dt_form),
                "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * K, "clocks": clk,
                "fp64_gpu_path": fp64, "larger_workloads": large, "other_s_transform": other, "steady_state": steady, "final_J": sc["J"], "final_J_arc": sc["J_arc"],
                "step_ms_median": statistics.median(step_ms)}
        print(json.dumps(line))
    curve.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
