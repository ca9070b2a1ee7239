#!/usr/bin/env python
"""Throughput of the adjoint-descent step on GB300.

Metric: curve-point adjoint-gradient evaluations per second, i.e. interior
curve points (M = N_s - 2 per curve) x descent steps / time.  One bench step is
one full descent step of the workload curve: the row phase (f, residual,
spatial adjoint, FP64 cost reductions), the s-contraction with the descent
update and |G|^2, and the s-contraction D_t u of the new state.

Workloads (`--workload`):
  mixed  L = 100, N_x = 256, N_s = 16384 (the default: the largest single-GPU
         curve, the mixed-precision workload): FP32 storage with FP64 reductions
         (`--precision fp32`), the x-transforms as split-BF16 tensor-core
         products (`bf16x2`, `bf16x3`), or plain FP64 (`fp64`);
  large  L = 44, N_x = 128, N_s = 4096;
  diff   L = 22, N_x = 64, N_s = 1024 (the differentiation workload);
  batch  256 curves, L ~ U[20,60], N_x in {32,64,128}, N_s ~ U[256,2048].
The single-curve workloads flush L2 (a 256 MiB write) before every timed step
and time each step alone with CUDA events on the curve's stream.

The JSON line carries, besides the throughput: the roofline of the dominant
kernel (algorithmic bytes and flops per launch after the per-point counts below,
over its mean event time), the HBM fraction of the whole step, the error of J,
J_arc, the gradient and the curve after ten steps against the FP64 oracle
(stored reference values), the plain FP64 GPU path at the same workload, an end
to end number through the C ABI with host buffers, and a CPU baseline (the
oracle on a bounded sample of the workload).

Per interior point and step (N = N_x, M = N_s - 2, b = bytes per stored word):
  flops  12.5 N log2 N (five real x-transforms) + 10 N log2(2(M+1)) (four real
         s-transforms) + 30 N (pointwise);
  bytes  2 N b (the state read and written; every intermediate can be recomputed).
Per kernel: the row phase reads U, D_t U and writes R, A (4 N b per section);
the update contraction reads R, A, U and writes U (4 N b); the D_t u contraction
reads U and writes D (2 N b); each contraction does half the s-transform flops.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mixed|large|diff|batch] [--precision ...]

Under torchrun (N > 1) every rank runs its own curve (independent replicas,
weak scaling); rank 0 prints the JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
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
WORKLOADS = {"diff": 1, "large": 2, "batch": 3, "mixed": 4}
BYTES = {"fp64": 8, "fp32": 4, "bf16x2": 4, "bf16x3": 4}
# the CUDA sources that define each kernel (a DRAM-traffic figure is used only
# while these are unchanged since its capture)
KERNEL_SOURCES = {
    "rows": ["ks_device.cuh", "ks_kernels.cu", "ks_internal.h"],
    "rows_tc": ["ks_rows_tc.cu", "ks_device.cuh", "ks_internal.h"],
    "fft4": ["ks_fft4.cu", "ks_device.cuh", "ks_internal.h"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mixed")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16x2", "bf16x3"], default=None,
                    help="default: the fastest form that meets the workload's J tolerance")
    ap.add_argument("--s-transform", choices=["auto", "dense", "fft", "dense_tc", "fft4", "fft4c"], default="auto")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the context measurements (other forms, "
                                                                 "FP64 path, other workloads, oracle errors)")
    return ap.parse_args()


def default_precision(workload):
    """The mixed-precision workload runs its x-transforms as split-BF16 tensor-core
    products with two parts (within 1e-5 of the FP64 oracle in J there, measured
    by tests/test_gpu_bf16.py); the others FP32."""
    return "bf16x2" if workload == "mixed" else "fp32"


def spec_of(workload):
    from paper_2301_11704_gb300 import gen
    return gen.workload(WORKLOADS[workload])[0]


def workload_name(spec, precision):
    prec = {"fp64": "FP64", "fp32": "FP32 storage and transforms, FP64 reductions",
            "bf16x2": "FP32 storage, x-transforms as 2-term split-BF16 tensor-core products, FP64 reductions",
            "bf16x3": "FP32 storage, x-transforms as 3-term split-BF16 tensor-core products, FP64 reductions"}
    return ("KSE curve L=%g N_x=%d N_s=%d (M=%d), S=%g, dtau=%g; %s"
            % (spec.L, spec.N, spec.Ns, spec.M, spec.S, spec.dtau, prec[precision]))


def config_of(spec, precision):
    """The workload's config, the same in both arms."""
    return {"workload": workload_name(spec, precision), "L": spec.L, "N_x": spec.N, "N_s": spec.Ns, "S": spec.S,
            "dtau": spec.dtau, "precision": precision, "adjoint": "paper", "curves_per_gpu": 1,
            "l2": "flushed before every timed step (256 MiB write); each step timed alone",
            "parallelism": "independent replicas (one curve per GPU)"}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def sources_digest(kind):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        p = os.path.join(ROOT, "paper_2301_11704_gb300", "csrc", name)
        if os.path.exists(p):
            with open(p, "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel_key, kind):
    """DRAM bytes (read + write) per launch of a kernel from the ncu captures
    summarised in profiles/dram_traffic.txt, when the kernel's sources are the
    ones captured (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = sources_digest(kind)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel_key and parts[2] == digest:
                return {"bytes_per_launch": float(parts[1]), "sources": digest,
                        "from": "ncu capture summarised in profiles/dram_traffic.txt"}
    return None


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


# ---------------------------------------------------------------------------- per-point counts
def flops_per_point(N, M):
    """Section 8(d) counts per interior point and step: x-side, s-side, pointwise."""
    fx = 12.5 * N * math.log2(N)
    fs = 10.0 * N * math.log2(2 * (M + 1))
    fp = 30.0 * N
    return fx, fs, fp


# ---------------------------------------------------------------------------- oracle (CPU)
ORACLE_COLS = 16     # complex Fourier columns of the s-direction sample (one per core on the box)
ORACLE_ROWS = 64     # sections of the x-direction sample


def oracle_sample_step(spec, U):
    """One descent step of the oracle on a bounded sample of the workload curve,
    scaled to the whole curve.  The oracle's step is an x-part per section (naive
    DFTs: f, residual, spatial adjoint) and an s-part per Fourier column (the two
    explicit trig sums of D_t applied to u and to r); each part is timed on a
    sample, through the oracle's own curve functions as they stand:
      s-part: curve_residual + curve_adjoint on the curve restricted to its first
              ORACLE_COLS complex columns (all N_s sections; D_t on those columns
              exactly as in the full step), scaled by (N/2) / ORACLE_COLS;
      x-part: curve_residual + curve_adjoint on ORACLE_ROWS of its sections at
              full N (the x-work of those sections), scaled by N_s / ORACLE_ROWS.
    Returns the estimated seconds of one full oracle step."""
    import numpy as np
    import oracle
    H = spec.N // 2
    Uc = np.ascontiguousarray(U[:, :ORACLE_COLS])
    t0 = time.perf_counter()
    R, _ = oracle.curve_residual(Uc, spec.L, spec.S)
    oracle.curve_adjoint(Uc, R, spec.L, spec.S)
    t_cols = time.perf_counter() - t0
    rows = np.linspace(0, spec.Ns - 1, ORACLE_ROWS).astype(int)
    Ur = np.ascontiguousarray(U[rows])
    t0 = time.perf_counter()
    R, _ = oracle.curve_residual(Ur, spec.L, spec.S)
    oracle.curve_adjoint(Ur, R, spec.L, spec.S)
    t_rows = time.perf_counter() - t0
    return t_cols * H / ORACLE_COLS + t_rows * spec.Ns / ORACLE_ROWS


def oracle_baseline(spec, nsamples):
    """(point-evals/s, per-sample step estimates, threads) of the oracle."""
    import oracle
    from paper_2301_11704_gb300 import gen
    oracle.build()
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    U = oracle.curve_init(spec.M, spec.S, up, um, s0=spec.s0, amps=amps, vp=vp)
    est = [oracle_sample_step(spec, U) for _ in range(nsamples)]
    return spec.M * len(est) / sum(est), est, oracle.num_threads()


def oracle_sample_text(spec):
    return ("oracle descent step (FP64, OpenMP) of the same curve, timed on a sample and scaled to the curve: "
            "the s-part (both D_t applications) on %d of %d complex Fourier columns x %d, the x-part on %d of %d "
            "sections x %d" % (ORACLE_COLS, spec.N // 2, spec.N // 2 // ORACLE_COLS, ORACLE_ROWS, spec.Ns,
                               spec.Ns // ORACLE_ROWS))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "batch":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the single-curve "
                                                             "workloads"}))
        return 0
    spec = spec_of(args.workload)
    precision = args.precision or default_precision(args.workload)
    W = max(0, args.warmup)
    oracle_baseline(spec, max(1, min(W, 1)))          # untimed warm-up (builds, pages in)
    value, est, cores = oracle_baseline(spec, args.steps)
    total = sum(est)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": len(est),
            "warmup": W, "ms_per_step": 1e3 * total / len(est), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(spec, precision),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_text(spec)},
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
    fp64 = None
    if not args.no_context:
        # the same batch in FP64 (storage, transforms and reductions), tuned and timed alike
        b64 = KSBatch(specs, [i[0][0] for i in ins], [i[0][1] for i in ins], precision="fp64", conv="jrel",
                      device=dev)
        b64.init_trial(np.array([i[1][0] for i in ins]), [i[1][1] for i in ins])
        t64 = b64.autotune(8)
        b64.descend_async(args.warmup)
        torch.cuda.synchronize(dev)
        e0.record()
        b64.descend_async(args.steps)
        e1.record()
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1)
        b64.close()
        fp64 = {"ms_per_step": ms64 / args.steps, "value": sum(s.M for s in specs) * args.steps / (ms64 / 1e3),
                "unit": UNIT, "fp32_speedup": ms64 / ms,
                "tuning": {k: (v if k != "splits" else {str(a): b2 for a, b2 in v.items()}) for k, v in t64.items()}}
    points = sum(s.M for s in specs)
    flops = sum(s.M * sum(flops_per_point(s.N, s.M)) for s in specs)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, src = read_peaks()
    mhz = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_alu = nsm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    ach = flops / (ms / args.steps / 1e3) / 1e12
    bytes_alg = sum(2.0 * s.M * s.N * 4 for s in specs)
    hbm_peak = float(peaks["hbm_gbs"])
    hbm_ach = bytes_alg / (ms / args.steps / 1e3) / 1e9
    sc = b.scalars()
    line = {"metric": METRIC, "value": points * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of 256 KSE curves, L~U[20,60], N_x in {32,64,128}, N_s~U[256,2048]",
                       "curves": len(specs), "points_per_step": points, "tuning": {k: (v if k != "splits" else {str(a): b2 for a, b2 in v.items()}) for k, v in chosen.items()},
                       "l2": "working set ~0.4 GB > L2; steps back to back (CUDA-graph replay)"},
            "roofline": {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_ach / hbm_peak, "traffic": None, "peak_source": src,
                         "kernel": "whole step of the batch",
                         "algorithmic_bytes_per_step": bytes_alg,
                         "alu": {"achieved": ach, "peak": peak_alu, "unit": "TFLOP/s", "frac": ach / peak_alu,
                                 "algorithmic_flops_per_step": flops}},
            "gpu_launches": None, "clocks": clk,
            "median_J_rel": float(np.median([x["J"] / max(x["Dnorm"], 1e-300) for x in sc])),
            "fp64_batch": fp64}
    print(json.dumps(line))
    b.close()
    return 0


# ---------------------------------------------------------------------------- errors against the oracle
def oracle_errors(spec, make_curve, precision):
    """J^2, J_arc, dJ^2/dl, |G|_W and sampled G of the trial curve, J, J_arc and
    sampled sections after ten steps, against the FP64 oracle's stored values
    (tests/golden/fullsize_*.json, written by tests/golden/make_fullsize_refs.py)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "fullsize_L%g_N%d_Ns%d.json" % (spec.L, spec.N, spec.Ns))
    if not os.path.exists(path):
        return None
    with open(path) as f:
        ref = json.load(f)
    rows = ref["rows"]

    def cx(rowsvals):
        a = np.array(rowsvals)
        return a[..., 0] + 1j * a[..., 1]

    k = 2 * np.pi * np.arange(spec.N // 2) / spec.L
    a = k ** 4 - k ** 2
    pw = spec.dtau / (1.0 + spec.dtau * a * a)

    def spec_rows(x):
        x = np.asarray(x, dtype=np.float64)
        return np.fft.rfft(x, axis=1)[:, : spec.N // 2] / spec.N

    c = make_curve(precision)
    J2, Ja = c.cost()
    g, dl = c.gradient()
    sc = c.scalars()
    Gs = spec_rows(g.double().cpu().numpy()[rows])
    Gr = cx(ref["trial"]["G_rows"])
    res = c.descend(ref["after_steps"]["steps"])
    u = c.get_state().double().cpu().numpy()
    Us = spec_rows(u[rows])
    Ur = cx(ref["after_steps"]["U_rows"])
    c.close()
    tr = ref["trial"]
    rel = lambda x, y: abs(x - y) / abs(y)
    return {"J2": rel(J2, tr["J2"]), "J_arc": rel(Ja, tr["J_arc"]),
            "dJ2_dlambda": rel(dl, tr["dJ2_dlambda"]), "Dnorm": rel(sc["Dnorm"], tr["Dnorm"]),
            "G_norm_W": rel(sc["G_norm"], math.sqrt(tr["G2"])),
            "G_sampled_precond": float(np.linalg.norm((Gs - Gr) * pw) / np.linalg.norm(Gr * pw)),
            "J_after_10": rel(res["J"], ref["after_steps"]["J"]),
            "J_arc_after_10": rel(res["J_arc"], ref["after_steps"]["J_arc"]),
            "u_sampled_after_10": float(np.linalg.norm(Us - Ur) / np.linalg.norm(Ur)),
            "sampled_sections": len(rows), "reference": os.path.relpath(path, ROOT)}


# ---------------------------------------------------------------------------- across ranks
def reduce_max_ms(total_ms, world, device):
    """The slowest rank's timed milliseconds (max over the ranks; every rank gets
    the same value).  One process per GPU; a single process returns its own."""
    if world <= 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, points_per_step, steps, total_ms_max):
    """Whole-job curve-point evaluations per second: every rank steps its own
    replica of the workload (weak scaling), timed by the slowest rank."""
    return world * points_per_step * steps / (total_ms_max / 1e3)


# ---------------------------------------------------------------------------- implicit stepping
def implicit_context(dev, timed_steps, K, dtau=0.5):
    """The L=44, N_x=128, N_s=4096 curve in FP32 stepped with every linear term of
    G implicit (eigenbases of the even and odd parts of the interior D_t^2) at a
    dtau 25x the IMEX limit, beside the IMEX scheme at the workload's dtau:
    device time per step, fictitious time per second, and the increment's two
    products against the FP32 CUDA-core peak."""
    from paper_2301_11704_gb300 import gen
    from paper_2301_11704_gb300.curve import KSCurve
    sl = spec_of("large")
    up, um = gen.end_points(sl)
    amps, vp = gen.perturbation(sl)
    out = {"workload": "L=%g N_x=%d N_s=%d FP32" % (sl.L, sl.N, sl.Ns)}
    for scheme, dt in (("imex", sl.dtau), ("implicit", dtau)):
        t0 = time.perf_counter()
        c = KSCurve(sl.L, sl.N, sl.Ns, sl.S, up, um, s0=sl.s0, dtau=dt, precision="fp32", scheme=scheme, device=dev)
        setup_s = time.perf_counter() - t0
        c.init_trial(0.0, None, amps, vp)
        ms, prof = timed_steps(c, K, 3, profile=K)
        sc = c.scalars()
        c.close()
        step = sum(ms) / K
        rec = {"dtau": dt, "ms_per_step": step, "tau_per_s": dt / (step / 1e3), "create_s": setup_s,
               "J_after": sc["J"], "steps": K, "phases_ms": {k: v["ms"] / v["launches"] for k, v in prof.items()
                                                             if isinstance(v, dict) and v.get("launches")}}
        if scheme == "implicit" and "implicit" in prof:
            # FP32 storage at N_x >= 32: the products on the tensor cores, operands in
            # two BF16 parts, three part products (against the measured bf16 peak)
            M = sl.Ns - 2
            ne, no = (M + 1) // 2, M // 2
            flops = 2 * 2.0 * (ne * ne + no * no) * sl.N
            t = prof["implicit"]["ms"] / prof["implicit"]["launches"]
            peaks, src = read_peaks()
            peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
            rec["products"] = {"ms": t, "algorithmic_flops": flops, "executed_tensor_flops": 3 * flops,
                               "achieved_tflops": flops / (t / 1e3) / 1e12,
                               "executed_tflops": 3 * flops / (t / 1e3) / 1e12, "peak_tflops": peak,
                               "frac": 3 * flops / (t / 1e3) / 1e12 / peak,
                               "bound": "tensor (tcgen05 kind::f16, split BF16)",
                               "peak_source": src + " bf16 sustained (MEASURED_PEAKS.json)",
                               "includes": "the two products, the split sum and the finishing pass"}
        out[scheme] = rec
    out["tau_rate_ratio"] = out["implicit"]["tau_per_s"] / out["imex"]["tau_per_s"]
    return out


def symmetric_context(dev, timed_steps, K):
    """Curves held in the odd subspace (Sec. V.B: real parts of every section's
    coefficients zero) beside the general run: symmetry = 1 keeps full storage
    (the three-launch four-step form then transforms the imaginary columns of two
    modes as one sequence); symmetry = 5 keeps only the sine coefficients (half
    the field bytes, half the columns of every s-contraction).  The L=44,
    N_x=128, N_s=4096 FP32 curve and the L=22, N_x=64, N_s=1024 curve in FP32 and
    FP64."""
    from paper_2301_11704_gb300 import gen
    from paper_2301_11704_gb300.curve import KSCurve
    out = {}
    for wl, prec in (("large", "fp32"), ("diff", "fp32"), ("diff", "fp64")):
        sl = spec_of(wl)
        up, um = gen.end_points(sl)
        amps, vp = gen.perturbation(sl)
        r = {}
        for name, sym in (("general", 0), ("odd_subspace", 1), ("sine_storage", 5)):
            c = KSCurve(sl.L, sl.N, sl.Ns, sl.S, up, um, s0=sl.s0, dtau=sl.dtau, precision=prec, symmetry=sym,
                        device=dev)
            c.init_trial(0.0, None, amps, vp)
            ms, prof = timed_steps(c, K, 3, profile=K)
            r[name] = {"ms_per_step": sum(ms) / K, "s_form": c.s_form, "workspace_bytes": c.workspace_bytes,
                       "phases_ms": {k: v["ms"] / v["launches"] for k, v in prof.items()
                                     if isinstance(v, dict) and v.get("launches")}}
            c.close()
        r["speedup_odd"] = r["general"]["ms_per_step"] / r["odd_subspace"]["ms_per_step"]
        r["speedup_sine"] = r["general"]["ms_per_step"] / r["sine_storage"]["ms_per_step"]
        out["L=%g N_x=%d N_s=%d %s" % (sl.L, sl.N, sl.Ns, prec.upper())] = r
    return out


def torch_sm_count(dev):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


# ---------------------------------------------------------------------------- single curve
def run_curve(args):
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

    spec = spec_of(args.workload)
    precision = args.precision or default_precision(args.workload)
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)

    def make_curve(prec, s_transform=args.s_transform):
        c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, s0=spec.s0, dtau=spec.dtau, precision=prec,
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

    curve = make_curve(precision)
    K, W = args.steps, max(3, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    # per-kernel events on the first 1/20 of the timed steps only (events between
    # kernels serialise them); the other steps run as a user's would
    step_ms, prof = timed_steps(curve, K, W, profile=max(3, K // 20))
    clk = clocks.stop()
    total_ms = sum(step_ms)
    total_ms_max = reduce_max_ms(total_ms, world, dev)
    M, N, b = spec.M, spec.N, BYTES[precision]
    value = job_throughput(world, M, K, total_ms_max)
    ms_step = total_ms_max / K

    # ---- roofline: the dominant kernel, bytes and flops after the per-point counts
    peaks, peak_src = read_peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_fp32 = nsm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    peak_alu = peak_fp32 if b == 4 else 1.25
    hbm_peak = float(peaks["hbm_gbs"])
    fx, fs, fpw = flops_per_point(N, M)
    F = curve.fft_length
    form = curve.s_form
    fused = form == "fft4c" and "dt_store" not in prof
    kernels = {}   # name -> (mean ms per launch, algorithmic bytes, algorithmic flops, traffic kind)
    rows_kind = "rows_tc" if precision.startswith("bf16") else "rows"
    if "rows" in prof:
        kernels["rows"] = (prof["rows"]["ms"] / prof["rows"]["launches"], 4.0 * N * b * spec.Ns,
                           (fx + fpw) * M, rows_kind)
    # the three-launch four-step form chains them: the update's third pass also
    # runs D_t u's first pass on the updated columns it holds, so D_t u itself
    # reads no field (it writes D)
    chained = form == "fft4"
    for key, nb in (("dt_update", 4.0), ("dt_store", 1.0 if chained else 2.0)):
        if key in prof:
            fl = fs / 2 * M * (2 if (key == "dt_update" and fused) else 1)
            by = (nb + (2.0 if (key == "dt_update" and fused) else 0.0)) * N * b * spec.Ns
            kernels[key] = (prof[key]["ms"] / prof[key]["launches"], by, fl, "fft4")
    dom = max(kernels, key=lambda k: kernels[k][0])
    t_dom, by_dom, fl_dom, kind = kernels[dom]
    kernel_names = {"rows": "row phase (k_rows%s)" % ("_tc" if rows_kind == "rows_tc" else ""),
                    "dt_update": "update contraction (%s)" % form, "dt_store": "D_t u contraction (%s)" % form}
    ach = by_dom / (t_dom / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": None, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
            "kernel": kernel_names[dom], "algorithmic_bytes_per_launch": by_dom,
            "ms_per_launch": t_dom,
            "alu": {"achieved": fl_dom / (t_dom / 1e3) / 1e12, "peak": peak_alu, "unit": "TFLOP/s",
                    "frac": fl_dom / (t_dom / 1e3) / 1e12 / peak_alu, "algorithmic_flops_per_launch": fl_dom,
                    "peak_source": ("%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (derived)" % (nsm, mhz))
                    if b == 4 else "nominal FP64 1.25 TFLOP/s"},
            "phase_ms_per_launch": {k: v[0] for k, v in kernels.items()}}
    if "passes" in prof:
        roof["pass_ms_per_launch"] = {k: [p["ms"] / max(p["launches"], 1) for p in v]
                                      for k, v in prof["passes"].items()}
        roof["note"] = ("a contraction of the three-launch four-step form counts as one kernel of three "
                        "launches (passes; the update's third also runs D_t u's first, which D_t u then "
                        "skips); its passes' times are listed")
    traf = None
    if dom == "rows":
        traf = recorded_traffic("rows:%s:N%d:Ns%d:%s" % (rows_kind, N, spec.Ns, precision), rows_kind)
    elif form == "fft4":
        traf = recorded_traffic("%s:fft4:N%d:Ns%d:%s" % (dom, N, spec.Ns, precision), "fft4")
    if traf:
        roof["traffic"] = traf["bytes_per_launch"]
        roof["traffic_source"] = traf
    if precision.startswith("bf16") and "rows" in kernels:
        nprod = 6 if precision == "bf16x3" else 3
        tfl = 4 * 2.0 * N * N * spec.Ns          # four real N x N DFT products per section
        tr = kernels["rows"][0]
        tpeak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        roof["tensor_rows"] = {"achieved": tfl / (tr / 1e3) / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                               "frac": tfl / (tr / 1e3) / 1e12 / tpeak,
                               "algorithmic_flops_per_launch": tfl,
                               "executed_tensor_flops_per_launch": tfl * nprod,
                               "executed_frac": tfl * nprod / (tr / 1e3) / 1e12 / tpeak,
                               "peak_source": peak_src + " bf16 sustained (MEASURED_PEAKS.json)"}
    bytes_step = 2.0 * N * b * M
    flops_step = (fx + fs + fpw) * M
    hbm_step = {"achieved": bytes_step / (ms_step / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": bytes_step / (ms_step / 1e3) / 1e9 / hbm_peak, "algorithmic_bytes_per_step": bytes_step,
                "alu": {"achieved": flops_step / (ms_step / 1e3) / 1e12, "peak": peak_alu, "unit": "TFLOP/s",
                        "frac": flops_step / (ms_step / 1e3) / 1e12 / peak_alu,
                        "algorithmic_flops_per_step": flops_step}}

    # ---- end to end through the public API with host buffers
    e2e = None
    if rank == 0 or world > 1:
        dt = curve.dtype
        host_in = torch.empty((spec.Ns, N), dtype=dt).pin_memory()
        host_in.copy_(curve.get_state().cpu())
        dev_in = [torch.empty((spec.Ns, N), dtype=dt, device=dev) for _ in range(2)]
        n_e2e = max(1, min(args.e2e_steps, K))
        nbytes = spec.Ns * N * b
        # every step: the curve from pinned host memory (set_state), one descent
        # step, and its result J read back to the host (ks_curve_descend copies the
        # device scalar record, 176 bytes, and synchronises).  Two device buffers:
        # the next step's copy runs on a copy stream while this step computes (the
        # buffer it fills was last read by the step before, which has completed).
        cur = torch.cuda.current_stream(dev)
        cps = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]

        def h2d(k):
            with torch.cuda.stream(cps):
                dev_in[k % 2].copy_(host_in, non_blocking=True)
                copied[k % 2].record(cps)

        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h2d(0)
        for k in range(n_e2e):
            cur.wait_event(copied[k % 2])
            if k + 1 < n_e2e:
                h2d(k + 1)
            curve.set_state(dev_in[k % 2], 1.0, 0.0)
            curve.descend(1)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": M * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": 176, "steps": n_e2e,
               "path": "pinned host curve -> set_state -> descend(1), J read back; each step's host-to-device "
                       "copy overlaps the step before (two device buffers, a copy stream)"}
    sc = curve.scalars()
    curve.close()

    ctx = {}
    if rank == 0 and not args.no_context:
        # ---- plain FP64 GPU path at the same workload
        if precision != "fp64":
            c64 = make_curve("fp64")
            k64 = max(3, min(20, K))
            ms64, _ = timed_steps(c64, k64, 3)
            ctx["fp64_gpu_path"] = {"value": M * k64 / (sum(ms64) / 1e3), "unit": UNIT,
                                    "ms_per_step": sum(ms64) / k64, "steps": k64, "s_form": c64.s_form}
            c64.close()
        # ---- the other precisions of this workload
        others = {}
        for prec in ("fp32", "bf16x3", "bf16x2"):
            if prec == precision:
                continue
            try:
                co = make_curve(prec)
            except Exception as exc:   # a precision this build or size does not support
                others[prec] = {"unavailable": str(exc)[:120]}
                continue
            ko = max(3, min(50, K))
            mso, _ = timed_steps(co, ko, 3)
            others[prec] = {"value": M * ko / (sum(mso) / 1e3), "unit": UNIT, "ms_per_step": sum(mso) / ko,
                            "steps": ko}
            co.close()
        ctx["other_precisions"] = others
        # ---- error against the FP64 oracle (stored reference values)
        errs = {}
        for prec in sorted({precision, "fp64", "fp32"} | ({"bf16x2", "bf16x3"} if spec.N >= 128 else set())):
            try:
                errs[prec] = oracle_errors(spec, make_curve, prec)
            except Exception as exc:
                errs[prec] = {"unavailable": str(exc)[:120]}
        ctx["error_vs_oracle"] = errs
        # ---- the differentiation workload (context)
        if args.workload != "diff":
            sd = spec_of("diff")
            upd, umd = gen.end_points(sd)
            ampd, vpd = gen.perturbation(sd)
            cd = KSCurve(sd.L, sd.N, sd.Ns, sd.S, upd, umd, s0=sd.s0, dtau=sd.dtau, precision="fp32", device=dev)
            cd.init_trial(0.0, None, ampd, vpd)
            kd = max(3, min(200, K))
            msd, _ = timed_steps(cd, kd, 3)
            ctx["diff_workload_fp32"] = {"workload": "L=%g N_x=%d N_s=%d FP32" % (sd.L, sd.N, sd.Ns),
                                         "value": sd.M * kd / (sum(msd) / 1e3), "unit": UNIT,
                                         "ms_per_step": sum(msd) / kd, "steps": kd, "s_form": cd.s_form}
            cd.close()
        # ---- full-linear-implicit stepping (Sec. V.C.3) on the single large curve
        try:
            ctx["implicit_scheme"] = implicit_context(dev, timed_steps, max(3, min(50, K)))
        except Exception as exc:
            ctx["implicit_scheme"] = {"unavailable": str(exc)[:160]}
        # ---- the odd subspace (Sec. V.B) on the same curve
        try:
            ctx["symmetric_subspace"] = symmetric_context(dev, timed_steps, max(3, min(50, K)))
        except Exception as exc:
            ctx["symmetric_subspace"] = {"unavailable": str(exc)[:160]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, est, cores = oracle_baseline(spec, 3)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": oracle_sample_text(spec),
               "seconds_per_step_estimates": est}

    if rank == 0:
        launches = {"fft4": 7, "fft4c": 2 if fused else 3}.get(form, 3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32"}.get(precision, precision + "+f32"),
                "data": "synthetic",
                "config": config_of(spec, precision),
                "s_transform": "%s%s" % (form, (", F=%d" % F) if F else ""),
                "roofline": roof, "hbm_step": hbm_step,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * K, "clocks": clk,
                "final_J": sc["J"], "final_J_arc": sc["J_arc"], "step_ms_median": statistics.median(step_ms)}
        line.update(ctx)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_curve(args)


if __name__ == "__main__":
    sys.exit(main())
