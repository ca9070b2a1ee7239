"""Runs descent steps of one synthetic workload curve and prints their device
time, for timing and profiling a configuration in isolation:

    python -m paper_2301_11704_gb300.steps --cfg 4 --steps 5 --precision fp32 --s-transform auto

Workloads (gen.workload): 0 L=22 N_x=32 N_s=128; 1 L=22 N_x=64 N_s=1024;
2 L=44 N_x=128 N_s=4096; 4 L=100 N_x=256 N_s=16384 (the first curve of each).
"""
from __future__ import annotations

import argparse
import json
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cfg", type=int, default=1, choices=[0, 1, 2, 4])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16x2", "bf16x3"])
    ap.add_argument("--s-transform", default="auto", choices=["auto", "dense", "fft", "dense_tc", "fft4", "fft4c"])
    ap.add_argument("--phases", action="store_true",
                    help="after the timed steps, time the phases of --steps more steps (rows, the two contractions)")
    args = ap.parse_args(argv)

    import torch
    from . import gen
    from .curve import KSCurve
    sp = gen.workload(args.cfg)[0]
    up, um = gen.end_points(sp)
    amps, vp = gen.perturbation(sp)
    c = KSCurve(sp.L, sp.N, sp.Ns, sp.S, up, um, s0=sp.s0, dtau=sp.dtau, precision=args.precision,
                s_transform=args.s_transform)
    c.init_trial(0.0, None, amps, vp)
    c.descend_async(args.warmup)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c.descend_async(1)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    phases = None
    if args.phases:
        c.profile(args.steps)
        c.descend_async(args.steps)
        torch.cuda.synchronize()
        phases = {k: v["ms"] / max(1, v["launches"]) for k, v in c.profile_read().items() if "launches" in v}
        c.profile(0)
    sc = c.scalars()
    c.close()
    out = {"L": sp.L, "N_x": sp.N, "N_s": sp.Ns, "precision": args.precision,
           "fft_length": c.fft_length, "ms_per_step": ms, "J": sc["J"]}
    if phases is not None:
        out["ms_per_phase_launch"] = phases
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
