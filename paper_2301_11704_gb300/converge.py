"""Runs a batch of workload curves towards convergence and reports, per curve,
the step at which J / |lambda D_t u|_W fell below the tolerance, or where it
stood when the step budget or the time budget ran out:

    python -m paper_2301_11704_gb300.converge --cfg 3 --scheme implicit --dtau 0.5 --budget-s 600

The batch runs in chunks of --chunk steps (each curve stops by itself at its
tolerance, Sec. V.C.3 and the FP32 criterion max(1e-8, 8 eps)); after each chunk
the per-curve scalars are read and one JSON line of progress is printed, and at
the end one JSON line with every curve's record.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cfg", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--scheme", default="implicit", choices=["imex", "implicit"])
    ap.add_argument("--dtau", type=float, default=None, help="default: each curve's own (IMEX) dtau")
    ap.add_argument("--chunk", type=int, default=2000)
    ap.add_argument("--max-steps", type=int, default=1_000_000)
    ap.add_argument("--budget-s", type=float, default=600.0)
    ap.add_argument("--tol", type=float, default=None, help="default: max(1e-8, 8 eps) of the storage type")
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    from . import gen
    from .batch import KSBatch

    specs = gen.workload(args.cfg)
    eps = np.finfo(np.float32 if args.precision == "fp32" else np.float64).eps
    tol = float(args.tol if args.tol is not None else max(1e-8, 8 * eps))
    ins = [(gen.end_points(s), gen.perturbation(s)) for s in specs]
    t0 = time.perf_counter()
    b = KSBatch(specs, [i[0][0] for i in ins], [i[0][1] for i in ins], precision=args.precision, conv="jrel",
                scheme=args.scheme, dtau=args.dtau)
    b.init_trial(np.array([i[1][0] for i in ins]), [i[1][1] for i in ins])
    setup_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    done_at = [None] * len(specs)
    steps = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_ms = 0.0
    while steps < args.max_steps and time.perf_counter() - t0 < args.budget_s:
        n = min(args.chunk, args.max_steps - steps)
        ev0.record()
        b.descend_async(n, tol)
        ev1.record()
        torch.cuda.synchronize()
        gpu_ms += ev0.elapsed_time(ev1)
        steps += n
        sc = b.scalars()
        jr = np.array([x["J"] / max(x["Dnorm"], 1e-300) for x in sc])
        for k, x in enumerate(sc):
            if x["converged"] and done_at[k] is None:
                done_at[k] = int(x["step"])
        bad = sum(1 for x in sc if x["status"] != 0)
        fin = jr[np.isfinite(jr)]
        print(json.dumps({"steps": steps, "wall_s": round(time.perf_counter() - t0, 1), "gpu_s": round(gpu_ms / 1e3, 2),
                          "converged": sum(d is not None for d in done_at), "nonfinite": bad,
                          "J_rel_quantiles_finite": [float(np.quantile(fin, q)) for q in (0, 0.1, 0.25, 0.5, 0.75, 0.9, 1.0)]
                          if fin.size else None}),
              flush=True)
        if all(d is not None or x["status"] != 0 for d, x in zip(done_at, sc)):
            break
    sc = b.scalars()
    b.close()
    recs = [{"curve": k, "L": float(s.L), "N_x": int(s.N), "N_s": int(s.Ns), "converged_at_step": done_at[k],
             "step": int(x["step"]), "tau": float(x["tau"]), "J_rel": float(x["J"] / max(x["Dnorm"], 1e-300)),
             "J_arc": float(x["J_arc"]), "G_norm": float(x["G_norm"]), "status": int(x["status"])}
            for k, (s, x) in enumerate(zip(specs, sc))]
    conv = [r["converged_at_step"] for r in recs if r["converged_at_step"] is not None]
    print(json.dumps({"cfg": args.cfg, "precision": args.precision, "scheme": args.scheme, "dtau": args.dtau,
                      "tol": tol, "setup_s": round(setup_s, 2), "steps_run": steps, "gpu_s": round(gpu_ms / 1e3, 2),
                      "ms_per_step": gpu_ms / max(1, steps), "converged": len(conv),
                      "steps_to_converge_quantiles": [int(np.quantile(conv, q)) for q in (0, 0.5, 1.0)] if conv else None,
                      "nonfinite": [r["curve"] for r in recs if r["status"] != 0],
                      "curves": recs}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
