"""Writes the end-point equilibria of the synthetic workloads.

Each nonzero end point u_+ is a Newton-converged equilibrium of the discretised
KSE (f(u_+) = 0), computed by the oracle's own Newton solver inside the
inversion-symmetric (odd) subspace from the seeded 4-mode guess of
``paper_2301_11704_gb300.gen.newton_guess`` (amplitude 1, raised to 2 and 3
after ten failed seeds each).  A start that collapses onto u = 0
(max |u| < 0.1) or fails to converge moves to the next seed block.

The result is stored as input data for the CUDA path, the tests and the
benchmark (which never call the oracle themselves):

    python oracle/make_equilibria.py  ->  paper_2301_11704_gb300/data/equilibria.json
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_2301_11704_gb300 import gen  # noqa: E402

OUT = os.path.join(_ROOT, "paper_2301_11704_gb300", "data", "equilibria.json")


def tolerance(N: int, L: float) -> float:
    """Newton stopping level on the sine coefficients of f: 1e-12 times the
    largest linear symbol k^4 on the grid (rounding floor of f)."""
    kmax = 2 * np.pi * (N // 2 - 1) / L
    return 1e-12 * max(1.0, kmax ** 4)


def solve(spec: gen.CurveSpec, max_attempts: int = 30):
    tol = tolerance(spec.N, spec.L)
    for attempt in range(max_attempts):
        seed = spec.seed(attempt)
        b0 = gen.newton_guess(spec.N, spec.L, seed, amplitude=gen.guess_amplitude(attempt))
        b, it, res = oracle.newton_odd(b0, spec.N, spec.L, maxit=200, tol=tol)
        if it < 0 or not np.isfinite(res) or res >= tol:
            continue
        u = oracle.inv(oracle.odd_to_spec(b, spec.N), spec.N)
        if np.abs(u).max() < 0.1:
            continue
        return dict(cfg=spec.cfg, index=spec.index, L=spec.L, N=spec.N, seed=seed, attempt=attempt,
                    newton_iters=it, residual=res, tol=tol, amplitude=gen.guess_amplitude(attempt), b=[float(x) for x in b])
    raise RuntimeError("no equilibrium for cfg %d curve %d" % (spec.cfg, spec.index))


def main():
    entries = []
    for cfg in range(5):
        for spec in gen.workload(cfg):
            e = solve(spec)
            entries.append(e)
            print("cfg %d curve %3d L=%.3f N=%3d seed=%d iters=%d res=%.2e" %
                  (cfg, spec.index, spec.L, spec.N, e["seed"], e["newton_iters"], e["residual"]))
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(dict(source="oracle/make_equilibria.py (oracle Newton solve, odd subspace)",
                       entries=entries), f, indent=0)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
