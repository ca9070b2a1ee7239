"""Writes the FP64 oracle's reference values for the two largest single-curve
workloads (L = 44, N_x = 128, N_s = 4096 and L = 100, N_x = 256, N_s = 16384) to
tests/golden/fullsize_<workload>.json.  Calls only the oracle (and the seeded
input generator); the GPU tests and the bench compare against these values
instead of re-running minutes of CPU work.

For the trial curve of each workload (eq. KSE_initial_curve plus the seeded
perturbation): J^2, J_arc, dJ^2/dlambda, |lambda D_t u|_W and |G|_W^2 of the
published adjoint (eq. KSE_G), with the residual and G at sampled sections;
after ten descent steps (Sec. V.C.3, dtau of the workload): J, J_arc, the
sampled sections of the state and norms of the whole state.

    python tests/golden/make_fullsize_refs.py [cfg ...]     (cfg = 2, 4)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_11704_gb300 import gen  # noqa: E402

STEPS = 10


def sample_rows(Ns):
    rows = sorted(set([1, 2, Ns // 7, Ns // 2 - 1, Ns // 2, (3 * Ns) // 4, Ns - 3, Ns - 2] +
                      [int(x) for x in np.linspace(1, Ns - 2, 16)]))
    return rows


def cplx_list(a):
    return [[float(v.real), float(v.imag)] for v in np.asarray(a).ravel()]


def make(cfg):
    spec = gen.workload(cfg)[0]
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    t0 = time.time()
    U0 = oracle.curve_init(spec.M, spec.S, up, um, amps=amps, vp=vp)
    R, D = oracle.curve_residual(U0, spec.L, spec.S)
    G, _ = oracle.curve_adjoint(U0, R, spec.L, spec.S, mode=oracle.PAPER)
    sc = oracle.curve_scalars(R, D, spec.L, spec.S, G=G)
    rows = sample_rows(spec.Ns)
    U10, steps, sc10, _ = oracle.curve_descend(U0, spec.L, spec.S, STEPS, dtau=spec.dtau)
    assert steps == STEPS
    out = {
        "workload": "L=%g N_x=%d N_s=%d S=%g dtau=%g" % (spec.L, spec.N, spec.Ns, spec.S, spec.dtau),
        "cfg": cfg, "L": spec.L, "N": spec.N, "Ns": spec.Ns, "S": spec.S, "dtau": spec.dtau,
        "rows": rows,
        "trial": {"J2": sc["J2"], "J_arc": sc["J_arc"], "dJ2_dlambda": sc["dJ2_dlambda"], "Dnorm": sc["Dnorm"],
                  "G2": sc["G2"],
                  "R_rows": [cplx_list(R[m]) for m in rows], "G_rows": [cplx_list(G[m]) for m in rows]},
        "after_steps": {"steps": STEPS, "J": sc10["J"], "J_arc": sc10["J_arc"],
                        "U_rows": [cplx_list(U10[m]) for m in rows],
                        "U_norm": float(np.linalg.norm(U10)), "dU_norm": float(np.linalg.norm(U10 - U0))},
        "oracle_seconds": time.time() - t0, "oracle_threads": oracle.num_threads(),
    }
    path = os.path.join(HERE, "fullsize_L%g_N%d_Ns%d.json" % (spec.L, spec.N, spec.Ns))
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, "%.0f s" % out["oracle_seconds"])


if __name__ == "__main__":
    for c in (sys.argv[1:] or ["2", "4"]):
        make(int(c))
