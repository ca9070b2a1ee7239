"""Shared test helpers: end points and trial curves of the synthetic workloads,
built from the seeded generator and the stored (oracle-computed) equilibria."""
import json
import os

import numpy as np

from paper_2301_11704_gb300 import gen

_EQ = None


def equilibria():
    global _EQ
    if _EQ is None:
        path = os.path.join(os.path.dirname(gen.__file__), "data", "equilibria.json")
        with open(path) as f:
            _EQ = {(e["cfg"], e["index"]): e for e in json.load(f)["entries"]}
    return _EQ


def end_points(spec):
    """(u_plus, u_minus) physical sections for a workload curve: u_+ is the stored
    Newton equilibrium (odd sine series), u_- = 0."""
    e = equilibria()[(spec.cfg, spec.index)]
    assert e["N"] == spec.N and abs(e["L"] - spec.L) < 1e-12
    x = gen.grid_x(spec.N, spec.L)
    b = np.array(e["b"])
    up = np.zeros(spec.N)
    for j, c in enumerate(b):
        up += c * np.sin(2 * np.pi * (j + 1) * x / spec.L)
    return up, np.zeros(spec.N)


def perturbation(spec):
    """(amps, fields[npert, N]) of the trial-curve perturbation."""
    v = gen.perturbation_fields(spec.N, spec.L, spec.seed(), spec.npert)
    return np.full(spec.npert, spec.amp), v


def random_smooth_curve(rng, M, N, decay=0.5, ends=True):
    """Random spectral curve [M+2, N/2] with decaying modes; zero end rows if ends=False."""
    U = (rng.standard_normal((M + 2, N // 2)) + 1j * rng.standard_normal((M + 2, N // 2)))
    U *= decay ** np.arange(N // 2)[None, :]
    th = np.arange(M + 2) * np.pi / (M + 1)
    U *= (0.3 + np.sin(th))[:, None]
    U[:, 0] = U[:, 0].real
    if not ends:
        U[0] = 0
        U[-1] = 0
    return U
