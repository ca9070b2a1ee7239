"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method itself: it only draws random
numbers and turns them into the raw ingredients of a workload (domain sizes,
Newton starting guesses for the end-point equilibria, and the smooth spatial
fields of the trial-curve perturbation).  Everything the method computes from
them (the curve, the residual, the gradient, the equilibria themselves) is
computed separately by the CUDA path and by the oracle.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to uniform doubles with
the top 53 bits and to normals with the Box-Muller transform.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import List, Optional

import numpy as np

SEED_BASE = 230111704
_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state advances by the golden-ratio increment; output is the
    published two-multiply finaliser of the state."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair; the other is discarded)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by the 53-bit uniform."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def seed_for(cfg: int, curve: int = 0, attempt: int = 0) -> int:
    """Seed of curve `curve` in workload `cfg`; `attempt` moves to the next
    seed block when a Newton start collapses onto u = 0."""
    return SEED_BASE + cfg * 1000 + curve + 100000 * attempt


def grid_x(N: int, L: float) -> np.ndarray:
    return np.arange(N) * (L / N)


def _sine_series(coef: np.ndarray, N: int, L: float) -> np.ndarray:
    x = grid_x(N, L)
    return sum(c * np.sin(2 * np.pi * (j + 1) * x / L) for j, c in enumerate(coef))


def newton_guess(N: int, L: float, seed: int, nmodes: int = 4, amplitude: float = 1.0) -> np.ndarray:
    """Starting guess for the end-point equilibrium: sine coefficients
    b_1..b_nmodes ~ N(0,1), scaled so that max_x |u| = amplitude (1 by default);
    returned as the N/2-1 sine coefficients b_j of u = sum_j b_j sin(k_j x)."""
    rng = SplitMix64(seed)
    b = np.array([rng.normal() for _ in range(nmodes)])
    amp = np.abs(_sine_series(b, N, L)).max()
    out = np.zeros(N // 2 - 1)
    out[:nmodes] = b * (amplitude / amp)
    return out


def guess_amplitude(attempt: int) -> float:
    """Amplitude of the Newton start for a given attempt: 1 for the first ten
    seeds, then 2, then 3 (a start of amplitude 1 often falls onto u = 0 on
    larger domains)."""
    return 1.0 + float(attempt // 10)


def perturbation_fields(N: int, L: float, seed: int, npert: int, nmodes: int = 4) -> np.ndarray:
    """Smooth spatial fields v_p(x_n), p = 1..npert: spatial modes j = 1..nmodes
    with N(0,1) cosine and sine coefficients, each normalised to max |v_p| = 1.
    Returns [npert, N]."""
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    x = grid_x(N, L)
    out = np.zeros((npert, N))
    for p in range(npert):
        v = np.zeros(N)
        for j in range(1, nmodes + 1):
            a, b = rng.normal(), rng.normal()
            v += a * np.cos(2 * np.pi * j * x / L) + b * np.sin(2 * np.pi * j * x / L)
        out[p] = v / np.abs(v).max()
    return out


@dataclasses.dataclass
class CurveSpec:
    """One synthetic curve: domain, resolution, mapping and descent settings."""
    cfg: int
    index: int
    L: float
    N: int            # Fourier modes = grid points per section (N_x)
    Ns: int           # sections including both ends (N_s = M + 2)
    S: float
    s0: float = 0.0
    dtau: float = 0.01
    npert: int = 4
    amp: float = 0.1
    steps: int = 0

    @property
    def M(self) -> int:
        return self.Ns - 2

    def seed(self, attempt: int = 0) -> int:
        return seed_for(self.cfg, self.index, attempt)


def mapping_scale(Ns: int) -> float:
    """S = 0.1 (M + 1): the ratio of the paper's E1 -> E2 run (M = 550, S = 55)."""
    return round(0.1 * (Ns - 1), 10)


def workload(cfg: int) -> List[CurveSpec]:
    """The five workloads:
    0 plain FP64          L=22, N=32,  Ns=128,   4 s-modes, amplitude 0.1, 2000 steps
    1 differentiation     L=22, N=64,  Ns=1024,  4 s-modes, amplitude 0.1
    2 single large curve  L=44, N=128, Ns=4096,  8 s-modes, amplitude 0.2, 10^4 steps
    3 batch of 256        L~U[20,60], N in {32,64,128}, Ns~U[256,2048]
    4 mixed precision     L=100, N=256, Ns=16384, 8 s-modes, amplitude 0.2, 10^4 steps
    """
    if cfg == 0:
        return [CurveSpec(0, 0, 22.0, 32, 128, mapping_scale(128), steps=2000)]
    if cfg == 1:
        return [CurveSpec(1, 0, 22.0, 64, 1024, mapping_scale(1024), steps=1)]
    if cfg == 2:
        return [CurveSpec(2, 0, 44.0, 128, 4096, mapping_scale(4096), npert=8, amp=0.2, steps=10000)]
    if cfg == 3:
        rng = SplitMix64(seed_for(3, 999))
        out = []
        for i in range(256):
            L = 20.0 + 40.0 * rng.uniform()
            N = (32, 64, 128)[rng.integer(0, 2)]
            Ns = rng.integer(256, 2048)
            out.append(CurveSpec(3, i, round(L, 6), N, Ns, mapping_scale(Ns), steps=0))
        return out
    if cfg == 4:
        return [CurveSpec(4, 0, 100.0, 256, 16384, mapping_scale(16384), npert=8, amp=0.2, steps=10000)]
    raise ValueError("unknown workload %d" % cfg)


def small_spec(L=22.0, N=8, Ns=16, S: Optional[float] = None, cfg=9, index=0) -> CurveSpec:
    """Tiny curve for brute-force checks (finite differences)."""
    return CurveSpec(cfg, index, L, N, Ns, S if S is not None else mapping_scale(Ns))


_EQ = None


def stored_equilibria() -> dict:
    """The stored end-point equilibria, keyed by (cfg, index).  They were computed
    once by the oracle's Newton solver (oracle/make_equilibria.py) and are read
    here as plain input data."""
    global _EQ
    if _EQ is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "equilibria.json")
        with open(path) as f:
            _EQ = {(e["cfg"], e["index"]): e for e in json.load(f)["entries"]}
    return _EQ


def end_points(spec: CurveSpec):
    """(u_plus, u_minus) physical sections of a workload curve: u_+ from the
    stored sine coefficients, u_- = 0."""
    e = stored_equilibria()[(spec.cfg, spec.index)]
    if e["N"] != spec.N or abs(e["L"] - spec.L) > 1e-12:
        raise ValueError("stored equilibrium does not match the workload")
    return _sine_series(np.array(e["b"]), spec.N, spec.L), np.zeros(spec.N)


def perturbation(spec: CurveSpec):
    """(amps, fields[npert, N]) of the trial-curve perturbation of a workload curve."""
    v = perturbation_fields(spec.N, spec.L, spec.seed(), spec.npert)
    return np.full(spec.npert, spec.amp), v


def stored_equilibria_paper() -> dict:
    """E1, E2, E3 at L = 22, N = 64 (stored Newton solutions), keyed by name."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "equilibria.json")
    with open(path) as f:
        return json.load(f)["paper"]
