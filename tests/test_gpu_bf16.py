"""Parity of the split-BF16 tensor-core row phase (precision bf16x3 / bf16x2:
the x-transforms of every section as products with the DFT matrices on the
tensor cores, Sec. V.C.1) with the FP64 oracle, on random smooth curves of
ragged sizes (N_s not a multiple of the 128-section tile, the one-interior-section
curve) and on the workload curves; with the FP32 GPU path beside it at the
largest workload, and against the oracle's stored values there.

Tolerances (relative): BF16X3 splits every operand into three BF16 parts
(about FP32 rounding), so it is held to the FP32 bounds of the other parity
tests; BF16X2 keeps two parts (about 2^-17 per product) and is held to the
bounds measured for it times two (they are printed by every test).
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.curve import KSCurve
from tests.test_gpu_parity import make_pair, oracle_eval, precond_2, rel_2

pytestmark = pytest.mark.gpu

# (J, residual 2-norm, preconditioned gradient 2-norm) bounds
TOL = {"bf16x3": (1e-5, 1e-5, 1e-5), "bf16x2": (2e-4, 2e-4, 2e-4)}


def smooth_curve(N, Ns, L, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((Ns, N))
    x = np.arange(N) * L / N
    for m in range(Ns):
        for j in range(1, min(6, N // 2)):
            X[m] += 0.5 * rng.standard_normal() * np.sin(2 * np.pi * j * x / L + rng.uniform(0, 6.28))
    return X


def report(tag, **errs):
    print("BF16 %s: %s" % (tag, " ".join("%s=%.3e" % kv for kv in errs.items())))


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x2"])
@pytest.mark.parametrize("N,Ns", [(64, 3), (64, 130), (128, 257), (256, 300), (256, 129)])
def test_bf16_evaluation_ragged_shapes(N, Ns, precision):
    L, S = 22.0 + N / 16.0, max(0.5, 0.1 * (Ns - 1))
    X = smooth_curve(N, Ns, L, N * 1000 + Ns).astype(np.float32).astype(np.float64)
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X).float(), precision=precision)
    # the GPU holds the FP64 transform of the FP32 input, rounded per coefficient
    U = oracle.curve_spectral(X)
    spec = gen.CurveSpec(0, 0, L, N, Ns, S)
    R, D, G, sc = oracle_eval(U, spec)
    J2, Ja = c.cost()
    r = c.residual().double().cpu().numpy()
    g, _ = c.gradient()
    e = dict(J=abs(np.sqrt(J2) - np.sqrt(sc["J2"])) / np.sqrt(sc["J2"]), J_arc=abs(Ja - sc["J_arc"]) / sc["J_arc"],
             r=rel_2(r, oracle.curve_physical(R)), g=precond_2(g.double().cpu().numpy(), G, spec))
    report("%s N=%d Ns=%d" % (precision, N, Ns), **e)
    tj, tr, tg = TOL[precision]
    assert e["J"] < tj and e["r"] < tr and e["g"] < tg
    assert e["J_arc"] < 3 * tj
    c.close()


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x2"])
def test_bf16_descent_matches_oracle(precision):
    """Twenty descent steps (dtau = 1e-3) of a ragged N = 128, N_s = 257 curve."""
    N, Ns, L = 128, 257, 30.0
    S = 0.1 * (Ns - 1)
    X = smooth_curve(N, Ns, L, 7).astype(np.float32).astype(np.float64)
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X).float(), dtau=1e-3, precision=precision)
    U = oracle.curve_spectral(X)
    out = c.descend(20)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 20, dtau=1e-3)
    e = dict(u=rel_2(c.get_state().double().cpu().numpy(), oracle.curve_physical(Uo)),
             J=abs(out["J"] - sco["J"]) / sco["J"])
    report("%s descent N=%d Ns=%d" % (precision, N, Ns), **e)
    tj, tr, _ = TOL[precision]
    assert e["J"] < tj and e["u"] < tr
    c.close()


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x2"])
def test_bf16_differentiation_workload(precision):
    """L = 22, N_x = 64, N_s = 1024 trial curve: one evaluation against the oracle."""
    spec = gen.workload(1)[0]
    c, U = make_pair(spec, precision=precision)
    R, D, G, sc = oracle_eval(U, spec)
    J2, Ja = c.cost()
    g, _ = c.gradient()
    e = dict(J=abs(np.sqrt(J2) - np.sqrt(sc["J2"])) / np.sqrt(sc["J2"]), J_arc=abs(Ja - sc["J_arc"]) / sc["J_arc"],
             r=rel_2(c.residual().double().cpu().numpy(), oracle.curve_physical(R)),
             g=precond_2(g.double().cpu().numpy(), G, spec))
    report("%s L=22 N=64 Ns=1024" % precision, **e)
    tj, tr, tg = TOL[precision]
    assert e["J"] < tj and e["r"] < tr and e["g"] < tg
    c.close()


def _golden(spec):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "fullsize_L%g_N%d_Ns%d.json" % (spec.L, spec.N, spec.Ns))
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for this workload")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x2", "fp32", "fp64"])
@pytest.mark.parametrize("cfg", [2, 4])
def test_large_workloads_against_stored_oracle(cfg, precision):
    """L = 44, N_x = 128, N_s = 4096 and L = 100, N_x = 256, N_s = 16384: J^2,
    J_arc, dJ^2/dl, |G|_W, G at sampled sections (trial curve), J and sampled
    sections after ten steps, against the oracle's values
    (tests/golden/make_fullsize_refs.py)."""
    spec = gen.workload(cfg)[0]
    ref = _golden(spec)
    rows = ref["rows"]
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, dtau=spec.dtau, precision=precision)
    c.init_trial(0.0, None, amps, vp)
    J2, Ja = c.cost()
    g, dl = c.gradient()
    sc = c.scalars()
    gs = g.double().cpu().numpy()[rows]
    res = c.descend(ref["after_steps"]["steps"])
    us = c.get_state().double().cpu().numpy()[rows]
    c.close()
    cx = lambda a: np.array(a)[..., 0] + 1j * np.array(a)[..., 1]
    tr, af = ref["trial"], ref["after_steps"]
    ur = np.stack([oracle.inv(v, spec.N) for v in cx(af["U_rows"])])
    e = dict(J2=abs(J2 - tr["J2"]) / tr["J2"], J_arc=abs(Ja - tr["J_arc"]) / tr["J_arc"],
             dJdl=abs(dl - tr["dJ2_dlambda"]) / abs(tr["dJ2_dlambda"]),
             Gnorm=abs(sc["G_norm"] - np.sqrt(tr["G2"])) / np.sqrt(tr["G2"]),
             g=precond_2(gs, cx(tr["G_rows"]), spec),
             J10=abs(res["J"] - af["J"]) / af["J"], Jarc10=abs(res["J_arc"] - af["J_arc"]) / af["J_arc"],
             u10=rel_2(us, ur))
    report("%s L=%g N=%d Ns=%d vs stored oracle" % (precision, spec.L, spec.N, spec.Ns), **e)
    if precision == "fp64":
        assert max(e["J2"], e["J_arc"], e["dJdl"], e["Gnorm"], e["J10"], e["Jarc10"]) < 1e-10
        assert e["g"] < 1e-10 and e["u10"] < 1e-10
        return
    # the raw |G|_W carries a_j^2 u^_j (a_j ~ k^4): FP32 rounding of the top modes,
    # amplified by k^8, dominates it, so it is reported only; the direction the
    # descent applies (preconditioned, `g`) is held to the bound
    tj = {"bf16x3": 1e-5, "fp32": 1e-5, "bf16x2": 2e-4}[precision]
    assert e["J2"] < 2 * tj and e["J10"] < 2 * tj and e["u10"] < tj
    assert e["J_arc"] < 4 * tj and e["Jarc10"] < 4 * tj
    assert e["g"] < 10 * tj and e["dJdl"] < 10 * tj
