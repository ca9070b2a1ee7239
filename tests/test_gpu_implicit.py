"""Parity of the full-linear-implicit stepping (scheme "implicit", Sec. V.C.3)
with the oracle's dense per-mode LU solve, through the C ABI.

The GPU applies the step through the eigenbases of the even and odd parts of
the interior D_t^2 (set up once in FP64); the oracle solves
(I (1 + dtau a_j^2) - dtau lambda^2 D~^2) delta = dtau G per mode by Gaussian
elimination.  FP64: states and J within 1e-10 relative after several steps at a
dtau far beyond the IMEX stability limit; FP32 storage: 1e-5.  Ragged sizes
cover odd and even M (the unpaired middle section of the even part).
"""
import numpy as np
import pytest

import oracle
from paper_2301_11704_gb300.curve import KSCurve

pytestmark = pytest.mark.gpu


def trial(N, Ns, L, seed, npert=3, amp=0.2):
    rng = np.random.default_rng(seed)
    x = np.arange(N) * L / N
    up = sum(0.6 * rng.standard_normal() * np.sin(2 * np.pi * q * x / L + rng.uniform(0, 6.3)) for q in (1, 2, 3))
    um = np.zeros(N)
    vp = np.stack([np.cos(2 * np.pi * (q + 1) * x / L + rng.uniform(0, 6.3)) for q in range(npert)])
    return up, um, np.full(npert, amp), vp


def pair(N, Ns, L, seed, dtau, precision="fp64", **kw):
    S = 0.1 * (Ns - 1)
    up, um, amps, vp = trial(N, Ns, L, seed)
    c = KSCurve(L, N, Ns, S, up, um, dtau=dtau, precision=precision, scheme="implicit", **kw)
    c.init_trial(0.0, None, amps, vp)
    U = oracle.curve_init(Ns - 2, S, up, um, amps=amps, vp=vp)
    return c, U, S


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def imex_limit(Ns):
    M = Ns - 2
    S = 0.1 * (M + 1)
    D = oracle.dt_matrix(M, S)[1:-1, 1:-1]
    return 2.0 / np.abs(np.linalg.eigvals(D @ D)).max()


@pytest.mark.parametrize("N,Ns,s_transform", [(16, 65, "auto"), (16, 66, "dense"), (32, 130, "fft"),
                                              (32, 301, "auto"), (64, 700, "fft4")])
def test_fp64_implicit_matches_oracle(N, Ns, s_transform):
    L = 22.0 + N / 8
    dtau = 20 * imex_limit(Ns)          # twenty times the IMEX limit
    c, U, S = pair(N, Ns, L, N + Ns, dtau, s_transform=s_transform)
    steps = 6
    Uo, so, sco, _ = oracle.curve_descend(U, L, S, steps, dtau=dtau, scheme=oracle.IMPLICIT)
    out = c.descend(steps)
    X = c.get_state().double().cpu().numpy()
    e_u = rel_max(X, oracle.curve_physical(Uo))
    e_j = abs(out["J"] - sco["J"]) / sco["J"]
    print("IMPLICIT fp64 N=%d Ns=%d %s dtau=%.3g: u %.2e J %.2e" % (N, Ns, s_transform, dtau, e_u, e_j))
    assert out["steps"] == so == steps
    assert e_u < 1e-10 and e_j < 1e-10
    c.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_fp32_implicit_matches_oracle(precision):
    N, Ns, L = 64, 257, 30.0
    dtau = 20 * imex_limit(Ns)
    c, U, S = pair(N, Ns, L, 11, dtau, precision=precision)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 6, dtau=dtau, scheme=oracle.IMPLICIT)
    out = c.descend(6)
    X = c.get_state().double().cpu().numpy()
    Xo = oracle.curve_physical(Uo)
    e_u = float(np.linalg.norm(X - Xo) / np.linalg.norm(Xo))
    e_j = abs(out["J"] - sco["J"]) / sco["J"]
    print("IMPLICIT %s: u %.2e J %.2e" % (precision, e_u, e_j))
    assert e_u < 1e-5 and e_j < 1e-5
    c.close()


def test_implicit_discrete_adjoint_and_free_lambda():
    N, Ns, L = 32, 129, 24.0
    dtau = 10 * imex_limit(Ns)
    c, U, S = pair(N, Ns, L, 5, dtau, adjoint="discrete", lambda_free=True, dtau_lambda=0.05)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 8, dtau=dtau, mode=oracle.DISCRETE, lambda_free=True,
                                        dtau_lambda=0.05, scheme=oracle.IMPLICIT)
    out = c.descend(8)
    X = c.get_state().double().cpu().numpy()
    assert rel_max(X, oracle.curve_physical(Uo)) < 1e-10
    assert abs(out["J"] - sco["J"]) < 1e-10 * sco["J"]
    lam, _ = c.get_lambda_tau()
    assert abs(lam - sco["lam"]) < 1e-12 and abs(lam - 1.0) > 1e-6
    c.close()


def test_implicit_stops_at_tolerance():
    N, Ns, L = 16, 97, 22.0
    dtau = 10 * imex_limit(Ns)
    c, U, S = pair(N, Ns, L, 2, dtau)
    _, _, _, hist = oracle.curve_descend(U, L, S, 40, dtau=dtau, scheme=oracle.IMPLICIT, history=True)
    tol = 0.5 * (hist[25, 3] + hist[26, 3])
    _, so, sco, _ = oracle.curve_descend(U, L, S, 500, dtau=dtau, tol=tol, scheme=oracle.IMPLICIT)
    out = c.descend(500, tol=tol)
    assert so == 26 and out["steps"] == 26
    assert abs(out["J_arc"] - sco["J_arc"]) < 1e-10 * sco["J_arc"]
    c.close()


def test_implicit_descent_is_stable_far_beyond_imex_limit():
    """200 graph-replayed steps at twenty times the IMEX limit (discrete adjoint,
    the exact gradient): J falls and matches the oracle's implicit descent.  (The
    nonlinear terms stay explicit, so dtau is still bounded: at fifty times the
    limit this curve diverges in the oracle and on the GPU alike.)"""
    N, Ns, L = 32, 200, 26.0
    dtau = 20 * imex_limit(Ns)
    c, U, S = pair(N, Ns, L, 8, dtau, adjoint="discrete")
    J = [c.descend(0)["J"]]
    for _ in range(20):
        J.append(c.descend(10)["J"])
    J = np.array(J)
    print("IMPLICIT J:", J[[0, 5, 10, 20]])
    assert np.all(np.isfinite(J)) and J[-1] < 0.5 * J[0]
    _, _, sco, _ = oracle.curve_descend(U, L, S, 200, dtau=dtau, mode=oracle.DISCRETE, scheme=oracle.IMPLICIT)
    assert abs(J[-1] - sco["J"]) < 1e-9 * sco["J"]
    c.close()


def test_implicit_full_size_fp32_tensor_cores_match_fp64():
    """The L = 44, N_x = 128, N_s = 4096 workload curve as the bench times it
    (FP32 storage: the increment's products on the tensor cores, K split over
    CTAs) against the FP64 implicit path on the CUDA cores (itself held to the
    oracle at 1e-13 above), five steps at dtau = 0.5."""
    from paper_2301_11704_gb300 import gen
    sp = gen.workload(2)[0]
    up, um = gen.end_points(sp)
    amps, vp = gen.perturbation(sp)
    out = {}
    for prec in ("fp32", "fp64"):
        c = KSCurve(sp.L, sp.N, sp.Ns, sp.S, up, um, dtau=0.5, precision=prec, scheme="implicit")
        c.init_trial(0.0, None, amps, vp)
        r = c.descend(5)
        out[prec] = (c.get_state().double().cpu().numpy(), r["J"])
        c.close()
    (x32, j32), (x64, j64) = out["fp32"], out["fp64"]
    e_u = float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64))
    e_j = abs(j32 - j64) / j64
    print("IMPLICIT full size fp32 vs fp64: u %.2e J %.2e" % (e_u, e_j))
    assert e_u < 1e-5 and e_j < 1e-5
