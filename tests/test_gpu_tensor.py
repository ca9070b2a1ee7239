"""The dense s-contraction on the tensor cores (FP32 storage: each operand split
exactly into three TF32 parts, six products, FP32 accumulation in tensor memory)
against the FP64 oracle and against the same contraction on the FP32 SIMT
pipes, on the same FP32 inputs, for every supported N_x, ragged N_s (not a
multiple of the 128-section tile or of the 32-section stage) and curves with and
without the cluster split of the section range."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.curve import KSCurve
from tests.test_gpu_parity import precond_2, rel_2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _curve(N, Ns, L, seed):
    """Random smooth curve in FP32 (the stored values are the inputs of both sides)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((Ns, N))
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    for j in range(1, min(6, N // 2)):
        a, b = rng.standard_normal(2)
        X += (0.6 ** j) * (a * np.cos(2 * np.pi * j * x / L) + b * np.sin(2 * np.pi * j * x / L))[None, :] * \
            (0.5 + np.sin(th * (1 + j % 3)))[:, None]
    return X.astype(np.float32).astype(np.float64)


SHAPES = [(8, 3), (16, 37), (32, 129), (64, 200), (64, 1024), (128, 300), (256, 70), (64, 1537)]


@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
@pytest.mark.parametrize("N,Ns", SHAPES)
def test_tensor_core_contraction_matches_oracle_and_simt(N, Ns, adjoint):
    L, S = 22.0 + N / 16.0, max(0.5, 0.1 * (Ns - 1))
    X = _curve(N, Ns, L, 17 * N + Ns)
    xt = torch.from_numpy(X).float()
    tc = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision="fp32", adjoint=adjoint, s_transform="dense_tc")
    simt = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision="fp32", adjoint=adjoint, s_transform="dense")
    assert tc.fft_length == 0 and simt.fft_length == 0
    U = oracle.curve_spectral(X)
    spec = gen.CurveSpec(0, 0, L, N, Ns, S)
    R, D = oracle.curve_residual(U, L, S, 1.0)
    G, _ = oracle.curve_adjoint(U, R, L, S, 1.0, mode=oracle.DISCRETE if adjoint == "discrete" else oracle.PAPER)
    ref = oracle.curve_physical(R)
    r_tc, r_simt = tc.residual().double().cpu().numpy(), simt.residual().double().cpu().numpy()
    assert rel_2(r_tc, ref) < TOL32
    assert rel_2(r_simt, ref) < TOL32
    assert rel_2(r_tc, r_simt) < 2e-6
    J_tc, J_simt = tc.cost(), simt.cost()
    sc = oracle.curve_scalars(R, D, L, S, 1.0)
    assert abs(np.sqrt(J_tc[0]) - np.sqrt(sc["J2"])) < TOL32 * np.sqrt(sc["J2"])
    assert abs(J_tc[1] - J_simt[1]) <= 2e-6 * J_simt[1]
    # the FP32 gradient's floor grows with k_max^5 (the FP32 rounding of the
    # pseudo-spectral products, amplified by the adjoint's linear part): the
    # tensor-core form must stay at the FP32 SIMT form's level
    g_tc, _ = tc.gradient()
    g_simt, _ = simt.gradient()
    e_tc = precond_2(g_tc.double().cpu().numpy(), G, spec)
    e_simt = precond_2(g_simt.double().cpu().numpy(), G, spec)
    assert e_tc < max(TOL32, 2.5 * e_simt), (e_tc, e_simt)
    tc.close()
    simt.close()


@pytest.mark.parametrize("N,Ns", [(32, 129), (64, 1024), (128, 300)])
def test_tensor_core_descent_tracks_simt(N, Ns):
    """30 descent steps: the two FP32 forms of the contraction stay within FP32
    rounding of each other, and of the FP64 oracle's descent."""
    L, S = 22.0, 0.1 * (Ns - 1)
    X = _curve(N, Ns, L, 5 * N + Ns)
    xt = torch.from_numpy(X).float()
    out = []
    for form in ("dense_tc", "dense"):
        c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision="fp32", dtau=1e-3, s_transform=form)
        r = c.descend(30)
        out.append((c.get_state().double().cpu().numpy(), r))
        c.close()
    (xa, ra), (xb, rb) = out
    assert ra["steps"] == rb["steps"] == 30
    assert rel_2(xa, xb) < 2e-6
    assert abs(ra["J"] - rb["J"]) < 1e-5 * rb["J"]
    Uo, _, sco, _ = oracle.curve_descend(oracle.curve_spectral(X), L, S, 30, dtau=1e-3)
    assert rel_2(xa, oracle.curve_physical(Uo)) < TOL32
    assert abs(ra["J"] - sco["J"]) < TOL32 * sco["J"]
