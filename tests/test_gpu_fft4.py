"""The four-step FFT form of the s-contraction (transforms longer than one CTA
holds: F = F1 F2 with warp-level line transforms and a scratch pass in between;
the three-launch form on the Toeplitz and Hankel parts of D_t with F >= 2P + 1,
the clustered one on the extended sequence with F >= 3P)
against the FP64 oracle and against the dense contraction on the same inputs:
every pair (F1, F2) the library uses, both adjoints, the descent, ragged N_s and
the symmetric subspace.

Tolerances: FP64 1e-10 relative; FP32 5e-6 (2-norm) on fields and 1e-5 on J
between the two FP32 forms (each within FP32 rounding of the exact result, about
2e-6 apart at these sizes).  J_arc, a variance of |D_t u| over the sections,
amplifies the FP32 rounding of D_t u about tenfold; the rounding of a length-F
FFT convolution grows with log2 F and the size of the cot kernel (up to 2P/pi),
so J_arc of the FP32 FFT form is held to 2e-5 relative: twice the worst
measured, 8.8e-6 (the clustered form at F = 65536 against the dense form; 8.5e-6
against the FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.curve import KSCurve
from tests.test_gpu_parity import assert_grad_close, rel_2, rel_max

pytestmark = pytest.mark.gpu


def _curve(N, Ns, L, seed, fp32=False):
    rng = np.random.default_rng(seed)
    X = np.zeros((Ns, N))
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    for j in range(1, min(6, N // 2)):
        a, b = rng.standard_normal(2)
        X += (0.6 ** j) * (a * np.cos(2 * np.pi * j * x / L) + b * np.sin(2 * np.pi * j * x / L))[None, :] * \
            (0.5 + np.sin(th * (1 + j % 3)))[:, None]
    return X.astype(np.float32).astype(np.float64) if fp32 else X


@pytest.mark.parametrize("form", ["fft", "fft4c"])
@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
def test_four_step_fp64_matches_oracle(adjoint, form):
    """N_s = 1500 in FP64 (above the single-CTA FP64 limit): the three-launch form
    on the Toeplitz and Hankel parts (F = 4096 = 64 x 64 >= 2P + 1) and the
    clustered one-launch form on the extended sequence (F = 8192 = 128 x 64 >= 3P)."""
    N, Ns, L = 32, 1500, 22.0
    S = 0.1 * (Ns - 1)
    X = _curve(N, Ns, L, 11)
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X), adjoint=adjoint, s_transform=form)
    assert c.fft_length == (4096 if form == "fft" else 8192)
    U = oracle.curve_spectral(X)
    spec = gen.CurveSpec(0, 0, L, N, Ns, S)
    mode = oracle.DISCRETE if adjoint == "discrete" else oracle.PAPER
    R, D = oracle.curve_residual(U, L, S, 1.0)
    G, _ = oracle.curve_adjoint(U, R, L, S, 1.0, mode=mode)
    sc = oracle.curve_scalars(R, D, L, S, 1.0)
    assert rel_max(c.residual().cpu().numpy(), oracle.curve_physical(R)) < 1e-10
    J2, Ja = c.cost()
    assert abs(J2 - sc["J2"]) < 1e-10 * sc["J2"] and abs(Ja - sc["J_arc"]) < 1e-10 * sc["J_arc"]
    g, _ = c.gradient()
    assert_grad_close(g.cpu().numpy(), G, U, spec, 1e-10)
    c.close()
    c2 = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X), adjoint=adjoint, dtau=1e-3, s_transform=form)
    out = c2.descend(20)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 20, dtau=1e-3, mode=mode)
    assert rel_max(c2.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < 1e-10
    assert abs(out["J"] - sco["J"]) < 1e-10 * sco["J"]
    c2.close()


@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
def test_fused_step_fp64_matches_oracle(adjoint):
    """N_x = 16, N_s = 1000 in FP64 (F = 4096): the clustered form, whose descent
    steps apply the update and D_t u of the updated state in one launch."""
    N, Ns, L = 16, 1000, 22.0
    S = 0.1 * (Ns - 1)
    X = _curve(N, Ns, L, 7)
    U = oracle.curve_spectral(X)
    mode = oracle.DISCRETE if adjoint == "discrete" else oracle.PAPER
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X), adjoint=adjoint, dtau=1e-3, s_transform="auto")
    assert c.s_form == "fft4c" and c.fft_length == 4096
    out = c.descend(20)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 20, dtau=1e-3, mode=mode)
    assert out["steps"] == 20
    assert rel_max(c.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < 1e-10
    assert abs(out["J"] - sco["J"]) < 1e-10 * sco["J"]
    R, D = oracle.curve_residual(Uo, L, S, 1.0)
    assert rel_max(c.residual().cpu().numpy(), oracle.curve_physical(R)) < 1e-10
    c.close()


@pytest.mark.parametrize("precision,N,Ns,F,form", [
    # the three-launch form (Toeplitz and Hankel parts, F >= 2P + 1): every (F1, F2)
    ("fp32", 64, 3000, 8192, "fft"),      # 128 x 64
    ("fp32", 64, 6000, 16384, "fft"),     # 128 x 128
    ("fp32", 32, 7001, 16384, "fft"),     # ragged
    ("fp32", 16, 12345, 32768, "fft"),    # 256 x 128, ragged
    ("fp32", 16, 20000, 65536, "fft"),    # 256 x 256
    ("fp32", 256, 16384, 32768, "fft4"),  # the largest workload's form
    ("fp64", 128, 2500, 8192, "fft"),     # 128 x 64
    ("fp64", 64, 5000, 16384, "fft"),
    ("fp32", 64, 1024, 4096, "fft4"),     # 64 x 64, where one CTA would also hold it
    ("fp64", 256, 700, 4096, "fft4"),
    # the clustered one-launch form: every (F1, F2), one and two FP32 modes per cluster
    ("fp32", 64, 1024, 4096, "fft4c"),
    ("fp32", 128, 2000, 8192, "fft4c"),   # 128 x 64, two modes per cluster
    ("fp32", 256, 3000, 16384, "fft4c"),  # 128 x 128
    ("fp32", 32, 7001, 32768, "fft4c"),   # 256 x 128, ragged
    ("fp32", 16, 12345, 65536, "fft4c"),  # 256 x 256, ragged
    ("fp64", 128, 2500, 8192, "fft4c"),
    ("fp64", 8, 10923, 32768, "fft4c"),   # the largest FP64 N_s of this form, the smallest N_x
])
def test_four_step_matches_dense(precision, N, Ns, F, form):
    L, S = 22.0 + N / 16.0, 0.1 * (Ns - 1)
    X = _curve(N, Ns, L, N + Ns, fp32=precision == "fp32")
    xt = torch.from_numpy(X)
    xt = xt.float() if precision == "fp32" else xt
    cf = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision=precision, dtau=1e-3, s_transform=form)
    cd = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision=precision, dtau=1e-3, s_transform="dense")
    assert cf.fft_length == F and cd.fft_length == 0
    ftol, jtol, atol = (5e-6, 1e-5, 2e-5) if precision == "fp32" else (1e-10, 1e-10, 1e-10)
    diff = rel_2 if precision == "fp32" else rel_max
    rf, rd = cf.residual().double().cpu().numpy(), cd.residual().double().cpu().numpy()
    assert diff(rf, rd) < ftol
    (J2f, Jaf), (J2d, Jad) = cf.cost(), cd.cost()
    print("FFT4 %s N=%d Ns=%d %s F=%d: r=%.3e J2=%.3e J_arc=%.3e" % (precision, N, Ns, form, F, diff(rf, rd),
                                                                      abs(J2f - J2d) / J2d, abs(Jaf - Jad) / Jad))
    assert abs(J2f - J2d) < jtol * J2d and abs(Jaf - Jad) < atol * Jad
    of, od = cf.descend(10), cd.descend(10)
    xf, xd = cf.get_state().double().cpu().numpy(), cd.get_state().double().cpu().numpy()
    assert diff(xf, xd) < ftol
    assert abs(of["J"] - od["J"]) < jtol * od["J"]
    cf.close()
    cd.close()


@pytest.mark.parametrize("Ns,F,form", [(20000, 65536, "fft"), (12345, 65536, "fft4c")])
def test_four_step_fp32_matches_oracle(Ns, F, form):
    """F = 65536 = 256 x 256 in FP32 against the FP64 oracle on the same (FP32)
    curve: the three-launch form (Toeplitz and Hankel parts) and the clustered one."""
    N = 16
    L, S = 22.0 + N / 16.0, 0.1 * (Ns - 1)
    X = _curve(N, Ns, L, N + Ns, fp32=True)
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X).float(), precision="fp32", s_transform=form)
    assert c.fft_length == F
    U = oracle.curve_spectral(X)
    R, D = oracle.curve_residual(U, L, S, 1.0)
    sc = oracle.curve_scalars(R, D, L, S, 1.0)
    er = rel_2(c.residual().double().cpu().numpy(), oracle.curve_physical(R))
    J2, Ja = c.cost()
    print("FFT4 fp32 vs oracle Ns=%d %s F=%d: r=%.3e J2=%.3e J_arc=%.3e" % (Ns, form, F, er, abs(J2 - sc["J2"]) / sc["J2"],
                                                                          abs(Ja - sc["J_arc"]) / sc["J_arc"]))
    assert er < 2e-6
    assert abs(J2 - sc["J2"]) < 1e-5 * sc["J2"]
    assert abs(Ja - sc["J_arc"]) < 2e-5 * sc["J_arc"]
    c.close()


@pytest.mark.parametrize("form", ["fft", "fft4c"])
@pytest.mark.parametrize("sym", [1, 3])
def test_four_step_holds_the_symmetric_subspace(sym, form):
    """Odd (and L/2-periodic) sections stay so exactly through the descent."""
    N, Ns, L = 32, 3000, 22.0
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    X = np.outer(np.sin(th / 2) + 0.2, np.sin(4 * np.pi * x / L)) + 0.3 * np.outer(np.sin(th), np.sin(8 * np.pi * x / L))
    if sym == 1:
        X += 0.2 * np.outer(np.sin(2 * th), np.sin(2 * np.pi * x / L))
    c = KSCurve(L, N, Ns, 0.1 * (Ns - 1), X[0], X[-1], u_init=torch.from_numpy(X), dtau=1e-3, symmetry=sym,
                s_transform=form)
    assert c.fft_length == (8192 if form == "fft" else 16384)
    c.descend(20)
    U = np.fft.rfft(c.get_state().cpu().numpy(), axis=1)
    assert np.abs(U.real).max() <= 1e-12 * np.abs(U).max()
    if sym == 3:
        assert np.abs(U[:, 1::2]).max() <= 1e-12 * np.abs(U).max()
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sym", [1, 3])
def test_paired_odd_columns_match_dense_and_oracle(precision, sym):
    """Odd sections (symmetry bit 0): the three-launch four-step form transforms
    the imaginary columns of two modes as one complex sequence, half the
    sequences of the general form; results equal the dense form's (and in FP64
    the oracle's descent, which has no projection and stays odd by itself)."""
    N, Ns, L = 64, 1500, 30.0
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    X = np.zeros((Ns, N))
    rng = np.random.default_rng(sym)
    for q in range(1, 9):
        if sym == 3 and q % 2:
            continue
        X += np.outer(0.4 * rng.standard_normal() * (np.sin(th * rng.integers(1, 4)) + 0.1 * q * np.cos(th)),
                      np.sin(2 * np.pi * q * x / L))
    if precision == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    xt = torch.from_numpy(X)
    xt = xt.float() if precision == "fp32" else xt
    S = 0.1 * (Ns - 1)
    cf = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision=precision, dtau=2e-3, symmetry=sym,
                 s_transform="fft4")
    cd = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision=precision, dtau=2e-3, symmetry=sym,
                 s_transform="dense")
    assert cf.fft_length == 4096
    (J2f, Jaf), (J2d, Jad) = cf.cost(), cd.cost()
    of, od = cf.descend(5), cd.descend(5)
    xf, xd = cf.get_state().double().cpu().numpy(), cd.get_state().double().cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-5
    e = dict(J2=abs(J2f - J2d) / J2d, J_arc=abs(Jaf - Jad) / Jad, u=rel_2(xf, xd), J5=abs(of["J"] - od["J"]) / od["J"])
    print("PAIRED %s sym=%d: %s" % (precision, sym, " ".join("%s=%.2e" % kv for kv in e.items())))
    assert e["J2"] < tol and e["u"] < tol and e["J5"] < tol and e["J_arc"] < 3 * tol
    if precision == "fp64":
        Uo, _, sco, _ = oracle.curve_descend(oracle.curve_spectral(X), L, S, 5, dtau=2e-3)
        assert rel_max(xf, oracle.curve_physical(Uo)) < 1e-10
        assert abs(of["J"] - sco["J"]) < 1e-10 * sco["J"]
    cf.close()
    cd.close()
