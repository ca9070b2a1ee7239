"""Sine storage (symmetry bit 2; Sec. V.B, eq. reflection): odd sections have
u^_j purely imaginary, so a curve may keep only Im u^_j, N_x/2 words per
section, and run every s-contraction on those N_x/2 columns.  Checked here
against full storage of the same odd curve (symmetry 1 or 3) in the same
s-form, and in FP64 against the oracle (which has no projection; an odd curve
stays odd under its descent), for the forms that take it (dense, one CTA per
column pair, the three-launch and the clustered four-step forms, auto), both precisions, both
adjoints, ragged N_s and the smallest width N_x = 16.

Tolerances: FP64 1e-10 relative (the two storages differ only in the
contraction's split of the sections, rounding order); FP32 1e-5 on J, the state
after five steps and the gradient, 3e-5 on J_arc (which amplifies the rounding
of D_t u about tenfold), as between the FP32 s-forms; dJ^2/dlambda, a sum with
cancellation, relative to its Cauchy-Schwarz bound 2 |D_t u|_W |r|_W."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300.curve import KSCurve
from tests.test_gpu_parity import rel_2, rel_max

pytestmark = pytest.mark.gpu


def _odd_curve(N, Ns, L, sym, seed, fp32):
    """Odd sections (and L/2-periodic for sym & 2), smooth in s, ends included."""
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    rng = np.random.default_rng(seed)
    X = np.zeros((Ns, N))
    for q in range(1, min(9, N // 2)):
        if (sym & 2) and q % 2:
            continue
        X += np.outer(0.4 * rng.standard_normal() * (np.sin(th * rng.integers(1, 4)) + 0.1 * q * np.cos(th)),
                      np.sin(2 * np.pi * q * x / L))
    return X.astype(np.float32).astype(np.float64) if fp32 else X


def _pair(N, Ns, L, sym, precision, form, adjoint="paper", seed=0):
    X = _odd_curve(N, Ns, L, sym, seed, precision == "fp32")
    xt = torch.from_numpy(X)
    xt = xt.float() if precision == "fp32" else xt
    S = 0.1 * (Ns - 1)
    kw = dict(u_init=xt, precision=precision, dtau=2e-3, s_transform=form, adjoint=adjoint)
    ch = KSCurve(L, N, Ns, S, X[0], X[-1], symmetry=sym | 4, **kw)
    cf = KSCurve(L, N, Ns, S, X[0], X[-1], symmetry=sym, **kw)
    return X, S, ch, cf


CASES = [  # (N_x, N_s, form): every form that takes sine storage, ragged N_s, several tiles
    (64, 301, "dense"),
    (64, 301, "fft"),       # one CTA per column pair, F = 1024
    (64, 1500, "fft4"),     # three-launch four-step, F = 4096
    (16, 1500, "fft4"),     # N_x = 16: one row sector of four FP32 column pairs
    (32, 2100, "fft4"),     # the row phase's tiles by TMA (N_s >= 2048), ragged last tile
    (64, 1024, "fft4c"),    # clustered four-step, F = 4096
    (128, 1024, "auto"),    # FP32 clustered in both storages; FP64 three-launch
    (256, 1024, "auto"),    # FP64: one CTA per mode in full storage, four-step on the 128 stored columns
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,Ns,form", CASES)
@pytest.mark.parametrize("sym", [1, 3])
def test_sine_storage_matches_full_storage(N, Ns, form, precision, sym):
    L = 30.0
    X, S, ch, cf = _pair(N, Ns, L, sym, precision, form, seed=N + Ns + sym)
    assert ch.s_form == cf.s_form or form == "auto"   # auto applies its rule to the stored columns
    assert ch.workspace_bytes < cf.workspace_bytes
    (J2h, Jah), (J2f, Jaf) = ch.cost(), cf.cost()
    rh, rf = ch.residual().double().cpu().numpy(), cf.residual().double().cpu().numpy()
    (gh, dlh), (gf, dlf) = ch.gradient(), cf.gradient()
    gh, gf = gh.double().cpu().numpy(), gf.double().cpu().numpy()
    # dJ^2/dlambda = -2 <D_t u, r>_W cancels: its error is measured on the bound
    # 2 |D_t u|_W |r|_W (lambda = 1)
    scf = cf.scalars()
    dl_scale = 2.0 * scf["J"] * scf["Dnorm"]
    oh, of = ch.descend(5), cf.descend(5)
    xh, xf = ch.get_state().double().cpu().numpy(), cf.get_state().double().cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-5
    e = dict(J2=abs(J2h - J2f) / J2f, J_arc=abs(Jah - Jaf) / Jaf, r=rel_2(rh, rf), g=rel_2(gh, gf),
             dl=abs(dlh - dlf) / dl_scale, u=rel_2(xh, xf), J5=abs(oh["J"] - of["J"]) / of["J"])
    print("SINE %s N=%d Ns=%d %s sym=%d form=%s: %s" % (precision, N, Ns, form, sym, ch.s_form,
                                                        " ".join("%s=%.2e" % kv for kv in e.items())))
    assert e["J2"] < tol and e["r"] < tol and e["g"] < tol and e["u"] < tol and e["J5"] < tol
    assert e["J_arc"] < 3 * tol and e["dl"] < 3 * tol
    # the state stays in the subspace: real parts (and odd modes for sym 3) zero,
    # up to the rounding of the physical values returned in the storage type
    U = np.fft.rfft(xh, axis=1)
    sub = 1e-12 if precision == "fp64" else 1e-6
    assert np.abs(U.real).max() <= sub * np.abs(U).max()
    if sym == 3:
        assert np.abs(U[:, 1::2]).max() <= sub * np.abs(U).max()
    ch.close()
    cf.close()


@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
@pytest.mark.parametrize("N,Ns,form", [(32, 301, "dense"), (32, 301, "fft"), (32, 1500, "fft4"), (32, 2100, "fft4")])
def test_sine_storage_fp64_matches_oracle(N, Ns, form, adjoint):
    """FP64 sine storage against the oracle: residual, J, J_arc, the gradient and
    five descent steps (the oracle keeps full coefficients; its odd curve stays odd)."""
    L = 22.0
    X, S, ch, cf = _pair(N, Ns, L, 1, "fp64", form, adjoint=adjoint, seed=7)
    cf.close()
    mode = oracle.DISCRETE if adjoint == "discrete" else oracle.PAPER
    U = oracle.curve_spectral(X)
    R, D = oracle.curve_residual(U, L, S, 1.0)
    G, dl = oracle.curve_adjoint(U, R, L, S, 1.0, mode=mode)
    sc = oracle.curve_scalars(R, D, L, S, 1.0)
    assert rel_max(ch.residual().cpu().numpy(), oracle.curve_physical(R)) < 1e-10
    J2, Ja = ch.cost()
    assert abs(J2 - sc["J2"]) < 1e-10 * sc["J2"] and abs(Ja - sc["J_arc"]) < 1e-10 * sc["J_arc"]
    g, _ = ch.gradient()
    assert rel_2(g.cpu().numpy(), oracle.curve_physical(G)) < 1e-10
    o = ch.descend(5)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 5, dtau=2e-3, mode=mode)
    assert rel_max(ch.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < 1e-10
    assert abs(o["J"] - sco["J"]) < 1e-10 * sco["J"]
    ch.close()


def test_sine_storage_set_state_round_trip():
    """set_state / get_state keep the physical layout: an odd curve comes back as
    given (to FP64 rounding), and its even part is dropped by the projection."""
    N, Ns, L = 32, 200, 22.0
    X = _odd_curve(N, Ns, L, 1, 3, False)
    c = KSCurve(L, N, Ns, 0.1 * (Ns - 1), X[0], X[-1], u_init=torch.from_numpy(X), symmetry=5)
    assert rel_max(c.get_state().cpu().numpy(), X) < 1e-14
    x = np.arange(N) * L / N
    Y = X + 0.3 * np.cos(2 * np.pi * x / L)[None, :]
    Y[0], Y[-1] = X[0], X[-1]
    c.set_state(torch.from_numpy(Y))
    assert rel_max(c.get_state().cpu().numpy(), X) < 1e-14
    c.close()
