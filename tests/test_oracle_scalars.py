"""Pins of the oracle's curve scalars (ko_curve_scalars, ko_curve_norm2_W)
against values the mathematics fixes, independent of the oracle's own formulas.

Each scalar is fed sections whose spatial norm is known in closed form
(|q|^2 = integral of q^2 over [0, L), eq. J_arc's norm) and whose profile in s
has a known integral over the real line, so the discrete value must reach the
integral to quadrature accuracy:

  * J^2 = integral |r|^2 ds                        (eq. cost_function_general)
  * J_arc = integral |r||l d| ds / integral |l d| ds   (eq. J_arc, l d = l D_t u)
  * dJ^2/dl = -2 integral <d, r> ds                 (derivative of J^2 in l)
  * |G|_W^2 = integral |G|^2 ds, |l D_t u|_W        (the W-norm of the scalars)

A dropped square root, a weight squared, l on one side of J_arc only, a wrong
dx or a factor 2 on the Fourier sums moves each of these far outside its
tolerance (checked in the last test by planting those mistakes in a copy of
the formulas).
"""
import numpy as np
import pytest

import oracle

L = 22.0
N = 16
M = 400
S = 8.0


def section(mode, amp, kind="sin"):
    """Spectral section of amp*sin(2 pi mode x / L) (or cos): the physical
    section is u^_0 + 2 Re sum_j u^_j e^{i k_j x}, so sin -> u^_mode = -i amp/2."""
    uh = np.zeros(N // 2, np.complex128)
    uh[mode] = (-0.5j if kind == "sin" else 0.5) * amp
    return uh


UNIT = np.sqrt(2.0 / L)    # amplitude with integral of (UNIT sin)^2 over [0, L) = 1


def curve_of(profile, sec):
    """Curve [M+2, N/2] with section m = profile(s_m) * sec, end rows 0."""
    _, s, _ = oracle.grid(M, S)
    U = np.zeros((M + 2, N // 2), np.complex128)
    U[1:-1] = profile(s[1:-1])[:, None] * sec[None, :]
    return U


def sech(x):
    e = np.exp(-np.abs(x))
    return 2.0 * e / (1.0 + e * e)


def test_section_norm_convention():
    """The unit section has |q| = 1 under the quadrature (one row, weight known)."""
    U = curve_of(lambda s: np.ones_like(s), section(1, UNIT))
    _, _, w = oracle.grid(M, S)
    assert abs(oracle.curve_norm2_W(U, L, S) - w[1:-1].sum()) < 1e-12 * w[1:-1].sum()


def test_J2_and_G2_of_a_sech_profile():
    """r = G = sech(s) sin(2 pi x / L): integral = 2 (in s) x L/2 (in x) = L."""
    X = curve_of(sech, section(1, 1.0))
    D = curve_of(sech, section(2, 1.0))
    sc = oracle.curve_scalars(X, D, L, S, lam=1.0, G=X)
    assert abs(sc["J2"] - L) < 1e-10 * L
    assert abs(sc["G2"] - L) < 1e-10 * L
    assert abs(oracle.curve_norm2_W(X, L, S) - L) < 1e-10 * L


def test_J_arc_of_constant_residual_norm_is_that_norm():
    """|r_m| = rho at every section: J_arc = rho exactly, whatever |d_m| and l."""
    rho = 0.37
    rng = np.random.default_rng(3)
    _, s, _ = oracle.grid(M, S)
    R = curve_of(lambda s: np.full_like(s, rho), section(1, UNIT))
    # |d_m| varies over the sections and mixes two modes
    D = curve_of(lambda s: 1.0 + 0.5 * np.tanh(s), section(2, UNIT))
    D[1:-1, 3] = 0.3 * rng.standard_normal(M)
    for lam in (1.0, -0.6, 2.5):
        sc = oracle.curve_scalars(R, D, L, S, lam=lam)
        assert abs(sc["J_arc"] - rho) < 1e-14 * rho


@pytest.mark.parametrize("lam", [1.0, 1.7, -0.8])
def test_J_arc_of_sech_profiles(lam):
    """|r| = sech^2 s, |d| = sech^2 s: J_arc = int sech^4 / int sech^2 = (4/3)/2."""
    R = curve_of(lambda s: sech(s) ** 2, section(1, UNIT))
    D = curve_of(lambda s: sech(s) ** 2, section(3, UNIT, "cos"))
    sc = oracle.curve_scalars(R, D, L, S, lam=lam)
    assert abs(sc["J_arc"] - 2.0 / 3.0) < 1e-10
    # |l d|_W = |l| sqrt(int sech^4) = |l| sqrt(4/3)
    assert abs(sc["Dnorm"] - abs(lam) * np.sqrt(4.0 / 3.0)) < 1e-10


def test_dJ2_dlambda_of_sech_profiles():
    """r = sech(s) e1, d = sech(s)(cos a e1 + sin a e2): -2 int <d, r> ds = -4 cos a."""
    a = 0.7
    R = curve_of(sech, section(1, UNIT))
    D = curve_of(sech, np.cos(a) * section(1, UNIT) + np.sin(a) * section(2, UNIT))
    sc = oracle.curve_scalars(R, D, L, S, lam=1.3)
    assert abs(sc["dJ2_dlambda"] + 4.0 * np.cos(a)) < 1e-10


def test_Dnorm_of_a_tanh_curve_through_D_t():
    """u = tanh(s) v(x): d u / d s = sech^2(s) v, so |l D_t u|_W = |l| sqrt(4/3) |v|;
    D_t from the oracle's own transform, the norm from the scalars."""
    _, s, _ = oracle.grid(M, S)
    v = section(1, UNIT) + section(2, 0.5 * UNIT, "cos")       # |v|^2 = 1 + 1/4
    U = np.zeros((M + 2, N // 2), np.complex128)
    U[1:-1] = np.tanh(s[1:-1])[:, None] * v[None, :]
    U[0], U[-1] = v, -v
    lam = 1.4
    R, D = oracle.curve_residual(U, L, S, lam)
    sc = oracle.curve_scalars(R, D, L, S, lam=lam)
    assert abs(sc["Dnorm"] - lam * np.sqrt(4.0 / 3.0 * 1.25)) < 1e-9


def _planted(R, D, lam, mistake):
    """Scalars by the same discrete formulas with one mistake planted."""
    _, _, w = oracle.grid(M, S)
    r, d = oracle.curve_physical(R)[1:-1], oracle.curve_physical(D)[1:-1]
    dx = L / N
    rr, dd, dr = (dx * (r * r).sum(1)), (dx * (d * d).sum(1)), (dx * (d * r).sum(1))
    w = w[1:-1]
    if mistake == "no_sqrt":
        ja = (w * rr * abs(lam) * np.sqrt(dd)).sum() / (w * abs(lam) * np.sqrt(dd)).sum()
    elif mistake == "weight_squared":
        ja = (w * w * np.sqrt(rr) * abs(lam) * np.sqrt(dd)).sum() / (w * abs(lam) * np.sqrt(dd)).sum()
    elif mistake == "lambda_one_side":
        ja = (w * np.sqrt(rr) * abs(lam) * np.sqrt(dd)).sum() / (w * np.sqrt(dd)).sum()
    else:
        ja = (w * np.sqrt(rr) * abs(lam) * np.sqrt(dd)).sum() / (w * abs(lam) * np.sqrt(dd)).sum()
    return ja


@pytest.mark.parametrize("mistake", ["no_sqrt", "weight_squared", "lambda_one_side"])
def test_the_J_arc_pins_catch_plausible_mistakes(mistake):
    """The sech-profile pin rejects each planted mistake (the correct formula passes)."""
    R = curve_of(lambda s: sech(s) ** 2, section(1, UNIT))
    D = curve_of(lambda s: sech(s) ** 2, section(3, UNIT, "cos"))
    lam = 1.7
    assert abs(_planted(R, D, lam, "none") - 2.0 / 3.0) < 1e-10
    assert abs(_planted(R, D, lam, mistake) - 2.0 / 3.0) > 1e-2
