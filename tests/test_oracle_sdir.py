"""Pins of the oracle's temporal direction (Sec. IV): grid, quadrature,
expansion coefficients (eq. rational_coeffs) and the differentiation matrix
(eq. rational_diff_matrix).

The references are: the exact derivative of each basis function cos(n theta)
with theta(s) from eq. Rational_domain, the exact derivative of smooth
functions of s, known integrals, and an independent closed form of D_t
(a Toeplitz-plus-Hankel matrix of cotangents derived by summing the series of
eq. rational_diff_matrix in closed form).
"""
import numpy as np
import pytest

import oracle


def test_grid_points_and_order():
    M, S, s0 = 21, 3.0, 0.7
    th, s, w = oracle.grid(M, S, s0)
    P = M + 1
    assert np.isposinf(s[0]) and np.isneginf(s[-1])
    assert np.all(np.diff(s[1:-1]) < 0)                 # s decreases with theta
    assert np.allclose(s[1:-1] - s0, -(s[1:-1][::-1] - s0), atol=1e-12)   # symmetric about s0
    assert abs(s[P // 2] - s0) < 1e-14 if P % 2 == 0 else True
    assert np.allclose(th, np.arange(M + 2) * np.pi / P)
    assert w[0] == 0 and w[-1] == 0 and np.all(w[1:-1] > 0)


@pytest.mark.parametrize("g,exact", [
    (lambda s: np.exp(-s * s), np.sqrt(np.pi)),
    (lambda s: 1.0 / np.cosh(s) ** 2, 2.0),
    (lambda s: np.exp(-(s - 1.5) ** 2 / 8.0), np.sqrt(8 * np.pi)),
])
def test_quadrature_integrates_decaying_functions(g, exact):
    M, S = 400, 6.0
    _, s, w = oracle.grid(M, S)
    approx = np.sum(w[1:-1] * g(s[1:-1]))
    assert abs(approx - exact) < 1e-10 * exact


@pytest.mark.parametrize("M", [5, 14, 31])
def test_expansion_coefficients_recover_basis_functions(M):
    P = M + 1
    th = np.arange(M + 2) * np.pi / P
    for n in range(P + 1):
        c = oracle.dt_coeffs(np.cos(n * th))
        e = np.zeros(M + 2)
        e[n] = 1.0
        assert np.abs(c - e).max() < 1e-13


@pytest.mark.parametrize("M,S", [(3, 1.0), (14, 1.5), (40, 4.1), (127, 12.8)])
def test_derivative_of_basis_functions_is_exact(M, S):
    """d/ds cos(n theta(s)) = n sin(n theta) sin^2(theta) / S for every n <= M+1."""
    P = M + 1
    th = np.arange(M + 2) * np.pi / P
    for n in range(P + 1):
        d = oracle.dt_apply(np.cos(n * th), S)
        ref = n * np.sin(n * th) * np.sin(th) ** 2 / S
        assert np.abs(d - ref).max() < 2e-13 * max(1, n)


def test_derivative_of_constant_is_zero_and_end_rows_vanish():
    M, S = 30, 3.1
    rng = np.random.default_rng(0)
    assert np.abs(oracle.dt_apply(np.full(M + 2, 2.5), S)).max() < 1e-13
    d = oracle.dt_apply(rng.standard_normal(M + 2), S)
    assert d[0] == 0.0 and abs(d[-1]) < 1e-15


def test_derivative_of_cos_theta_of_s():
    """q(s) = (s - s0)/sqrt((s - s0)^2 + S^2) = cos(theta); dq/ds = sin^3(theta)/S."""
    M, S, s0 = 60, 5.0, 0.0
    th, s, _ = oracle.grid(M, S, s0)
    q = np.cos(th)
    ref = np.sin(th) ** 3 / S
    assert np.abs(oracle.dt_apply(q, S) - ref).max() < 1e-13


def test_spectral_convergence_on_tanh():
    """D_t tanh(s) -> sech^2(s), error falling fast with M (Sec. IV)."""
    errs = []
    S = 2.0            # fixed map scale: refining M refines every part of the s-axis
    for M in (16, 32, 64, 128):
        th, s, _ = oracle.grid(M, S)
        q = np.tanh(s)
        q[0], q[-1] = 1.0, -1.0
        d = oracle.dt_apply(q, S)
        ref = np.zeros(M + 2)
        ref[1:-1] = 1.0 / np.cosh(s[1:-1]) ** 2
        errs.append(np.abs(d - ref).max())
    assert errs[-1] < 1e-12
    assert all(b < a for a, b in zip(errs, errs[1:]))


def _dt_closed_form(M, S):
    """D_t from the closed form of the k-sum in eq. rational_diff_matrix:
    sum_{k=1}^{P-1} k sin(k pi n / P) = (-1)^(n+1) (P/2) cot(pi n / (2P)), so
    D_{j,m} = -(-1)^(j+m) sin^2(j pi/P) / (2 S cbar_m)
              * [cot(pi (j+m)/(2P)) + cot(pi (j-m)/(2P))], a cot with an argument
    that is a multiple of pi contributing 0."""
    P = M + 1
    t = np.arange(2 * P)
    cot = np.zeros(2 * P)
    cot[1:] = np.cos(np.pi * t[1:] / (2 * P)) / np.sin(np.pi * t[1:] / (2 * P))
    j = np.arange(M + 2)[:, None]
    m = np.arange(M + 2)[None, :]
    cb = np.where((m == 0) | (m == P), 2.0, 1.0)
    sign = np.where((j + m) % 2 == 0, -1.0, 1.0)
    return sign * np.sin(j * np.pi / P) ** 2 / (2 * S * cb) * (cot[(j + m) % (2 * P)] + cot[(j - m) % (2 * P)])


@pytest.mark.parametrize("M,S", [(3, 1.0), (14, 1.5), (41, 4.2), (100, 10.1)])
def test_explicit_matrix_equals_closed_form(M, S):
    D = oracle.dt_matrix(M, S)
    C = _dt_closed_form(M, S)
    assert np.abs(D - C).max() < 1e-12 * np.abs(C).max()


@pytest.mark.parametrize("M,S", [(14, 1.5), (63, 6.4)])
def test_two_sum_form_and_transpose_equal_the_matrix(M, S):
    D = oracle.dt_matrix(M, S)
    rng = np.random.default_rng(M)
    for _ in range(3):
        x = rng.standard_normal(M + 2)
        assert np.abs(oracle.dt_apply(x, S) - D @ x).max() < 1e-12 * np.abs(D).max() * np.abs(x).sum()
        assert np.abs(oracle.dtT_apply(x, S) - D.T @ x).max() < 1e-12 * np.abs(D).max() * np.abs(x).sum()


def test_single_rows_equal_the_explicit_matrix():
    M, S = 41, 4.2
    D = oracle.dt_matrix(M, S)
    for j in (0, 1, 7, 20, M, M + 1):
        assert np.abs(oracle.dt_row(M, S, j) - D[j]).max() < 1e-13 * np.abs(D).max()
