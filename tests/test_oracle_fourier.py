"""Pins of the oracle's Fourier direction and spatial operators (Sec. V.C.1, eq. KSE).

Each check compares the oracle with something other than itself: a library FFT,
closed forms of f for one- and two-mode fields, finite differences, and the
transpose identity of the spatial adjoint (App. A).
"""
import numpy as np
import pytest

import oracle


def _grid(N, L):
    return np.arange(N) * L / N


def _round_tol(N, L, scale):
    """Rounding floor of f on the grid: noise of size eps * N * scale in every
    coefficient, amplified by the largest linear symbol k_max^4."""
    kmax = 2 * np.pi * (N // 2 - 1) / L
    return 4e-16 * N * max(1.0, kmax ** 4) * scale


@pytest.mark.parametrize("N", [8, 32, 64])
def test_forward_transform_matches_library_fft(N):
    rng = np.random.default_rng(N)
    u = rng.standard_normal(N)
    ref = np.fft.fft(u)[: N // 2] / N
    assert np.abs(oracle.fwd(u) - ref).max() < 1e-14


@pytest.mark.parametrize("N", [8, 32, 64])
def test_inverse_transform_roundtrip_and_library(N):
    rng = np.random.default_rng(7 + N)
    uh = rng.standard_normal(N // 2) + 1j * rng.standard_normal(N // 2)
    uh[0] = uh[0].real
    u = oracle.inv(uh, N)
    full = np.zeros(N, complex)
    full[: N // 2] = uh
    full[N // 2 + 1:] = np.conj(uh[1:][::-1])
    assert np.abs(u - np.real(np.fft.ifft(full)) * N).max() < 1e-13
    assert np.abs(oracle.fwd(u) - uh).max() < 1e-14


def test_single_modes_have_textbook_coefficients():
    N, L = 32, 22.0
    x = _grid(N, L)
    for j in (1, 3, 7):
        k = 2 * np.pi * j / L
        c = oracle.fwd(np.cos(k * x))
        s = oracle.fwd(np.sin(k * x))
        e = np.zeros(N // 2, complex)
        e[j] = 0.5
        assert np.abs(c - e).max() < 1e-15
        assert np.abs(s - (-1j) * e).max() < 1e-15


def test_rhs_of_trivial_equilibrium_is_exactly_zero():
    for N in (8, 32, 64):
        assert np.all(oracle.rhs(np.zeros(N // 2, complex), N, 22.0) == 0)


@pytest.mark.parametrize("j,a,L", [(1, 0.7, 22.0), (2, -1.3, 22.0), (3, 0.4, 44.0), (5, 2.0, 100.0)])
def test_rhs_single_sine_closed_form(j, a, L):
    """u = a sin(kx):  f = -(a^2 k / 2) sin 2kx + a (k^2 - k^4) sin kx."""
    N = 64
    x = _grid(N, L)
    k = 2 * np.pi * j / L
    f = oracle.inv(oracle.rhs(oracle.fwd(a * np.sin(k * x)), N, L), N)
    ref = -(a * a * k / 2) * np.sin(2 * k * x) + a * (k ** 2 - k ** 4) * np.sin(k * x)
    assert np.abs(f - ref).max() < _round_tol(N, L, abs(a) + a * a)


def test_rhs_two_mode_closed_form():
    """u = a cos(p x) + b sin(q x): the quadratic term produces sum and
    difference wavenumbers with known coefficients."""
    N, L = 64, 22.0
    x = _grid(N, L)
    p, q = 2 * np.pi * 2 / L, 2 * np.pi * 5 / L
    a, b = 0.8, -1.1
    u = a * np.cos(p * x) + b * np.sin(q * x)
    half_dx_u2 = 0.5 * (-a * a * p * np.sin(2 * p * x)
                        + 2 * a * b * ((q + p) * np.cos((q + p) * x) + (q - p) * np.cos((q - p) * x)) / 2
                        + b * b * q * np.sin(2 * q * x))
    lin = a * (p ** 2 - p ** 4) * np.cos(p * x) + b * (q ** 2 - q ** 4) * np.sin(q * x)
    ref = -half_dx_u2 + lin
    f = oracle.inv(oracle.rhs(oracle.fwd(u), N, L), N)
    assert np.abs(f - ref).max() < _round_tol(N, L, 4.0)


def _rand_spec(rng, N, decay=0.6):
    uh = (rng.standard_normal(N // 2) + 1j * rng.standard_normal(N // 2)) * decay ** np.arange(N // 2)
    uh[0] = uh[0].real
    return uh


def test_linearisation_matches_finite_differences():
    N, L = 32, 22.0
    rng = np.random.default_rng(3)
    uh, vh = _rand_spec(rng, N), _rand_spec(rng, N)
    h = 1e-6
    fd = (oracle.rhs(uh + h * vh, N, L) - oracle.rhs(uh - h * vh, N, L)) / (2 * h)
    jv = oracle.jac_apply(uh, vh, N, L)
    assert np.abs(fd - jv).max() < 1e-7 * np.abs(jv).max()


def test_spatial_adjoint_is_transpose_of_linearisation():
    """sum_n (Df v)_n r_n == sum_n v_n ((Df)^T r)_n on the grid (App. A, spatial part)."""
    N, L = 32, 22.0
    rng = np.random.default_rng(4)
    for _ in range(5):
        uh, vh, rh = _rand_spec(rng, N), _rand_spec(rng, N), _rand_spec(rng, N)
        lhs = np.dot(oracle.inv(oracle.jac_apply(uh, vh, N, L), N), oracle.inv(rh, N))
        rhs = np.dot(oracle.inv(vh, N), oracle.inv(oracle.jac_adjoint_apply(uh, rh, N, L), N))
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
