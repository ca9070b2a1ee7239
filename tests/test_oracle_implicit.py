"""Pins of the oracle's full-linear-implicit step (Sec. V.C.3: semi-implicit
forward Euler with every term of G that is linear in u taken at the new level).

On the interior rows the linear part of G is (lambda^2 Dt~^2 - a_j^2) u per
spatial mode j (Dt~ the interior block of the rational-Chebyshev derivative
matrix).  The pins do not re-derive the oracle's LU solve:
  * curves made of one eigenvector x of Dt~^2 (eigenvalue mu < 0, from
    numpy's eigensolver) in the mean mode, where G is exactly linear, must be
    scaled by 1 / (1 - dtau lambda^2 mu) in one step (closed form);
  * the same with a small amplitude in a mode j >= 1, where G is linear up to
    O(amplitude), must be scaled by 1 / (1 + dtau (a_j^2 - lambda^2 mu));
  * as dtau -> 0 the implicit and the diagonal-implicit (IMEX) steps agree to
    second order in dtau (both are consistent first-order schemes);
  * at a dtau fifty times the IMEX stability limit the implicit descent lowers
    J^2 at every step while the IMEX descent blows up.
"""
import numpy as np
import pytest

import oracle


def interior_D2(M, S):
    D = oracle.dt_matrix(M, S)[1:-1, 1:-1]
    return D @ D


def eig_pairs(M, S):
    """Real eigenpairs of Dt~^2 whose eigenvalue is simple (the even and odd
    parts of the s-reflection share most eigenvalues, so numpy's vectors are
    only real for the unpaired ones; a pair is combined back to a real vector)."""
    w, V = np.linalg.eig(interior_D2(M, S))
    out = []
    for i in np.argsort(w.real):
        x = V[:, i]
        x = x.real if np.abs(x.real).max() >= np.abs(x.imag).max() else x.imag
        x = x / np.abs(x).max()
        out.append((float(w[i].real), x))
    return out


def eigvec_checked(M, S, which):
    D2 = interior_D2(M, S)
    for mu, x in eig_pairs(M, S)[which:]:
        if np.linalg.norm(D2 @ x - mu * x) < 1e-11 * abs(mu) * np.linalg.norm(x) and mu < -1e-6:
            return mu, x
    raise AssertionError("no real eigenvector found")


@pytest.mark.parametrize("lam", [1.0, 1.7])
@pytest.mark.parametrize("which", [0, 5, 40])
def test_mean_mode_eigenvector_closed_form(lam, which):
    M, N, L = 62, 16, 22.0
    S = 0.1 * (M + 1)
    mu, x = eigvec_checked(M, S, which)
    U = np.zeros((M + 2, N // 2), np.complex128)
    U[1:-1, 0] = x
    dtau = 0.3
    Uo, steps, _, _ = oracle.curve_descend(U, L, S, 1, dtau=dtau, lam=lam, scheme=oracle.IMPLICIT)
    assert steps == 1
    expect = x / (1.0 - dtau * lam * lam * mu)
    assert np.abs(Uo[1:-1, 0] - expect).max() < 1e-12 * np.abs(expect).max()
    # the other modes only see the naive DFTs' rounding
    assert np.abs(Uo[:, 1:]).max() < 1e-14 and Uo[0, 0] == 0 and Uo[-1, 0] == 0


@pytest.mark.parametrize("j", [1, 3, 6])
def test_single_mode_small_amplitude_closed_form(j):
    M, N, L, lam = 62, 16, 22.0, 1.0
    S = 0.1 * (M + 1)
    mu, x = eigvec_checked(M, S, 3)
    eps = 1e-9
    U = np.zeros((M + 2, N // 2), np.complex128)
    U[1:-1, j] = eps * (0.6 - 0.8j) * x
    k = 2 * np.pi * j / L
    a = k ** 4 - k ** 2
    dtau = 0.5
    Uo, _, _, _ = oracle.curve_descend(U, L, S, 1, dtau=dtau, lam=lam, scheme=oracle.IMPLICIT)
    expect = U[1:-1, j] / (1.0 + dtau * (a * a - lam * lam * mu))
    assert np.abs(Uo[1:-1, j] - expect).max() < 1e-6 * np.abs(expect).max()
    others = np.delete(Uo[1:-1], j, axis=1)
    assert np.abs(others).max() < 1e-6 * np.abs(expect).max()


def trial_curve(M, N, L, seed):
    rng = np.random.default_rng(seed)
    S = 0.1 * (M + 1)
    x = np.arange(N) * L / N
    up = sum(rng.standard_normal() * np.sin(2 * np.pi * q * x / L) for q in (1, 2, 3))
    um = np.zeros(N)
    vp = np.stack([np.cos(2 * np.pi * (q + 1) * x / L + rng.uniform(0, 6.3)) for q in range(3)])
    U = oracle.curve_init(M, S, up, um, amps=np.full(3, 0.2), vp=vp)
    return U, S


def test_agrees_with_imex_to_second_order_as_dtau_vanishes():
    M, N, L = 30, 16, 22.0
    U, S = trial_curve(M, N, L, 3)
    diffs = []
    for dtau in (4e-3, 2e-3, 1e-3):
        Ui, _, _, _ = oracle.curve_descend(U, L, S, 1, dtau=dtau, scheme=oracle.IMPLICIT)
        Ue, _, _, _ = oracle.curve_descend(U, L, S, 1, dtau=dtau, scheme=oracle.IMEX_X)
        diffs.append(np.linalg.norm(Ui - Ue))
        assert np.linalg.norm(Ui - U) > 100 * diffs[-1]
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, (r1, r2)


def test_stable_far_beyond_the_imex_limit():
    M, N, L = 62, 16, 22.0
    U, S = trial_curve(M, N, L, 5)
    D = oracle.dt_matrix(M, S)[1:-1, 1:-1]
    rho = np.abs(np.linalg.eigvals(D @ D)).max()
    dtau = 50 * 2.0 / rho           # fifty times the IMEX limit dtau rho(Dt~^2) < 2
    _, _, _, hist_i = oracle.curve_descend(U, L, S, 60, dtau=dtau, scheme=oracle.IMPLICIT, mode=oracle.DISCRETE,
                                          history=True)
    J = hist_i[:, 2]
    assert np.all(np.isfinite(J)) and np.all(np.diff(J) < 0) and J[-1] < 0.5 * J[0]
    _, _, _, hist_e = oracle.curve_descend(U, L, S, 60, dtau=dtau, scheme=oracle.IMEX_X, mode=oracle.DISCRETE,
                                          history=True)
    Je = hist_e[:, 2]
    assert not np.all(np.isfinite(Je)) or Je[-1] > 1e3 * Je[0]


def test_increment_form_matches_curve_descend():
    """implicit_update (the single-step entry point) is the step curve_descend takes."""
    M, N, L = 30, 16, 22.0
    U, S = trial_curve(M, N, L, 9)
    R, _ = oracle.curve_residual(U, L, S)
    G, _ = oracle.curve_adjoint(U, R, L, S)
    U1 = oracle.implicit_update(U, G, L, S, 0.2)
    U2, _, _, _ = oracle.curve_descend(U, L, S, 1, dtau=0.2, scheme=oracle.IMPLICIT)
    assert np.abs(U1 - U2).max() == 0.0
