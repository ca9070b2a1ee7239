"""Curve-level pins of the oracle: symmetry (Sec. V.B), the adjoint identity
(eq. adjoint_definition), the linearisation (eq. directional_derivative),
brute-force finite differences of J^2 (eq. cost_function_general), monotone
descent (eq. monotonic_decrase_of_J_general) and the trial curve
(eq. KSE_initial_curve)."""
import numpy as np
import pytest

import oracle
from paper_2301_11704_gb300 import gen
from tests.curves import end_points, perturbation, random_smooth_curve


def inner_W(A, B, L, S):
    """<a,b>_W = dx sum_m w_m sum_n a_{m,n} b_{m,n} on the interior rows."""
    M, N = A.shape[0] - 2, 2 * A.shape[1]
    _, _, w = oracle.grid(M, S)
    a, b = oracle.curve_physical(A), oracle.curve_physical(B)
    return (L / N) * np.sum(w[1:-1, None] * a[1:-1] * b[1:-1])


def J2(U, L, S, lam=1.0):
    R, D = oracle.curve_residual(U, L, S, lam)
    return oracle.curve_scalars(R, D, L, S, lam)["J2"]


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(11)
    M, N, L, S = 14, 16, 22.0, 1.5
    return M, N, L, S, random_smooth_curve(rng, M, N)


# ---------------------------------------------------------------- symmetry (P4)

def test_cost_invariant_under_grid_shift_and_inversion(small):
    M, N, L, S, U = small
    j = np.arange(N // 2)
    ref = J2(U, L, S)
    for n0 in (1, 3, 7):
        Us = U * np.exp(2j * np.pi * j * n0 / N)[None, :]
        assert abs(J2(Us, L, S) - ref) < 1e-13 * ref
    assert abs(J2(-np.conj(U), L, S) - ref) < 1e-13 * ref


@pytest.mark.parametrize("mode", [oracle.PAPER, oracle.DISCRETE])
def test_descent_direction_is_equivariant(small, mode):
    M, N, L, S, U = small
    j = np.arange(N // 2)
    R, _ = oracle.curve_residual(U, L, S)
    G, _ = oracle.curve_adjoint(U, R, L, S, mode=mode)
    # inversion sigma: u^ -> -conj(u^)
    Rs, _ = oracle.curve_residual(-np.conj(U), L, S)
    Gs, _ = oracle.curve_adjoint(-np.conj(U), Rs, L, S, mode=mode)
    assert np.abs(Gs - (-np.conj(G))).max() < 1e-12 * np.abs(G).max()
    # translation by 3 grid points
    ph = np.exp(2j * np.pi * j * 3 / N)[None, :]
    Rt, _ = oracle.curve_residual(U * ph, L, S)
    Gt, _ = oracle.curve_adjoint(U * ph, Rt, L, S, mode=mode)
    assert np.abs(Gt - G * ph).max() < 1e-12 * np.abs(G).max()


def test_inversion_symmetric_curve_stays_symmetric_under_descent():
    """A curve with all sections odd (imaginary coefficients) stays odd (Sec. V.B)."""
    rng = np.random.default_rng(5)
    M, N, L, S = 30, 16, 22.0, 3.1
    U = 1j * random_smooth_curve(rng, M, N).imag
    Uf, steps, _, _ = oracle.curve_descend(U, L, S, 25, dtau=0.01)
    assert steps == 25
    assert np.abs(Uf.real).max() < 1e-13 * np.abs(Uf).max()
    assert np.abs(Uf - U).max() > 1e-6


# ---------------------------------------------------------------- linearisation and adjoint (P6)

def test_linearised_residual_matches_finite_differences(small):
    M, N, L, S, U = small
    rng = np.random.default_rng(2)
    G = random_smooth_curve(rng, M, N, ends=False)
    h = 1e-6
    fd = (oracle.curve_residual(U + h * G, L, S, 0.8)[0] - oracle.curve_residual(U - h * G, L, S, 0.8)[0]) / (2 * h)
    lin = oracle.curve_linearised(U, G, L, S, 0.8)
    assert np.abs(fd - lin).max() < 1e-7 * np.abs(lin).max()


def test_discrete_adjoint_identity_is_exact(small):
    """<L(u;G), r>_W = <G, L^dagger(u;r)>_W with L^dagger = -G_DISCRETE(u; r)."""
    M, N, L, S, U = small
    rng = np.random.default_rng(3)
    for lam in (1.0, 0.7):
        for _ in range(4):
            G = random_smooth_curve(rng, M, N, ends=False)
            r = random_smooth_curve(rng, M, N, ends=False)
            lhs = inner_W(oracle.curve_linearised(U, G, L, S, lam), r, L, S)
            Gd, _ = oracle.curve_adjoint(U, r, L, S, lam, mode=oracle.DISCRETE)
            rhs = inner_W(G, -Gd, L, S)
            assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_published_adjoint_differs_only_by_a_spectrally_small_term():
    """The s-term of eq. KSE_G (+lambda D_t r) is the continuous adjoint; on smooth
    fields it agrees with the discrete adjoint up to a gap that shrinks with M."""
    gaps = []
    for M in (14, 30, 62):
        S = 0.1 * (M + 1)
        th = np.arange(M + 2) * np.pi / (M + 1)
        N, L = 8, 22.0
        env = np.exp(-(S / np.tan(np.clip(th, 1e-9, np.pi - 1e-9))) ** 2 / 4.0)
        env[0] = env[-1] = 0.0
        U = np.zeros((M + 2, N // 2), complex)
        U[:, 1] = -0.5j * env
        U[:, 2] = 0.3 * env
        r = U.copy()
        Gp, _ = oracle.curve_adjoint(U, r, L, S, mode=oracle.PAPER)
        Gd, _ = oracle.curve_adjoint(U, r, L, S, mode=oracle.DISCRETE)
        gaps.append(np.sqrt(inner_W(Gp - Gd, Gp - Gd, L, S) / inner_W(Gd, Gd, L, S)))
    assert gaps[0] < 0.1 and gaps[1] < 1e-3 and gaps[2] < 1e-9
    assert gaps[0] > gaps[1] > gaps[2]


# ---------------------------------------------------------------- finite differences (P7)

def test_gradient_matches_central_finite_differences():
    """N_x = 8, N_s = 16: dJ^2/du along 64 seeded directions (h = 1e-6) equals the
    Euclidean gradient -2 dx w_m G_DISCRETE; dJ^2/dlambda likewise."""
    spec = gen.small_spec(L=22.0, N=8, Ns=16, S=1.5)
    M, N, L, S = spec.M, spec.N, spec.L, spec.S
    rng = gen.SplitMix64(spec.seed())
    U = np.zeros((M + 2, N // 2), complex)
    for m in range(M + 2):
        for j in range(N // 2):
            U[m, j] = complex(rng.normal(), rng.normal() if j else 0.0) * 0.6 ** j
    lam = 1.0
    R, D = oracle.curve_residual(U, L, S, lam)
    G, _ = oracle.curve_adjoint(U, R, L, S, lam, mode=oracle.DISCRETE)
    _, _, w = oracle.grid(M, S)
    grad = -2.0 * (L / N) * w[:, None] * oracle.curve_physical(G)
    X = oracle.curve_physical(U)
    h = 1e-6
    scale = np.linalg.norm(grad)
    for _ in range(64):
        dlt = np.array([[rng.normal() for _ in range(N)] for _ in range(M + 2)])
        dlt[0] = dlt[-1] = 0.0
        jp = J2(oracle.curve_spectral(X + h * dlt), L, S, lam)
        jm = J2(oracle.curve_spectral(X - h * dlt), L, S, lam)
        fd = (jp - jm) / (2 * h)
        an = np.sum(grad * dlt)
        assert abs(fd - an) <= 1e-7 * scale * np.linalg.norm(dlt), (fd, an)
    fdl = (J2(U, L, S, lam + h) - J2(U, L, S, lam - h)) / (2 * h)
    dl = oracle.curve_scalars(R, D, L, S, lam)["dJ2_dlambda"]
    assert abs(fdl - dl) <= 1e-7 * max(abs(dl), 1.0)


# ---------------------------------------------------------------- descent (P8) and trial curve

def test_descent_decreases_cost_monotonically():
    spec = gen.workload(0)[0]
    up, um = end_points(spec)
    amps, vp = perturbation(spec)
    U = oracle.curve_init(spec.M, spec.S, up, um, amps=amps, vp=vp)
    _, steps, sc, hist = oracle.curve_descend(U, spec.L, spec.S, 100, dtau=spec.dtau,
                                              mode=oracle.DISCRETE, history=True)
    J = hist[:, 2]
    assert steps == 100 and np.all(np.diff(J) < 0)
    assert J[-1] < 0.9 * J[0]
    assert abs(sc["J"] - J[-1]) < 1e-15 * J[-1]


def test_trial_curve_end_rows_and_center():
    N, L, M, S = 32, 22.0, 21, 2.2       # P = 22 is even: theta = pi/2 gives s = s0 = 0
    rng = np.random.default_rng(1)
    up, um = rng.standard_normal(N), rng.standard_normal(N)
    v = rng.standard_normal((2, N))
    U = oracle.curve_init(M, S, up, um, amps=[0.1, 0.2], vp=v)
    X = oracle.curve_physical(U)
    proj = lambda y: oracle.inv(oracle.fwd(y), N)      # the Nyquist mode is not represented
    assert np.allclose(X[0], proj(up), atol=1e-13) and np.allclose(X[-1], proj(um), atol=1e-13)
    center = 0.5 * (up + um) + 0.1 * np.sin(np.pi / 2) * v[0] + 0.2 * np.sin(np.pi) * v[1]
    assert np.allclose(X[(M + 1) // 2], proj(center), atol=1e-13)
    # tanh weighting away from the center
    _, s, _ = oracle.grid(M, S)
    m = 5
    t = np.tanh(s[m])
    th = m * np.pi / (M + 1)
    ref = 0.5 * ((1 + t) * up + (1 - t) * um) + 0.1 * np.sin(th) * v[0] + 0.2 * np.sin(2 * th) * v[1]
    assert np.allclose(X[m], proj(ref), atol=1e-13)


def test_single_section_residual_equals_the_curve_residual(small):
    M, N, L, S, U = small
    R, _ = oracle.curve_residual(U, L, S, 0.9)
    for j in (0, 1, 6, M, M + 1):
        assert np.abs(oracle.section_residual(U, j, L, S, 0.9) - R[j]).max() < 1e-13 * np.abs(R).max()
