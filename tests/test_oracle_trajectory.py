"""Trajectory pin: a curve sampled from a finely time-stepped KS trajectory is
(nearly) an integral curve, so its residual r = f(u) - du/ds is nearly zero
(Sec. II: J = 0 exactly on a connecting orbit).

Inside the subspace U of odd, L/2-periodic fields (even-j sine modes) at
L = 22, the trivial equilibrium E0 has a single unstable direction, sin(4 pi x/L)
with eigenvalue k_2^2 - k_2^4 = 0.2198 (Table tab:KSE_eigenvals).  Its unstable
manifold is a one-dimensional trajectory that leaves E0 and settles on an
equilibrium of U (E2, which is odd and L/2-periodic, Sec. V.D).  Sampling that
trajectory at s_m and measuring J with the oracle pins f, D_t and the
quadrature together: a wrong sign, factor or index anywhere gives J_rel = O(1).
The time stepper itself is pinned first against the exact linear solution and
its fourth-order convergence.
"""
import numpy as np
import pytest

import oracle

N, L = 32, 22.0
K2 = 2 * np.pi * 2 / L
LAM2 = K2 ** 2 - K2 ** 4          # 0.2198
SYM = 3                           # odd and L/2-periodic


def _mode2(eps):
    uh = np.zeros(N // 2, complex)
    uh[2] = -0.5j * eps           # eps sin(4 pi x / L)
    return uh


def test_time_stepper_reproduces_linear_growth():
    eps, T = 1e-10, 12.0
    out = oracle.ks_integrate(_mode2(eps), N, L, T, 5e-3, SYM)
    assert abs(out[2] / _mode2(eps)[2] - np.exp(LAM2 * T)) < 1e-8 * np.exp(LAM2 * T)
    assert np.abs(np.delete(out, 2)).max() < 1e-18


def test_time_stepper_is_fourth_order():
    rng = np.random.default_rng(0)
    uh = np.zeros(N // 2, complex)
    uh[1:6] = 1j * rng.standard_normal(5) * 0.3
    ref = oracle.ks_integrate(uh, N, L, 2.0, 1e-3, 1)
    e1 = np.abs(oracle.ks_integrate(uh, N, L, 2.0, 0.04, 1) - ref).max()
    e2 = np.abs(oracle.ks_integrate(uh, N, L, 2.0, 0.02, 1) - ref).max()
    assert 12 < e1 / e2 < 20


@pytest.fixture(scope="module")
def trajectory():
    """Integrate until |f(u)| stops falling: the discrete scheme's own fixed point
    sits O(dt^4) away from f = 0 (about 1e-8 here)."""
    eps, dt, chunk = 1e-6, 1e-3, 1.0
    cur, t = _mode2(eps), 0.0
    ts, vs = [], []
    while t < 600.0:
        cur = oracle.ks_integrate(cur, N, L, chunk, dt, SYM)
        t += chunk
        v = np.linalg.norm(oracle.inv(oracle.rhs(cur, N, L), N))
        ts.append(t)
        vs.append(v)
        if t > 100.0 and v > 0.9 * vs[-11]:
            break
    return dict(eps=eps, dt=dt, t_end=t, t_peak=ts[int(np.argmax(vs))], u_end=cur, v_end=vs[-1])


def test_trajectory_settles_on_an_equilibrium_of_the_subspace(trajectory):
    u = trajectory["u_end"]
    assert trajectory["v_end"] < 1e-7
    assert np.abs(u.real).max() < 1e-15 and np.abs(u[1::2]).max() < 1e-15
    assert np.abs(oracle.inv(u, N)).max() > 1.0
    b, it, res = oracle.newton_odd(-2.0 * u[1:].imag, N, L, maxit=20, tol=1e-13)
    assert it >= 0 and res < 1e-13
    assert np.abs(oracle.odd_to_spec(b, N) - u).max() < 1e-7


def test_sampled_trajectory_has_near_zero_cost(trajectory):
    M, S = 200, 15.0
    s0 = trajectory["t_peak"]
    th, s, _ = oracle.grid(M, S, s0)
    U = np.zeros((M + 2, N // 2), complex)
    U[0] = trajectory["u_end"]          # s -> +inf
    U[-1] = 0.0                         # s -> -inf: E0
    start = _mode2(trajectory["eps"])
    cur, tc = start.copy(), 0.0
    for m in sorted(range(1, M + 1), key=lambda i: s[i]):
        sm = s[m]
        if sm <= 0.0:                   # before the start: linear growth out of E0
            U[m] = start * np.exp(LAM2 * sm)
        elif sm >= trajectory["t_end"]:
            U[m] = trajectory["u_end"]
        else:
            cur = oracle.ks_integrate(cur, N, L, sm - tc, trajectory["dt"], SYM)
            tc = sm
            U[m] = cur
    R, D = oracle.curve_residual(U, L, S)
    sc = oracle.curve_scalars(R, D, L, S)
    J_rel = np.sqrt(sc["J2"]) / sc["Dnorm"]
    assert J_rel < 1e-5, J_rel
    # the same curve with the s-derivative sign flipped is far from an orbit
    R2, D2 = oracle.curve_residual(U, L, S, -1.0)
    sc2 = oracle.curve_scalars(R2, D2, L, S, -1.0)
    assert np.sqrt(sc2["J2"]) / sc2["Dnorm"] > 1.0
