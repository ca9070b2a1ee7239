"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.

Tolerances: FP64 results within 1e-10 relative (max-norm error over max-norm of
the oracle value, per field; plain relative error for scalars).  FP32 storage
with FP64 reductions: J within 1e-5 relative, fields within 1e-5 relative in
the 2-norm, both on the trial curve where J is far above the FP32 floor.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.curve import KSCurve
from tests.curves import end_points, perturbation

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def rel_max(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def rel_2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def make_pair(spec, precision="fp64", adjoint="paper", lam=1.0, lambda_free=False, dtau_lambda=0.0,
              s_transform="auto"):
    """GPU curve and oracle spectral curve of the same workload trial curve."""
    up, um = end_points(spec)
    amps, vp = perturbation(spec)
    c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, s0=spec.s0, lam=lam, lambda_free=lambda_free,
                dtau=spec.dtau, dtau_lambda=dtau_lambda, precision=precision, adjoint=adjoint,
                s_transform=s_transform)
    c.init_trial(0.0, None, amps, vp)
    U = oracle.curve_init(spec.M, spec.S, up, um, s0=spec.s0, amps=amps, vp=vp)
    return c, U


def precond_2(g_phys, G_spec, spec):
    """Relative 2-norm error of the gradient in the norm the descent applies it in:
    each Fourier mode weighted by dtau / (1 + dtau a_j^2) (Sec. V.C.3).  FP32
    rounding noise of the pseudo-spectral products reaches every mode of r and is
    amplified by k^4 in the adjoint's linear part; the semi-implicit step damps
    exactly those modes."""
    k = 2 * np.pi * np.arange(spec.N // 2) / spec.L
    a = k ** 4 - k ** 2
    pw = spec.dtau / (1.0 + spec.dtau * a * a)
    gh = np.fft.rfft(np.asarray(g_phys, dtype=np.float64), axis=1)[:, : spec.N // 2] / spec.N
    return rel_2(gh * pw[None, :], np.asarray(G_spec) * pw[None, :])


def assert_grad_close(g_phys, G_spec, U_spec, spec, tol):
    """G = -(Df)^T r - l s-term contains a_j^2 u^_j (through -a_j r^, a_j = k_j^4 - k_j^2),
    so a rounding-level difference eps |u| between the two sides' transforms of the
    same input curve reaches G amplified by a_j^2 (k^8).  The check is therefore:
      * the preconditioned direction dtau G_j / (1 + dtau a_j^2) that the descent
        applies (Sec. V.C.3), max-norm relative, within `tol`;
      * raw G within tol + 8 eps a_max^2 max|u| / max|G| (its conditioning)."""
    k = 2 * np.pi * np.arange(spec.N // 2) / spec.L
    a = k ** 4 - k ** 2
    pw = spec.dtau / (1.0 + spec.dtau * a * a)
    g = np.asarray(g_phys, dtype=np.float64)
    gh = np.fft.rfft(g, axis=1)[:, : spec.N // 2] / spec.N
    assert rel_max(gh * pw[None, :], np.asarray(G_spec) * pw[None, :]) < tol
    Gp = oracle.curve_physical(G_spec)
    eps = np.finfo(g.dtype).eps if g.dtype == np.float64 else 2.0 ** -52
    umax = np.abs(oracle.curve_physical(U_spec)).max()
    cond = 8 * eps * a.max() ** 2 * umax / max(np.abs(Gp).max(), 1e-300)
    assert rel_max(g, Gp) < tol + cond


def oracle_eval(U, spec, lam=1.0, mode=oracle.PAPER):
    R, D = oracle.curve_residual(U, spec.L, spec.S, lam)
    G, _ = oracle.curve_adjoint(U, R, spec.L, spec.S, lam, mode=mode)
    sc = oracle.curve_scalars(R, D, spec.L, spec.S, lam, G=G)
    return R, D, G, sc


@pytest.fixture(scope="module")
def cfg0():
    return gen.workload(0)[0]


@pytest.mark.parametrize("s_transform", ["dense", "fft"])
@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
def test_single_evaluation_fp64(cfg0, adjoint, s_transform):
    spec = cfg0
    mode = oracle.PAPER if adjoint == "paper" else oracle.DISCRETE
    c, U = make_pair(spec, adjoint=adjoint, s_transform=s_transform)
    assert rel_max(c.get_state().cpu().numpy(), oracle.curve_physical(U)) < 1e-13
    R, D, G, sc = oracle_eval(U, spec, mode=mode)
    r = c.residual().cpu().numpy()
    assert rel_max(r, oracle.curve_physical(R)) < TOL64
    J2, Ja = c.cost()
    assert abs(J2 - sc["J2"]) < TOL64 * sc["J2"]
    assert abs(Ja - sc["J_arc"]) < TOL64 * sc["J_arc"]
    g, dl = c.gradient(euclidean=False)
    assert_grad_close(g.cpu().numpy(), G, U, spec, TOL64)
    assert abs(dl - sc["dJ2_dlambda"]) < TOL64 * abs(sc["dJ2_dlambda"])
    s = c.scalars()
    assert abs(s["G_norm"] ** 2 - sc["G2"]) < TOL64 * sc["G2"]
    assert abs(s["Dnorm"] - sc["Dnorm"]) < TOL64 * sc["Dnorm"]
    c.close()


def test_euclidean_gradient_fp64(cfg0):
    spec = cfg0
    c, U = make_pair(spec, adjoint="paper")
    R, D = oracle.curve_residual(U, spec.L, spec.S)
    Gd, _ = oracle.curve_adjoint(U, R, spec.L, spec.S, mode=oracle.DISCRETE)
    _, _, w = oracle.grid(spec.M, spec.S)
    g, _ = c.gradient(euclidean=True)
    gd = g.cpu().numpy()
    scale = np.zeros_like(w)
    scale[1:-1] = 1.0 / (-2.0 * (spec.L / spec.N) * w[1:-1])
    assert np.all(gd[0] == 0) and np.all(gd[-1] == 0)
    assert_grad_close(gd * scale[:, None], Gd, U, spec, TOL64)
    c.close()


@pytest.mark.parametrize("adjoint,s_transform", [("paper", "dense"), ("paper", "fft"), ("discrete", "fft")])
def test_descent_2000_steps_fp64(cfg0, adjoint, s_transform):
    """cfg 0 end to end: 2000 semi-implicit descent steps from the same trial curve."""
    spec = cfg0
    mode = oracle.PAPER if adjoint == "paper" else oracle.DISCRETE
    c, U = make_pair(spec, adjoint=adjoint, s_transform=s_transform)
    Uo, steps_o, sco, _ = oracle.curve_descend(U, spec.L, spec.S, spec.steps, dtau=spec.dtau, mode=mode)
    out = c.descend(spec.steps)
    assert out["steps"] == steps_o == spec.steps
    assert rel_max(c.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < TOL64
    assert abs(out["J"] - sco["J"]) < TOL64 * sco["J"]
    assert abs(out["J_arc"] - sco["J_arc"]) < TOL64 * sco["J_arc"]
    s = c.scalars()
    assert abs(s["tau"] - spec.steps * spec.dtau) < 1e-9 and s["step"] == spec.steps
    c.close()


def test_descent_with_free_lambda_fp64(cfg0):
    spec = cfg0
    c, U = make_pair(spec, adjoint="discrete", lam=1.0, lambda_free=True, dtau_lambda=0.05)
    Uo, _, sco, _ = oracle.curve_descend(U, spec.L, spec.S, 300, dtau=spec.dtau, lam=1.0, lambda_free=True,
                                         dtau_lambda=0.05, mode=oracle.DISCRETE)
    out = c.descend(300)
    lam, _ = c.get_lambda_tau()
    assert abs(lam - sco["lam"]) < TOL64 * abs(sco["lam"]) and abs(lam - 1.0) > 1e-6
    assert rel_max(c.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < TOL64
    assert abs(out["J"] - sco["J"]) < TOL64 * sco["J"]
    c.close()


def test_descent_stops_at_tolerance(cfg0):
    spec = cfg0
    c, U = make_pair(spec)
    _, _, _, hist = oracle.curve_descend(U, spec.L, spec.S, 60, dtau=spec.dtau, history=True)
    tol = 0.5 * (hist[40, 3] + hist[41, 3])        # between J_arc after 40 and 41 steps
    Uo, steps_o, sco, _ = oracle.curve_descend(U, spec.L, spec.S, 1000, dtau=spec.dtau, tol=tol)
    out = c.descend(1000, tol=tol)
    assert steps_o == 41 and out["steps"] == 41
    assert abs(out["J_arc"] - sco["J_arc"]) < TOL64 * sco["J_arc"]
    assert c.scalars()["converged"] == 1
    c.close()


@pytest.mark.parametrize("s_transform", ["dense", "fft"])
def test_fp32_matches_fp64_oracle(cfg0, s_transform):
    spec = cfg0
    c, U = make_pair(spec, precision="fp32", s_transform=s_transform)
    R, D, G, sc = oracle_eval(U, spec)
    J2, Ja = c.cost()
    assert abs(np.sqrt(J2) - np.sqrt(sc["J2"])) < TOL32 * np.sqrt(sc["J2"])
    assert abs(Ja - sc["J_arc"]) < TOL32 * sc["J_arc"]
    assert rel_2(c.residual().double().cpu().numpy(), oracle.curve_physical(R)) < TOL32
    g, _ = c.gradient()
    assert precond_2(g.double().cpu().numpy(), G, spec) < TOL32
    c.close()


@pytest.mark.parametrize("s_transform", ["dense", "fft"])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_config1_single_evaluation(precision, tol, s_transform):
    """N_x = 64, N_s = 1024 (the differentiation workload): one evaluation."""
    spec = gen.workload(1)[0]
    c, U = make_pair(spec, precision=precision, s_transform=s_transform)
    R, D, G, sc = oracle_eval(U, spec)
    J2, Ja = c.cost()
    assert abs(np.sqrt(J2) - np.sqrt(sc["J2"])) < tol * np.sqrt(sc["J2"])
    assert abs(Ja - sc["J_arc"]) < tol * sc["J_arc"]
    g, _ = c.gradient()
    if precision == "fp64":
        assert rel_max(c.residual().cpu().numpy(), oracle.curve_physical(R)) < tol
        assert_grad_close(g.cpu().numpy(), G, U, spec, tol)
    else:
        assert rel_2(c.residual().double().cpu().numpy(), oracle.curve_physical(R)) < tol
        assert precond_2(g.double().cpu().numpy(), G, spec) < tol
    c.close()


@pytest.mark.parametrize("s_transform", ["dense", "fft"])
@pytest.mark.parametrize("N,Ns", [(8, 3), (8, 16), (16, 37), (32, 33), (64, 65), (128, 31), (256, 20), (32, 129),
                                  (16, 2053)])   # the last: row tiles by TMA, ragged last tile
def test_edge_shapes_fp64(N, Ns, s_transform):
    """Smallest curve (one interior section), ragged N_s (odd, not a tile multiple),
    every supported N_x, on a random smooth curve; includes 20 descent steps."""
    L, S = 22.0 + N / 16.0, max(0.5, 0.1 * (Ns - 1))
    rng = np.random.default_rng(N * 1000 + Ns)
    X = np.zeros((Ns, N))
    x = np.arange(N) * L / N
    for m in range(Ns):
        for j in range(1, min(5, N // 2)):
            X[m] += 0.5 * rng.standard_normal() * np.sin(2 * np.pi * j * x / L + rng.uniform(0, 6.28))
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X), s_transform=s_transform)
    U = oracle.curve_spectral(X)
    spec = gen.CurveSpec(0, 0, L, N, Ns, S)
    R, D, G, sc = oracle_eval(U, spec)
    assert rel_max(c.residual().cpu().numpy(), oracle.curve_physical(R)) < TOL64
    g, _ = c.gradient()
    assert_grad_close(g.cpu().numpy(), G, U, spec, TOL64)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 20, dtau=1e-3)
    c2 = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=torch.from_numpy(X), dtau=1e-3, s_transform=s_transform)
    out = c2.descend(20)
    assert rel_max(c2.get_state().cpu().numpy(), oracle.curve_physical(Uo)) < TOL64
    assert abs(out["J"] - sco["J"]) < TOL64 * max(sco["J"], 1e-300)
    c.close()
    c2.close()


def test_descent_is_deterministic_and_resumable(cfg0):
    """Fixed reduction order: two identical runs agree bit for bit; a run resumed
    from get_state/set_state (a physical round trip, exact to rounding) agrees
    with the uninterrupted run to 1e-12."""
    spec = cfg0
    a, _ = make_pair(spec)
    b, _ = make_pair(spec)
    a.descend(80)
    b.descend(80)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.scalars()["J"] == b.scalars()["J"]
    c, _ = make_pair(spec)
    c.descend(50)
    u = c.get_state().clone()
    lam, tau = c.get_lambda_tau()
    d, _ = make_pair(spec)
    d.set_state(u, lam, tau)
    d.descend(30)
    assert rel_max(d.get_state().cpu().numpy(), a.get_state().cpu().numpy()) < 1e-12
    assert abs(d.get_lambda_tau()[1] - 80 * spec.dtau) < 1e-12
    for x in (a, b, c, d):
        x.close()


@pytest.mark.parametrize("N,Ns,L", [(64, 1024, 22.0), (256, 600, 100.0)])
def test_set_state_fp32_matches_the_fp64_transform(N, Ns, L):
    """FP32 storage: set_state transforms its input in double-float arithmetic;
    the state it makes equals, to one FP32 rounding per coefficient, the state
    that create's FP64 transform makes of the same curve, so J (whose linear term
    weighs each coefficient by a_j ~ k_j^4) agrees to 1e-6 relative (an FP32
    transform in set_state put J of the autograd test's curve 3.6e-4 off)."""
    rng = np.random.default_rng(N + Ns)
    x = np.arange(N) * L / N
    th = np.arange(Ns) * np.pi / (Ns - 1)
    X = np.zeros((Ns, N))
    for j in range(1, N // 2):   # a spectrum decaying over the whole range of modes
        a, b = rng.standard_normal(2) * np.exp(-0.35 * j)
        X += np.outer(0.5 + np.sin(th * (1 + j % 3)), a * np.cos(2 * np.pi * j * x / L) + b * np.sin(2 * np.pi * j * x / L))
    X = X.astype(np.float32).astype(np.float64)
    xt = torch.from_numpy(X).float()
    S = 0.1 * (Ns - 1)
    c = KSCurve(L, N, Ns, S, X[0], X[-1], u_init=xt, precision="fp32")
    d = KSCurve(L, N, Ns, S, X[0], X[-1], precision="fp32")
    d.set_state(xt.cuda(), 1.0, 0.0)
    (J2c, Jac), (J2d, Jad) = c.cost(), d.cost()
    gc, gd = c.gradient()[0].double().cpu().numpy(), d.gradient()[0].double().cpu().numpy()
    e = dict(J2=abs(J2d - J2c) / J2c, J_arc=abs(Jad - Jac) / Jac, g=rel_2(gd, gc),
             u=rel_max(d.get_state().double().cpu().numpy(), c.get_state().double().cpu().numpy()))
    print("SET_STATE fp32 N=%d Ns=%d: %s" % (N, Ns, " ".join("%s=%.2e" % kv for kv in e.items())))
    assert e["J2"] < 1e-6 and e["J_arc"] < 1e-6 and e["g"] < 1e-6 and e["u"] < 1e-6
    c.close()
    d.close()


@pytest.mark.parametrize("s_transform", ["dense", "fft"])
@pytest.mark.parametrize("sym", [1, 3])
def test_symmetric_subspace_is_held_exactly(sym, s_transform):
    """Sections restricted to odd (and L/2-periodic) fields keep exactly zero
    coefficients outside the subspace and agree with the oracle's unrestricted
    descent, whose off-subspace coefficients stay at rounding level (Sec. V.B)."""
    from paper_2301_11704_gb300 import replay
    M, S, N, L = 60, 6.1, 32, 22.0
    e2 = replay.equilibrium("E2", 64, L)[::2]          # E2 on the N = 32 grid
    up, um = e2, np.zeros(N)
    c = KSCurve(L, N, M + 2, S, up, um, symmetry=sym, s_transform=s_transform)
    U = oracle.curve_init(M, S, up, um)
    Uo, _, sco, _ = oracle.curve_descend(U, L, S, 100, dtau=0.01)
    out = c.descend(100)
    x = c.get_state().cpu().numpy()
    h = np.fft.rfft(x, axis=1)[:, : N // 2]
    assert np.abs(h.real).max() < 1e-12 * np.abs(h).max()         # odd: cosine parts vanish
    if sym & 2:
        assert np.abs(h[:, 1::2]).max() < 1e-12 * np.abs(h).max()  # L/2-periodic: odd modes vanish
    xo = oracle.curve_physical(Uo)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()
    assert abs(out["J_arc"] - sco["J_arc"]) <= 1e-10 * sco["J_arc"]
    c.close()
