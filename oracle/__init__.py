"""FP64 CPU oracle for the adjoint-descent step (Ashtari & Schneider, arXiv 2301.11704).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path in ``paper_2301_11704_gb300``: the arithmetic lives in plain C
(``ks_oracle.c``: naive DFT sums, the two explicit trig sums that define the
rational-Chebyshev derivative, explicit loops), compiled with gcc, and this
module only marshals numpy arrays in and out.

Layout conventions (Sec. V.C.1):
  * a time section is N/2 complex Fourier coefficients u^_j, j = 0..N/2-1
    (the Nyquist coefficient is held at zero);
  * a curve is a complex array [M+2, N/2]; row 0 is s -> +inf (u_+), row M+1
    is s -> -inf (u_-).

Pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "libks_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ks_oracle.c with gcc (plain C11 + OpenMP) into oracle/_build."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        p = ctypes.c_void_p
        sig = {
            "ko_version": (i, []),
            "ko_num_threads": (i, []),
            "ko_fwd": (None, [i, p, p]),
            "ko_inv": (None, [i, p, p]),
            "ko_rhs": (None, [i, d, p, p]),
            "ko_jac_apply": (None, [i, d, p, p, p]),
            "ko_jac_adjoint_apply": (None, [i, d, p, p, p]),
            "ko_grid": (None, [i, d, d, p, p, p]),
            "ko_dt_coeffs": (None, [i, p, p]),
            "ko_dt_apply": (None, [i, d, p, p]),
            "ko_dtT_apply": (None, [i, d, p, p]),
            "ko_dt_matrix": (None, [i, d, p]),
            "ko_dt_row": (None, [i, d, i, p]),
            "ko_curve_residual": (None, [i, i, d, d, d, p, p, p]),
            "ko_curve_rhs": (None, [i, i, d, p, p]),
            "ko_curve_linearised": (None, [i, i, d, d, d, p, p, p]),
            "ko_curve_adjoint": (None, [i, i, d, d, d, i, p, p, p, p]),
            "ko_curve_scalars": (None, [i, i, d, d, d, p, p, p, p]),
            "ko_curve_norm2_W": (d, [i, i, d, d, p]),
            "ko_curve_descend": (l, [i, i, d, d, d, i, d, d, i, i, l, d, i, p, p, p]),
            "ko_implicit_update": (None, [i, i, d, d, d, d, p, p]),
            "ko_curve_init": (None, [i, i, d, d, p, p, d, p, i, p, p, p]),
            "ko_newton_odd": (i, [i, d, p, i, d, p]),
            "ko_jacobian_zero_mean": (None, [i, d, p, p]),
            "ko_ks_integrate": (None, [i, d, p, d, d, i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().ko_num_threads())


# ----------------------------------------------------------------------------
# Fourier direction
# ----------------------------------------------------------------------------

def fwd(u):
    """Physical section u[N] -> spectral u^[N/2] (forward DFT with 1/N)."""
    u = _c(u, np.float64)
    N = u.shape[-1]
    out = np.empty(N // 2, np.complex128)
    _load().ko_fwd(N, _ptr(u), _ptr(out))
    return out


def inv(uh, N):
    """Spectral u^[N/2] -> physical section u[N]."""
    uh = _c(uh, np.complex128)
    out = np.empty(N, np.float64)
    _load().ko_inv(N, _ptr(uh), _ptr(out))
    return out


def rhs(uh, N, L):
    """KSE right-hand side f(u) of one section, spectral in and out."""
    uh = _c(uh, np.complex128)
    out = np.empty(N // 2, np.complex128)
    _load().ko_rhs(N, L, _ptr(uh), _ptr(out))
    return out


def jac_apply(uh, vh, N, L):
    uh, vh = _c(uh, np.complex128), _c(vh, np.complex128)
    out = np.empty(N // 2, np.complex128)
    _load().ko_jac_apply(N, L, _ptr(uh), _ptr(vh), _ptr(out))
    return out


def jac_adjoint_apply(uh, rh, N, L):
    uh, rh = _c(uh, np.complex128), _c(rh, np.complex128)
    out = np.empty(N // 2, np.complex128)
    _load().ko_jac_adjoint_apply(N, L, _ptr(uh), _ptr(rh), _ptr(out))
    return out


# ----------------------------------------------------------------------------
# Temporal direction
# ----------------------------------------------------------------------------

def grid(M, S, s0=0.0):
    """(theta, s, w) on the M+2 rational-Chebyshev points."""
    th, s, w = (np.empty(M + 2) for _ in range(3))
    _load().ko_grid(M, S, s0, _ptr(th), _ptr(s), _ptr(w))
    return th, s, w


def dt_coeffs(q):
    q = _c(q, np.float64)
    M = q.shape[0] - 2
    out = np.empty(M + 2)
    _load().ko_dt_coeffs(M, _ptr(q), _ptr(out))
    return out


def dt_apply(q, S):
    q = _c(q, np.float64)
    M = q.shape[0] - 2
    out = np.empty(M + 2)
    _load().ko_dt_apply(M, S, _ptr(q), _ptr(out))
    return out


def dtT_apply(y, S):
    y = _c(y, np.float64)
    M = y.shape[0] - 2
    out = np.empty(M + 2)
    _load().ko_dtT_apply(M, S, _ptr(y), _ptr(out))
    return out


def dt_row(M, S, j):
    """Row j of the D_t matrix, entry by entry from its explicit k-sum."""
    out = np.empty(M + 2)
    _load().ko_dt_row(M, S, int(j), _ptr(out))
    return out


def section_residual(U, j, L, S, lam=1.0):
    """Residual of section j alone: f(u_j) - lam sum_m D_t[j, m] u_m, with the
    row of D_t from its explicit sum (for sampled checks of large curves)."""
    U = _c(U, np.complex128)
    M, N = U.shape[0] - 2, 2 * U.shape[1]
    if j == 0 or j == M + 1:
        return np.zeros(N // 2, np.complex128)
    return rhs(U[j], N, L) - lam * (dt_row(M, S, j) @ U)


def dt_matrix(M, S):
    out = np.empty((M + 2, M + 2))
    _load().ko_dt_matrix(M, S, _ptr(out))
    return out


# ----------------------------------------------------------------------------
# Curve
# ----------------------------------------------------------------------------

def _curve(U):
    U = _c(U, np.complex128)
    return U, U.shape[0] - 2, 2 * U.shape[1]


def curve_residual(U, L, S, lam=1.0):
    """Returns (R, Dtu): residual r^ and D_t u^ (without lambda)."""
    U, M, N = _curve(U)
    R, D = np.empty_like(U), np.empty_like(U)
    _load().ko_curve_residual(M, N, L, S, lam, _ptr(U), _ptr(R), _ptr(D))
    return R, D


def curve_rhs(U, L):
    U, M, N = _curve(U)
    F = np.empty_like(U)
    _load().ko_curve_rhs(M, N, L, _ptr(U), _ptr(F))
    return F


def curve_linearised(U, G, L, S, lam=1.0):
    U, M, N = _curve(U)
    G = _c(G, np.complex128)
    out = np.empty_like(U)
    _load().ko_curve_linearised(M, N, L, S, lam, _ptr(U), _ptr(G), _ptr(out))
    return out


PAPER, DISCRETE = 0, 1


def curve_adjoint(U, R, L, S, lam=1.0, mode=PAPER):
    """Returns (G, A): descent direction G = -L^dagger(u;r) and spatial part (Df)^T r."""
    U, M, N = _curve(U)
    R = _c(R, np.complex128)
    G, A = np.empty_like(U), np.empty_like(U)
    _load().ko_curve_adjoint(M, N, L, S, lam, mode, _ptr(U), _ptr(R), _ptr(G), _ptr(A))
    return G, A


def curve_scalars(R, Dtu, L, S, lam=1.0, G=None):
    """dict(J2, J_arc, dJ2_dlambda, G2, Dnorm)."""
    R, M, N = _curve(R)
    Dtu = _c(Dtu, np.complex128)
    G = None if G is None else _c(G, np.complex128)
    out = np.zeros(5)
    _load().ko_curve_scalars(M, N, L, S, lam, _ptr(R), _ptr(Dtu), _ptr(G), _ptr(out))
    return dict(J2=out[0], J_arc=out[1], dJ2_dlambda=out[2], G2=out[3], Dnorm=out[4])


def curve_norm2_W(X, L, S):
    X, M, N = _curve(X)
    return float(_load().ko_curve_norm2_W(M, N, L, S, _ptr(X)))


CONV_JARC, CONV_J, CONV_JREL = 0, 1, 2


IMEX_X, IMPLICIT = 0, 1


def curve_descend(U, L, S, nsteps, dtau=0.01, lam=1.0, lambda_free=False, dtau_lambda=0.0,
                  mode=PAPER, tol=0.0, conv=CONV_JARC, history=False, scheme=IMEX_X):
    """Runs the descent in place on a copy of U.  scheme IMEX_X takes only the
    diagonal -a_j^2 u term of G implicitly; IMPLICIT every linear term
    (lambda^2 Dt~^2 - a_j^2) u, by a dense LU solve per spatial mode.

    Returns (U_final, steps_done, scalars dict, history array [steps+1, 6] or None).
    """
    U, M, N = _curve(U)
    U = U.copy()
    hist = np.zeros((nsteps + 1, 6)) if history else None
    out = np.zeros(5)
    steps = _load().ko_curve_descend(M, N, L, S, lam, int(bool(lambda_free)), dtau, dtau_lambda,
                                     mode, int(scheme), int(nsteps), tol, conv, _ptr(U), _ptr(hist), _ptr(out))
    sc = dict(J=out[0], J_arc=out[1], dJ2_dlambda=out[2], G=out[3], lam=out[4])
    if hist is not None:
        hist = hist[: steps + 1]
    return U, int(steps), sc, hist


def implicit_update(U, G, L, S, dtau, lam=1.0):
    """One full-linear-implicit increment of the interior rows of a copy of U:
    (I (1 + dtau a_j^2) - dtau lam^2 Dt~^2) delta_j = dtau G_j, U + delta."""
    U, M, N = _curve(U)
    U = U.copy()
    G = _c(G, np.complex128)
    _load().ko_implicit_update(M, N, L, S, dtau, lam, _ptr(G), _ptr(U))
    return U


def curve_init(M, S, up, um, s0=0.0, a=0.0, v=None, amps=None, vp=None):
    """Trial curve of eq. KSE_initial_curve (+ optional perturbation sum), spectral."""
    up, um = _c(up, np.float64), _c(um, np.float64)
    N = up.shape[0]
    v = None if v is None else _c(v, np.float64)
    npert = 0 if amps is None else len(amps)
    amps = None if amps is None else _c(amps, np.float64)
    vp = None if vp is None else _c(vp, np.float64)
    U = np.empty((M + 2, N // 2), np.complex128)
    _load().ko_curve_init(M, N, S, s0, _ptr(up), _ptr(um), a, _ptr(v), npert, _ptr(amps), _ptr(vp),
                          _ptr(U))
    return U


def curve_physical(U):
    """Spectral curve [M+2, N/2] -> physical [M+2, N] (row by row, naive DFT)."""
    U, M, N = _curve(U)
    return np.stack([inv(U[m], N) for m in range(M + 2)])


def curve_spectral(X):
    """Physical curve [M+2, N] -> spectral [M+2, N/2]."""
    X = _c(X, np.float64)
    return np.stack([fwd(X[m]) for m in range(X.shape[0])])


# ----------------------------------------------------------------------------
# Equilibria and time stepping
# ----------------------------------------------------------------------------

def newton_odd(b0, N, L, maxit=100, tol=1e-12):
    """Damped Newton for f(u)=0 in the odd subspace; returns (b, iters, resnorm)."""
    b = _c(b0, np.float64).copy()
    assert b.shape[0] == N // 2 - 1
    res = ctypes.c_double(0.0)
    it = _load().ko_newton_odd(N, L, _ptr(b), maxit, tol, ctypes.byref(res))
    return b, int(it), float(res.value)


def odd_to_spec(b, N):
    """Sine coefficients b_j (j=1..N/2-1) -> spectral section."""
    uh = np.zeros(N // 2, np.complex128)
    uh[1:] = -0.5j * np.asarray(b)
    return uh


def jacobian_zero_mean(uh, N, L):
    uh = _c(uh, np.complex128)
    out = np.empty((N - 2, N - 2))
    _load().ko_jacobian_zero_mean(N, L, _ptr(uh), _ptr(out))
    return out


def ks_integrate(uh, N, L, T, dt, sym=0):
    uh = _c(uh, np.complex128).copy()
    _load().ko_ks_integrate(N, L, _ptr(uh), T, dt, sym)
    return uh
