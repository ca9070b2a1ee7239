"""KSCurve: a curve of KSE states joining two equilibria, held on the GPU.

PyTorch supplies the device memory (the workspace and the output tensors) and
the CUDA stream; every step of the method runs in libksconn.so.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _native
from ._native import KSParams, KSScalars, check, dptr

_PREC = {"fp64": _native.KS_FP64, "fp32": _native.KS_FP32, "bf16x2": _native.KS_BF16X2,
         "bf16x3": _native.KS_BF16X3}
_ADJ = {"paper": _native.KS_ADJ_PAPER, "discrete": _native.KS_ADJ_DISCRETE}
_CONV = {"jarc": _native.KS_CONV_JARC, "j": _native.KS_CONV_J, "jrel": _native.KS_CONV_JREL}
_STR = {"auto": 0, "dense": 1, "fft": 2, "dense_tc": 3, "fft4": 4, "fft4c": 5}
_FORM_NAME = {1: "dense", 2: "fft", 3: "dense_tc", 4: "fft4", 5: "fft4c"}
_LAUNCH = {"auto": 0, "kernels": 0, "persistent": 1}
_SCHEME = {"imex": _native.KS_SCHEME_IMEX, "implicit": _native.KS_SCHEME_IMPLICIT}


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class KSCurve:
    """One curve u(x_n, s_m), n < nx, m < ns (ns = M + 2 sections incl. both ends).

    Physical arrays exchanged with the curve are torch tensors [ns, nx] on the
    curve's device in its storage dtype (float64 for "fp64", float32 for "fp32").
    Row 0 is s = +inf (u_plus), row ns-1 is s = -inf (u_minus).
    symmetry: 1 holds every section odd, 2 holds it L/2-periodic, 3 both (the
    symmetric subspaces the descent preserves, Sec. V.B); adding 4 to an odd
    value (5, 7) also stores only the sine coefficients Im u^_j (half the field
    bytes and half the columns of every s-contraction; FP64 or FP32, nx >= 16,
    s_transform "auto", "dense", "fft", "fft4" or "fft4c").
    s_transform: how D_t is applied along s (same results to rounding): "auto"
    (the form measured fastest for the size), "dense", "dense_tc" (FP32, tensor
    cores), "fft" (one CTA per mode; four-step above its limit), "fft4" (four-step
    FFT, three launches), "fft4c" (four-step FFT, one clustered launch); the form
    in use is in `s_form`, the FFT length in `fft_length`.
    launch: "auto" / "kernels" run descent steps as kernels per phase (row phase
    and the two contractions; one launch for both contractions in the clustered
    form), "persistent" runs many steps of a dense-form curve in one cooperative
    kernel (same results; slower on GB300 at the sizes measured).
    scheme: "imex" takes only the diagonal term -a_j^2 u of G implicitly (stable
    while dtau rho(lambda^2 D_t^2) < 2); "implicit" every linear term of G,
    (lambda^2 D~^2 - a_j^2) u, through the eigenbases of the interior D_t^2 set
    up once at creation (Sec. V.C.3), which allows far larger dtau.
    """

    def __init__(self, L: float, nx: int, ns: int, S: float, u_plus, u_minus=None, *, s0: float = 0.0,
                 lam: float = 1.0, lambda_free: bool = False, dtau: float = 0.01, dtau_lambda: float = 0.0,
                 precision: str = "fp64", adjoint: str = "paper", conv: str = "jarc", u_init=None,
                 check_ends: bool = False, symmetry: int = 0, s_transform: str = "auto", launch: str = "auto",
                 scheme: str = "imex", device=None, stream: Optional[torch.cuda.Stream] = None):
        self.lib = _native.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.nx, self.ns, self.L, self.S = int(nx), int(ns), float(L), float(S)
        self.params = KSParams(L=L, nx=nx, ns=ns, S=S, s0=s0, lam=lam, lambda_free=int(bool(lambda_free)),
                               dtau=dtau, dtau_lambda=dtau_lambda, precision=_PREC[precision],
                               adjoint=_ADJ[adjoint], conv=_CONV[conv], check_ends=int(bool(check_ends)),
                               symmetry=int(symmetry), s_transform=_STR[s_transform],
                               launch=_LAUNCH[launch], scheme=_SCHEME[scheme])
        nbytes = self.lib.ks_curve_workspace_bytes(ctypes.byref(self.params))
        if nbytes == 0:
            raise _native.KSError(_native.KS_EINVAL, self.lib.ks_last_error().decode())
        self.workspace_bytes = int(nbytes)
        # length of the FFT that applies D_t along s (0: dense contraction)
        self.fft_length = int(self.lib.ks_curve_fft_length(ctypes.byref(self.params)))
        self.s_form = _FORM_NAME.get(int(self.lib.ks_curve_s_form(ctypes.byref(self.params))))
        # descent steps run as one persistent kernel (dense form) or as three kernels per step
        self.persistent = self.fft_length == 0 and _LAUNCH[launch] == 1
        self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        up = _f64(u_plus, nx)
        um = _f64(u_minus, nx) if u_minus is not None else np.zeros(nx)
        init_ptr = None
        if u_init is not None:
            u_init = self._as_curve_tensor(u_init)
            init_ptr = u_init.data_ptr()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.ks_curve_create(ctypes.byref(self.params), dptr(up), dptr(um), init_ptr,
                                           self._ws_ptr, self.workspace_bytes, self.stream.cuda_stream,
                                           ctypes.byref(h)))
        self.handle = h

    # ------------------------------------------------------------------ helpers
    def _as_curve_tensor(self, u):
        u = torch.as_tensor(u, device=self.device, dtype=self.dtype).contiguous()
        if tuple(u.shape) != (self.ns, self.nx):
            raise ValueError("expected a [%d, %d] curve, got %s" % (self.ns, self.nx, tuple(u.shape)))
        return u

    def _new(self):
        return torch.empty((self.ns, self.nx), dtype=self.dtype, device=self.device)

    def _live(self):
        if self.handle is None:
            raise RuntimeError("curve is closed")
        return self.handle

    # ------------------------------------------------------------------ API
    def init_trial(self, a: float = 0.0, v=None, amps=None, vp=None):
        """Trial curve of eq. KSE_initial_curve plus sum_p amps[p] sin((p+1) theta) vp[p](x)."""
        v = _f64(v, self.nx)
        amps = _f64(amps)
        npert = 0 if amps is None else int(amps.size)
        vp = _f64(vp, npert * self.nx) if npert else None
        check(self.lib.ks_curve_init_trial(self._live(), float(a), dptr(v), npert, dptr(amps), dptr(vp)))

    def residual(self) -> torch.Tensor:
        out = self._new()
        check(self.lib.ks_curve_residual(self._live(), out.data_ptr()))
        return out

    def cost(self):
        j2, ja = ctypes.c_double(), ctypes.c_double()
        check(self.lib.ks_curve_cost(self._live(), ctypes.byref(j2), ctypes.byref(ja)))
        return j2.value, ja.value

    def gradient(self, euclidean: bool = False):
        out = self._new()
        dl = ctypes.c_double()
        check(self.lib.ks_curve_gradient(self._live(), int(bool(euclidean)), out.data_ptr(), ctypes.byref(dl)))
        return out, dl.value

    def descend(self, nsteps: int, tol: float = 0.0, raise_on_notconv: bool = False):
        steps, J, Ja = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        st = self.lib.ks_curve_descend(self._live(), int(nsteps), float(tol), ctypes.byref(steps),
                                       ctypes.byref(J), ctypes.byref(Ja))
        allow = () if raise_on_notconv else (_native.KS_ENOTCONV,)
        check(st, allow=allow)
        return dict(steps=steps.value, J=J.value, J_arc=Ja.value, status=st)

    def descend_async(self, nsteps: int, tol: float = 0.0):
        check(self.lib.ks_curve_descend_async(self._live(), int(nsteps), float(tol)))

    def scalars(self) -> dict:
        s = KSScalars()
        check(self.lib.ks_curve_scalars(self._live(), ctypes.byref(s)))
        return s.as_dict()

    def get_state(self) -> torch.Tensor:
        out = self._new()
        check(self.lib.ks_curve_get_state(self._live(), out.data_ptr(), None, None))
        return out

    def get_lambda_tau(self):
        lam, tau = ctypes.c_double(), ctypes.c_double()
        check(self.lib.ks_curve_get_state(self._live(), None, ctypes.byref(lam), ctypes.byref(tau)))
        return lam.value, tau.value

    def set_state(self, u, lam: float = 1.0, tau: float = 0.0):
        """Asynchronous on the curve's stream (like the C call): u is read by the
        curve's kernels; on another stream than torch's current one its memory is
        kept from reuse until that stream has read it."""
        u = self._as_curve_tensor(u)
        check(self.lib.ks_curve_set_state(self._live(), u.data_ptr(), float(lam), float(tau)))
        if self.stream != torch.cuda.current_stream(self.device):
            u.record_stream(self.stream)

    def profile(self, max_steps: int):
        """Start (max_steps > 0) or stop (0) per-phase event timing of descent steps."""
        check(self.lib.ks_curve_profile(self._live(), int(max_steps)))

    def profile_read(self) -> dict:
        pr = _native.KSProfile()
        check(self.lib.ks_curve_profile_read(self._live(), ctypes.byref(pr)))
        names = ("rows", "dt_update", "dt_store")
        out = {n: dict(ms=pr.ms[i], launches=pr.launches[i]) for i, n in enumerate(names) if pr.launches[i]}
        if pr.step_launches:
            out["step"] = dict(ms=pr.step_ms, launches=pr.step_launches, steps=pr.step_steps)
        # three-launch four-step form: the passes of each contraction, timed one by one
        passes = {}
        for i, n in enumerate(("dt_update", "dt_store")):
            if pr.pass_launches[i][0]:
                passes[n] = [dict(ms=pr.pass_ms[i][q], launches=pr.pass_launches[i][q]) for q in range(3)]
        if passes:
            out["passes"] = passes
        if pr.impl_launches:
            out["implicit"] = dict(ms=pr.impl_ms, launches=pr.impl_launches)
        return out

    def debug_wait_limit(self, cycles: int):
        """Bound (clock cycles) of each kernel's first device-side mbarrier wait
        (0: the default; < 0: give up at once).  A test hook for the KS_ETIMEOUT
        path; ks_curve_init_trial restores the default."""
        check(self.lib.ks_curve_debug_wait_limit(self._live(), int(cycles)))

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.stream.synchronize()
            self.lib.ks_curve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
