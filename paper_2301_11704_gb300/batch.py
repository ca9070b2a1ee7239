"""KSBatch: many independent curves (uneven N_s, N, L) descending together on
one GPU through the batched C ABI (ks_batch_*)."""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _native
from ._native import KSParams, KSScalars, check, dptr

_PREC = {"fp64": _native.KS_FP64, "fp32": _native.KS_FP32}
_ADJ = {"paper": _native.KS_ADJ_PAPER, "discrete": _native.KS_ADJ_DISCRETE}
_CONV = {"jarc": _native.KS_CONV_JARC, "j": _native.KS_CONV_J, "jrel": _native.KS_CONV_JREL}
_STR = {"auto": 0, "dense": 1, "fft": 2}
_SCHEME = {"imex": _native.KS_SCHEME_IMEX, "implicit": _native.KS_SCHEME_IMPLICIT}


class KSBatch:
    """specs: sequence of objects with L, N, Ns, S, s0, dtau (e.g. gen.CurveSpec);
    u_plus / u_minus: per-curve physical end sections.  scheme "implicit" steps
    every curve with all linear terms of G implicit (its eigenbases are set up
    at creation, in parallel host threads); dtau, when given, replaces every
    spec's dtau.  symmetry: one value for every curve, or one per curve (the
    subspaces of KSCurve; 5 and 7 store only the sine coefficients)."""

    def __init__(self, specs: Sequence, u_plus, u_minus, *, precision="fp32", adjoint="paper", conv="jrel",
                 s_transform="auto", scheme="imex", dtau=None, symmetry=0, device=None, stream=None):
        self.lib = _native.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.specs = list(specs)
        self.nb = len(self.specs)
        arr = (KSParams * self.nb)()
        syms = [int(symmetry)] * self.nb if np.ndim(symmetry) == 0 else [int(v) for v in symmetry]
        for i, s in enumerate(self.specs):
            arr[i] = KSParams(L=s.L, nx=s.N, ns=s.Ns, S=s.S, s0=getattr(s, "s0", 0.0), lam=1.0, lambda_free=0,
                              dtau=s.dtau if dtau is None else dtau, dtau_lambda=0.0, precision=_PREC[precision],
                              adjoint=_ADJ[adjoint], conv=_CONV[conv], check_ends=0, symmetry=syms[i],
                              s_transform=_STR[s_transform], launch=0, scheme=_SCHEME[scheme])
        self.params = arr
        nbytes = self.lib.ks_batch_workspace_bytes(self.nb, arr)
        if nbytes == 0:
            raise _native.KSError(_native.KS_EINVAL, self.lib.ks_last_error().decode())
        self.workspace_bytes = int(nbytes)
        self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        ptr = (self._ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        up = np.ascontiguousarray(np.concatenate([np.asarray(u, dtype=np.float64) for u in u_plus]))
        um = np.ascontiguousarray(np.concatenate([np.asarray(u, dtype=np.float64) for u in u_minus]))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.ks_batch_create(self.nb, arr, dptr(up), dptr(um), ptr, self.workspace_bytes,
                                           self.stream.cuda_stream, ctypes.byref(h)))
        self.handle = h

    def init_trial(self, amps, vps):
        """amps [nb][npert]; vps: per curve an array [npert, N_i]."""
        amps = np.ascontiguousarray(np.asarray(amps, dtype=np.float64))
        npert = amps.shape[1] if amps.ndim == 2 else 0
        vp = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in vps]))
        check(self.lib.ks_batch_init_trial(self.handle, npert, dptr(amps), dptr(vp)))

    def descend(self, nsteps: int, tol: float = 0.0):
        steps = (ctypes.c_int64 * self.nb)()
        J = np.zeros(self.nb)
        Ja = np.zeros(self.nb)
        st = self.lib.ks_batch_descend(self.handle, int(nsteps), float(tol), steps, dptr(J), dptr(Ja))
        check(st, allow=(_native.KS_ENOTCONV,))
        return dict(steps=np.array(steps[:]), J=J, J_arc=Ja, status=st)

    def descend_async(self, nsteps: int, tol: float = 0.0):
        check(self.lib.ks_batch_descend_async(self.handle, int(nsteps), float(tol)))

    def scalars(self):
        out = (KSScalars * self.nb)()
        check(self.lib.ks_batch_scalars(self.handle, out))
        return [o.as_dict() for o in out]

    def get_state(self, i: int) -> torch.Tensor:
        s = self.specs[i]
        out = torch.empty((s.Ns, s.N), dtype=self.dtype, device=self.device)
        check(self.lib.ks_batch_get_state(self.handle, int(i), out.data_ptr()))
        self.stream.synchronize()
        return out

    def autotune(self, steps: int = 8) -> dict:
        """Tunes the launch shapes (sections per row CTA, the four-step split of each
        transform length, the dense tile width) on real descent steps; returns the
        choices (see tuning())."""
        chosen = ctypes.c_int32()
        check(self.lib.ks_batch_autotune(self.handle, int(steps), ctypes.byref(chosen)))
        return self.tuning()

    def tuning(self) -> dict:
        t = _native.KSBatchTuning()
        check(self.lib.ks_batch_get_tuning(self.handle, ctypes.byref(t)))
        return dict(row_sections=t.row_sections, dense_tile=t.dense_tile,
                    splits={int(t.F[i]): (int(t.F1[i]), int(t.F[i] // t.F1[i])) for i in range(t.nlen)},
                    ms_per_step=t.ms_per_step)

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.stream.synchronize()
            self.lib.ks_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
