"""ks_cost_noalloc: the allocation-free cost evaluation, checked through the C ABI
against the workspace-based entry points (ks_curve_create + ks_curve_cost) on
the same curve, on two calls in a row.

The entry point exists for callers that cannot allocate device memory (a host
program that owns every device allocation, a time-critical loop that must not
pay for cudaMalloc, a process with its device memory reserved up front); its
scratch is a static device array shared by all calls.  This file is collected
last so that a stop at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2301_11704_gb300 import _native, gen
from paper_2301_11704_gb300.curve import KSCurve

pytestmark = pytest.mark.gpu


def _curve(cfg, precision):
    spec = gen.workload(cfg)[0]
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, dtau=spec.dtau, precision=precision)
    c.init_trial(0.0, None, amps, vp)
    return spec, c


def _reference(spec, precision, u):
    """J^2, J_arc of the physical curve u from the workspace entry points
    (ks_curve_create with u as the initial curve, then ks_curve_cost)."""
    x = u.cpu().double().numpy()
    r = KSCurve(spec.L, spec.N, spec.Ns, spec.S, x[0], x[-1], dtau=spec.dtau, precision=precision, u_init=u)
    out = r.cost()
    r.close()
    return out


def _noalloc(lib, c, u):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=u.device)
    st = lib.ks_cost_noalloc(ctypes.byref(c.params), ctypes.c_void_p(u.data_ptr()),
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(c.stream.cuda_stream))
    _native.check(st)
    c.stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_noalloc_cost_matches_the_workspace_entry_points(precision, tol):
    lib = _native.load()
    refs = []
    for cfg in (0, 1):
        spec, c = _curve(cfg, precision)
        c.descend(3)
        u = c.get_state().clone()
        refs.append((c, u, _reference(spec, precision, u)))
    # calls in a row on two curve sizes, so the shared scratch is reused
    for c, u, (J2, Ja) in refs + refs[::-1]:
        got = _noalloc(lib, c, u)
        assert np.all(np.isfinite(got))
        assert abs(got[0] - J2) <= tol * J2 and abs(got[1] - Ja) <= tol * Ja, (got, J2, Ja)
    for c, _, _ in refs:
        c.close()


def test_noalloc_call_allocates_no_device_memory():
    """After a first (module-loading) call, further calls leave the device's free
    memory unchanged: the entry point allocates nothing."""
    lib = _native.load()
    spec, c = _curve(1, "fp32")
    u = c.get_state().clone()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=u.device)
    args = (ctypes.byref(c.params), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(c.stream.cuda_stream))
    _native.check(lib.ks_cost_noalloc(*args))
    c.stream.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _native.check(lib.ks_cost_noalloc(*args))
    c.stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.all(np.isfinite(out.cpu().numpy()))
    c.close()


def test_noalloc_rejects_curves_larger_than_its_scratch():
    lib = _native.load()
    p = _native.KSParams(L=100.0, nx=256, ns=16384, S=1638.3, s0=0.0, lam=1.0, lambda_free=0, dtau=0.01,
                         dtau_lambda=0.0, precision=1, adjoint=0, conv=0, check_ends=0, symmetry=0, s_transform=0, launch=0)
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.ks_cost_noalloc(ctypes.byref(p), ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                             None)
    assert st == _native.KS_ENOMEM
    assert b"scratch" in lib.ks_last_error()


def test_noalloc_cost_in_sine_storage():
    """A curve in sine storage (symmetry 5) evaluated by the allocation-free entry
    point: the same J^2 and J_arc as its workspace curve and as full storage."""
    lib = _native.load()
    spec, c = _curve(1, "fp64")
    u = c.get_state().clone()   # odd end points; the projection of both curves drops the rest
    c.close()
    x = u.cpu().double().numpy()
    outs = []
    for sym in (1, 5):
        r = KSCurve(spec.L, spec.N, spec.Ns, spec.S, x[0], x[-1], dtau=spec.dtau, precision="fp64", u_init=u,
                    symmetry=sym)
        ref = r.cost()
        got = _noalloc(lib, r, u)
        outs.append(got)
        assert abs(got[0] - ref[0]) <= 1e-12 * ref[0] and abs(got[1] - ref[1]) <= 1e-12 * ref[1]
        r.close()
    assert abs(outs[0][0] - outs[1][0]) <= 1e-12 * outs[0][0]
