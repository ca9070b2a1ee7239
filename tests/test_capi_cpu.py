"""The C-ABI library builds, loads and exports every entry point declared in
include/ksconn.h; argument validation runs on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2301_11704_gb300 import _native
from paper_2301_11704_gb300._native import KSParams

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ks_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(_native.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.ks_version() >> 16 == 1


def _params(**kw):
    base = dict(L=22.0, nx=32, ns=128, S=12.7, s0=0.0, lam=1.0, lambda_free=0, dtau=0.01, dtau_lambda=0.0,
                precision=0, adjoint=0, conv=0, check_ends=0, symmetry=0, s_transform=0, launch=0)
    base.update(kw)
    return KSParams(**base)


def test_workspace_size_scales_with_the_curve(lib):
    a = lib.ks_curve_workspace_bytes(ctypes.byref(_params()))
    b = lib.ks_curve_workspace_bytes(ctypes.byref(_params(ns=256)))
    c = lib.ks_curve_workspace_bytes(ctypes.byref(_params(precision=1)))
    assert a > 6 * 128 * 32 * 8 and b > a and c < a
    # linear, not quadratic, in ns
    big = lib.ks_curve_workspace_bytes(ctypes.byref(_params(ns=16384, nx=256)))
    assert big < 16 * 16384 * 256 * 8   # fields, FP64 scratch and the four-step scratch (about 4 fields)


@pytest.mark.parametrize("bad", [dict(nx=24), dict(nx=4), dict(nx=512), dict(ns=2), dict(L=0.0), dict(S=-1.0),
                                 dict(dtau=0.0), dict(precision=7), dict(adjoint=3), dict(conv=9),
                                 dict(symmetry=4), dict(s_transform=5), dict(s_transform=4, ns=500), dict(s_transform=3, precision=0), dict(launch=2), dict(L=float("nan"))])
def test_invalid_parameters_are_rejected_on_the_host(lib, bad):
    p = _params(**bad)
    assert lib.ks_curve_workspace_bytes(ctypes.byref(p)) == 0
    assert lib.ks_last_error()
    h = ctypes.c_void_p()
    st = lib.ks_curve_create(ctypes.byref(p), None, None, None, None, 0, None, ctypes.byref(h))
    assert st == _native.KS_EINVAL and h.value is None


def test_missing_pointers_and_small_workspace_are_rejected(lib):
    import numpy as np
    p = _params()
    up = np.zeros(32)
    h = ctypes.c_void_p()
    st = lib.ks_curve_create(ctypes.byref(p), None, _native.dptr(up), None, None, 0, None, ctypes.byref(h))
    assert st == _native.KS_EINVAL
    st = lib.ks_curve_create(ctypes.byref(p), _native.dptr(up), _native.dptr(up), None, 256, 16, None,
                             ctypes.byref(h))
    assert st == _native.KS_ENOMEM
    assert b"needed" in lib.ks_last_error()
    st = lib.ks_curve_create(ctypes.byref(p), _native.dptr(up), _native.dptr(up), None, 257, 1 << 30, None,
                             ctypes.byref(h))
    assert st == _native.KS_EINVAL and b"aligned" in lib.ks_last_error()


def test_null_handle_is_rejected(lib):
    assert lib.ks_curve_cost(None, None, None) == _native.KS_EINVAL
    assert lib.ks_curve_destroy(None) == _native.KS_OK


@pytest.mark.parametrize("kw,F", [
    (dict(precision=1, nx=64, ns=1024), 0),                  # FP32, N_s N_x = 65536: dense
    (dict(precision=1, nx=128, ns=1024), 4096),              # FP32, N_s N_x = 131072: FFT, F >= 3 (N_s - 1)
    (dict(precision=1, nx=32, ns=2731), 8192),               # FP32, N_s > 2048
    (dict(precision=1, nx=256, ns=4096), 16384),             # above one CTA: the four-step form
    (dict(precision=1, nx=256, ns=16384), 65536),
    (dict(precision=1, nx=64, ns=30000), 0),                 # above the four-step limit: dense
    (dict(precision=0, nx=64, ns=1024), 4096),               # FP64, N_x >= 64
    (dict(precision=0, nx=32, ns=1024), 4096),               # FP64, N_s >= 684: four-step
    (dict(precision=0, nx=32, ns=600), 0),                   # FP64, N_x = 32, small
    (dict(precision=0, nx=32, ns=128), 512),                 # FP64, N_s <= 128
    (dict(precision=1, nx=64, ns=1024, s_transform=2), 4096),
    (dict(precision=1, nx=128, ns=1024, s_transform=1), 0),
    (dict(nx=24), -1),
])
def test_s_transform_rule(lib, kw, F):
    assert lib.ks_curve_fft_length(ctypes.byref(_params(**kw))) == F
