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


def test_sine_storage_halves_the_fields(lib):
    """Symmetry bit 2 keeps N_x/2 words per section in each of the five fields (and
    half the four-step scratch); the FP64 physical scratch and the tables stay."""
    for kw in (dict(), dict(precision=1, nx=64, ns=1500, s_transform=4)):
        full = lib.ks_curve_workspace_bytes(ctypes.byref(_params(symmetry=1, **kw)))
        sine = lib.ks_curve_workspace_bytes(ctypes.byref(_params(symmetry=5, **kw)))
        p = _params(**kw)
        b = 8 if p.precision == 0 else 4
        half_field = p.ns * p.nx // 2 * b
        assert 0 < sine < full and full - sine >= 5 * half_field - 5 * 256


@pytest.mark.parametrize("bad", [dict(nx=24), dict(nx=4), dict(nx=512), dict(ns=2), dict(L=0.0), dict(S=-1.0),
                                 dict(dtau=0.0), dict(precision=7), dict(precision=4), dict(precision=2, nx=32), dict(precision=3, nx=16), dict(adjoint=3), dict(conv=9),
                                 dict(symmetry=4), dict(symmetry=6), dict(symmetry=8), dict(symmetry=5, nx=8),
                                 dict(symmetry=5, precision=2, nx=64), dict(symmetry=5, precision=1, s_transform=3),
                                 dict(symmetry=5, launch=1), dict(symmetry=5, scheme=1), dict(s_transform=6), dict(s_transform=4, ns=500), dict(s_transform=5, ns=500), dict(s_transform=5, ns=12000, precision=0), dict(s_transform=3, precision=0), dict(launch=2), dict(L=float("nan"))])
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


@pytest.mark.parametrize("kw,F,form", [
    (dict(precision=1, nx=64, ns=600), 0, 1),                # FP32 below N_s = 684: dense
    (dict(precision=1, nx=64, ns=1024), 4096, 5),            # FP32 from N_s = 684: clustered four-step
    (dict(precision=1, nx=64, ns=5462), 16384, 5),           # N_x <= 64 up to F = 16384
    (dict(precision=1, nx=64, ns=5463), 16384, 4),           # three-launch: F >= 2P + 1
    (dict(precision=1, nx=128, ns=2731), 8192, 5),           # N_x = 128 up to F = 8192
    (dict(precision=1, nx=128, ns=2732), 8192, 4),
    (dict(precision=1, nx=256, ns=700), 4096, 4),            # N_x = 256: three-launch four-step
    (dict(precision=1, nx=256, ns=16384), 32768, 4),
    (dict(precision=1, nx=256, ns=16385), 65536, 4),         # 2P + 1 = 32769
    (dict(precision=1, nx=64, ns=30000), 0, 3),              # above the four-step limit: tensor-core dense
    (dict(precision=0, nx=16, ns=1366), 4096, 5),            # FP64 clustered at F = 4096, N_x <= 16
    (dict(precision=0, nx=32, ns=1024), 4096, 4),            # FP64 N_s >= 684: four-step
    (dict(precision=0, nx=256, ns=1024), 4096, 2),           # FP64 N_x = 256: one CTA per mode while it fits
    (dict(precision=0, nx=256, ns=2048), 4096, 4),
    (dict(precision=0, nx=64, ns=600), 2048, 2),             # FP64 below N_s = 684, N_x >= 64: one-CTA FFT
    (dict(precision=0, nx=32, ns=600), 0, 1),                # FP64, N_x = 32, small: dense
    (dict(precision=0, nx=32, ns=128), 512, 2),              # FP64, N_s <= 128
    (dict(precision=1, nx=64, ns=1024, s_transform=2), 4096, 2),
    (dict(precision=1, nx=64, ns=1024, s_transform=4), 4096, 4),
    (dict(precision=1, nx=128, ns=1024, s_transform=1), 0, 1),
    (dict(precision=1, nx=128, ns=1024, s_transform=3), 0, 3),
    (dict(precision=1, nx=64, ns=1024, symmetry=5), 4096, 5),   # sine storage: the rule on the 32 stored columns
    (dict(precision=1, nx=256, ns=2731, symmetry=5), 8192, 5),  # 128 stored columns: clustered (full rows: three-launch)
    (dict(precision=1, nx=256, ns=2731, symmetry=1), 8192, 4),
    (dict(precision=0, nx=256, ns=1024, symmetry=5), 4096, 4),  # FP64, 128 columns: four-step (full rows: one CTA per mode)
    (dict(precision=1, nx=64, ns=30000, symmetry=5), 0, 1),     # sine storage: SIMT dense, not the tensor-core form
    (dict(precision=0, nx=64, ns=600, symmetry=7), 0, 1),       # FP64, 32 stored columns below N_s = 684: dense
    (dict(precision=0, nx=128, ns=600, symmetry=5), 2048, 2),   # 64 stored columns: one CTA per column pair
    (dict(nx=24), -1, -1),
])
def test_s_transform_rule(lib, kw, F, form):
    assert lib.ks_curve_fft_length(ctypes.byref(_params(**kw))) == F
    assert lib.ks_curve_s_form(ctypes.byref(_params(**kw))) == form


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("nx", [64, 128, 256])
def test_split_bf16_workspace_holds_the_dft_matrices(lib, prec, nx):
    """Split-BF16 x-transforms: FP32 storage plus the two N x N DFT matrices in
    three BF16 parts (12 N^2 bytes); same s-form as FP32."""
    ws32 = lib.ks_curve_workspace_bytes(ctypes.byref(_params(precision=1, nx=nx, ns=1024)))
    wsb = lib.ks_curve_workspace_bytes(ctypes.byref(_params(precision=prec, nx=nx, ns=1024)))
    assert wsb - ws32 == ((12 * nx * nx + 255) // 256) * 256
    assert lib.ks_curve_s_form(ctypes.byref(_params(precision=prec, nx=nx, ns=1024))) == \
        lib.ks_curve_s_form(ctypes.byref(_params(precision=1, nx=nx, ns=1024)))


def test_split_bf16_batches_are_rejected(lib):
    ps = (KSParams * 2)(_params(precision=3, nx=64), _params(precision=3, nx=64))
    assert lib.ks_batch_workspace_bytes(2, ps) == 0
    assert b"batch" in lib.ks_last_error()


@pytest.mark.parametrize("bad", [dict(scheme=2), dict(scheme=-1), dict(scheme=1, launch=1), dict(scheme=1, ns=3),
                                 dict(scheme=1, ns=16385, nx=64)])
def test_invalid_implicit_parameters_are_rejected(lib, bad):
    p = _params(**bad)
    assert lib.ks_curve_workspace_bytes(ctypes.byref(p)) == 0
    assert lib.ks_last_error()


@pytest.mark.parametrize("prec,b", [(0, 8), (1, 4), (2, 4)])
@pytest.mark.parametrize("ns", [129, 130, 1000])
def test_implicit_workspace_holds_the_eigenbases(lib, prec, b, ns):
    """Full-linear-implicit stepping: V and V^-1 of the even (ceil(M/2) square) and
    odd (floor(M/2) square) parts of D~^2 in the storage type, their eigenvalues
    in FP64, the split partials of the two products (2 x 8 x M x N), and in FP32
    storage V^-1 and V as split-BF16 tensor-core operands (two parts, padded to
    128-row tiles and 32-wide K chunks); same s-form as the IMEX scheme."""
    nx = 64
    imex = lib.ks_curve_workspace_bytes(ctypes.byref(_params(precision=prec, nx=nx, ns=ns)))
    impl = lib.ks_curve_workspace_bytes(ctypes.byref(_params(precision=prec, nx=nx, ns=ns, scheme=1)))
    M = ns - 2
    ne, no = (M + 1) // 2, M // 2
    al = lambda x: (x + 255) // 256 * 256
    blk = lambda n: ((n + 127) // 128) * ((n + 31) // 32) * 2 * (128 * 32 * 2)   # tensor-core operand blocks
    tc = al(2 * (blk(ne) + blk(no))) if b == 4 else 0
    assert impl - imex == 2 * al((ne * ne + no * no) * b) + al(M * 8) + al(2 * 8 * M * nx * b) + tc
    assert lib.ks_curve_s_form(ctypes.byref(_params(precision=prec, nx=nx, ns=ns, scheme=1))) == \
        lib.ks_curve_s_form(ctypes.byref(_params(precision=prec, nx=nx, ns=ns)))


def test_batches_with_mixed_schemes_are_rejected(lib):
    ps = (KSParams * 2)(_params(scheme=1), _params(scheme=0))
    assert lib.ks_batch_workspace_bytes(2, ps) == 0
    assert b"scheme" in lib.ks_last_error()
    ok = (KSParams * 2)(_params(scheme=1), _params(scheme=1, ns=200))
    plain = (KSParams * 2)(_params(), _params(ns=200))
    assert lib.ks_batch_workspace_bytes(2, ok) > lib.ks_batch_workspace_bytes(2, plain) > 0


def test_sine_storage_batches_take_half_fields(lib):
    """A batch may mix sine and full storage curve by curve; each sine curve's five
    fields take half the bytes (the FP64 scratch and the tables stay); the
    implicit scheme keeps full storage."""
    full = (KSParams * 3)(_params(symmetry=1, precision=1, nx=64, ns=700), _params(symmetry=1, ns=300),
                          _params(symmetry=1, precision=1, nx=128, ns=1500))
    mixed = (KSParams * 3)(_params(symmetry=5, precision=1, nx=64, ns=700), _params(symmetry=1, ns=300),
                           _params(symmetry=5, precision=1, nx=128, ns=1500))
    # batches take one precision: make the middle curve FP32 too
    full[1].precision = mixed[1].precision = 1
    bf, bm = lib.ks_batch_workspace_bytes(3, full), lib.ks_batch_workspace_bytes(3, mixed)
    assert 0 < bm < bf
    assert bf - bm >= 5 * (700 * 32 + 1500 * 64) * 4 - 10 * 256
    bad = (KSParams * 2)(_params(symmetry=5, scheme=1), _params(symmetry=5, scheme=1))
    assert lib.ks_batch_workspace_bytes(2, bad) == 0
