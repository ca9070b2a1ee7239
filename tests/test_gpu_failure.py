"""Failure detection on the GPU without a GPU fault: a non-finite curve handed in
from the host stops the descent with KS_ENONFINITE, and a device-side bounded
wait that runs out (its bound set to give up at once through the test hook
ks_curve_debug_wait_limit) makes the kernel flag the launch as invalid, finish
the copies and products in flight, free its tensor memory and return: the host
reads KS_ETIMEOUT and the context stays usable (the same curve, re-initialised,
then gives the cost of a fresh curve)."""
import numpy as np
import pytest
import torch

from paper_2301_11704_gb300 import _native, gen
from paper_2301_11704_gb300.curve import KSCurve

pytestmark = pytest.mark.gpu


def _curve(N, Ns, precision, s_transform="auto", scheme="imex"):
    L = 22.0 + N / 16.0
    spec = gen.CurveSpec(0, 0, L, N, Ns, 0.1 * (Ns - 1))
    up = np.zeros(N)
    amps = np.full(4, 0.1)
    vp = gen.perturbation_fields(N, L, 11, 4)
    c = KSCurve(L, N, Ns, spec.S, up, np.zeros(N), dtau=1e-3, precision=precision, s_transform=s_transform,
                scheme=scheme)
    c.init_trial(0.0, None, amps, vp)
    return c, (amps, vp)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3"])
def test_nonfinite_state_stops_the_descent(precision):
    c, _ = _curve(64, 200, precision)
    u = c.get_state()
    good = u.clone()
    u[57, 11] = float("nan")
    c.set_state(u, 1.0, 0.0)
    with pytest.raises(_native.KSError) as err:
        c.descend(5)
    assert err.value.status == _native.KS_ENONFINITE
    sc = c.scalars()
    assert sc["status"] == _native.KS_ENONFINITE and sc["step"] == 0
    # the curve takes a finite state again and descends
    c.set_state(good, 1.0, 0.0)
    out = c.descend(3)
    assert out["steps"] == 3 and np.isfinite(out["J"])
    c.close()


@pytest.mark.parametrize("precision,s_transform,N,Ns,call,scheme", [
    ("bf16x3", "auto", 128, 257, "cost", "imex"),        # the split-BF16 row phase (tcgen05, bulk copies)
    ("bf16x2", "auto", 256, 130, "cost", "imex"),
    ("fp64", "fft", 32, 128, "descend", "imex"),         # the FFT form with one CTA per mode (bulk-copied twiddles)
    ("fp32", "dense_tc", 64, 256, "descend", "imex"),    # the tensor-core s-contraction
    ("fp32", "dense", 64, 300, "descend", "implicit"),   # the implicit increment's tensor-core products
])
def test_expired_device_wait_reports_timeout(precision, s_transform, N, Ns, call, scheme):
    c, (amps, vp) = _curve(N, Ns, precision, s_transform, scheme)
    ref, _ = _curve(N, Ns, precision, s_transform, scheme)
    J2_ref = ref.cost()[0]
    out_ref = ref.descend(1)
    ref.close()
    c.debug_wait_limit(-1)
    with pytest.raises(_native.KSError) as err:
        if call == "cost":
            c.cost()
        else:
            c.descend(1)
    assert err.value.status == _native.KS_ETIMEOUT
    # every later read of the scalars reports it until the curve is re-initialised
    with pytest.raises(_native.KSError):
        c.scalars()
    c.init_trial(0.0, None, amps, vp)
    assert c.cost()[0] == J2_ref
    out = c.descend(1)
    assert out["J"] == out_ref["J"]
    c.close()
    torch.cuda.synchronize()
