"""The persistent step kernel (one cooperative launch for many descent steps,
grid-wide barriers between the phases of a step) against the three-kernel step
on the same inputs: the state u and D_t u are bit-identical (the same
arithmetic in the same order; only the FP64 reductions of the scalars are
grouped differently), the curves stop at a tolerance after the same number of
steps, and with a free lambda (whose update reads the FP64 reductions) the two
stay within rounding.  The three-kernel step itself is checked against the
oracle in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.curve import KSCurve
from tests.curves import end_points, perturbation

pytestmark = pytest.mark.gpu


def _spec(N, Ns, L=22.0, dtau=0.01):
    return gen.CurveSpec(0, 0, L, N, Ns, gen.mapping_scale(Ns), dtau=dtau, steps=0)


def _pair(spec, **kw):
    up, um = end_points(gen.workload(0)[0]) if spec.N == 32 else (None, None)
    if up is None:
        x = np.arange(spec.N) * spec.L / spec.N
        up = 0.4 * np.sin(2 * np.pi * x / spec.L) - 0.2 * np.sin(4 * np.pi * x / spec.L)
        um = np.zeros(spec.N)
    amps, vp = perturbation(spec)
    out = []
    for launch in ("persistent", "kernels"):
        c = KSCurve(spec.L, spec.N, spec.Ns, spec.S, up, um, dtau=spec.dtau, s_transform="dense", launch=launch, **kw)
        c.init_trial(0.0, None, amps, vp)
        out.append(c)
    assert out[0].persistent and not out[1].persistent
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("adjoint", ["paper", "discrete"])
@pytest.mark.parametrize("N,Ns", [(32, 128), (64, 1024), (16, 37), (8, 3), (128, 300), (256, 70)])
def test_persistent_matches_three_kernel_step(precision, adjoint, N, Ns):
    spec = _spec(N, Ns, dtau=0.002)
    a, b = _pair(spec, precision=precision, adjoint=adjoint)
    ra = a.descend(37)
    rb = b.descend(37)
    assert ra["steps"] == rb["steps"] == 37
    assert torch.equal(a.get_state(), b.get_state())
    assert abs(ra["J"] - rb["J"]) <= 1e-12 * rb["J"]
    sa, sb = a.scalars(), b.scalars()
    assert sa["step"] == sb["step"] and sa["tau"] == sb["tau"]
    assert abs(sa["G_norm"] - sb["G_norm"]) <= 1e-12 * sb["G_norm"]
    # D_t u of the final state: the next residual is the same too
    assert torch.equal(a.residual(), b.residual())
    a.close()
    b.close()


def test_persistent_many_launches_and_tolerance_stop():
    spec = _spec(32, 128)
    a, b = _pair(spec)
    J0 = a.cost()[1]
    tol = 0.5 * J0
    ra = a.descend(3000, tol)       # three persistent launches; stops inside the first
    rb = b.descend(3000, tol)
    assert ra["steps"] == rb["steps"] and 0 < ra["steps"] < 3000
    assert ra["J_arc"] < tol
    assert torch.equal(a.get_state(), b.get_state())
    # a further call on a converged curve does nothing
    again = a.descend(10, tol)
    assert again["steps"] == 0
    a.close()
    b.close()


def test_persistent_free_lambda_stays_within_rounding():
    spec = _spec(32, 128)
    a, b = _pair(spec, lambda_free=True, dtau_lambda=0.01, lam=1.3)
    a.descend(200)
    b.descend(200)
    la, _ = a.get_lambda_tau()
    lb, _ = b.get_lambda_tau()
    assert abs(la - lb) <= 1e-12 * abs(lb)
    xa, xb = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
    assert np.abs(xa - xb).max() <= 1e-11 * np.abs(xb).max()
    a.close()
    b.close()


def test_profile_reports_persistent_launches():
    spec = _spec(64, 1024)
    a, _b = _pair(spec, precision="fp32")
    _b.close()
    a.profile(4)
    a.descend_async(1)
    a.descend_async(5)
    p = a.profile_read()
    assert p["step"]["launches"] == 2 and p["step"]["steps"] == 6 and p["step"]["ms"] > 0
    assert "rows" not in p
    a.close()
