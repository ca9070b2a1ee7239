"""Batched descent (ks_batch_*): curves of uneven N_s, N and L in one set of
launches must behave exactly like independent curves (each checked against a
single-curve run and the oracle), stop independently at their own tolerance,
and survive the tile autotuner; the 256-curve batch workload runs end to end."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_11704_gb300 import gen
from paper_2301_11704_gb300.batch import KSBatch
from paper_2301_11704_gb300.curve import KSCurve

pytestmark = pytest.mark.gpu


def _mixed_specs():
    """Seven curves from the batch workload recipe, cut to small sizes (uneven
    N_s, N, L; N_s ragged with respect to every tile size)."""
    base = gen.workload(3)
    picks = [0, 1, 2, 3, 5, 8, 13]
    out = []
    for k, i in enumerate(picks):
        s = base[i]
        Ns = [37, 130, 65, 200, 19, 96, 151][k]
        out.append(gen.CurveSpec(3, i, s.L, s.N, Ns, gen.mapping_scale(Ns), dtau=0.002, steps=0))
    return out


def _inputs(spec):
    up, um = gen.end_points(spec)
    amps, vp = gen.perturbation(spec)
    return up, um, amps, vp


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_independent_curves(precision):
    specs = _mixed_specs()
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision=precision, conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    out = b.descend(40)
    assert np.all(out["steps"] == 40)
    tol = 1e-11 if precision == "fp64" else 2e-5
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        c = KSCurve(s.L, s.N, s.Ns, s.S, up, um, dtau=s.dtau, precision=precision)
        c.init_trial(0.0, None, amps, vp)
        ref = c.descend(40)
        xb = b.get_state(k).double().cpu().numpy()
        xc = c.get_state().double().cpu().numpy()
        assert np.abs(xb - xc).max() <= tol * np.abs(xc).max(), (k, s)
        assert abs(out["J"][k] - ref["J"]) <= tol * ref["J"]
        c.close()
    b.close()


def test_batch_matches_the_oracle_fp64():
    specs = _mixed_specs()[:3]
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp64", conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    out = b.descend(25)
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        U = oracle.curve_init(s.M, s.S, up, um, amps=amps, vp=vp)
        Uo, _, sco, _ = oracle.curve_descend(U, s.L, s.S, 25, dtau=s.dtau)
        xo = oracle.curve_physical(Uo)
        assert np.abs(b.get_state(k).cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()
        assert abs(out["J_arc"][k] - sco["J_arc"]) <= 1e-10 * sco["J_arc"]
    b.close()


def test_curves_stop_at_their_own_tolerance_and_autotune_keeps_results():
    specs = _mixed_specs()
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp64", conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    first = b.descend(0)
    tol = float(np.median(first["J_arc"]))          # about half of the curves are already below it
    out = b.descend(30, tol)
    below = first["J_arc"] < tol
    assert np.all(out["steps"][below] == 0) and np.all(out["steps"][~below] > 0)
    tune = b.autotune(4)
    assert tune["row_sections"] in (8, 16) and tune["dense_tile"] in (0, 32, 64)
    sc = b.scalars()
    assert all(np.isfinite(x["J"]) for x in sc)
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_autotuned_four_step_batch_matches_independent_curves(precision, tol):
    """Curves in the batched four-step form (F = 1024, 2048, 4096; N_s = 2000 is
    the longest FP64 curve that fits it): the autotuner switches the row-phase
    width and the split of every length (recomputing the spectra); the tuned
    batch still equals independent curves run for the same number of steps."""
    base = gen.workload(3)
    specs = [gen.CurveSpec(3, i, base[i].L, base[i].N, Ns, gen.mapping_scale(Ns), dtau=0.002, steps=0)
             for i, Ns in zip((4, 6, 7, 9, 11), (400, 700, 1100, 1300, 2000))]
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision=precision, conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    tune = b.autotune(3)
    print("batch tuning:", tune)
    assert set(tune["splits"]) == {1024, 2048, 4096}
    assert all(f1 * f2 == F for F, (f1, f2) in tune["splits"].items())
    out = b.descend(10)
    steps = [x["step"] for x in b.scalars()]
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        c = KSCurve(s.L, s.N, s.Ns, s.S, up, um, dtau=s.dtau, precision=precision)
        c.init_trial(0.0, None, amps, vp)
        ref = c.descend(steps[k])
        xb = b.get_state(k).double().cpu().numpy()
        xc = c.get_state().double().cpu().numpy()
        assert np.abs(xb - xc).max() <= tol * np.abs(xc).max(), (k, s.Ns)
        assert abs(out["J"][k] - ref["J"]) <= tol * ref["J"]
        c.close()
    b.close()


def test_batch_workload_256_curves_fp32():
    specs = gen.workload(3)
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp32", conv="jrel")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    j0 = b.descend(0)["J"]
    # three curves' trial-curve cost against the FP64 oracle (J within 1e-5)
    for k in (0, 100, 255):
        s = specs[k]
        up, um, amps, vp = ins[k]
        R, D = oracle.curve_residual(oracle.curve_init(s.M, s.S, up, um, amps=amps, vp=vp), s.L, s.S)
        J = np.sqrt(oracle.curve_scalars(R, D, s.L, s.S)["J2"])
        assert abs(j0[k] - J) <= 1e-5 * J
    out = b.descend(64)
    assert np.all(np.isfinite(out["J"])) and np.all(out["steps"] == 64)
    assert np.median(out["J"] / j0) < 1.0
    b.close()


def _four_step_specs(sizes):
    """Curves of the batch recipe with the given N (their stored end points) and N_s."""
    base = gen.workload(3)
    out, used = [], set()
    for N, Ns in sizes:
        i = next(i for i, s in enumerate(base) if s.N == N and i not in used)
        used.add(i)
        out.append(gen.CurveSpec(3, i, base[i].L, N, Ns, gen.mapping_scale(Ns), dtau=0.002, steps=0))
    return out


def test_batch_four_step_items_match_independent_curves_fp32():
    """Curves whose transform length is 1024 to 8192 run the batch's
    one-CTA-per-mode four-step form; each tracks its own single-curve run."""
    specs = _four_step_specs([(32, 700), (64, 1500), (128, 2100), (32, 1200), (32, 300), (64, 600)])
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp32", conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    out = b.descend(20)
    assert np.all(out["steps"] == 20)
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        c = KSCurve(s.L, s.N, s.Ns, s.S, up, um, dtau=s.dtau, precision="fp32")
        c.init_trial(0.0, None, amps, vp)
        ref = c.descend(20)
        xb = b.get_state(k).double().cpu().numpy()
        xc = c.get_state().double().cpu().numpy()
        assert np.abs(xb - xc).max() <= 2e-5 * np.abs(xc).max(), (k, s)
        assert abs(out["J"][k] - ref["J"]) <= 2e-5 * ref["J"]
        c.close()
    b.close()


def test_batch_four_step_items_match_the_oracle_fp64():
    """FP64 batch curves with F = 1024, 2048 and 4096 (the one-CTA-per-mode
    four-step form) against the oracle's descent."""
    specs = _four_step_specs([(32, 700), (64, 1200), (32, 300), (64, 500)])
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp64", conv="jarc")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    out = b.descend(10)
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        U = oracle.curve_init(s.M, s.S, up, um, amps=amps, vp=vp)
        Uo, _, sco, _ = oracle.curve_descend(U, s.L, s.S, 10, dtau=s.dtau)
        xo = oracle.curve_physical(Uo)
        assert np.abs(b.get_state(k).cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()
        assert abs(out["J_arc"][k] - sco["J_arc"]) <= 1e-10 * sco["J_arc"]
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_implicit_batch_matches_independent_curves(precision, tol):
    """Full-linear-implicit stepping in a batch (its eigenbases set up in parallel
    host threads; one K chunk per product) at dtau = 0.2, far beyond the IMEX
    limit of every curve: each curve equals its single-curve implicit run, and
    the FP64 curves the oracle's implicit descent."""
    base = gen.workload(3)
    specs = [gen.CurveSpec(3, i, base[i].L, base[i].N, Ns, gen.mapping_scale(Ns), dtau=0.2, steps=0)
             for i, Ns in zip((0, 1, 2, 3, 5, 6, 9), (19, 130, 65, 200, 400, 1100, 1300))]
    ins = [_inputs(s) for s in specs]
    b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision=precision, conv="jarc", scheme="implicit")
    b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    out = b.descend(20)
    for k, s in enumerate(specs):
        up, um, amps, vp = ins[k]
        c = KSCurve(s.L, s.N, s.Ns, s.S, up, um, dtau=s.dtau, precision=precision, scheme="implicit")
        c.init_trial(0.0, None, amps, vp)
        ref = c.descend(20)
        xb = b.get_state(k).double().cpu().numpy()
        xc = c.get_state().double().cpu().numpy()
        assert np.abs(xb - xc).max() <= tol * np.abs(xc).max(), (k, s.Ns)
        assert abs(out["J"][k] - ref["J"]) <= tol * ref["J"]
        c.close()
        if precision == "fp64" and s.Ns <= 200:
            U = oracle.curve_init(s.M, s.S, up, um, amps=amps, vp=vp)
            Uo, _, sco, _ = oracle.curve_descend(U, s.L, s.S, 20, dtau=s.dtau, scheme=oracle.IMPLICIT)
            assert np.abs(xb - oracle.curve_physical(Uo)).max() <= 1e-10 * np.abs(xb).max()
    b.close()


def test_batch_converges_per_curve_to_the_papers_criterion():
    """The paper's searches from E0 to E1 and E2 at L = 22 (Sec. V.D, Table
    tab:parameters: their (M, S), N = 64, a = 0) in one FP64 batch with the
    full-linear-implicit step (dtau = 0.2): every curve stops by itself at
    J_arc < 1e-11 (eq. J_arc), at the step its single-curve run stops at, and the
    oracle confirms the cost of each final state.  (E0 -> E3, which converges at
    the paper's dtau = 0.01, ends at dtau = 0.2 near a local minimum, J_arc ~ 0.1:
    the step size changes the path in tau, not the fixed points.)"""
    from paper_2301_11704_gb300 import replay
    orbits = ["E0-E1", "E0-E2"]
    specs, ups, ums = [], [], []
    for o in orbits:
        M, S = replay.ORBITS[o]
        um, up = replay.end_points(o)
        specs.append(gen.CurveSpec(3, 0, 22.0, 64, M + 2, S, dtau=0.2, steps=0))
        ups.append(up)
        ums.append(um)
    b = KSBatch(specs, ups, ums, precision="fp64", conv="jarc", scheme="implicit")
    tol = 1e-11
    out = b.descend(40000, tol)
    sc = b.scalars()
    print("CONVERGED steps:", list(out["steps"]), "J_arc:", [x["J_arc"] for x in sc])
    for k, (o, s) in enumerate(zip(orbits, specs)):
        assert sc[k]["converged"] == 1 and sc[k]["J_arc"] < tol, o
        c = KSCurve(22.0, 64, s.Ns, s.S, ups[k], ums[k], dtau=0.2, precision="fp64", conv="jarc", scheme="implicit")
        ref = c.descend(40000, tol)
        c.close()
        assert ref["steps"] == out["steps"][k], (o, ref["steps"], out["steps"][k])
        X = b.get_state(k).double().cpu().numpy()
        R, D = oracle.curve_residual(oracle.curve_spectral(X), 22.0, s.S)
        assert oracle.curve_scalars(R, D, 22.0, s.S)["J_arc"] < 1e-10, o
    b.close()


@pytest.mark.parametrize("precision,tol,tol_tuned", [("fp64", 1e-12, 1e-11), ("fp32", 2e-6, 2e-5)])
def test_sine_storage_batch_matches_full_storage(precision, tol, tol_tuned):
    """A batch of odd curves (the workload's end points are odd; the projection
    makes the trial curves so) in which every other curve keeps only the sine
    coefficients (symmetry 5) against the same batch in full storage (symmetry
    1), curve by curve, in the dense, one-CTA FFT and batched four-step forms,
    before and after the tile autotuner (which may pick other splits for the two
    batches: then the tolerance between s-forms)."""
    specs = _mixed_specs() + _four_step_specs([(32, 700), (64, 1500), (128, 600)])
    ins = [_inputs(s) for s in specs]
    syms = [5 if k % 2 == 0 else 1 for k in range(len(specs))]
    bh = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision=precision, conv="jarc", symmetry=syms)
    bf = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision=precision, conv="jarc", symmetry=1)
    assert bh.workspace_bytes < bf.workspace_bytes
    for b in (bh, bf):
        b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
    oh, of = bh.descend(20), bf.descend(20)
    for k in range(len(specs)):
        xh, xf = bh.get_state(k).double().cpu().numpy(), bf.get_state(k).double().cpu().numpy()
        assert np.abs(xh - xf).max() <= tol * np.abs(xf).max(), (k, specs[k])
        assert abs(oh["J"][k] - of["J"][k]) <= tol * of["J"][k]
        U = np.fft.rfft(xh, axis=1)
        assert np.abs(U.real).max() <= (1e-12 if precision == "fp64" else 1e-6) * np.abs(U).max()
    bh.autotune(4)
    bf.autotune(4)
    oh, of = bh.descend(10), bf.descend(10)
    for k in range(len(specs)):
        assert abs(oh["J"][k] - of["J"][k]) <= tol_tuned * of["J"][k], k
    bh.close()
    bf.close()


def test_sine_storage_batch_dense_form():
    """The dense batched contraction (s_transform "dense") in sine storage against
    full storage, FP64, curve by curve."""
    specs = _mixed_specs()
    ins = [_inputs(s) for s in specs]
    out = []
    for sym in (5, 1):
        b = KSBatch(specs, [i[0] for i in ins], [i[1] for i in ins], precision="fp64", conv="jarc",
                    s_transform="dense", symmetry=sym)
        b.init_trial(np.array([i[2] for i in ins]), [i[3] for i in ins])
        o = b.descend(15)
        out.append((o["J"].copy(), [b.get_state(k).cpu().numpy() for k in range(len(specs))]))
        b.close()
    (jh, xh), (jf, xf) = out
    for k in range(len(specs)):
        assert np.abs(xh[k] - xf[k]).max() <= 1e-12 * np.abs(xf[k]).max(), k
        assert abs(jh[k] - jf[k]) <= 1e-12 * jf[k], k
