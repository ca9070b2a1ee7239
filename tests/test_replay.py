"""The paper-replay set-up (Sec. V.D, Table tab:parameters): end points, shifts,
and (GPU) the first descent steps of a replayed orbit against the oracle."""
import numpy as np
import pytest

from paper_2301_11704_gb300 import replay


def test_orbit_table_matches_the_golden_copy(golden_dir):
    rows = {}
    for line in open(golden_dir + "/paper_run_parameters.txt"):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b, M, S = line.split()
        rows.setdefault((a, b), []).append((int(M), float(S)))
    assert replay.ORBITS["E1-E2"] == rows[("E1", "E2")][0] == (550, 55.0)
    assert replay.ORBITS["E0-E1"] == rows[("E0", "E1")][0]
    assert replay.ORBITS["E2-g14E2"] == rows[("E2", "g14E2")][0]


def test_end_points_are_the_stored_equilibria_and_shifts_are_exact():
    um, up = replay.end_points("E1-E2")
    assert np.abs(um).max() > 1 and np.abs(up).max() > 1
    x = np.arange(64)
    for u in (um, up):
        assert np.abs(u + u[(-x) % 64]).max() < 1e-12          # odd (inversion symmetric)
    e2 = replay.equilibrium("E2")
    g = replay.shifted(e2, 0.25)
    assert np.abs(g - np.roll(e2, -16)).max() == 0
    assert np.abs(g + g[(-x) % 64]).max() < 1e-12               # gamma(1/4) E2 is odd as well
    assert np.abs(g - e2).max() > 1.0
    with pytest.raises(ValueError):
        replay.shifted(e2, 0.3)


@pytest.mark.gpu
def test_replayed_orbit_first_steps_match_the_oracle():
    import oracle
    from paper_2301_11704_gb300.curve import KSCurve
    M, S = replay.ORBITS["E0-E1"]
    um, up = replay.end_points("E0-E1")
    c = KSCurve(22.0, 64, M + 2, S, up, um, dtau=0.01, check_ends=True)
    U = oracle.curve_init(M, S, up, um)
    Uo, _, sco, hist = oracle.curve_descend(U, 22.0, S, 200, dtau=0.01, history=True)
    out = c.descend(200)
    assert abs(out["J_arc"] - sco["J_arc"]) < 1e-10 * sco["J_arc"]
    x = c.get_state().cpu().numpy()
    xo = oracle.curve_physical(Uo)
    assert np.abs(x - xo).max() < 1e-10 * np.abs(xo).max()
    assert hist[-1, 3] < hist[0, 3]
    c.close()
