"""Pins of the oracle's linearisation and end-point equilibria against the
values the paper prints (Table tab:KSE_eigenvals, L = 22) and the facts it
states about E1, E2, E3 (Sec. V.D: inversion symmetric; E2 and E3 invariant
under shifts by L/2 and L/3; one zero eigenvalue each).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2301_11704_gb300 import gen

L22 = 22.0


def _table(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "kse_eigenvalues_L22.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, re_, im_, mult = line.split()
            rows.setdefault(name, []).extend([complex(float(re_), float(im_))] * int(mult))
    return rows


def _unstable(uh, N, L):
    ev = np.linalg.eigvals(oracle.jacobian_zero_mean(uh, N, L))
    return ev, sorted(ev[ev.real > 1e-6], key=lambda z: (-z.real, z.imag))


def _match(found, expected, tol=5e-5):
    expected = sorted(expected, key=lambda z: (-z.real, z.imag))
    assert len(found) == len(expected), (found, expected)
    for a, b in zip(found, expected):
        assert abs(a.real - b.real) < tol and abs(abs(a.imag) - abs(b.imag)) < tol, (a, b)


def test_trivial_equilibrium_spectrum(golden_dir):
    """Df(0) at L = 22: unstable eigenvalues 0.2198, 0.1952, 0.0749 (each twice),
    equal to k^2 - k^4 for j = 2, 3, 1."""
    N = 64
    ev, unst = _unstable(np.zeros(N // 2, complex), N, L22)
    _match(unst, _table(golden_dir)["E0"])
    k = 2 * np.pi * np.arange(1, N // 2) / L22
    assert np.allclose(np.sort(ev.real), np.sort(np.repeat(k ** 2 - k ** 4, 2)), atol=1e-9)


def _classify(b):
    """E2: only even j (period L/2); E3: only j = 0 mod 3 (period L/3); E1: neither."""
    j = np.arange(1, len(b) + 1)
    big = np.abs(b) > 1e-8
    if np.all(j[big] % 2 == 0):
        return "E2"
    if np.all(j[big] % 3 == 0):
        return "E3"
    return "E1"


@pytest.fixture(scope="module")
def equilibria_L22():
    """Newton equilibria at L = 22, N = 64 from seeded starts: random 4-mode starts
    (generator recipe) and, for E3, starts in modes 3, 6, 9."""
    N = 64
    found = {}
    for seed in range(60):
        if seed < 40:
            b0 = gen.newton_guess(N, L22, gen.seed_for(7, seed), amplitude=1.0 + (seed % 2))
        else:
            rng = gen.SplitMix64(gen.seed_for(8, seed))
            b0 = np.zeros(N // 2 - 1)
            b0[[2, 5, 8]] = [2.0 + rng.normal(), rng.normal(), 0.1 * rng.normal()]
        b, it, res = oracle.newton_odd(b0, N, L22, maxit=100, tol=1e-12)
        if it < 0 or res > 1e-12:
            continue
        if np.abs(oracle.inv(oracle.odd_to_spec(b, N), N)).max() < 0.1:
            continue
        found.setdefault(_classify(b), b)
        if len(found) == 3:
            break
    return N, found


def test_newton_finds_all_three_nontrivial_equilibria(equilibria_L22):
    _, found = equilibria_L22
    assert set(found) == {"E1", "E2", "E3"}


@pytest.mark.parametrize("name", ["E1", "E2", "E3"])
def test_equilibrium_spectrum_matches_table(name, equilibria_L22, golden_dir):
    N, found = equilibria_L22
    uh = oracle.odd_to_spec(found[name], N)
    assert np.abs(oracle.rhs(uh, N, L22)).max() < 1e-12
    ev, unst = _unstable(uh, N, L22)
    _match(unst, _table(golden_dir)[name])
    # exactly one (translational) zero eigenvalue, all others stable
    assert np.sum(np.abs(ev) < 1e-7) == 1
    rest = ev[(np.abs(ev) >= 1e-7) & (ev.real <= 1e-6)]
    assert len(rest) + len(unst) + 1 == len(ev)


def test_symmetries_of_the_equilibria(equilibria_L22):
    """E1..E3 are odd (sigma-invariant); E2 is gamma(1/2)- and E3 gamma(1/3)-invariant."""
    N, found = equilibria_L22
    x = np.arange(N)
    for name, b in found.items():
        u = oracle.inv(oracle.odd_to_spec(b, N), N)
        assert np.abs(u + u[(-x) % N]).max() < 1e-12
        if name == "E2":
            assert np.abs(u - np.roll(u, N // 2)).max() < 1e-10
    b3 = found["E3"]
    Nb = 96                                       # 3 | N for an exact grid shift by L/3
    b3big = np.zeros(Nb // 2 - 1)
    b3big[: len(b3)] = b3
    u3 = oracle.inv(oracle.odd_to_spec(b3big, Nb), Nb)
    assert np.abs(u3 - np.roll(u3, Nb // 3)).max() < 1e-10


def test_stored_end_points_are_equilibria():
    """The stored u_+ of every workload satisfies f(u_+) = 0 to its Newton tolerance."""
    path = os.path.join(os.path.dirname(gen.__file__), "data", "equilibria.json")
    with open(path) as f:
        entries = json.load(f)["entries"]
    assert len(entries) == 1 + 1 + 1 + 256 + 1
    for e in entries[:3] + entries[3:259:37] + entries[-1:]:
        uh = oracle.odd_to_spec(np.array(e["b"]), e["N"])
        fh = oracle.rhs(uh, e["N"], e["L"])
        assert np.abs(-2 * fh[1:].imag).max() < e["tol"]
        assert np.abs(oracle.inv(uh, e["N"])).max() >= 0.1
