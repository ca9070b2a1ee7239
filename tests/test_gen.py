"""The seeded input generator: published SplitMix64 outputs, determinism and
the shapes and statistics of the synthetic workloads."""
import os

import numpy as np

from paper_2301_11704_gb300 import gen


def test_splitmix64_published_outputs(golden_dir):
    with open(os.path.join(golden_dir, "splitmix64_seed0.txt")) as f:
        ref = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    r = gen.SplitMix64(0)
    assert [r.next_u64() for _ in range(len(ref))] == ref


def test_normals_have_unit_variance_and_are_reproducible():
    a = gen.SplitMix64(12345)
    x = np.array([a.normal() for _ in range(20000)])
    assert abs(x.mean()) < 0.03 and abs(x.std() - 1) < 0.03
    b = gen.SplitMix64(12345)
    assert b.normal() == x[0]


def test_workload_shapes():
    c0, = gen.workload(0)
    assert (c0.L, c0.N, c0.Ns, c0.steps) == (22.0, 32, 128, 2000) and abs(c0.S - 12.7) < 1e-12
    c1, = gen.workload(1)
    assert (c1.L, c1.N, c1.Ns) == (22.0, 64, 1024) and abs(c1.S - 102.3) < 1e-12
    c2, = gen.workload(2)
    assert (c2.L, c2.N, c2.Ns, c2.npert, c2.amp) == (44.0, 128, 4096, 8, 0.2)
    batch = gen.workload(3)
    assert len(batch) == 256
    assert all(20 <= c.L <= 60 and c.N in (32, 64, 128) and 256 <= c.Ns <= 2048 for c in batch)
    assert len({c.N for c in batch}) == 3
    c4, = gen.workload(4)
    assert (c4.L, c4.N, c4.Ns) == (100.0, 256, 16384)


def test_perturbation_fields_are_smooth_and_normalised():
    N, L = 64, 22.0
    v = gen.perturbation_fields(N, L, 99, 4)
    assert v.shape == (4, N)
    assert np.allclose(np.abs(v).max(axis=1), 1.0)
    spec = np.abs(np.fft.rfft(v, axis=1))
    assert spec[:, 0].max() < 1e-12 and spec[:, 5:].max() < 1e-12


def test_newton_guess_amplitude():
    N, L = 32, 22.0
    b = gen.newton_guess(N, L, 5, amplitude=2.0)
    x = gen.grid_x(N, L)
    u = sum(b[j] * np.sin(2 * np.pi * (j + 1) * x / L) for j in range(len(b)))
    assert abs(np.abs(u).max() - 2.0) < 1e-12 and np.all(b[4:] == 0)
