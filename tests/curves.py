"""Shared test helpers: end points and trial curves of the synthetic workloads,
built from the seeded generator and the stored (oracle-computed) equilibria."""
import numpy as np

from paper_2301_11704_gb300 import gen

end_points = gen.end_points
perturbation = gen.perturbation


def random_smooth_curve(rng, M, N, decay=0.5, ends=True):
    """Random spectral curve [M+2, N/2] with decaying modes; zero end rows if ends=False."""
    U = (rng.standard_normal((M + 2, N // 2)) + 1j * rng.standard_normal((M + 2, N // 2)))
    U *= decay ** np.arange(N // 2)[None, :]
    th = np.arange(M + 2) * np.pi / (M + 1)
    U *= (0.3 + np.sin(th))[:, None]
    U[:, 0] = U[:, 0].real
    if not ends:
        U[0] = 0
        U[-1] = 0
    return U
