"""GB300-native adjoint descent for connecting orbits of the Kuramoto-Sivashinsky
equation (Ashtari & Schneider, arXiv 2301.11704).

The compute path is the CUDA library libksconn.so (include/ksconn.h), built for
sm_103a; ``KSCurve`` wraps it with PyTorch-owned device memory and streams.
"""
from . import build  # noqa: F401

__all__ = ["KSCurve", "build"]


def __getattr__(name):
    if name == "KSCurve":
        from .curve import KSCurve
        return KSCurve
    raise AttributeError(name)
