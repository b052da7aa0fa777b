"""GB300-native uniform-grid mechanical interactions of spherical cell agents
(after Hesam et al., "GPU Acceleration of 3D Agent-Based Biological
Simulations", arXiv 2105.00039).

  ugmech      ctypes binding of the C ABI (include/ugmech.h)
  autograd    differentiable trajectories over the library's adjoint
  populations seeded synthetic populations
"""
from . import populations  # noqa: F401

__all__ = ["populations", "ugmech", "autograd"]


def __getattr__(name):
    if name in ("ugmech", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
