"""GB300 (sm_103a) implementation of the weakly compressible SPH time step of
Dominguez, Crespo & Gomez-Gesteira (DualSPHysics): NL, PI and SU as CUDA kernels
behind the C ABI of ``include/sph.h``.

Importing the package does not load the shared library; ``sph.lib()`` does, and
raises when it has not been built.
"""
from . import build  # noqa: F401

__all__ = ["build", "sph"]
