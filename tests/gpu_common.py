"""Helpers shared by the GPU tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_3711_gb300 import build
    build.build()
    return torch


def make_sim(case, precision, **kw):
    """Simulation of a case through the C ABI (kw: device, stream, pi_kernel)."""
    from paper_1110_3711_gb300.sph import Simulation
    return Simulation.from_case(case, precision=precision, **kw)


def rel_err(a, b, scale):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / scale)
