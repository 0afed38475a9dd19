"""The C-ABI library loads on a CPU-only host and exports every call that
include/sph.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsph():
    from paper_1110_3711_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libsph):
    names = _declared("sph.h")
    assert "sph_interact" in names and "sph_create" in names
    for n in names:
        assert hasattr(libsph, n), n


def test_binding_covers_header():
    from paper_1110_3711_gb300 import sph
    assert set(_declared("sph.h")) == set(sph.exported_symbols())


def test_error_strings_and_workspace_on_cpu(libsph):
    from paper_1110_3711_gb300 import sph
    from sphcases import dam_break
    assert sph.lib().sph_error_string(-6).decode().startswith("call out of order")
    c = dam_break(0.02)
    p = sph.make_params(c.params, "fp32")
    ws = sph.sph_workspace_bytes(p, c.n_f, c.n_b)
    p64 = sph.make_params(c.params, "fp64")
    assert sph.sph_workspace_bytes(p64, c.n_f, c.n_b) > ws > c.n * 100
    bad = sph.make_params(c.params, "fp32")
    bad.cell_size = c.params.h  # below the support 2h
    with pytest.raises(sph.SphError):
        sph.sph_workspace_bytes(bad, c.n_f, c.n_b)
    g5 = sph.make_params(c.params, "fp32")
    g5.gamma = 5.0  # the float32 sound speed is the gamma = 7 form
    with pytest.raises(sph.SphError):
        sph.sph_workspace_bytes(g5, c.n_f, c.n_b)
    g5 = sph.make_params(c.params, "fp64")
    g5.gamma = 5.0
    assert sph.sph_workspace_bytes(g5, c.n_f, c.n_b) > 0
    # cells of edge h (125-cell search): float64 and the thread-per-particle
    # kernel only; below h the support spans more than two cells
    for prec, kern, ok in (("fp64", "warp", True), ("fp32", "thread", True),
                           ("fp32", "warp", False), ("fp32", "thread_fastcells", False)):
        q = sph.make_params(c.params, prec, kern)
        q.cell_size = c.params.h
        if ok:
            assert sph.sph_workspace_bytes(q, c.n_f, c.n_b) > ws
        else:
            with pytest.raises(sph.SphError):
                sph.sph_workspace_bytes(q, c.n_f, c.n_b)
    # the symmetric warp kernel: cells >= 2h and no tensile correction
    q = sph.make_params(c.params, "fp32", "warp_sym")
    assert sph.sph_workspace_bytes(q, c.n_f, c.n_b) == ws
    q.cell_size = c.params.h
    with pytest.raises(sph.SphError):
        sph.sph_workspace_bytes(q, c.n_f, c.n_b)
    q = sph.make_params(c.params, "fp32", "warp_sym")
    q.tensile_eps, q.tensile_pos = 0.2, 0.01
    with pytest.raises(sph.SphError):
        sph.sph_workspace_bytes(q, c.n_f, c.n_b)
    q = sph.make_params(c.params, "fp64")
    q.cell_size = 0.99 * c.params.h
    with pytest.raises(sph.SphError):
        sph.sph_workspace_bytes(q, c.n_f, c.n_b)
    # float64: the warp-per-item design or one thread per particle
    for kern, ok in (("warp", True), ("thread", True), ("thread_fastcells", False),
                     ("warp_sym", False)):
        q = sph.make_params(c.params, "fp64", kern)
        if ok:
            assert sph.sph_workspace_bytes(q, c.n_f, c.n_b) > ws
        else:
            with pytest.raises(sph.SphError):
                sph.sph_workspace_bytes(q, c.n_f, c.n_b)


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    """The binding refuses to run when libsph.so is missing."""
    from paper_1110_3711_gb300 import sph, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(sph, "_lib", None)
    with pytest.raises(RuntimeError):
        sph.lib()


def test_fma_rate_rejects_bad_arguments_before_any_cuda_call(libsph):
    """sph_fma_rate checks its arguments on the host: no scratch, no output or
    an unknown precision give SPH_ERR_INVALID_ARG without touching a GPU."""
    import ctypes as C
    from paper_1110_3711_gb300 import sph
    L = sph.lib()
    out = C.c_double(0.0)
    assert L.sph_fma_rate(1, None, None, C.byref(out)) == -1
    assert L.sph_fma_rate(1, C.c_void_p(16), None, None) == -1
    assert L.sph_fma_rate(7, C.c_void_p(16), None, C.byref(out)) == -1
    assert out.value == 0.0
