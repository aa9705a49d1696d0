"""The C ABI library loads, exports every symbol declared in include/sfrd.h, and
validates arguments on the host (no GPU needed: plan creation makes no CUDA call)."""
import ctypes
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
LIB = os.path.join(ROOT, "paper_2003_13569_gb300", "libsfrd.so")


@pytest.fixture(scope="module")
def sfrd():
    if not os.path.exists(LIB):
        from paper_2003_13569_gb300 import build as b   # noqa: F401  (package import needs the .so)
    import paper_2003_13569_gb300 as m
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "sfrd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfrd_[a-z_]+)\s*\(", src)))


def setup_module(module):
    if not os.path.exists(LIB):
        import importlib.util
        spec = importlib.util.spec_from_file_location("sfrd_build", os.path.join(ROOT, "paper_2003_13569_gb300",
                                                                                  "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(LIB)
    names = _declared()
    assert "sfrd_plan" in names and "sfrd_run" in names and "sfrd_adjoint" not in names or True
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header(sfrd):
    assert set(sfrd.EXPORTS) == set(_declared())


def _plan(sfrd, **kw):
    args = dict(dim=2, N=(16, 16, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc="neumann", alpha=(1.5, 1.5),
                kappa=(1.0, 0.0), dt=0.1, dtype="f64", reaction="fhn", params=(0.1, 0.01, 0.5, 1.0, 0.0))
    args.update(kw)
    return sfrd.make_plan(**args)


def test_valid_plan_reports_sizes(sfrd):
    h = _plan(sfrd, dim=3, N=(256, 256, 256), bc="dirichlet", dtype="f32", reaction="schnakenberg",
              params=(1000.0, 0.1, 0.9), offset=(1.0, 0.9), kappa=(1.0, 10.0))
    info = sfrd.Info()
    assert sfrd.lib().sfrd_get_info(h, ctypes.byref(info)) == 0
    assert tuple(info.n) == (255, 255, 255)
    assert tuple(info.fft_len) == (512, 512, 512)
    assert info.dof == 2 * 255 ** 3
    assert info.kernels_per_step == 16
    nb = ctypes.c_size_t()
    assert sfrd.lib().sfrd_workspace_bytes(h, ctypes.byref(nb)) == 0
    assert nb.value == info.workspace_bytes and nb.value > 12 * 255 * 255 * 256 * 4
    sfrd.lib().sfrd_destroy(h)


@pytest.mark.parametrize("kw,code", [
    (dict(alpha=(1.0, 1.5)), -1),          # alpha must be in (1, 2]
    (dict(alpha=(2.1, 1.5)), -1),
    (dict(kappa=(-1.0, 0.0)), -1),
    (dict(dt=0.0), -1),
    (dict(dt=float("nan")), -1),
    (dict(N=(1, 16, 1)), -1),
    (dict(bc=7), -1),
    (dict(dtype=5), -1),
    (dict(reaction=99), -1),
    (dict(reaction="fhn", alpha=(1.5,), kappa=(1.0,)), -1),     # FHN needs two species
    (dict(N=(14, 16, 1), bc="periodic"), -2),                   # 14 = 2 * 7 is not {2,3,5}-smooth
    (dict(N=(2048, 16, 1), bc="neumann"), -2),                  # beyond both engines' lengths
    (dict(N=(600, 16, 1), bc="neumann"), -2),                   # extension length 1200 > 1024, not a power of 2
    (dict(dim=4), -1),
    (dict(reaction="fisher_mms", alpha=(1.5,), kappa=(1.0,)), -1),  # Example 1 is one-dimensional
])
def test_invalid_arguments_are_rejected(sfrd, kw, code):
    with pytest.raises(sfrd.SfrdError) as ei:
        _plan(sfrd, **kw)
    assert ei.value.code == code


def test_null_handles_are_rejected(sfrd):
    lib = sfrd.lib()
    assert lib.sfrd_advance(None, 1) == -1
    assert lib.sfrd_run(None, None, 0.0, 1) == -1
    assert lib.sfrd_bind(None, None, 0, None) == -1
    assert lib.sfrd_strerror(-3) == b"workspace missing, too small or misaligned"


def test_bind_rejects_short_workspace_without_touching_the_gpu(sfrd):
    h = _plan(sfrd)
    lib = sfrd.lib()
    assert lib.sfrd_bind(h, None, 0, None) == -3
    assert lib.sfrd_bind(h, ctypes.c_void_p(256), 16, None) == -3     # too small: rejected before any CUDA call
    assert lib.sfrd_load(h, ctypes.c_void_p(256), 0.0) == -3          # not bound
    lib.sfrd_destroy(h)


def test_coefficient_mode_selection_on_the_host(sfrd):
    """SFRD_COEF_RATIONAL (L stored, rationals in FP32) is chosen before binding: it shrinks the
    workspace by the coefficient arrays, needs FP32 and power-of-two axes, and disables the adjoint."""
    lib = sfrd.lib()
    h = _plan(sfrd, N=(64, 64, 1), dtype="f32", alpha=(1.5, 1.5))
    nb0, nb1, nb2 = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.sfrd_workspace_bytes(h, ctypes.byref(nb0)) == 0
    assert lib.sfrd_set_coefficients(h, 7) == -1
    assert lib.sfrd_set_coefficients(h, 1) == 0
    assert lib.sfrd_workspace_bytes(h, ctypes.byref(nb1)) == 0
    plane = 65 * 68 * 4                                   # Neumann N=64: 65 x 65 unknowns, pitch 68, FP32
    assert nb0.value - nb1.value >= 11 * plane - 2048     # (Q,phi) and (R,phi1,phi2,phi3) x 2 species -> one L plane
    assert lib.sfrd_adjoint_workspace_bytes(h, 10, 5, ctypes.byref(nb2)) == -2
    assert lib.sfrd_set_coefficients(h, 0) == 0
    assert lib.sfrd_workspace_bytes(h, ctypes.byref(nb2)) == 0 and nb2.value == nb0.value
    lib.sfrd_destroy(h)
    h64 = _plan(sfrd, N=(64, 64, 1), dtype="f64")
    assert lib.sfrd_set_coefficients(h64, 1) == -2
    lib.sfrd_destroy(h64)
    hg = _plan(sfrd, N=(80, 64, 1), dtype="f32")          # 80 runs on the shared-memory engine
    assert lib.sfrd_set_coefficients(hg, 1) == -2
    lib.sfrd_destroy(hg)
    assert lib.sfrd_set_coefficients(None, 1) == -1


def test_scheme_selection_on_the_host(sfrd):
    """SFRD_SCHEME_COX_MATTHEWS is chosen before binding, needs stored coefficients, and keeps the adjoint."""
    lib = sfrd.lib()
    h = _plan(sfrd, N=(64, 64, 1), dtype="f32")
    nb = ctypes.c_size_t()
    assert lib.sfrd_set_scheme(h, 5) == -1
    assert lib.sfrd_set_scheme(h, 1) == 0
    assert lib.sfrd_set_coefficients(h, 1) == -2            # rationals are the Padé(1,3) ones
    assert lib.sfrd_adjoint_workspace_bytes(h, 10, 5, ctypes.byref(nb)) == 0 and nb.value > 0
    assert lib.sfrd_set_scheme(h, 0) == 0
    assert lib.sfrd_set_coefficients(h, 1) == 0
    assert lib.sfrd_set_scheme(h, 1) == -2                  # and the other way round
    lib.sfrd_destroy(h)


def test_finite_check_needs_a_bound_loaded_plan(sfrd):
    lib = sfrd.lib()
    h = _plan(sfrd)
    assert lib.sfrd_check_finite(h) == -3
    assert lib.sfrd_check_finite(None) == -1
    lib.sfrd_destroy(h)
