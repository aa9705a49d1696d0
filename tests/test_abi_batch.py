"""Host-side contract of the batched C ABI (no GPU: batch plan creation makes no CUDA call).
Argument validation, sizes, and the state errors of calls made before a workspace is bound."""
import ctypes
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

sf = pytest.importorskip("paper_2003_13569_gb300")
L = sf.lib()
BC = {"periodic": 0, "dirichlet": 1, "neumann": 2}


def _batch(sides, bcs, dims=None, alpha=1.5, dtype="f32", reaction=None):
    n = len(sides)
    dims = dims or [2] * n
    grids = (sf.Grid * n)()
    for i, (N, d) in enumerate(zip(sides, dims)):
        grids[i].dim = d
        for a in range(3):
            grids[i].N[a] = N if a < d else 1
            grids[i].lo[a] = 0.0
            grids[i].hi[a] = 50.0 if a < d else 1.0
    b = (ctypes.c_int32 * n)(*[BC[x] for x in bcs])
    al = (ctypes.c_double * (2 * n))(*([alpha] * (2 * n)))
    ka = (ctypes.c_double * (2 * n))(*([1.0, 30.0] * n))
    r = reaction or sf.Reaction()
    if reaction is None:
        r.kind, r.nspecies = sf.REACTION["gierer_meinhardt"], 2
        for i in range(4):
            r.p[i] = 1.0
        r.offset[0] = r.offset[1] = 1.0
    h = ctypes.c_void_p()
    code = L.sfrd_batch_plan(ctypes.byref(h), n, grids, b, al, ka, 0.05, sf.DTYPE[dtype], ctypes.byref(r))
    return code, h


def _unknowns(N, bc, dim=2):
    return (N + {"periodic": 0, "dirichlet": -1, "neumann": 1}[bc]) ** dim


def test_valid_batch_reports_count_unknowns_and_launches():
    sides, bcs = [96, 128, 200], ["periodic", "dirichlet", "neumann"]
    code, h = _batch(sides, bcs)
    assert code == 0 and h.value
    cnt, dof, lps = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert L.sfrd_batch_info(h, ctypes.byref(cnt), ctypes.byref(dof), ctypes.byref(lps)) == 0
    assert cnt.value == 3 and lps.value == 4 * 2 * 3        # one launch per axis length and pass
    assert dof.value == 2 * sum(_unknowns(N, b) for N, b in zip(sides, bcs))
    assert L.sfrd_batch_info(h, None, None, None) == 0                 # NULL outputs are skipped
    nb = ctypes.c_size_t()
    assert L.sfrd_batch_workspace_bytes(h, ctypes.byref(nb)) == 0
    assert nb.value % 256 == 0 and nb.value > 4 * dof.value * 4       # at least state + stored spectra
    L.sfrd_batch_destroy(h)


def test_3d_batch_launches_per_step():
    """Four passes per stage (middle, x, middle, slow), each one launch per engine group: here the
    shared-memory engine (32 intervals) and the register engine at 64."""
    code, h = _batch([32, 64], ["dirichlet", "neumann"], dims=[3, 3])
    assert code == 0
    lps = ctypes.c_int64()
    assert L.sfrd_batch_info(h, None, None, ctypes.byref(lps)) == 0 and lps.value == 4 * 4 * 2
    L.sfrd_batch_destroy(h)


@pytest.mark.parametrize("kw,code", [
    (dict(sides=[64], bcs=["periodic"], dims=[1]), -2),                      # 1D batches: unsupported
    (dict(sides=[64, 64], bcs=["periodic", "periodic"], dims=[2, 3]), -1),   # mixed dimensions
    (dict(sides=[64, 1024], bcs=["periodic", "periodic"]), -2),              # more than 512 intervals
    (dict(sides=[64, 64], bcs=["periodic", "neumann"], alpha=2.5), -1),      # alpha outside (1, 2]
    (dict(sides=[77], bcs=["periodic"]), -2),                                # 77 = 7 x 11 is not {2,3,5}-smooth
])
def test_invalid_batches_are_rejected(kw, code):
    got, h = _batch(**kw)
    assert got == code and not h.value


def test_null_arguments_are_rejected():
    g = (sf.Grid * 1)()
    b = (ctypes.c_int32 * 1)(0)
    a = (ctypes.c_double * 2)(1.5, 1.5)
    r = sf.Reaction()
    h = ctypes.c_void_p()
    assert L.sfrd_batch_plan(None, 1, g, b, a, a, 0.1, 1, ctypes.byref(r)) == -1
    assert L.sfrd_batch_plan(ctypes.byref(h), 0, g, b, a, a, 0.1, 1, ctypes.byref(r)) == -1
    assert L.sfrd_batch_plan(ctypes.byref(h), 1, None, b, a, a, 0.1, 1, ctypes.byref(r)) == -1
    assert L.sfrd_batch_plan(ctypes.byref(h), 1, g, b, None, a, 0.1, 1, ctypes.byref(r)) == -1
    assert L.sfrd_batch_plan(ctypes.byref(h), 1, g, b, a, a, 0.1, 1, None) == -1
    assert L.sfrd_batch_workspace_bytes(None, None) == -1
    assert L.sfrd_batch_info(None, None, None, None) == -1


def test_calls_before_bind_report_missing_workspace():
    code, h = _batch([64], ["neumann"])
    assert code == 0
    ptrs = (ctypes.c_void_p * 1)(None)
    assert L.sfrd_batch_advance(h, 1) == -3                             # SFRD_ENOWS
    assert L.sfrd_batch_load(h, ptrs, 0.0) in (-1, -3)
    assert L.sfrd_batch_store(h, ptrs) in (-1, -3)
    assert L.sfrd_batch_bind(h, None, 0, None) == -3                    # NULL workspace
    assert L.sfrd_batch_bind(h, ctypes.c_void_p(4096 + 16), 1 << 40, None) == -3   # misaligned
    L.sfrd_batch_destroy(h)
