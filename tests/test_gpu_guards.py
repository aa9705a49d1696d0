"""Out-of-bounds detection without a sanitizer: the workspace and the caller's fields are placed
between guard bands of a known byte pattern, the plan (or batch) is bound there and run through
every entry point that writes device memory, and the guard bytes must be unchanged afterwards."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _rand_fields  # noqa: E402

GUARD = 1 << 16
PATTERN = 0xA5


class Guarded:
    """A device buffer of `nbytes` (256-byte aligned) between two guard bands."""

    def __init__(self, nbytes):
        self.nbytes = int(nbytes)
        self.raw = torch.full((GUARD + self.nbytes + GUARD + 256,), PATTERN, dtype=torch.uint8, device="cuda")
        base = self.raw.data_ptr()
        self.ptr = (base + GUARD + 255) // 256 * 256
        self.off = self.ptr - base

    def intact(self):
        torch.cuda.synchronize()
        raw = self.raw.cpu().numpy()
        return bool((raw[:self.off] == PATTERN).all() and (raw[self.off + self.nbytes:] == PATTERN).all())


CASES = [(2, (64, 48), "neumann", "fhn"), (2, (96, 200), "periodic", "gray_scott"),
         (3, (16, 12, 10), "dirichlet", "schnakenberg"), (3, (64, 64, 64), "periodic", "gray_scott"),
         (1, (64,), "dirichlet", "fhn"), (1, (100,), "neumann", "gierer_meinhardt"),
         (2, (64, 1024), "periodic", "gray_scott"), (2, (64, 1024), "neumann", "fhn")]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dim,N,bc,kind", CASES)
def test_no_write_outside_workspace_or_fields(dim, N, bc, kind, dtype):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    s = sf.Solver(cfg, dtype=dtype)
    lib = sf.lib()
    ws = Guarded(s.info.workspace_bytes)
    assert lib.sfrd_bind(s.handle, ctypes.c_void_p(ws.ptr), ws.nbytes, ctypes.c_void_p(s.stream.cuda_stream)) == 0
    esize = 8 if dtype == "f64" else 4
    nbytes = int(np.prod(s.shape)) * esize
    u0 = np.stack(_rand_fields(cfg, seed=8, lo=0.0 if kind in ("fhn", "gray_scott") else -0.05,
                               hi=1.0 if kind in ("fhn", "gray_scott") else 0.05))
    fin, fout, fhat = Guarded(nbytes), Guarded(nbytes), Guarded(nbytes)
    src = torch.as_tensor(u0).to(device="cuda", dtype=s.tdtype).contiguous()
    # copy the field into the guarded input buffer
    dst = torch.as_strided(fin.raw, (nbytes,), (1,), fin.off)
    dst.copy_(src.view(torch.uint8).reshape(-1))
    assert lib.sfrd_load(s.handle, ctypes.c_void_p(fin.ptr), 0.0) == 0
    assert lib.sfrd_advance(s.handle, 3) == 0
    assert lib.sfrd_store(s.handle, ctypes.c_void_p(fout.ptr)) == 0
    assert lib.sfrd_forward(s.handle, ctypes.c_void_p(fin.ptr), ctypes.c_void_p(fhat.ptr)) == 0
    assert lib.sfrd_inverse(s.handle, ctypes.c_void_p(fhat.ptr), ctypes.c_void_p(fout.ptr)) == 0
    for w in sf.COEFFICIENTS:
        assert lib.sfrd_coefficients(s.handle, sf.COEFFICIENTS.index(w), ctypes.c_void_p(fhat.ptr)) == 0
    assert lib.sfrd_check_finite(s.handle) == 0
    for g, name in ((ws, "workspace"), (fin, "input"), (fout, "output"), (fhat, "spectrum")):
        assert g.intact(), name


def test_batch_writes_stay_inside_its_workspace():
    cfgs = W.gm_instances(12, seed=7)
    b = sf.Batch(cfgs, dtype="f32")
    nb = ctypes.c_size_t()
    lib = sf.lib()
    assert lib.sfrd_batch_workspace_bytes(b.handle, ctypes.byref(nb)) == 0
    ws = Guarded(nb.value)
    assert lib.sfrd_batch_bind(b.handle, ctypes.c_void_p(ws.ptr), ws.nbytes, ctypes.c_void_p(b.stream.cuda_stream)) == 0
    b.load([np.stack(W.initial_fields(c)) for c in cfgs])
    b.advance(3)
    b.store()
    assert ws.intact()
