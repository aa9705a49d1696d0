"""The allocation-free forward transform against the workspace-bound one.

sfrd_forward_noalloc serves callers that may not allocate device memory (a
component inside a host application that owns the GPU memory budget, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation):
its scratch is a fixed device array inside the library.  The plan used here is
created but never bound to a workspace.  Each case calls the entry point twice
in a row with different inputs, since every call reuses the array the previous
call left behind.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
import workloads as W  # noqa: E402


def _cfg(dim, N, bc):
    return dict(dim=dim, N=tuple(N), lo=(0.0,) * dim, hi=(2.0,) * dim, bc=bc, alpha=(1.5, 1.8), kappa=(0.5, 0.1),
                dt=0.1, nsteps=1, reaction=dict(kind="none", p=[], offset=[0, 0]), dtype="f64", seed=0)


def _rel_max(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("dim,N,bc", [(2, (64, 48), "neumann"), (2, (40, 128), "periodic"),
                                      (3, (32, 24, 64), "dirichlet")])
def test_noalloc_forward_matches_bound_forward_on_two_calls(dim, N, bc, dtype, tol):
    cfg = _cfg(dim, N, bc)
    bound = sf.Solver(cfg, dtype=dtype)
    r = cfg["reaction"]
    plan = sf.make_plan(dim, N, cfg["lo"], cfg["hi"], bc, cfg["alpha"], cfg["kappa"], cfg["dt"], dtype,
                        r["kind"], r["p"], r["offset"], nspecies=2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            u = torch.as_tensor(rng.uniform(-1, 1, bound.shape)).to(device="cuda", dtype=bound.tdtype)
            uhat = torch.empty_like(u)
            rc = sf.lib().sfrd_forward_noalloc(plan, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(uhat.data_ptr()),
                                               stream)
            assert rc == 0, sf.lib().sfrd_last_error()
            assert _rel_max(uhat, bound.forward(u)) < tol
    finally:
        sf.lib().sfrd_destroy(plan)


def test_noalloc_forward_rejects_problems_beyond_its_scratch():
    cfg = W.config("schnak256")
    r = cfg["reaction"]
    plan = sf.make_plan(3, cfg["N"], cfg["lo"], cfg["hi"], cfg["bc"], cfg["alpha"], cfg["kappa"], cfg["dt"], "f32",
                        r["kind"], r["p"], r["offset"])
    try:
        dummy = torch.empty(16, device="cuda")
        rc = sf.lib().sfrd_forward_noalloc(plan, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                           None)
        assert rc == -2
    finally:
        sf.lib().sfrd_destroy(plan)
