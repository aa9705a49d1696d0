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


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_noalloc_forward_on_a_bound_plan_leaves_the_plan_bound(dtype, tol):
    """A caller may also hold a bound plan: the allocation-free call borrows the plan's tables for
    the duration of the call only, so the bound plan's own transform and time steps afterwards equal
    those of a fresh plan."""
    cfg = _cfg(2, (64, 40), "dirichlet")
    cfg["reaction"] = dict(kind="gray_scott", p=[0.04, 0.06], offset=[0, 0])
    s = sf.Solver(cfg, dtype=dtype)
    fresh = sf.Solver(cfg, dtype=dtype)
    rng = np.random.default_rng(7)
    u = torch.as_tensor(rng.uniform(0, 1, s.shape)).to(device="cuda", dtype=s.tdtype)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        uhat = torch.empty_like(u)
        rc = sf.lib().sfrd_forward_noalloc(s.handle, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(uhat.data_ptr()),
                                           stream)
        assert rc == 0, sf.lib().sfrd_last_error()
        assert _rel_max(uhat, fresh.forward(u)) < tol
    torch.testing.assert_close(s.forward(u), fresh.forward(u), rtol=0, atol=0)
    torch.testing.assert_close(s.run(u, nsteps=3), fresh.run(u, nsteps=3), rtol=0, atol=0)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_noalloc_forward_1d_and_writes_only_its_output(bc):
    """1D plans (the transform is the x pass alone), with the output between guard bands of a known byte
    pattern: the call writes the whole output and nothing next to it."""
    cfg = _cfg(1, (128,), bc)
    bound = sf.Solver(cfg, dtype="f64")
    r = cfg["reaction"]
    plan = sf.make_plan(1, cfg["N"], cfg["lo"], cfg["hi"], bc, cfg["alpha"], cfg["kappa"], cfg["dt"], "f64",
                        r["kind"], r["p"], r["offset"], nspecies=2)
    guard, pattern = 1 << 16, 0xA5
    nbytes = int(np.prod(bound.shape)) * 8
    raw = torch.full((2 * guard + nbytes,), pattern, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for call in range(2):
            u = torch.as_tensor(np.random.default_rng(200 + call).uniform(-1, 1, bound.shape)).cuda()
            rc = sf.lib().sfrd_forward_noalloc(plan, ctypes.c_void_p(u.data_ptr()),
                                               ctypes.c_void_p(raw.data_ptr() + guard), stream)
            assert rc == 0, sf.lib().sfrd_last_error()
            uhat = raw[guard:guard + nbytes].view(torch.float64).reshape(bound.shape)
            assert _rel_max(uhat, bound.forward(u)) < 1e-12
            host = raw.cpu().numpy()
            assert (host[:guard] == pattern).all() and (host[guard + nbytes:] == pattern).all()
    finally:
        sf.lib().sfrd_destroy(plan)
