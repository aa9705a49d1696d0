"""GPU discrete adjoint (checkpointed) against the oracle's adjoint and central differences.

Tolerances: FP64 gradients within 1e-6 relative of central differences (h = 1e-6)
and within 1e-8 of the oracle's reverse-mode derivative of the same step; the FP32
adjoint is compared with the FP64 one and its error reported (loose bound).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.bridge import problem as oracle_problem, reaction_fns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402


def _cfg(N, bc, kind, dim=2, alpha=(1.5, 1.7), kappa=(0.3, 0.05), dt=0.05):
    p = {"fhn": [0.1, 0.01, 0.5, 1.0, 0.0], "gray_scott": [0.04, 0.06], "schnakenberg": [5.0, 0.1, 0.9],
         "gierer_meinhardt": [1.0, 1.0, 1.0, 1.0]}[kind]
    off = {"schnakenberg": [1.0, 0.9], "gierer_meinhardt": [1.0, 1.0]}.get(kind, [0.0, 0.0])
    return dict(dim=dim, N=tuple(N), lo=(0.0,) * dim, hi=tuple(3.0 + d for d in range(dim)), bc=bc, alpha=alpha,
                kappa=kappa, dt=dt, nsteps=1, reaction=dict(kind=kind, p=p, offset=off), dtype="f64", seed=0)


def _fields(cfg, seed, kind):
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    rng = np.random.default_rng(seed)
    shp = W.field_shape(cfg)
    return np.stack([rng.uniform(lo, hi, shp) for _ in range(2)])


def _loss(cfg, u0, target, nsteps, dtype="f64"):
    uT = sf.Solver(cfg, dtype=dtype).run(u0, nsteps=nsteps).double().cpu().numpy()
    return 0.5 * float(np.sum((uT - target) ** 2))


def _grads(cfg, u0, target, nsteps, K, dtype="f64"):
    s = sf.Solver(cfg, dtype=dtype)
    uT = s.run_checkpointed(u0, 0.0, nsteps, K)
    g = uT - torch.as_tensor(target, device=uT.device, dtype=uT.dtype)
    du0, da, dk, dp = s.adjoint(g, 0.0, nsteps, K)
    return du0.double().cpu().numpy(), da, dk, dp


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


CASES = [((64, 64), "neumann", "fhn", 2), ((64, 128), "periodic", "gray_scott", 2),
         ((64, 64), "dirichlet", "schnakenberg", 2), ((128, 64), "neumann", "gierer_meinhardt", 2),
         ((64, 64, 64), "dirichlet", "schnakenberg", 3),
         # register-engine lengths 3 * 2^5, 5^2 * 2^3 and 3 * 2^7
         ((96, 200), "dirichlet", "fhn", 2), ((200, 96), "periodic", "gierer_meinhardt", 2),
         ((384, 96), "neumann", "gray_scott", 2),
         # 1D plans: the reverse combinations act on the x spectra directly
         ((128,), "neumann", "fhn", 1), ((96,), "dirichlet", "gray_scott", 1), ((256,), "periodic", "schnakenberg", 1)]


@pytest.mark.parametrize("scheme", ["p13", "cox_matthews"])
@pytest.mark.parametrize("N,bc,dim", [((64, 128), "neumann", 2), ((96, 64), "dirichlet", 2),
                                      ((64, 64, 64), "periodic", 3), ((128,), "neumann", 1)])
def test_adjoint_is_the_transpose_of_the_linear_run(N, bc, dim, scheme):
    """Dot-product test through the C ABI: with a linear reaction the checkpointed run u0 -> u_M is a
    linear map J, and sfrd_adjoint with dl/du_M = w must return J^T w: <J v, w> = <v, J^T w> to
    rounding, for random v, w (FP64).  With the library's diagonal linear reaction J is symmetric for
    periodic and Dirichlet grids, where the test checks scaling and coefficients; the Neumann cases
    (weighted DCT-I, not symmetric) also tell J from J^T."""
    cfg = dict(_cfg(N, bc, "fhn", dim=dim, alpha=(1.5, 1.8), kappa=(0.4, 0.1), dt=0.02), scheme=scheme)
    cfg["reaction"] = dict(kind="linear", p=[-0.7], offset=[0.0, 0.0])
    rng = np.random.default_rng(23)
    shp = (2,) + W.field_shape(cfg)
    v, w = rng.standard_normal(shp), rng.standard_normal(shp)
    nsteps, K = 5, 2
    s = sf.Solver(cfg, dtype="f64")
    Jv = s.run_checkpointed(v, 0.0, nsteps, K)
    JTw = s.adjoint(torch.as_tensor(w, device=Jv.device), 0.0, nsteps, K)[0].double().cpu().numpy()
    Jv = Jv.double().cpu().numpy()
    lhs, rhs = float(np.sum(Jv * w)), float(np.sum(v * JTw))
    assert abs(lhs - rhs) <= 1e-12 * float(np.linalg.norm(Jv) * np.linalg.norm(w))


@pytest.mark.parametrize("N,bc,kind,dim", CASES)
def test_adjoint_matches_oracle_adjoint(N, bc, kind, dim):
    cfg = _cfg(N, bc, kind, dim=dim, dt=0.02 if dim == 3 else 0.05)
    nsteps, K = (4, 3) if dim == 3 else (7, 3)
    u0 = _fields(cfg, 1, kind)
    target = _fields(cfg, 2, kind)
    du0, da, dk, dp = _grads(cfg, u0, target, nsteps, K)
    s = O.ETDRK4P13(oracle_problem(cfg))
    uT = s.run(list(u0), 0.0, nsteps)
    dparams = reaction_fns(cfg)[2]
    ref = O.adjoint_run(s, list(u0), 0.0, nsteps, [a - b for a, b in zip(uT, target)], dparams=dparams)
    ref_u0 = np.stack(ref["u0"])
    assert float(np.max(np.abs(du0 - ref_u0)) / np.max(np.abs(ref_u0))) < 1e-9
    for sp in range(2):
        assert _rel(da[sp], ref["alpha"][sp]) < 1e-8
        assert _rel(dk[sp], ref["kappa"][sp]) < 1e-8 or abs(dk[sp] - ref["kappa"][sp]) < 1e-12
    if kind == "fhn":
        assert _rel(dp[0], ref["params"]) < 1e-8


@pytest.mark.parametrize("N,bc,kind,dim", CASES[:4] + CASES[5:6] + CASES[8:10])
def test_adjoint_matches_central_differences(N, bc, kind, dim):
    cfg = _cfg(N, bc, kind, dim=dim)
    nsteps, K = 6, 4
    u0 = _fields(cfg, 3, kind)
    target = _fields(cfg, 4, kind)
    du0, da, dk, dp = _grads(cfg, u0, target, nsteps, K)
    h = 1e-6

    def with_(alpha=None, kappa=None, p0=None):
        c = dict(cfg)
        if alpha is not None:
            c["alpha"] = alpha
        if kappa is not None:
            c["kappa"] = kappa
        if p0 is not None:
            r = dict(cfg["reaction"])
            r["p"] = [p0] + list(r["p"][1:])
            c["reaction"] = r
        return c

    a0, a1 = cfg["alpha"]
    k0, k1 = cfg["kappa"]
    fd = (_loss(with_(alpha=(a0 + h, a1)), u0, target, nsteps) - _loss(with_(alpha=(a0 - h, a1)), u0, target,
                                                                         nsteps)) / (2 * h)
    assert _rel(da[0], fd) < 1e-6
    fd = (_loss(with_(kappa=(k0, k1 + h)), u0, target, nsteps) - _loss(with_(kappa=(k0, k1 - h)), u0, target,
                                                                         nsteps)) / (2 * h)
    assert _rel(dk[1], fd) < 1e-6
    p0 = cfg["reaction"]["p"][0]
    fd = (_loss(with_(p0=p0 + h), u0, target, nsteps) - _loss(with_(p0=p0 - h), u0, target, nsteps)) / (2 * h)
    assert _rel(dp[0], fd) < 1e-6
    v = np.random.default_rng(9).standard_normal(u0.shape)
    fd = (_loss(cfg, u0 + h * v, target, nsteps) - _loss(cfg, u0 - h * v, target, nsteps)) / (2 * h)
    assert _rel(float(np.sum(du0 * v)), fd) < 1e-6


@pytest.mark.parametrize("N,bc,kind,dim", [((64, 64), "neumann", "fhn", 2), ((96, 128), "dirichlet", "schnakenberg", 2),
                                          ((64, 64, 64), "periodic", "gray_scott", 3)])
def test_cox_matthews_adjoint_matches_oracle_and_central_differences(N, bc, kind, dim):
    """The adjoint of the Cox-Matthews scheme: the same reverse sweep over its coefficient arrays,
    with dC/dL of the exact-exponential coefficients for the kappa and alpha gradients."""
    cfg = dict(_cfg(N, bc, kind, dim=dim, dt=0.02 if dim == 3 else 0.05), scheme="cox_matthews")
    nsteps, K = (4, 3) if dim == 3 else (6, 4)
    u0 = _fields(cfg, 5, kind)
    target = _fields(cfg, 6, kind)
    du0, da, dk, dp = _grads(cfg, u0, target, nsteps, K)
    s = O.ETDRK4P13(oracle_problem(cfg), scheme="cox_matthews")
    uT = s.run(list(u0), 0.0, nsteps)
    ref = O.adjoint_run(s, list(u0), 0.0, nsteps, [a - b for a, b in zip(uT, target)],
                        dparams=reaction_fns(cfg)[2])
    ref_u0 = np.stack(ref["u0"])
    assert float(np.max(np.abs(du0 - ref_u0)) / np.max(np.abs(ref_u0))) < 1e-9
    for sp in range(2):
        assert _rel(da[sp], ref["alpha"][sp]) < 1e-8
        assert _rel(dk[sp], ref["kappa"][sp]) < 1e-8 or abs(dk[sp] - ref["kappa"][sp]) < 1e-12
    h = 1e-6
    a0, a1 = cfg["alpha"]
    fd = (_loss(dict(cfg, alpha=(a0, a1 + h)), u0, target, nsteps)
          - _loss(dict(cfg, alpha=(a0, a1 - h)), u0, target, nsteps)) / (2 * h)
    assert _rel(da[1], fd) < 1e-6
    k0, k1 = cfg["kappa"]
    fd = (_loss(dict(cfg, kappa=(k0 + h, k1)), u0, target, nsteps)
          - _loss(dict(cfg, kappa=(k0 - h, k1)), u0, target, nsteps)) / (2 * h)
    assert _rel(dk[0], fd) < 1e-6


def test_checkpoint_interval_does_not_change_gradients():
    cfg = _cfg((64, 64), "neumann", "fhn")
    u0, target = _fields(cfg, 5, "fhn"), _fields(cfg, 6, "fhn")
    a = _grads(cfg, u0, target, 9, 9)
    b = _grads(cfg, u0, target, 9, 2)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-13 * np.max(np.abs(a[0])))
    for x, y in zip(a[1] + a[2] + a[3], b[1] + b[2] + b[3]):
        assert abs(x - y) <= 1e-12 * max(abs(x), 1e-300) + 1e-15


def test_fp32_adjoint_error_is_reported():
    cfg = _cfg((128, 128), "periodic", "gray_scott")
    u0, target = _fields(cfg, 7, "gray_scott"), _fields(cfg, 8, "gray_scott")
    g64 = _grads(cfg, u0, target, 10, 5, "f64")
    g32 = _grads(cfg, u0, target, 10, 5, "f32")
    e = float(np.linalg.norm(g32[0] - g64[0]) / np.linalg.norm(g64[0]))
    print("fp32 adjoint dL/du0 rel l2 error %.2e; dalpha %.2e" % (e, _rel(g32[1][0], g64[1][0])))
    assert e < 1e-3 and _rel(g32[1][0], g64[1][0]) < 1e-2


def test_autograd_function_matches_direct_adjoint():
    cfg = _cfg((64, 64), "neumann", "fhn")
    u0 = torch.as_tensor(_fields(cfg, 10, "fhn"), device="cuda").requires_grad_(True)
    target = torch.as_tensor(_fields(cfg, 11, "fhn"), device="cuda")
    alpha = torch.tensor(cfg["alpha"], dtype=torch.float64, requires_grad=True)
    kappa = torch.tensor(cfg["kappa"], dtype=torch.float64, requires_grad=True)
    params = torch.tensor(cfg["reaction"]["p"], dtype=torch.float64, requires_grad=True)
    uT = sf.run(u0, alpha, kappa, params, cfg, nsteps=5, ckpt_every=2)
    loss = 0.5 * ((uT - target) ** 2).sum()
    loss.backward()
    du0, da, dk, dp = _grads(cfg, u0.detach().cpu().numpy(), target.cpu().numpy(), 5, 2)
    np.testing.assert_allclose(u0.grad.cpu().numpy(), du0, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(alpha.grad.numpy(), da, rtol=1e-12)
    np.testing.assert_allclose(kappa.grad.numpy(), dk, rtol=1e-12)
    np.testing.assert_allclose(params.grad.numpy()[:1], dp[:1], rtol=1e-12)


def test_adjoint_workload_fhn257_central_differences():
    """2D FitzHugh-Nagumo on 257^2 Neumann nodes, 500 steps, checkpoints every 50: gradients of
    0.5 ||u_T - target||^2 w.r.t. alpha (both species), kappa_u, mu and u0; the target comes from
    the same solver at alpha = 1.6 from another seed."""
    cfg = W.config("fhn256_adjoint")
    n, K = cfg["nsteps"], cfg["checkpoint_every"]
    tg = cfg["target"]
    u0 = np.stack(W.initial_fields(cfg))
    tcfg = dict(cfg, alpha=(tg["alpha"], tg["alpha"]), kappa=(tg["kappa_u"], cfg["kappa"][1]))
    target = sf.Solver(tcfg, dtype="f64").run(np.stack(W.initial_fields(cfg, seed=tg["seed"])),
                                              nsteps=n).cpu().numpy()
    du0, da, dk, dp = _grads(cfg, u0, target, n, K)
    h = 1e-6
    a = cfg["alpha"][0]
    fd = (_loss(dict(cfg, alpha=(a + h, a + h)), u0, target, n)
          - _loss(dict(cfg, alpha=(a - h, a - h)), u0, target, n)) / (2 * h)
    assert _rel(da[0] + da[1], fd) < 1e-6
    k = cfg["kappa"]
    fd = (_loss(dict(cfg, kappa=(k[0] + h, k[1])), u0, target, n)
          - _loss(dict(cfg, kappa=(k[0] - h, k[1])), u0, target, n)) / (2 * h)
    assert _rel(dk[0], fd) < 1e-6
    r = cfg["reaction"]
    fd = (_loss(dict(cfg, reaction=dict(r, p=[r["p"][0] + h] + r["p"][1:])), u0, target, n)
          - _loss(dict(cfg, reaction=dict(r, p=[r["p"][0] - h] + r["p"][1:])), u0, target, n)) / (2 * h)
    assert _rel(dp[0], fd) < 1e-6
    v = np.random.default_rng(12).standard_normal(u0.shape)
    fd = (_loss(cfg, u0 + h * v, target, n) - _loss(cfg, u0 - h * v, target, n)) / (2 * h)
    assert _rel(float(np.sum(du0 * v)), fd) < 1e-6


def test_adjoint_workload_fhn257_matches_oracle_adjoint_20_steps():
    cfg = W.config("fhn256_adjoint")
    n, K = 20, 8
    u0 = np.stack(W.initial_fields(cfg))
    target = np.stack(W.initial_fields(cfg, seed=cfg["target"]["seed"]))
    du0, da, dk, dp = _grads(cfg, u0, target, n, K)
    s = O.ETDRK4P13(oracle_problem(cfg))
    uT = s.run(list(u0), 0.0, n)
    ref = O.adjoint_run(s, list(u0), 0.0, n, [a - b for a, b in zip(uT, target)], dparams=reaction_fns(cfg)[2])
    ref_u0 = np.stack(ref["u0"])
    assert float(np.max(np.abs(du0 - ref_u0)) / np.max(np.abs(ref_u0))) < 1e-9
    assert _rel(da[0] + da[1], ref["alpha"][0] + ref["alpha"][1]) < 1e-8
    assert _rel(dk[0], ref["kappa"][0]) < 1e-8
    assert _rel(dp[0], ref["params"]) < 1e-8
