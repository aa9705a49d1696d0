"""The 1D path: per stage the x pass (inverse transform, reaction, forward transform) and a pointwise
spectral combination.  Checked against the FP64 oracle (whole runs, transforms) and, through
Example 1's manufactured solution, against the paper's Table 1."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.bridge import solver as oracle_solver
from tests.helpers import library_forward, rel_max
from tests.test_oracle_pins import _same_to_printed_digits, _table

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _np, _rand_fields  # noqa: E402


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [64, 48, 100])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_1d_transform_matches_dense_matrices(bc, N, dtype):
    cfg = _cfg(1, (N,), bc, kind="none")
    s = sf.Solver(cfg, dtype=dtype)
    u = _rand_fields(cfg, seed=3)
    got = _np(s.forward(u))
    tol = 1e-12 if dtype == "f64" else 2e-6 * math.sqrt(N)
    for sp in range(2):
        assert rel_max(got[sp], library_forward(u[sp], bc, (N,))) < tol
    back = _np(s.inverse(got))
    for sp in range(2):
        assert rel_max(back[sp], u[sp]) < tol


@pytest.mark.parametrize("N", [64, 48])
@pytest.mark.parametrize("bc,kind", [("periodic", "gray_scott"), ("dirichlet", "schnakenberg"),
                                     ("neumann", "fhn"), ("neumann", "gierer_meinhardt")])
def test_1d_runs_match_oracle(bc, kind, N):
    cfg = _cfg(1, (N,), bc, kind=kind, dt=0.02)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=13, lo=lo, hi=hi)
    ref = oracle_solver(cfg).run(u0, 0.0, 6)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=6))
    assert O.rel_max(list(g64), ref) < 1e-11
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=6)).astype(np.float64)
    assert O.rel_l2(list(g32), ref) < 1e-4


def test_1d_variants_match_oracle():
    """Cox-Matthews scheme (FP64) and rational coefficients (FP32) on a 1D grid."""
    cfg = _cfg(1, (64,), "dirichlet", kind="fhn", dt=0.02, scheme="cox_matthews")
    u0 = _rand_fields(cfg, seed=17, lo=0.0, hi=1.0)
    ref = oracle_solver(cfg).run(u0, 0.0, 5)
    assert O.rel_max(list(_np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=5))), ref) < 1e-11
    cfg2 = dict(cfg, scheme="p13", alpha=(1.5, 1.5))
    ref2 = oracle_solver(cfg2).run(u0, 0.0, 5)
    rat = _np(sf.Solver(cfg2, dtype="f32", coefficients="rational").run(u0, nsteps=5)).astype(np.float64)
    assert O.rel_l2(list(rat), ref2) < 1e-4


def _example1_error_gpu(Ninv):
    kappa, alpha = 10.0, 1.8
    tau = (1.0 / Ninv) / (4 * kappa)
    cfg = dict(dim=1, N=(Ninv,), lo=(0.0,), hi=(1.0,), bc="dirichlet", alpha=(alpha,), kappa=(kappa,), dt=tau,
               reaction=dict(kind="fisher_mms", p=[]), dtype="f64")
    x = np.arange(1, Ninv) / Ninv
    exact = lambda t: math.exp(-t) * np.sin(2 * np.pi * x) ** 3   # noqa: E731
    M = int(round(1.0 / tau))
    u = _np(sf.Solver(cfg, dtype="f64").run([exact(0.0)], nsteps=M))[0]
    return float(np.max(np.abs(u - exact(M * tau))))


@pytest.mark.parametrize("row", _table("table1.txt"))
def test_table1_example1_errors_on_gpu(row):
    """Example 1 (1D fractional Fisher equation, Dirichlet, alpha = 1.8, kappa = 10, tau = h/(4 kappa),
    T = 1): the GPU's maximum-norm errors equal the paper's Table 1 to its printed digits."""
    Ninv, printed = int(row[0]), row[1]
    assert _same_to_printed_digits(_example1_error_gpu(Ninv), printed)
