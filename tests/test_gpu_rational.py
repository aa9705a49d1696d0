"""Rational-coefficient mode (SFRD_COEF_RATIONAL): only L = kappa tau Lambda^{alpha/2} is stored
(computed in FP64, rounded to FP32) and the passes evaluate the Padé(1,3) coefficients of
Algorithm 1 as rationals of L in FP32.  Checked against the FP64 oracle (coefficients and whole
runs, at the FP32 tolerance) and against the stored-coefficient FP32 path."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.bridge import solver as oracle_solver
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _np, _rand_fields  # noqa: E402


@pytest.mark.parametrize("alpha", [(1.5, 1.5), (1.3, 1.9)])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_rational_coefficients_match_algorithm1(bc, alpha):
    """The six coefficient arrays evaluated from the stored L (FP32 rationals) against the
    oracle's FP64 Algorithm 1 arrays; one shared L plane when the orders are equal."""
    cfg = _cfg(3, (64, 64, 128), bc, kind="none", alpha=alpha, kappa=(0.7, 3.0), dt=0.3)
    s = sf.Solver(cfg, dtype="f32", coefficients="rational")
    ora = oracle_solver(cfg)
    for which in sf.COEFFICIENTS:
        got = _np(s.coefficients(which)).astype(np.float64)
        for sp in range(2):
            ref = ora.coef[sp][which]
            err = np.max(np.abs(got[sp] - ref)) / np.max(np.abs(ref))
            assert err < 2e-6, (which, sp, err)


def test_rational_mode_needs_less_workspace_and_shares_l():
    cfg = _cfg(3, (64, 64, 64), "dirichlet", kind="none", alpha=(1.5, 1.5))
    stored = sf.Solver(cfg, dtype="f32")
    shared = sf.Solver(cfg, dtype="f32", coefficients="rational")
    cfg2 = dict(cfg, alpha=(1.5, 1.7))
    per_species = sf.Solver(cfg2, dtype="f32", coefficients="rational")
    plane = 63 * 63 * 64 * 4
    assert stored.info.workspace_bytes - shared.info.workspace_bytes >= 12 * plane - 4096 - plane
    assert per_species.info.workspace_bytes - shared.info.workspace_bytes >= plane - 256


@pytest.mark.parametrize("dim,N,bc,kind,alpha", [
    (2, (64, 128), "periodic", "gray_scott", (1.7, 1.7)),
    (2, (128, 64), "dirichlet", "schnakenberg", (1.5, 1.8)),
    (2, (64, 64), "neumann", "fhn", (1.5, 1.5)),
    (3, (64, 64, 64), "dirichlet", "schnakenberg", (1.5, 1.5)),
    (3, (64, 128, 64), "periodic", "gray_scott", (1.4, 1.9)),
    (3, (64, 64, 64), "neumann", "fhn", (1.5, 1.5)),
])
def test_rational_runs_match_oracle_and_stored_path(dim, N, bc, kind, alpha):
    cfg = _cfg(dim, N, bc, kind=kind, alpha=alpha, dt=0.02)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=21, lo=lo, hi=hi)
    nsteps = 5
    ref = oracle_solver(cfg).run(u0, 0.0, nsteps)
    rat = _np(sf.Solver(cfg, dtype="f32", coefficients="rational").run(u0, nsteps=nsteps)).astype(np.float64)
    sto = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps)).astype(np.float64)
    assert O.rel_l2(list(rat), ref) < 1e-4
    assert rel_l2(rat, sto) < 1e-5


def test_rational_schnakenberg_scaled_workload_tracks_fp64():
    """The 3D Schnakenberg workload (Dirichlet, alpha 1.5 for both species: one shared L plane) at
    N = 64, 20 steps: rational FP32 against the FP64 path."""
    cfg = W.scaled("schnak256", 64, nsteps=20)
    u0 = list(W.initial_fields(cfg))
    r64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=20))
    rat = _np(sf.Solver(cfg, dtype="f32", coefficients="rational").run(u0, nsteps=20)).astype(np.float64)
    assert O.rel_l2(list(rat), list(r64)) < 1e-4


def test_rational_mode_has_no_adjoint():
    cfg = _cfg(2, (64, 64), "neumann", kind="fhn", alpha=(1.5, 1.5))
    s = sf.Solver(cfg, dtype="f32", coefficients="rational")
    with pytest.raises(sf.SfrdError) as e:
        s.run_checkpointed(list(_rand_fields(cfg, seed=2, lo=0.0, hi=1.0)), nsteps=4, ckpt_every=2)
    assert e.value.code == -2
