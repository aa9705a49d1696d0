"""Cox-Matthews scheme (SFRD_SCHEME_COX_MATTHEWS): Algorithm 1's stages with the exact-exponential
coefficients (FP64 on the GPU: Taylor series of the phi-functions for L < 1, closed forms otherwise)
against the oracle's contour-integral coefficients and its step, and the exact decay of an
eigenmode without reaction."""
import numpy as np
import pytest

import oracle as O
from oracle.bridge import solver as oracle_solver
from tests.helpers import rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _np, _rand_fields  # noqa: E402


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_cox_matthews_coefficients_match_contour_integrals(bc, dtype):
    cfg = _cfg(3, (10, 12, 8), bc, kind="none", alpha=(1.3, 1.9), kappa=(0.7, 3.0), dt=0.3, scheme="cox_matthews")
    s = sf.Solver(cfg, dtype=dtype)
    ora = oracle_solver(cfg)
    for which in sf.COEFFICIENTS:
        got = _np(s.coefficients(which))
        for sp in range(2):
            ref = ora.coef[sp][which]
            err = np.max(np.abs(got[sp] - ref)) / np.max(np.abs(ref))
            assert err < (1e-13 if dtype == "f64" else 1e-7), (which, sp, err)


@pytest.mark.parametrize("dim,N,bc,kind", [(2, (20, 12), "periodic", "gray_scott"),
                                           (2, (20, 12), "dirichlet", "schnakenberg"),
                                           (2, (64, 64), "neumann", "fhn"),
                                           (3, (10, 8, 6), "dirichlet", "gierer_meinhardt"),
                                           (3, (64, 64, 64), "periodic", "gray_scott")])
def test_cox_matthews_steps_match_oracle(dim, N, bc, kind):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02, scheme="cox_matthews")
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=41, lo=lo, hi=hi)
    ref = oracle_solver(cfg).run(u0, 0.0, 4)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=4))
    assert O.rel_max(list(g64), ref) < 1e-11
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=4)).astype(np.float64)
    assert O.rel_l2(list(g32), ref) < 1e-4
    p13 = _np(sf.Solver(dict(cfg, scheme="p13"), dtype="f64").run(u0, nsteps=4))
    assert rel_max(p13, g64) > 0      # a different scheme, not the default by mistake


@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_single_mode_decays_exactly_on_gpu(bc):
    """No reaction: every eigen-coefficient of u_M equals exp(-kappa Lambda^{alpha/2} M tau) times
    that of u_0, with the exponential from the oracle's eigenvalues."""
    cfg = _cfg(2, (64, 48), bc, kind="linear", S=1, alpha=(1.7,), kappa=(0.3,), dt=0.2, scheme="cox_matthews")
    cfg["reaction"]["p"] = [0.0]
    s = sf.Solver(cfg, dtype="f64")
    M = 7
    u0 = _rand_fields(cfg, seed=5)
    uM = s.run(u0, nsteps=M)
    ora = oracle_solver(cfg)
    decay = np.exp(-ora.L[0] * M)
    got, expect = _np(s.forward(uM))[0], _np(s.forward(u0))[0] * decay
    assert np.max(np.abs(got - expect)) <= 1e-12 * np.max(np.abs(expect))
