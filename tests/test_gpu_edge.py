"""GPU edge case: a run of zero steps is the load transform followed by the store transform, so it
returns the input up to the transforms' rounding (register engine and shared-memory engine, both
precisions).  The kernels are those of every run; only the step count is degenerate."""
import numpy as np
import pytest

from tests.helpers import rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _np, _rand_fields  # noqa: E402


@pytest.mark.parametrize("dim,N,bc,kind", [(3, (64, 64, 64), "dirichlet", "schnakenberg"),
                                           (2, (64, 128), "neumann", "fhn"),
                                           (2, (20, 12), "periodic", "gray_scott"),
                                           (3, (10, 8, 6), "dirichlet", "schnakenberg")])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 2e-4)])
def test_zero_steps_return_the_input(dim, N, bc, kind, dtype, tol):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    u0 = np.stack(_rand_fields(cfg, seed=31, lo=-0.5, hi=1.0))
    got = _np(sf.Solver(cfg, dtype=dtype).run(u0, nsteps=0)).astype(np.float64)
    assert got.shape == u0.shape
    assert rel_max(got, u0) < tol


@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
@pytest.mark.parametrize("Ns", [(2,), (3,), (5,), (2, 2), (2, 3), (4, 5), (2, 3, 4), (4, 2, 3), (5, 5, 2)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_smallest_grids_match_the_oracle(bc, Ns, dtype, tol):
    """Degenerate sizes: 2-5 intervals per axis (one to six unknowns), 1D to 3D, every boundary condition,
    a two-species reaction, several steps, against the oracle (the shared-memory engine's smallest
    transforms, single-row and single-column tiles)."""
    import oracle as O
    from oracle.bridge import solver as oracle_solver
    cfg = _cfg(len(Ns), Ns, bc, kind="fhn", dt=0.05)
    u0 = _rand_fields(cfg, seed=sum(Ns), lo=0.0, hi=1.0)
    got = _np(sf.Solver(cfg, dtype=dtype).run(np.stack(u0), nsteps=5)).astype(np.float64)
    ref = oracle_solver(cfg).run(u0, 0.0, 5)
    err = O.rel_max(list(got), ref) if dtype == "f64" else O.rel_l2(list(got), ref)
    assert err < tol, err
