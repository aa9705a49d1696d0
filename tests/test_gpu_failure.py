"""Failure detection without a GPU fault: a non-finite value in the state is reported as
SFRD_ENONFINITE by a host-polled device flag (no device waits, traps or asserts).  The fault is
injected on the host: a NaN in the initial field."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402
from tests.test_gpu_parity import _cfg, _rand_fields  # noqa: E402


@pytest.mark.parametrize("dim,N,bc", [(2, (64, 48), "neumann"), (3, (16, 12, 10), "dirichlet"), (1, (64,), "periodic")])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_nan_in_the_initial_field_is_reported(dim, N, bc, dtype):
    cfg = _cfg(dim, N, bc, kind="fhn", dt=0.02)
    u0 = _rand_fields(cfg, seed=9, lo=0.0, hi=1.0)
    s = sf.Solver(cfg, dtype=dtype)
    s.load(u0)
    s.advance(2)
    assert s.check_finite()
    bad = [x.copy() for x in u0]
    bad[1].flat[bad[1].size // 3] = np.nan
    s.load(bad)
    assert not s.check_finite()
    s.advance(1)
    assert not s.check_finite()
    s.load(u0)                       # a clean load clears it: the flag is not sticky
    assert s.check_finite()


def test_debug_checks_make_advance_fail(monkeypatch):
    monkeypatch.setenv("SFRD_DEBUG_CHECKS", "1")
    cfg = _cfg(2, (32, 32), "periodic", kind="gray_scott", dt=0.02)
    u0 = _rand_fields(cfg, seed=4, lo=0.0, hi=1.0)
    s = sf.Solver(cfg, dtype="f64")
    s.run(u0, nsteps=3)              # finite: no error
    bad = [x.copy() for x in u0]
    bad[0][3, 5] = np.inf
    with pytest.raises(sf.SfrdError) as e:
        s.run(bad, nsteps=1)
    assert e.value.code == -5
