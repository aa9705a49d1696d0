"""Autotuner of the radix/tile schedule (shared-memory engine axes) and of the batched persistent
launches: every schedule it picks computes the same result as the default one, and the cache file
named by SFRD_AUTOTUNE_CACHE is written and reused."""
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


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dim,N,bc,kind", [(2, (120, 100), "periodic", "gray_scott"),
                                           (2, (100, 48), "neumann", "fhn"),
                                           (3, (30, 24, 40), "dirichlet", "schnakenberg")])
def test_autotuned_schedule_gives_the_same_run(dim, N, bc, kind, dtype, monkeypatch, tmp_path):
    monkeypatch.setenv("SFRD_AUTOTUNE_CACHE", str(tmp_path / "cache.txt"))
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=31, lo=lo, hi=hi)
    plain = _np(sf.Solver(cfg, dtype=dtype).run(u0, nsteps=4))
    s = sf.Solver(cfg, dtype=dtype)
    cc, rule = s.autotune(steps=2)
    assert cc in ((16, 8, 4) if dtype == "f32" else (8, 4, 2)) and 0 <= rule <= 3
    tuned = _np(s.run(u0, nsteps=4))
    assert rel_l2(tuned, plain) < (1e-12 if dtype == "f64" else 1e-5)
    ref = oracle_solver(cfg).run(u0, 0.0, 4)
    if dtype == "f64":
        assert O.rel_max(list(tuned), ref) < 1e-11
    else:
        assert O.rel_l2(list(tuned.astype(np.float64)), ref) < 1e-4
    # the choice is recorded and reused by a new plan of the same problem
    text = (tmp_path / "cache.txt").read_text().split()
    assert text[-2:] == [str(cc), str(rule)]
    again = sf.Solver(cfg, dtype=dtype).autotune(steps=2)
    assert again == (cc, rule)


def test_register_engine_plan_has_nothing_to_tune():
    cfg = _cfg(2, (64, 128), "dirichlet", kind="schnakenberg", dt=0.02)
    s = sf.Solver(cfg, dtype="f32")
    s.autotune(steps=1)
    u0 = _rand_fields(cfg, seed=2, lo=-0.05, hi=0.05)
    assert O.rel_l2(list(_np(s.run(u0, nsteps=2)).astype(np.float64)), oracle_solver(cfg).run(u0, 0.0, 2)) < 1e-4


def test_batch_autotune_keeps_every_instance_exact():
    cfgs = W.gm_instances(24, seed=5)
    u0 = [np.stack(W.initial_fields(c)) for c in cfgs]
    b = sf.Batch(cfgs, dtype="f32")
    k, rule = b.autotune(steps=1)
    assert 1 <= k <= 4 and 0 <= rule <= 3
    b.load(u0)
    b.advance(3)
    got = b.store()
    for i in range(0, 24, 3):
        single = sf.Solver(cfgs[i], dtype="f32").run(u0[i], nsteps=3)
        assert float((got[i] - single).abs().max() / single.abs().max()) < 1e-5, i
