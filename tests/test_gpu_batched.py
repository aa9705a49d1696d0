"""Batched instances (one persistent launch per pass for all instances) against the
single-instance path and the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.bridge import solver as oracle_solver

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402


def _mixed(count, sides, seed=21):
    out = []
    rng = np.random.default_rng(seed)
    for i in range(count):
        cfg = W.gm_instances(1, seed=seed + i)[0]
        N = int(sides[i % len(sides)])
        cfg["N"] = (N, N)
        cfg["bc"] = ("periodic", "dirichlet", "neumann")[i % 3]
        a = float(rng.uniform(1.25, 2.0))
        cfg["alpha"] = (a, a)
        out.append(cfg)
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_equals_single_instance_runs(dtype):
    cfgs = _mixed(9, (96, 128, 200, 64, 256, 40))
    u0 = [np.stack(W.initial_fields(c)) for c in cfgs]
    b = sf.Batch(cfgs, dtype=dtype)
    b.load(u0)
    b.advance(5)
    got = [x.double().cpu().numpy() for x in b.store()]
    for c, u, g in zip(cfgs, u0, got):
        single = sf.Solver(c, dtype=dtype).run(u, nsteps=5).double().cpu().numpy()
        tol = 1e-12 if dtype == "f64" else 1e-5
        assert float(np.max(np.abs(g - single)) / np.max(np.abs(single))) < tol, (c["N"], c["bc"])


def test_batch_fp64_matches_oracle():
    cfgs = _mixed(6, (64, 96, 40, 128, 32, 48), seed=33)
    u0 = [np.stack(W.initial_fields(c)) for c in cfgs]
    b = sf.Batch(cfgs, dtype="f64")
    b.load(u0)
    b.advance(4)
    got = [x.cpu().numpy() for x in b.store()]
    for c, u, g in zip(cfgs, u0, got):
        ref = oracle_solver(c).run(list(u), 0.0, 4)
        assert O.rel_max(list(g), ref) < 1e-11, (c["N"], c["bc"])


def test_batch_resumes_and_fp32_tracks_fp64():
    cfgs = _mixed(6, (96, 128, 200), seed=44)
    u0 = [np.stack(W.initial_fields(c)) for c in cfgs]
    b64 = sf.Batch(cfgs, dtype="f64")
    b64.load(u0)
    b64.advance(3)
    b64.advance(4)
    g64 = [x.cpu().numpy() for x in b64.store()]
    b64.load(u0)
    b64.advance(7)
    again = [x.cpu().numpy() for x in b64.store()]
    for x, y in zip(g64, again):
        np.testing.assert_array_equal(x, y)
    b32 = sf.Batch(cfgs, dtype="f32")
    b32.load(u0)
    b32.advance(7)
    for x, y in zip(b32.store(), g64):
        assert O.rel_l2(list(x.double().cpu().numpy()), list(y)) < 1e-4


def test_gierer_meinhardt_256_instance_workload_sampled():
    """The 256-instance Gierer-Meinhardt workload (sides {96,128,200,256,384}, BC and alpha drawn per
    instance) in one batch: 2 steps, every 16th instance compared with its single-instance run."""
    cfgs = W.gm_instances(256, seed=3)
    u0 = [np.stack(W.initial_fields(c)) for c in cfgs]
    b = sf.Batch(cfgs, dtype="f32")
    # one launch per pass for each axis length (96, 128, 200, 256, 384), 4 stages x 2 passes
    assert b.count == 256 and b.launches_per_step == 4 * 2 * 5
    b.load(u0)
    b.advance(2)
    got = b.store()
    for i in range(0, 256, 16):
        single = sf.Solver(cfgs[i], dtype="f32").run(u0[i], nsteps=2)
        assert float((got[i] - single).abs().max() / single.abs().max()) < 1e-5, i
