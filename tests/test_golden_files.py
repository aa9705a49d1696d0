"""The stored full-run oracle results (tests/golden/fullrun_*.npz, written by make_fullrun.py from the
oracle alone) belong to the workloads the GPU tests run: same steps, grid, boundary condition and seed as
the workload definition today, sample indices inside the field and covering its last unknown on every
axis, and norms consistent with the stored samples.  A changed input recipe fails here, on the CPU,
instead of as a silent mismatch in the GPU comparison."""
import glob
import os

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "fullrun_*.npz")))


def _workload(name):
    if name == "schnak128":
        return W.scaled("schnak256", 128)
    if name.startswith("gm"):
        return W.gm_instances(256, seed=3)[int(name[2:])]
    return W.config(name)


def test_there_are_stored_runs():
    names = [os.path.basename(f)[len("fullrun_"):-len(".npz")] for f in FILES]
    assert {"schnak128", "schnak256", "gs1024"} <= set(names)
    assert sum(n.startswith("gm") for n in names) == len(W.GM_SIDES) * len(W.GM_BCS)


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_stored_run_matches_its_workload(path):
    g = np.load(path)
    cfg = _workload(os.path.basename(path)[len("fullrun_"):-len(".npz")])
    assert int(g["nsteps"]) == cfg["nsteps"]
    assert tuple(int(n) for n in g["N"]) == tuple(cfg["N"])
    assert str(g["bc"]) == cfg["bc"]
    assert int(g["seed"]) == cfg["seed"]
    shape = W.field_shape(cfg)
    idx = [g["idx%d" % d] for d in range(len(shape))]
    for ix, n in zip(idx, shape):
        assert ix.min() >= 0 and ix.max() == n - 1 and np.all(np.diff(ix) > 0)
    vals = g["values"]
    assert vals.shape == (len(cfg["alpha"]),) + tuple(len(ix) for ix in idx)
    assert np.all(np.isfinite(vals))
    # the full-field norms bound the samples' (max-norm: at least the largest sample; L2: at least the
    # samples' L2, and at most sqrt(unknowns) times the max-norm)
    assert float(g["max_abs"]) >= float(np.max(np.abs(vals)))
    l2s = float(np.linalg.norm(vals.ravel()))
    assert l2s <= float(g["l2"]) * (1 + 1e-12)
    assert float(g["l2"]) <= float(g["max_abs"]) * np.sqrt(len(cfg["alpha"]) * np.prod(shape)) * (1 + 1e-12)
