"""Whole-run parity of the named workloads: the CUDA path through the C ABI after the workload's
full number of steps, against the FP64 CPU oracle.

Bars (the ones every parity test uses): FP64 within 1e-11 relative max-norm of the oracle, FP32
(FP64-computed coefficients) within 1e-4 relative L2.  The 63^3 Schnakenberg run is compared with
the oracle live on every unknown.  The larger runs (127^3 and 255^3 Schnakenberg for 500 steps,
1024^2 Gray-Scott for 2000 steps, one Gierer-Meinhardt instance per side and boundary condition
for 400 steps) take the oracle minutes to hours, so tests/golden/make_fullrun.py stores its result
on a strided subgrid (every axis's last unknown included) with the full-field norms; the library
runs the whole workload and is compared at those points: max-norm differences over the samples
divided by the full field's max-norm, L2 over the samples.
"""
import os

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

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL64, TOL32 = 1e-11, 1e-4


def _np(t):
    return t.detach().double().cpu().numpy()


def _golden(name):
    path = os.path.join(GOLDEN, "fullrun_%s.npz" % name)
    if not os.path.exists(path):
        pytest.skip("no stored oracle run %s (tests/golden/make_fullrun.py)" % name)
    return np.load(path)


def _sampled(u, g):
    """The library's fields (species-major array) at the stored sample points."""
    idx = [g["idx%d" % d] for d in range(u.ndim - 1)]
    return np.stack([x[np.ix_(*idx)] for x in u])


def _rel_max_sampled(u, g):
    return float(np.max(np.abs(_sampled(u, g) - g["values"])) / float(g["max_abs"]))


def _rel_l2_sampled(u, g):
    ref = g["values"]
    return float(np.linalg.norm((_sampled(u, g) - ref).ravel()) / np.linalg.norm(ref.ravel()))


def _workload(name):
    if name == "schnak128":
        return W.scaled("schnak256", 128)
    if name.startswith("gm"):
        return W.gm_instances(256, seed=3)[int(name[2:])]
    return W.config(name)


GM_NAMES = sorted(f[len("fullrun_"):-len(".npz")] for f in os.listdir(GOLDEN)
                  if f.startswith("fullrun_gm") and f.endswith(".npz"))


def test_schnakenberg_63_full_run_against_live_oracle():
    """3D Schnakenberg, Dirichlet, 63^3 interior (N = 64), all 500 steps of the workload, every unknown."""
    cfg = W.scaled("schnak256", 64)
    assert cfg["nsteps"] == 500
    u0 = W.initial_fields(cfg)
    ref = oracle_solver(cfg).run(u0, 0.0, cfg["nsteps"])
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_l2(list(g32), ref) < TOL32


@pytest.mark.parametrize("name", ["schnak128", "schnak256", "gs1024"])
def test_full_run_against_stored_oracle(name):
    """127^3 and 255^3 Schnakenberg (500 steps; 255^3 is the bench's launch configuration) and
    1024^2 Gray-Scott (2000 steps; its slow axis is the N = 1024 element-pair pass), FP64 and FP32."""
    g = _golden(name)
    cfg = _workload(name)
    assert int(g["nsteps"]) == cfg["nsteps"] and tuple(g["N"]) == tuple(cfg["N"])
    u0 = W.initial_fields(cfg)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=cfg["nsteps"]))
    e64 = _rel_max_sampled(g64, g)
    torch.cuda.empty_cache()
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=cfg["nsteps"]))
    e32 = _rel_l2_sampled(g32, g)
    torch.cuda.empty_cache()
    print("%s: FP64 rel max %.2e, FP32 rel L2 %.2e after %d steps" % (name, e64, e32, cfg["nsteps"]))
    assert e64 < TOL64
    assert e32 < TOL32


@pytest.mark.parametrize("name", GM_NAMES)
def test_gierer_meinhardt_instance_full_run_against_stored_oracle(name):
    """One instance of the batched workload per side (96, 128, 200, 256, 384) and boundary condition,
    all 400 steps, single-instance plans in FP64 and FP32."""
    g = _golden(name)
    cfg = _workload(name)
    assert int(g["nsteps"]) == cfg["nsteps"] == 400 and tuple(g["N"]) == tuple(cfg["N"])
    u0 = W.initial_fields(cfg)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=cfg["nsteps"]))
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=cfg["nsteps"]))
    e64, e32 = _rel_max_sampled(g64, g), _rel_l2_sampled(g32, g)
    print("%s N=%d %s: FP64 rel max %.2e, FP32 rel L2 %.2e after 400 steps" % (name, cfg["N"][0], cfg["bc"], e64, e32))
    assert e64 < TOL64
    assert e32 < TOL32


def test_batched_workload_full_run_against_stored_oracle():
    """The 256-instance Gierer-Meinhardt batch (FP32, one persistent launch per pass) for its 400 steps;
    the instances with a stored oracle run (one per side and boundary condition) are compared."""
    if not GM_NAMES:
        pytest.skip("no stored oracle runs of the Gierer-Meinhardt instances")
    cfgs = W.gm_instances(256, seed=3)
    b = sf.Batch(cfgs, dtype="f32")
    b.load([np.stack(W.initial_fields(c)) for c in cfgs])
    b.advance(400)
    got = b.store()
    for name in GM_NAMES:
        g = _golden(name)
        assert _rel_l2_sampled(_np(got[int(name[2:])]), g) < TOL32, name
    del b, got
    torch.cuda.empty_cache()
    # the same instances batched in FP64
    sel = [int(n[2:]) for n in GM_NAMES]
    b64 = sf.Batch([cfgs[i] for i in sel], dtype="f64")
    b64.load([np.stack(W.initial_fields(cfgs[i])) for i in sel])
    b64.advance(400)
    for name, x in zip(GM_NAMES, b64.store()):
        assert _rel_max_sampled(_np(x), _golden(name)) < TOL64, name


@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_slow_axis_of_1024_intervals(bc):
    """2D grids whose slow (y) axis has 1024 intervals: the element-pair slow-axis pass at N = 1024
    (tile width 8 in FP32, 4 in FP64), a few steps against the oracle on every unknown."""
    cfg = W.scaled("gs1024", (64, 1024), nsteps=3, bc=bc)
    u0 = W.initial_fields(cfg)
    ref = oracle_solver(cfg).run(u0, 0.0, cfg["nsteps"])
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_l2(list(g32), ref) < TOL32


def test_gray_scott_1024_fp32_tracks_fp64_over_the_whole_run():
    """1024^2 Gray-Scott, 2000 steps: the FP32 path against the FP64 path on the GPU, every unknown,
    checked every 250 steps (the FP64 path is itself checked against the oracle above)."""
    cfg = W.config("gs1024")
    u0 = torch.as_tensor(np.stack(W.initial_fields(cfg)))
    s64 = sf.Solver(cfg, dtype="f64")
    s32 = sf.Solver(cfg, dtype="f32")
    s64.load(u0.cuda(), 0.0)
    s32.load(u0.cuda().float(), 0.0)
    errs = []
    for _ in range(cfg["nsteps"] // 250):
        s64.advance(250)
        s32.advance(250)
        a, b = s64.store(), s32.store().double()
        errs.append(float(torch.linalg.vector_norm(b - a) / torch.linalg.vector_norm(a)))
    print("FP32 vs FP64 relative L2 every 250 steps:", " ".join("%.2e" % e for e in errs))
    assert max(errs) < TOL32
