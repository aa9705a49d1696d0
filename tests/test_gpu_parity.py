"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 path within 1e-11 relative max-norm of the oracle after the
whole run; FP32 path (FP64-computed coefficients) within 1e-4 relative L2;
transforms alone FP64 <= 1e-12, FP32 <= 2e-6 relative max-norm.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import library_forward, rel_l2, rel_max
from oracle.bridge import solver as oracle_solver

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2003_13569_gb300 as sf  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL64, TOL32 = 1e-11, 1e-4


def _cfg(dim, N, bc, kind="none", S=2, alpha=(1.5, 1.7), kappa=(0.7, 0.2), dt=0.05, lo=None, hi=None, **kw):
    p = {"none": [], "linear": [0.3], "fhn": [0.1, 0.01, 0.5, 1.0, 0.0], "gray_scott": [0.04, 0.06],
         "schnakenberg": [5.0, 0.1, 0.9], "gierer_meinhardt": [1.0, 1.0, 1.0, 1.0]}[kind]
    off = {"schnakenberg": [1.0, 0.9], "gierer_meinhardt": [1.0, 1.0]}.get(kind, [0.0, 0.0])
    return dict(dim=dim, N=tuple(N), lo=lo or (0.0,) * dim, hi=hi or tuple(2.0 + d for d in range(dim)), bc=bc,
                alpha=tuple(alpha[:S]), kappa=tuple(kappa[:S]), dt=dt, nsteps=1,
                reaction=dict(kind=kind, p=p, offset=off), dtype="f64", seed=7, **kw)


def _rand_fields(cfg, seed=0, lo=-1.0, hi=1.0):
    shp = W.field_shape(cfg)
    rng = np.random.default_rng(seed)
    return [rng.uniform(lo, hi, shp) for _ in range(len(cfg["alpha"]))]


def _np(t):
    return t.detach().cpu().numpy()


# ---- transforms -----------------------------------------------------------------

SHAPES = [(2, (20, 12), "periodic"), (2, (20, 12), "dirichlet"), (2, (20, 12), "neumann"),
          (2, (30, 40), "periodic"), (2, (48, 10), "neumann"), (2, (50, 16), "dirichlet"),
          (3, (10, 8, 6), "periodic"), (3, (10, 8, 6), "dirichlet"), (3, (12, 10, 8), "neumann"),
          (3, (16, 6, 20), "dirichlet")]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dim,N,bc", SHAPES)
@pytest.mark.parametrize("S", [2, 1])
def test_forward_transform_matches_dense_matrices(dim, N, bc, dtype, S):
    cfg = _cfg(dim, N, bc, kind="none" if S == 2 else "linear", S=S)
    s = sf.Solver(cfg, dtype=dtype)
    u = _rand_fields(cfg, seed=1)
    got = _np(s.forward(u))
    for sp in range(S):
        ref = library_forward(u[sp], bc, N)
        assert rel_max(got[sp], ref) < (1e-12 if dtype == "f64" else 2e-6)
    back = _np(s.inverse(got))
    for sp in range(S):
        assert rel_max(back[sp], u[sp]) < (1e-12 if dtype == "f64" else 2e-6)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet", "neumann"])
def test_coefficient_arrays_match_algorithm1(bc, dtype):
    cfg = _cfg(3, (10, 12, 8), bc, kind="none", alpha=(1.3, 1.9), kappa=(0.7, 3.0), dt=0.3)
    s = sf.Solver(cfg, dtype=dtype)
    ora = oracle_solver(cfg)
    for which in sf.COEFFICIENTS:
        got = _np(s.coefficients(which))
        for sp in range(2):
            ref = ora.coef[sp][which]
            assert rel_max(got[sp], ref) < (1e-13 if dtype == "f64" else 1e-7), (which, sp)


SHAPES_V2 = [(2, (64, 128), "periodic"), (2, (64, 128), "dirichlet"), (2, (64, 128), "neumann"),
             (2, (256, 64), "dirichlet"), (2, (256, 64), "neumann"), (2, (512, 64), "periodic"),
             (2, (1024, 64), "periodic"), (2, (1024, 64), "neumann"), (2, (512, 64), "dirichlet"),
             (3, (64, 64, 128), "dirichlet"), (3, (128, 64, 64), "neumann"), (3, (64, 128, 64), "periodic"),
             (3, (64, 48, 80), "dirichlet"),
             # lengths 3 * 2^5, 5^2 * 2^3, 3 * 2^7 on the register engine (mixed-radix in-register DFTs)
             (2, (96, 200), "periodic"), (2, (200, 96), "dirichlet"), (2, (384, 96), "neumann"),
             (2, (96, 384), "dirichlet"), (3, (96, 200, 64), "neumann"), (3, (200, 64, 384), "periodic")]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dim,N,bc", SHAPES_V2)
@pytest.mark.parametrize("S", [2, 1])
def test_forward_transform_register_engine(dim, N, bc, dtype, S):
    """Power-of-two axes (64..1024) run on the register FFT engine (length-N packed FFT with the
    sine/cosine pre- and post-processing); mixed shapes combine both engines."""
    cfg = _cfg(dim, N, bc, kind="none" if S == 2 else "linear", S=S)
    s = sf.Solver(cfg, dtype=dtype)
    u = _rand_fields(cfg, seed=11)
    got = _np(s.forward(u))
    # FP32: the odd-index sine/cosine outputs are running sums of DFT values, whose rounding
    # errors add up like a random walk over N/2 terms (max-norm ~ sqrt(N) eps per axis).
    tol = 1e-12 if dtype == "f64" else (4e-6 if bc == "periodic" else 3e-6 * np.sqrt(max(N)))
    for sp in range(S):
        assert rel_max(got[sp], library_forward(u[sp], bc, N)) < tol
        if dtype == "f32":
            assert rel_l2(got[sp], library_forward(u[sp], bc, N)) < 3e-6
    back = _np(s.inverse(got))
    for sp in range(S):
        assert rel_max(back[sp], u[sp]) < tol


@pytest.mark.parametrize("kind,bc", [("none", "periodic"), ("linear", "dirichlet"), ("fhn", "neumann"),
                                     ("gray_scott", "periodic"), ("schnakenberg", "dirichlet"),
                                     ("gierer_meinhardt", "neumann")])
def test_contiguous_axis_of_1024_intervals_every_reaction_kind(kind, bc):
    """2D grids whose contiguous (x) axis has 1024 intervals: the FP32 reaction pass at that length is
    compiled once per two-species reaction kind, so each kind runs its own kernel; a few steps against
    the oracle on every unknown, FP64 and FP32."""
    cfg = _cfg(2, (1024, 64), bc, kind=kind, dt=0.02)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=13, lo=lo, hi=hi)
    nsteps = 3
    ref = oracle_solver(cfg).run(u0, 0.0, nsteps)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
    assert O.rel_l2(list(g32), ref) < TOL32


@pytest.mark.parametrize("dim,N,bc,kind", [(2, (64, 128), "periodic", "gray_scott"),
                                           (2, (128, 64), "dirichlet", "schnakenberg"),
                                           (2, (64, 64), "neumann", "fhn"),
                                           (2, (256, 128), "neumann", "gierer_meinhardt"),
                                           (3, (64, 64, 64), "dirichlet", "schnakenberg"),
                                           (3, (64, 64, 64), "neumann", "fhn"),
                                           (2, (96, 200), "periodic", "gierer_meinhardt"),
                                           (2, (384, 96), "dirichlet", "gray_scott"),
                                           (2, (200, 384), "neumann", "schnakenberg")])
def test_register_engine_steps_match_oracle_and_generic_engine(dim, N, bc, kind, monkeypatch):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    lo, hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=12, lo=lo, hi=hi)
    nsteps = 5
    ref = oracle_solver(cfg).run(u0, 0.0, nsteps)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
    assert O.rel_l2(list(g32), ref) < TOL32
    monkeypatch.setenv("SFRD_ENGINE", "generic")
    gen = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert rel_max(g64, gen) < 1e-12


# ---- whole steps -----------------------------------------------------------------

STEP_CASES = [
    (2, (20, 12), "periodic", "gray_scott"), (2, (20, 12), "dirichlet", "schnakenberg"),
    (2, (20, 12), "neumann", "fhn"), (2, (24, 30), "neumann", "gierer_meinhardt"),
    (2, (32, 16), "periodic", "fhn"), (3, (10, 8, 6), "periodic", "gray_scott"),
    (3, (10, 8, 6), "dirichlet", "schnakenberg"), (3, (12, 10, 8), "neumann", "fhn"),
    (3, (8, 10, 12), "dirichlet", "gierer_meinhardt"),
]


@pytest.mark.parametrize("dim,N,bc,kind", STEP_CASES)
def test_steps_fp64_match_oracle(dim, N, bc, kind):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    rng_lo, rng_hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=3, lo=rng_lo, hi=rng_hi)
    nsteps = 6
    ref = oracle_solver(cfg).run(u0, 0.25, nsteps)
    s = sf.Solver(cfg, dtype="f64")
    got = _np(s.run(u0, t0=0.25, nsteps=nsteps))
    assert O.rel_max(list(got), ref) < TOL64


@pytest.mark.parametrize("dim,N,bc,kind", STEP_CASES[:5] + STEP_CASES[6:7])
def test_steps_fp32_match_oracle(dim, N, bc, kind):
    cfg = _cfg(dim, N, bc, kind=kind, dt=0.02)
    rng_lo, rng_hi = (0.0, 1.0) if kind in ("fhn", "gray_scott") else (-0.05, 0.05)
    u0 = _rand_fields(cfg, seed=4, lo=rng_lo, hi=rng_hi)
    ref = oracle_solver(cfg).run(u0, 0.0, 6)
    s = sf.Solver(cfg, dtype="f32")
    got = _np(s.run(u0, nsteps=6))
    assert O.rel_l2(list(got), ref) < TOL32


def test_load_advance_store_equals_run_and_state_is_resumable():
    cfg = _cfg(2, (20, 24), "neumann", kind="fhn", dt=0.05)
    u0 = _rand_fields(cfg, seed=5, lo=0.0, hi=1.0)
    s = sf.Solver(cfg, dtype="f64")
    a = _np(s.run(u0, t0=0.0, nsteps=7))
    s.load(u0, 0.0)
    s.advance(3)
    mid = _np(s.store())
    s.advance(4)
    b = _np(s.store())
    np.testing.assert_array_equal(a, b)
    ref_mid = oracle_solver(cfg).run(u0, 0.0, 3)
    assert O.rel_max(list(mid), ref_mid) < TOL64


def test_graph_and_direct_launches_agree(monkeypatch):
    cfg = _cfg(3, (10, 8, 6), "dirichlet", kind="schnakenberg", dt=0.01)
    u0 = _rand_fields(cfg, seed=6, lo=-0.01, hi=0.01)
    s = sf.Solver(cfg, dtype="f64")
    a = _np(s.run(u0, nsteps=5))
    monkeypatch.setenv("SFRD_NO_GRAPH", "1")
    s2 = sf.Solver(cfg, dtype="f64")
    b = _np(s2.run(u0, nsteps=5))
    np.testing.assert_array_equal(a, b)


def test_single_mode_decays_by_r13_power_on_gpu():
    """f = 0: the library spectrum of u_M is R13(L)^M times that of u_0 (Section 4)."""
    cfg = _cfg(2, (16, 20), "dirichlet", kind="none", dt=0.2)
    s = sf.Solver(cfg, dtype="f64")
    u0 = _rand_fields(cfg, seed=8)
    M = 9
    uM = s.run(u0, nsteps=M)
    got = _np(s.forward(uM))
    expect = _np(s.forward(u0)) * _np(s.coefficients("R13")) ** M
    assert rel_max(got, expect) < 1e-12


def test_host_entry_point_round_trip():
    cfg = _cfg(2, (20, 12), "periodic", kind="gray_scott", dt=0.1)
    u0 = np.ascontiguousarray(np.stack(_rand_fields(cfg, seed=9, lo=0.0, hi=1.0)))
    s = sf.Solver(cfg, dtype="f64")
    dev = _np(s.run(u0, nsteps=4))
    host = s.run_host(u0, nsteps=4)
    np.testing.assert_array_equal(dev, host)


def test_advance_before_load_is_an_error():
    cfg = _cfg(2, (20, 12), "periodic", kind="gray_scott")
    s = sf.Solver(cfg, dtype="f64")
    with pytest.raises(sf.SfrdError) as ei:
        s.advance(1)
    assert ei.value.code == -6


# ---- the paper's own numbers on the GPU --------------------------------------------

def _table2():
    rows = []
    for line in open(os.path.join(GOLDEN, "table2.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", [r for r in _table2() if r[1] <= 40])
@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_table2_errors_reproduced_on_gpu(row, bc):
    alpha, Ninv = row[0], int(row[1])
    printed = row[2] if bc == "neumann" else row[3]
    cfg = dict(dim=2, N=(Ninv, Ninv), lo=(0.0, 0.0), hi=(1.0, 1.0), bc=bc, alpha=(alpha,), kappa=(1.0,),
               dt=0.1 / Ninv, reaction=dict(kind="huxley_mms", p=[], offset=[0, 0]), dtype="f64")
    s = sf.Solver(cfg, dtype="f64")
    X, Y = W.mesh(cfg)
    g = np.cos(2 * np.pi * X) ** 3 * np.cos(2 * np.pi * Y) ** 3
    M = int(round(1.0 / cfg["dt"]))
    u = _np(s.run([0.0 * g], t0=0.0, nsteps=M))[0]
    err = float(np.max(np.abs(u - (M * cfg["dt"]) ** alpha * g)))
    assert float("%.4e" % err) == printed


# ---- the named workloads ---------------------------------------------------------

def _oracle_run(cfg, u0, nsteps):
    return oracle_solver(cfg).run(u0, 0.0, nsteps)


def test_fhn64_full_run_fp64_and_fp32():
    """2D FitzHugh-Nagumo, Neumann, 65^2 nodes, 200 steps: the whole workload."""
    cfg = W.config("fhn64")
    u0 = W.initial_fields(cfg)
    ref = _oracle_run(cfg, u0, cfg["nsteps"])
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=cfg["nsteps"]))
    assert O.rel_l2(list(g32), ref) < TOL32


@pytest.mark.parametrize("N,nsteps", [(64, 40), (128, 10)])
def test_gray_scott_scaled_fp64_and_fp32(N, nsteps):
    cfg = W.scaled("gs1024", N)
    u0 = W.initial_fields(cfg)
    ref = _oracle_run(cfg, u0, nsteps)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
    assert O.rel_l2(list(g32), ref) < TOL32


@pytest.mark.parametrize("N,nsteps", [(16, 20), (32, 6)])
def test_schnakenberg_scaled_fp64_and_fp32(N, nsteps):
    cfg = W.scaled("schnak256", N)
    u0 = W.initial_fields(cfg)
    ref = _oracle_run(cfg, u0, nsteps)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert O.rel_max(list(g64), ref) < TOL64
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
    assert O.rel_l2(list(g32), ref) < TOL32


def test_gierer_meinhardt_instances():
    for cfg in W.gm_instances(6, seed=3):
        cfg = dict(cfg)
        u0 = W.initial_fields(cfg)
        nsteps = 5
        ref = _oracle_run(cfg, u0, nsteps)
        g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
        assert O.rel_max(list(g64), ref) < TOL64, (cfg["N"], cfg["bc"])
        g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
        assert O.rel_l2(list(g32), ref) < TOL32


def test_schnakenberg_full_size_two_steps():
    """3D Schnakenberg at 255^3 interior (N = 256, FFT length 512): the bench launch configuration."""
    cfg = W.config("schnak256")
    u0 = W.initial_fields(cfg)
    nsteps = 2
    ref = _oracle_run(cfg, u0, nsteps)
    g64 = _np(sf.Solver(cfg, dtype="f64").run(u0, nsteps=nsteps))
    assert O.rel_max(list(g64), ref) < TOL64
    torch.cuda.empty_cache()
    g32 = _np(sf.Solver(cfg, dtype="f32").run(u0, nsteps=nsteps))
    assert O.rel_l2(list(g32), ref) < TOL32
