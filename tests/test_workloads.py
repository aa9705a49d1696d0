"""The seeded synthetic inputs: shapes per boundary condition, determinism, and the initial-condition
recipes (amplitudes, regions, parameter ranges) of the workloads that stand in for the paper's Section 5
experiments."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402


@pytest.mark.parametrize("name,shape", [("fhn64", (65, 65)), ("gs1024", (1024, 1024)),
                                        ("schnak256", (255, 255, 255)), ("fhn256_adjoint", (257, 257))])
def test_field_shapes_follow_the_unknowns_of_each_boundary_condition(name, shape):
    assert W.field_shape(W.config(name)) == shape


def test_scaled_grids_and_node_coordinates():
    cfg = W.scaled("schnak256", (8, 10, 12), nsteps=3)
    assert W.field_shape(cfg) == (11, 9, 7) and cfg["nsteps"] == 3
    X, Y, Z = W.mesh(cfg)
    assert X.shape == Y.shape == Z.shape == (11, 9, 7)
    np.testing.assert_allclose(X[0, 0, :], np.arange(1, 8) / 8.0)       # Dirichlet: interior nodes 1..N-1
    np.testing.assert_allclose(Z[:, 0, 0], np.arange(1, 12) / 12.0)
    assert list(W.node_indices("neumann", 4)) == [0, 1, 2, 3, 4]
    assert list(W.node_indices("periodic", 4)) == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        W.node_indices("robin", 4)


@pytest.mark.parametrize("name", ["fhn64", "schnak256", "gs1024"])
def test_initial_fields_are_deterministic_per_seed(name):
    cfg = W.scaled(name, 16)
    a, b = W.initial_fields(cfg), W.initial_fields(cfg)
    c = W.initial_fields(cfg, seed=cfg["seed"] + 1)
    for x, y, z in zip(a, b, c):
        assert x.dtype == np.float64 and x.shape == W.field_shape(cfg)
        assert np.array_equal(x, y) and not np.array_equal(x, z)


def test_fitzhugh_nagumo_recipe():
    cfg = W.config("fhn64")
    u, v = W.initial_fields(cfg)
    X, Y = W.mesh(cfg)
    assert np.all(np.abs(u - np.where(X < 50.0, 1.0, 0.0)) <= 1e-3)
    assert np.all(np.abs(v - np.where(Y > 50.0, 0.1, 0.0)) <= 1e-3)


def test_gray_scott_recipe():
    cfg = W.scaled("gs1024", 64)
    u, v = W.initial_fields(cfg)
    X, Y = W.mesh(cfg)
    sq = (np.abs(X - 1.25) <= 0.125) & (np.abs(Y - 1.25) <= 0.125)
    assert sq.sum() > 0 and (~sq).sum() > 0
    assert np.all(np.abs(u - np.where(sq, 0.5, 1.0)) <= 0.01)
    assert np.all(np.abs(v - np.where(sq, 0.25, 0.0)) <= 0.01)


def test_perturbation_recipes_are_small_and_centred():
    w = W.initial_fields(W.scaled("schnak256", 32))
    for x in w:
        assert np.abs(x).max() <= 0.01 and abs(x.mean()) < 1e-3 and x.std() > 0.005
    assert W.config("schnak256")["reaction"]["offset"] == [1.0, 0.9]      # steady state (a + b, b / (a + b)^2)


def test_gierer_meinhardt_instances():
    cfgs = W.gm_instances(256, seed=3)
    assert len(cfgs) == 256
    assert {c["N"][0] for c in cfgs} == set(W.GM_SIDES)
    assert {c["bc"] for c in cfgs} == set(W.GM_BCS)
    alphas = np.array([c["alpha"][0] for c in cfgs])
    assert np.all((alphas > 1.2) & (alphas <= 2.0)) and alphas.std() > 0.15
    assert len({c["seed"] for c in cfgs}) == 256
    assert all(c["alpha"][0] == c["alpha"][1] and c["kappa"] == (1.0, 30.0) for c in cfgs)
    assert W.gm_instances(256, seed=3) == cfgs                            # reproducible
    w = W.initial_fields(W.gm_instances(1, seed=3)[0])
    assert all(np.abs(x).max() <= 0.05 for x in w)
