"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the bench.

This module holds problem sizes, parameters and seeded initial fields only.  It
contains none of the method's arithmetic (no transforms, eigenvalues, Pade
coefficients or reaction terms): each side -- the CPU oracle and the CUDA
library -- implements those on its own.

Grid convention: `N` is the number of intervals per axis, h = (hi - lo) / N.
The unknowns per axis are the nodes 0..N-1 (periodic), 1..N-1 (homogeneous
Dirichlet) or 0..N (homogeneous Neumann).  Fields are float64 numpy arrays of
shape (n_z, n_y, n_x) / (n_y, n_x) / (n_x,), x fastest, one per species.
"""

from __future__ import annotations

import copy

import numpy as np

PERIODIC, DIRICHLET, NEUMANN = "periodic", "dirichlet", "neumann"


def node_indices(bc: str, N: int) -> np.ndarray:
    if bc == PERIODIC:
        return np.arange(0, N)
    if bc == DIRICHLET:
        return np.arange(1, N)
    if bc == NEUMANN:
        return np.arange(0, N + 1)
    raise ValueError(bc)


def field_shape(cfg: dict) -> tuple:
    return tuple(len(node_indices(cfg["bc"], n)) for n in reversed(cfg["N"]))


def mesh(cfg: dict) -> list:
    """[X, Y, (Z)] node coordinates broadcast to the field shape."""
    axes = []
    for d in reversed(range(len(cfg["N"]))):
        h = (cfg["hi"][d] - cfg["lo"][d]) / cfg["N"][d]
        axes.append(cfg["lo"][d] + node_indices(cfg["bc"], cfg["N"][d]) * h)
    g = np.meshgrid(*axes, indexing="ij")
    return list(reversed(g))


# Reaction descriptors: kind name + parameter vector + offsets (the steady state
# about which a Dirichlet perturbation is taken).  Parameter order:
#   fhn:               [mu, eps, beta, gamma, delta]
#   gray_scott:        [F, K]
#   schnakenberg:      [gamma, a, b]
#   gierer_meinhardt:  [c1, c2, c3, c4]   f_u = c1 u^2/v - c2 u, f_v = c3 u^2 - c4 v
#   huxley_mms:        []   (Example 2, single species)
#   fisher_mms:        []   (Example 1, single species)
#   linear:            [gamma]
#   none:              []

CONFIGS = {
    # 2D fractional FitzHugh-Nagumo, Neumann, 65^2 nodes, FP64.
    "fhn64": dict(
        dim=2, N=(64, 64), lo=(0.0, 0.0), hi=(100.0, 100.0), bc=NEUMANN,
        alpha=(1.5, 1.5), kappa=(1.0, 0.0), dt=0.1, nsteps=200,
        reaction=dict(kind="fhn", p=[0.1, 0.01, 0.5, 1.0, 0.0], offset=[0.0, 0.0]),
        dtype="f64", seed=0),
    # 2D fractional Gray-Scott, periodic, 1024^2.
    "gs1024": dict(
        dim=2, N=(1024, 1024), lo=(0.0, 0.0), hi=(2.5, 2.5), bc=PERIODIC,
        alpha=(1.7, 1.7), kappa=(2e-5, 1e-5), dt=1.0, nsteps=2000,
        reaction=dict(kind="gray_scott", p=[0.04, 0.06], offset=[0.0, 0.0]),
        dtype="f32", seed=1),
    # 3D fractional Schnakenberg, Dirichlet on the perturbation, 255^3 interior.
    "schnak256": dict(
        dim=3, N=(256, 256, 256), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=DIRICHLET,
        alpha=(1.5, 1.5), kappa=(1.0, 10.0), dt=1e-4, nsteps=500,
        reaction=dict(kind="schnakenberg", p=[1000.0, 0.1, 0.9], offset=[1.0, 0.9]),
        dtype="f32", seed=2),
    # 2D FHN on 257^2 Neumann nodes for the adjoint.
    "fhn256_adjoint": dict(
        dim=2, N=(256, 256), lo=(0.0, 0.0), hi=(100.0, 100.0), bc=NEUMANN,
        alpha=(1.5, 1.5), kappa=(1.0, 0.0), dt=0.1, nsteps=500,
        reaction=dict(kind="fhn", p=[0.1, 0.01, 0.5, 1.0, 0.0], offset=[0.0, 0.0]),
        dtype="f64", seed=4, checkpoint_every=50,
        target=dict(alpha=1.6, kappa_u=1.0, mu=0.1, seed=5)),
}

GM_SIDES = (96, 128, 200, 256, 384)
GM_BCS = (PERIODIC, DIRICHLET, NEUMANN)


def config(name: str, **over) -> dict:
    cfg = copy.deepcopy(CONFIGS[name])
    cfg.update(over)
    return cfg


def scaled(name: str, N, nsteps=None, **over) -> dict:
    """The named workload on a smaller grid (same domain, parameters and IC recipe)."""
    cfg = config(name, **over)
    cfg["N"] = tuple(N) if not isinstance(N, int) else (N,) * cfg["dim"]
    if nsteps is not None:
        cfg["nsteps"] = nsteps
    return cfg


def initial_fields(cfg: dict, seed: int | None = None) -> list:
    """Seeded float64 initial fields for one of the workloads (one array per species)."""
    rng = np.random.default_rng(cfg["seed"] if seed is None else seed)
    kind = cfg["reaction"]["kind"]
    shp = field_shape(cfg)
    M = mesh(cfg)
    if kind == "fhn":
        X, Y = M[0], M[1]
        mid = 0.5 * (cfg["lo"][0] + cfg["hi"][0])
        midy = 0.5 * (cfg["lo"][1] + cfg["hi"][1])
        u = np.where(X < mid, 1.0, 0.0)
        v = np.where(Y > midy, 0.1, 0.0)
        amp = 1e-3
        return [u + rng.uniform(-amp, amp, shp), v + rng.uniform(-amp, amp, shp)]
    if kind == "gray_scott":
        X, Y = M[0], M[1]
        cx = 0.5 * (cfg["lo"][0] + cfg["hi"][0])
        cy = 0.5 * (cfg["lo"][1] + cfg["hi"][1])
        sq = (np.abs(X - cx) <= 0.125) & (np.abs(Y - cy) <= 0.125)
        u = np.where(sq, 0.5, 1.0)
        v = np.where(sq, 0.25, 0.0)
        return [u + rng.uniform(-0.01, 0.01, shp), v + rng.uniform(-0.01, 0.01, shp)]
    if kind == "schnakenberg":
        return [rng.uniform(-0.01, 0.01, shp), rng.uniform(-0.01, 0.01, shp)]
    if kind == "gierer_meinhardt":
        # perturbation about the homogeneous steady state (1, 1)
        return [rng.uniform(-0.05, 0.05, shp), rng.uniform(-0.05, 0.05, shp)]
    if kind in ("linear", "none"):
        return [rng.uniform(-1.0, 1.0, shp) for _ in range(len(cfg["alpha"]))]
    raise ValueError(kind)


def gm_instances(count: int = 256, seed: int = 3) -> list:
    """The batched Gierer-Meinhardt workload: per-instance side, BC and alpha drawn from `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice(GM_SIDES))
        bc = GM_BCS[int(rng.integers(0, 3))]
        a = float(2.0 - rng.uniform(0.0, 0.8))     # uniform in (1.2, 2]
        cfg = dict(dim=2, N=(N, N), lo=(0.0, 0.0), hi=(50.0, 50.0), bc=bc,
                   alpha=(a, a), kappa=(1.0, 30.0), dt=0.05, nsteps=400,
                   reaction=dict(kind="gierer_meinhardt", p=[1.0, 1.0, 1.0, 1.0],
                                 offset=[1.0, 1.0]),
                   dtype="f32", seed=seed * 100003 + i)
        out.append(cfg)
    return out


def random_field(shape, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, shape)
