"""Placement of independent instances on ranks (one process per GPU), and the one reduction the
timing needs.

The instances of a batched run share nothing: each is its own grid, boundary condition, fractional order
and diffusivity (e.g. a sweep of the Gierer-Meinhardt model of Section 5.2 over grids, boundary
conditions and orders), stepped by the same ETDRK4-P13 scheme (Section 4).  So whole instances go to
ranks and no collective touches the data path; every rank computes the same deterministic placement on
its own, and only a timing is reduced across ranks (the maximum: the job ends when its slowest rank
does).
"""
from __future__ import annotations

import math

_UNKNOWN_OFFSET = {"periodic": 0, "dirichlet": -1, "neumann": 1}


def instance_dof(cfg: dict) -> int:
    """Unknowns per species times species: N per axis for periodic, N-1 for Dirichlet, N+1 for
    Neumann (N = intervals per axis)."""
    off = _UNKNOWN_OFFSET[cfg["bc"]]
    n = 1
    for d in range(cfg["dim"]):
        n *= int(cfg["N"][d]) + off
    return n * len(cfg["alpha"])


def instance_cost(cfg: dict) -> float:
    """Relative cost of one step: every pass streams the instance's unknowns and a line of a length-n
    transform costs about log2 n per point (n = N for periodic, the 2N extension for Dirichlet and
    Neumann)."""
    ext = 1 if cfg["bc"] == "periodic" else 2
    depth = sum(math.log2(ext * int(cfg["N"][d])) for d in range(cfg["dim"]))
    return instance_dof(cfg) * depth


def shard_instances(cfgs: list, world: int, rank: int | None = None):
    """Longest-processing-time-first placement of `cfgs` on `world` ranks: instances in decreasing cost
    (ties by index) each go to the rank with the least load so far (ties to the lowest rank).  The
    largest load is within 4/3 of the best possible placement (Graham's bound for this greedy rule).

    Returns the per-rank lists of instance indices, each ascending, or with `rank` only that rank's list.
    Raises ValueError for world < 1 or a rank outside [0, world)."""
    if world < 1:
        raise ValueError("world size must be at least 1, got %d" % world)
    if rank is not None and not 0 <= rank < world:
        raise ValueError("rank %d outside [0, %d)" % (rank, world))
    costs = [instance_cost(c) for c in cfgs]
    order = sorted(range(len(cfgs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    parts = [sorted(p) for p in parts]
    return parts if rank is None else parts[rank]


def max_over_ranks(x: float) -> float:
    """The maximum of `x` over the ranks of the default process group (`x` itself when no group is
    initialised).  The reduction runs on the current CUDA device under NCCL and on the host under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
