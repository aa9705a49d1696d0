"""The N>1 host logic on the CPU: placement of whole batched instances on ranks (no data-path collective)
and the max-over-ranks timing reduction, run as two gloo ranks on 127.0.0.1."""
import itertools
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_2003_13569_gb300.shard import (instance_cost, instance_dof, max_over_ranks,  # noqa: E402
                                          shard_instances)


def _cfg(N, bc, dim=2, S=2):
    return dict(dim=dim, N=(N,) * dim, bc=bc, alpha=(1.5,) * S)


def test_instance_dof_counts_unknowns_per_boundary_condition():
    assert instance_dof(_cfg(64, "periodic")) == 64 * 64 * 2
    assert instance_dof(_cfg(64, "dirichlet")) == 63 * 63 * 2
    assert instance_dof(_cfg(64, "neumann")) == 65 * 65 * 2
    assert instance_dof(_cfg(256, "dirichlet", dim=3)) == 255 ** 3 * 2
    assert instance_dof(_cfg(10, "neumann", dim=1, S=1)) == 11


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_placement_is_a_partition(world):
    cfgs = W.gm_instances(256, seed=3)
    parts = shard_instances(cfgs, world)
    assert len(parts) == world
    flat = [i for p in parts for i in p]
    assert sorted(flat) == list(range(len(cfgs)))
    for r, p in enumerate(parts):
        assert p == sorted(p)
        assert shard_instances(cfgs, world, r) == p
    costs = [instance_cost(c) for c in cfgs]
    loads = [sum(costs[i] for i in p) for p in parts]
    # on this workload (many small items) the greedy placement is within 1 % of the mean load
    assert max(loads) <= 1.01 * sum(loads) / world


def test_equal_instances_spread_evenly():
    cfgs = [_cfg(128, "periodic") for _ in range(13)]
    for world in range(1, 8):
        sizes = [len(p) for p in shard_instances(cfgs, world)]
        assert max(sizes) - min(sizes) <= 1


def test_largest_load_within_graham_bound_of_brute_force_optimum():
    """Longest-first greedy placement is within (4/3 - 1/(3m)) of the optimal makespan on m ranks
    (Graham, 1969); the optimum here is found by trying every assignment of 7 instances."""
    rng = np.random.default_rng(11)
    for trial in range(30):
        bcs = ["periodic", "dirichlet", "neumann"]
        cfgs = [_cfg(int(rng.choice([16, 24, 32, 48, 64, 96])), bcs[int(rng.integers(3))]) for _ in range(7)]
        costs = [instance_cost(c) for c in cfgs]
        for m in (2, 3):
            best = min(max(sum(costs[i] for i in range(7) if a[i] == r) for r in range(m))
                       for a in itertools.product(range(m), repeat=7))
            got = max(sum(costs[i] for i in p) for p in shard_instances(cfgs, m))
            assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * best * (1 + 1e-12), (trial, m)


def test_placement_rejects_bad_world_and_rank():
    cfgs = [_cfg(32, "periodic")]
    with pytest.raises(ValueError):
        shard_instances(cfgs, 0)
    with pytest.raises(ValueError):
        shard_instances(cfgs, 2, 2)
    with pytest.raises(ValueError):
        shard_instances(cfgs, 2, -1)


def test_max_over_ranks_without_a_process_group_is_the_identity():
    assert max_over_ranks(3.25) == 3.25


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        cfgs = W.gm_instances(256, seed=3)
        mine = shard_instances(cfgs, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(10.0 + 1.5 * rank)
        dof_mine = sum(instance_dof(cfgs[i]) for i in mine)
        dist.barrier()
        with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
            json.dump({"mine": mine, "gathered": gathered, "max": t, "dof": dof_mine}, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_placement_and_reduce_the_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    cfgs = W.gm_instances(256, seed=3)
    expect = shard_instances(cfgs, world)
    for r in range(world):
        assert res[r]["mine"] == expect[r]
        assert res[r]["gathered"] == expect          # every rank computed the same placement on its own
        assert res[r]["max"] == 11.5                 # the slowest rank's time, seen by every rank
    # the ranks together step every unknown of the workload exactly once
    assert sum(r["dof"] for r in res) == sum(instance_dof(c) for c in cfgs)
