"""Writes the full-run expected values of the named workloads (tests/golden/fullrun_*.npz).

Each file holds the FP64 CPU oracle's result after the workload's whole run (Algorithm 1,
M steps from the seeded initial fields of workloads/), sampled on a strided subgrid that
includes the last unknown of every axis, plus the full-field norms the relative errors divide
by.  Nothing here comes from the CUDA library: the script imports only oracle/ and the input
generators.  The GPU tests (tests/test_gpu_fullrun.py) run the same workload through the C ABI
and compare at the same points.

  python tests/golden/make_fullrun.py [case ...]      (default: every case; hours for the
                                                       255^3 and 1024^2 cases on a few cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.bridge import solver  # noqa: E402


def sample_axis(n: int, stride: int) -> np.ndarray:
    """Every stride-th unknown along an axis of n unknowns, and the last one."""
    return np.unique(np.r_[np.arange(0, n, stride), n - 1])


def gm_cases() -> list:
    """The first instance of the 256-instance Gierer-Meinhardt draw for every (side, BC) pair."""
    seen, out = set(), []
    for i, cfg in enumerate(W.gm_instances(256, seed=3)):
        key = (cfg["N"][0], cfg["bc"])
        if key not in seen:
            seen.add(key)
            out.append((i, cfg))
    return sorted(out, key=lambda t: (t[1]["N"][0], t[1]["bc"]))


# case name -> (workload config, stride of the sampled subgrid)
def cases() -> dict:
    c = {
        "schnak128": (W.scaled("schnak256", 128), 8),      # 127^3 interior, 500 steps
        "schnak256": (W.config("schnak256"), 16),          # 255^3 interior, 500 steps
        "gs1024": (W.config("gs1024"), 16),                # 1024^2 periodic, 2000 steps
    }
    for i, cfg in gm_cases():
        c["gm%03d" % i] = (cfg, max(1, cfg["N"][0] // 32))
    return c


def write_case(name: str, cfg: dict, stride: int) -> str:
    u0 = W.initial_fields(cfg)
    t0 = time.time()
    u = solver(cfg).run(u0, 0.0, cfg["nsteps"])
    el = time.time() - t0
    shape = u[0].shape
    idx = [sample_axis(n, stride) for n in shape]
    sel = np.ix_(*idx)
    vals = np.stack([np.asarray(x)[sel] for x in u])
    path = os.path.join(HERE, "fullrun_%s.npz" % name)
    np.savez_compressed(
        path, values=vals, **{"idx%d" % d: idx[d] for d in range(len(idx))},
        max_abs=np.array(max(float(np.max(np.abs(x))) for x in u)),
        l2=np.array(float(np.sqrt(sum(float(np.sum(np.asarray(x) ** 2)) for x in u)))),
        nsteps=np.array(cfg["nsteps"]), N=np.array(cfg["N"]), bc=np.array(cfg["bc"]),
        seed=np.array(cfg["seed"]), oracle_seconds=np.array(el))
    return path


def main(argv):
    all_cases = cases()
    names = argv or list(all_cases)
    for nm in names:
        cfg, stride = all_cases[nm]
        t = time.time()
        p = write_case(nm, cfg, stride)
        print("%s: %s steps of N=%s %s -> %s (%.0f s)" % (nm, cfg["nsteps"], cfg["N"], cfg["bc"], p, time.time() - t),
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
