"""The benchmark's command-line contract on the CPU: the reference arm (the FP64 oracle on a bounded sample)
prints one JSON line with the required keys on rank 0 and nothing on other ranks, and the product arm and the
package refuse to run without the CUDA library and a GPU instead of falling back to anything."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, BENCH] + args, capture_output=True, text=True, env=env, timeout=timeout,
                          cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"], {"SFRD_REF_N": "8"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "DOF-steps/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["data"] == "synthetic" and d["dtype"] == "f64" and d["vs_baseline"] is None
    assert "255^3" in d["config"]["workload"] and d["config"]["sample_grid"] == [8, 8, 8]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "N=8" in d["cpu_baseline"]["sample"]
    assert isinstance(d["cpu_baseline"]["cpu_model"], str) and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_nothing_on_other_ranks():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"SFRD_REF_N": "8", "RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_product_arm_without_a_gpu_fails_without_a_result_line():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the product arm would run")
    r = _run(["--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--fp64-steps", "0", "--batched-steps", "0",
              "--rational-steps", "0"])
    assert r.returncode != 0
    assert not any(ln.lstrip().startswith("{") for ln in r.stdout.splitlines())


def test_package_refuses_to_import_without_the_library(tmp_path):
    pkg = tmp_path / "sfrd_copy"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2003_13569_gb300", "__init__.py"), pkg / "__init__.py")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n    import sfrd_copy\nexcept ImportError as e:\n    print('refused:', e)\n    sys.exit(0)\n"
            "sys.exit(1)\n" % str(tmp_path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "libsfrd.so is not built" in r.stdout


def test_clock_summary_keeps_the_samples_of_the_timed_region():
    import datetime
    sys.path.insert(0, ROOT)
    import bench
    t = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def row(dt, sm, hw="Not Active", cap="Not Active"):
        ts = (t + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return [ts, "0", str(sm), "2070", "900.5", "0x0", hw, "Not Active", "Not Active", cap]

    rows = [row(0.0, 1400), row(0.2, 2070), row(0.4, 2055, cap="Active"), row(0.6, 2070), row(0.8, 1500,
                                                                                              hw="Active")]
    t0, t1 = (t + datetime.timedelta(seconds=0.1)).timestamp(), (t + datetime.timedelta(seconds=0.7)).timestamp()
    c = bench.summarise_clocks(rows, t0, t1)
    assert c["samples_in_timed_region"] == 3 and c["samples"] == 3
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]                 # the hw_slowdown sample lies after the region
    c = bench.summarise_clocks(rows)                         # no interval: every sample
    assert c["samples"] == 5 and c["samples_in_timed_region"] == 0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"] and c["sm_mhz"] == 2055
    bad = [["not a time"] + r[1:] for r in rows]             # unparsable timestamps: every sample, none dropped
    assert bench.summarise_clocks(bad, t0, t1)["samples"] == 5


def test_pass_model_and_committed_traffic():
    sys.path.insert(0, ROOT)
    import bench
    launches_3d = {0: 4, 1: 8, 2: 1, 3: 1, 4: 1, 5: 1}       # x, middle, stages a-c, update
    launches_2d = {0: 4, 2: 1, 3: 1, 4: 1, 5: 1}
    assert sum(bench.WORDS[k] * n for k, n in launches_3d.items()) == 54
    assert sum(bench.WORDS[k] * n for k, n in launches_2d.items()) == 38
    dof = 2 * 255 ** 3
    for kind, name in bench.KIND_NAME.items():
        t = bench.ncu_traffic(name)
        assert t is not None, name
        # the captured DRAM bytes of a launch lie within [0.5, 1.2] x its algorithmic bytes (no re-reads;
        # below 1 where the input was still in L2)
        assert 0.5 < t / (bench.WORDS[kind] * dof * 4) < 1.2, (name, t)
    assert bench.ncu_traffic("no_such_kernel") is None
    peak, src = bench.peaks()
    assert peak > 1000 and src in ("measured", "fallback")


def test_timed_regions_span_the_clock_sampler():
    """The bench times at least --repeats regions of K steps, and enough of them to span about a second
    (the 200 ms clock sampler then lands samples inside them): 20 steps of 1.6 ms need 32 regions, 500
    steps keep the 7 asked for, no warm-up estimate keeps --repeats, and the count is capped."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.timed_regions(7, 1.0, 1.6, 20) == 32
    assert bench.timed_regions(7, 1.0, 1.6, 500) == 7
    assert bench.timed_regions(7, 1.0, None, 20) == 7
    assert bench.timed_regions(0, 1.0, None, 20) == 1
    assert bench.timed_regions(7, 1.0, 1e-6, 1) == 1000
