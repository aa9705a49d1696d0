"""Throughput of the ETDRK4-P13 time step on GB300: DOF-steps/s and HBM roofline fraction.

Workload: 3D fractional Schnakenberg, homogeneous Dirichlet BC on the
perturbation (DST-I), N = 256 intervals per axis (255^3 interior unknowns, FFT
length 512), 2 species, alpha = 1.5, kappa = (1, 10), gamma = 1000, dt = 1e-4,
seeded U(-0.01, 0.01) perturbation.  One bench step = one ETDRK4-P13 time step
of the resident spectral state (all four stages: transforms, Pade-(1,3)
combination, reaction) -- launched as the library's captured CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank advances its own replica:
the method has no data-parallel exchange for one grid, so this is replicas-only
weak scaling.  --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ETDRK4 DOF-steps/s, FP32 vs FP64, 3D 255^3, and % of HBM roofline"
WORKLOAD = "schnak256"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=20,
                    help="steps timed on the FP64 path of the same workload (0: skip FP64)")
    ap.add_argument("--err-steps", type=int, default=500,
                    help="steps after which FP32 is compared with FP64 on the GPU (the workload's whole run)")
    ap.add_argument("--repeats", type=int, default=7,
                    help="timed regions of --steps steps each (at least; more are taken until the regions span "
                         "about --clock-span seconds); the line reports their median")
    ap.add_argument("--clock-span", type=float, default=1.0,
                    help="seconds the timed regions span at least, so that the 200 ms clock sampler lands "
                         "samples inside them")
    ap.add_argument("--gs-steps", type=int, default=200,
                    help="steps timed on the 2D Gray-Scott 1024^2 workload, FP32 and FP64 (0: skip)")
    ap.add_argument("--gs-err-steps", type=int, default=2000,
                    help="steps after which the Gray-Scott FP32 path is compared with FP64 (its whole run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--adjoint-steps", type=int, default=500,
                    help="steps of the timed checkpointed forward + adjoint run (0: skip)")
    ap.add_argument("--fhn-steps", type=int, default=200,
                    help="steps timed on the 2D FitzHugh-Nagumo workload, FP64 and FP32 (0: skip)")
    ap.add_argument("--rational-steps", type=int, default=50,
                    help="steps timed for the rational-coefficient variant (0: skip)")
    return ap.parse_args()


def workload_desc(cfg):
    return ("3D fractional Schnakenberg, Dirichlet (DST-I), N=%d (%d^3 interior, FFT length %d), 2 species, "
            "alpha=%.1f, kappa=(%g,%g), gamma=%g, dt=%g" % (cfg["N"][0], cfg["N"][0] - 1, 2 * cfg["N"][0],
                                                            cfg["alpha"][0], cfg["kappa"][0], cfg["kappa"][1],
                                                            cfg["reaction"]["p"][0], cfg["dt"]))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def timed_regions(repeats, span_s, ms_per_step, steps, cap=1000):
    """Number of timed regions of `steps` steps: at least `repeats`, and enough to span `span_s` seconds
    at `ms_per_step` (the warm-up's step time; None when there was no warm-up), at most `cap`."""
    n = max(1, repeats)
    if ms_per_step and ms_per_step > 0 and steps > 0:
        n = max(n, min(cap, math.ceil(span_s * 1e3 / (ms_per_step * steps))))
    return n


def summarise_clocks(rows, t0=None, t1=None):
    """Median SM clock, maximum SM clock and the throttle reasons seen in nvidia-smi rows
    (timestamp, index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap), keeping the samples taken inside the
    wall-clock interval [t0, t1] (all samples when none fall inside or no interval is given)."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    parsed = []
    for r in rows:
        try:
            vals = (float(r[2]), float(r[3]),
                    [nm for i, nm in enumerate(names) if r[6 + i].strip().lower() == "active"])
        except (ValueError, IndexError):
            continue
        try:
            ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        parsed.append((ts,) + vals)
    inside = [p for p in parsed if None not in (p[0], t0, t1) and t0 <= p[0] <= t1]
    use = inside if inside else parsed
    sm = [p[1] for p in use]
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(p[2] for p in use) if use else None,
            "reasons": sorted(set(nm for p in use for nm in p[3])), "samples": len(use),
            "samples_in_timed_region": len(inside)}


class Clocks:
    """nvidia-smi sampling (every 200 ms) around the timed region; the summary keeps the samples
    taken between mark() and stop()."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.t0 = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def mark(self):
        """Start of the timed region (wall clock)."""
        self.t0 = time.time()

    def stop(self):
        t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)   # the sample that covers the end of the region
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        return summarise_clocks(rows, self.t0, t1)


# Algorithmic HBM words per unknown (per species element) of each pass kind (fixed pass model).
# x pass: read + write the field (the reaction needs no extra traffic);
# middle pass: read + write; slow passes: field in/out + stored spectra + coefficients.
WORDS = {0: 2, 1: 2, 2: 6, 3: 6, 4: 7, 5: 11}
KIND_NAME = {0: "x_pass_react", 1: "y_pass_middle", 2: "z_pass_stage_a", 3: "z_pass_stage_b",
             4: "z_pass_stage_c", 5: "z_pass_update"}


def ncu_traffic(kind_name):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if one exists for it."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 2 and parts[0] == kind_name:
            try:
                return float(parts[1])
            except ValueError:
                return None
    return None


def cpu_model():
    """The host CPU's model name (lscpu), for the baseline records."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(cfg, seconds):
    """The FP64 oracle (dense per-axis transforms, Algorithm 1) timed on the host cores."""
    from oracle.bridge import solver as oracle_solver
    u0 = W.initial_fields(cfg)
    s = oracle_solver(cfg)
    t0 = time.perf_counter()
    n = 0
    u = u0
    while True:
        u = s.step(u, n * cfg["dt"])
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 50:
            break
    el = time.perf_counter() - t0
    dof = int(np.prod(W.field_shape(cfg))) * 2
    return {"value": dof * n / el, "unit": "DOF-steps/s", "cores": os.cpu_count(), "cpu_model": cpu_model(),
            "kind": "oracle", "role": "the stated host baseline: whole steps of the full workload",
            "sample": "%d ETDRK4-P13 step(s) of the full %s workload, FP64 dense-matrix oracle, %.1f s"
                      % (n, "x".join(str(x) for x in W.field_shape(cfg)), el)}


def reference_arm(args):
    """--impl reference: the CPU oracle on the workload per step, timed on the host cores.

    The full 255^3 grid is used when the whole --warmup/--steps run fits in about four minutes at the
    measured time of one oracle step (one untimed step first); otherwise the largest of the reduced grids
    N = 128, 64 that fits, named in config.sample_grid (same_config false)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.bridge import solver as oracle_solver
    budget = float(os.environ.get("SFRD_REF_SECONDS", "240"))
    nrun = args.warmup + args.steps
    cfg = None
    sizes = (W.config(WORKLOAD)["N"][0], 128, 64)
    if os.environ.get("SFRD_REF_N"):             # a fixed sample size (the CPU tests use a tiny one)
        sizes = (int(os.environ["SFRD_REF_N"]),)
    for Nsample in sizes:
        c = W.scaled(WORKLOAD, Nsample)
        s = oracle_solver(c)
        u = W.initial_fields(c)
        t0 = time.perf_counter()
        u = s.step(u, 0.0)                       # untimed: the cost of one step at this size
        if (time.perf_counter() - t0) * nrun <= budget or Nsample == sizes[-1]:
            cfg = c
            break
    for k in range(args.warmup):
        u = s.step(u, (k + 1) * cfg["dt"])
    t0 = time.perf_counter()
    for k in range(args.steps):
        u = s.step(u, (args.warmup + 1 + k) * cfg["dt"])
    el = time.perf_counter() - t0
    dof = int(np.prod(W.field_shape(cfg))) * 2
    v = dof * args.steps / el
    full = cfg["N"] == W.config(WORKLOAD)["N"]
    n1 = cfg["N"][0] - 1
    line = {"metric": METRIC, "value": v, "unit": "DOF-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(W.config(WORKLOAD)),
                       "sample_grid": list(cfg["N"]), "same_config": full, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "DOF-steps/s", "cores": os.cpu_count(), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": "one FP64 oracle step per bench step on the same workload at N=%d "
                                       "(%d^3 interior)" % (cfg["N"][0], n1)},
            "e2e": {"value": v, "unit": "DOF-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    import paper_2003_13569_gb300 as sf
    from paper_2003_13569_gb300.shard import instance_dof, max_over_ranks, shard_instances

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    cfg = W.config(WORKLOAD)
    u0 = W.initial_fields(cfg, seed=cfg["seed"] + rank)
    solver = sf.Solver(cfg, dtype=args.dtype)
    dof = solver.dof
    stream = solver.stream
    u0_dev = torch.as_tensor(np.stack(u0)).to(device="cuda", dtype=solver.tdtype)
    solver.load(u0_dev, 0.0)
    w0 = torch.cuda.Event(enable_timing=True)
    w1 = torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    solver.advance(args.warmup)
    w1.record(stream)
    torch.cuda.synchronize()
    # regions: --repeats, or as many as span --clock-span seconds at the warm-up's step time (same on every rank)
    est_ms = max_over_ranks(w0.elapsed_time(w1) / args.warmup) if args.warmup > 0 else None
    nreg = timed_regions(args.repeats, args.clock_span, est_ms, args.steps)

    clocks = Clocks(local) if rank == 0 else None
    time.sleep(0.3 if clocks else 0.0)
    # R timed regions of exactly K steps each (barrier + synchronize on both sides of every region, CUDA
    # events on the solver's stream, max over ranks); the line reports the median region
    regions = []
    if clocks:
        clocks.mark()
    for _ in range(nreg):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.advance(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        regions.append(max_over_ranks(e0.elapsed_time(e1)))
    clk = clocks.stop() if clocks else None
    ms = statistics.median(regions)
    value = dof * args.steps * world / (ms * 1e-3)
    repeats = {"regions": len(regions), "steps_per_region": args.steps, "min_span_s": args.clock_span,
               "ms_per_step_median": ms / args.steps,
               "ms_per_step_min": min(regions) / args.steps, "ms_per_step_max": max(regions) / args.steps,
               "value_min": dof * args.steps * world / (max(regions) * 1e-3),
               "value_max": dof * args.steps * world / (min(regions) * 1e-3)}

    # per-launch profile of the same step (events on the launching stream)
    prof = {}
    nprof = max(3, min(args.steps, 10))
    for _ in range(nprof):
        for kd, t in solver.profile_step():
            prof.setdefault(kd, []).append(t)
    esize = 4 if args.dtype == "f32" else 8
    per_kind = {}
    tot = sum(sum(v) for v in prof.values())
    for kd, ts in prof.items():
        avg = sum(ts) / len(ts)
        algo = WORDS[kd] * dof * esize
        per_kind[KIND_NAME[kd]] = {"launches_per_step": len(ts) // nprof, "avg_ms": avg,
                                   "share": sum(ts) / tot, "algo_bytes": algo,
                                   "gbs": algo / (avg * 1e-3) / 1e9}
    dom = max(per_kind.items(), key=lambda kv: kv[1]["share"])
    peak, peak_kind = peaks()
    roof = {"bound": "hbm", "achieved": dom[1]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": dom[1]["gbs"] / peak, "traffic": ncu_traffic(dom[0]), "kernel": dom[0],
            "peak_source": peak_kind}
    step_words = sum(WORDS[kd] * len(ts) / nprof for kd, ts in prof.items())
    model_bytes = step_words * dof * esize
    step_roof = {"model_words_per_dof_step": step_words, "model_bytes_per_step": model_bytes,
                 "achieved_gbs": model_bytes / (ms * 1e-3 / args.steps) / 1e9,
                 "frac_of_" + peak_kind: model_bytes / (ms * 1e-3 / args.steps) / 1e9 / peak}

    # FP64 path on the same workload, and the FP32-vs-FP64 error after the workload's whole run
    extra = {}
    ref = None
    if rank == 0 and args.dtype == "f32" and args.fp64_steps > 0:
        s64 = sf.Solver(cfg, dtype="f64")
        s64.load(u0_dev.double(), 0.0)
        s64.advance(1)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s64.stream)
        s64.advance(args.fp64_steps)
        a1.record(s64.stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1)
        extra["fp64"] = {"value": dof * args.fp64_steps / (ms64 * 1e-3), "unit": "DOF-steps/s",
                         "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps}
        if args.err_steps > 0:
            ref = s64.run(u0_dev.double(), nsteps=args.err_steps)
            got = solver.run(u0_dev, nsteps=args.err_steps).double()
            err = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
            extra["fp32_vs_fp64_rel_l2"] = {"value": err, "steps": args.err_steps,
                                            "whole_run": args.err_steps == cfg["nsteps"]}
        del s64
        torch.cuda.empty_cache()

        # the rational-coefficient variant: L = kappa tau Lambda^(alpha/2) computed in FP64 and stored in
        # FP32 (one plane shared by the species when their orders agree), the Pade(1,3) coefficients
        # evaluated in FP32 inside the slow-axis passes; its own pass model (fewer coefficient words)
        if args.rational_steps > 0:
            sr = sf.Solver(cfg, dtype="f32", coefficients="rational")
            sr.load(u0_dev, 0.0)
            sr.advance(args.warmup)
            torch.cuda.synchronize()
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(sr.stream)
            sr.advance(args.rational_steps)
            r1.record(sr.stream)
            torch.cuda.synchronize()
            msr = r0.elapsed_time(r1)
            errr = None
            if ref is not None:
                gotr = sr.run(u0_dev, nsteps=args.err_steps).double()
                errr = float(torch.linalg.vector_norm(gotr - ref) / torch.linalg.vector_norm(ref))
            shared = len(cfg["alpha"]) == 2 and cfg["alpha"][0] == cfg["alpha"][1]
            lw = 0.5 if shared else 1.0            # words of L per unknown, per slow-axis pass
            coef_words = {2: 2, 3: 2, 4: 2, 5: 4}  # stored coefficient words per pass kind
            rwords = sum((WORDS[kd] - coef_words.get(kd, 0) + (lw if kd in coef_words else 0)) * len(ts) / nprof
                         for kd, ts in prof.items())
            rbytes = rwords * dof * esize
            extra["rational_coefficients"] = {
                "value": dof * args.rational_steps / (msr * 1e-3), "unit": "DOF-steps/s",
                "ms_per_step": msr / args.rational_steps, "steps": args.rational_steps,
                "model_words_per_dof_step": rwords,
                "frac_of_" + peak_kind: rbytes / (msr * 1e-3 / args.rational_steps) / 1e9 / peak,
                "fp32_vs_fp64_rel_l2": {"value": errr, "steps": args.err_steps},
                "shared_l_plane": shared}
            del sr
            torch.cuda.empty_cache()
    ref = None

    # the batched workload: 256 Gierer-Meinhardt instances, one persistent launch per pass; with several
    # ranks each takes whole instances (no data-path collective) and the slowest rank sets the time
    if args.batched_steps > 0:
        cfgs_all = W.gm_instances(256, seed=3)
        mine = shard_instances(cfgs_all, world, rank)
        cfgs = [cfgs_all[i] for i in mine]
        bt = sf.Batch(cfgs, dtype="f32")
        sched = bt.autotune(steps=2)          # blocks per SM and radix order (shared-memory engine sides)
        bt.load([np.stack(W.initial_fields(c)) for c in cfgs])
        bt.advance(3)
        torch.cuda.synchronize()
        barrier()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(bt.stream)
        bt.advance(args.batched_steps)
        b1.record(bt.stream)
        torch.cuda.synchronize()
        barrier()
        msb = max_over_ranks(b0.elapsed_time(b1))
        sides = sorted(set(int(c["N"][0]) for c in cfgs_all))
        dof_all = sum(instance_dof(c) for c in cfgs_all)
        extra["batched"] = {"value": dof_all * args.batched_steps / (msb * 1e-3), "unit": "DOF-steps/s",
                            "ms_per_step": msb / args.batched_steps, "steps": args.batched_steps,
                            "instances": len(cfgs_all), "dof": dof_all, "instances_per_rank": len(mine),
                            "placement": "whole instances per rank, longest first (no collective)",
                            "launches_per_step": bt.launches_per_step,
                            "schedule": {"blocks_per_sm": sched[0], "radix_order_rule": sched[1],
                                         "chosen_by": "sfrd_batch_autotune (2 timed steps per candidate)"},
                            "workload": "2D fractional Gierer-Meinhardt, 256 instances, sides %s, BC P/D/N and "
                                        "alpha U(1.2,2] per instance, dt=0.05, FP32" % sides}
        del bt
        torch.cuda.empty_cache()

    # end to end through host memory: pinned input -> device -> K steps -> pinned output
    host_in = torch.as_tensor(np.stack(u0)).to(dtype=solver.tdtype).contiguous().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    solver.run_host_ptr(host_in.data_ptr(), host_out.data_ptr(), 0.0, args.steps)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    ncalls = 2
    for _ in range(ncalls):
        solver.run_host_ptr(host_in.data_ptr(), host_out.data_ptr(), 0.0, args.steps)
    el = time.perf_counter() - t0
    barrier()
    el = max_over_ranks(el)
    fbytes = host_in.numel() * host_in.element_size()
    e2e = {"value": dof * args.steps * ncalls * world / el, "unit": "DOF-steps/s",
           "h2d_bytes_per_step": fbytes / args.steps, "d2h_bytes_per_step": fbytes / args.steps,
           "steps_per_call": args.steps, "api": "sfrd_run_host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, args.cpu_seconds)

    # the 2D Gray-Scott workload (1024^2 periodic, FP32 and FP64): throughput, its 38-word pass model against
    # the HBM peak (the FP32 working set, about 0.1 GB, may stay in the 126 MB L2: context, not a gate), and the
    # FP32-vs-FP64 error after its whole 2000-step run
    if rank == 0 and args.gs_steps > 0:
        gcfg = W.config("gs1024")
        gu0 = torch.as_tensor(np.stack(W.initial_fields(gcfg)))
        extra["gs1024"] = {"workload": "2D fractional Gray-Scott, periodic (Hartley), N=1024 (1024^2), alpha=1.7, "
                                       "kappa=(2e-5,1e-5), F=0.04, K=0.06, dt=1", "steps": args.gs_steps}
        finals = {}
        try:
            for dt in ("f32", "f64"):
                sg = sf.Solver(gcfg, dtype=dt)
                sg.load(gu0.cuda(), 0.0)
                sg.advance(3)
                torch.cuda.synchronize()
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(sg.stream)
                sg.advance(args.gs_steps)
                g1.record(sg.stream)
                torch.cuda.synchronize()
                msg = g0.elapsed_time(g1) / args.gs_steps
                es = 4 if dt == "f32" else 8
                words = sum(WORDS[k] for k, _ in sg.profile_step())   # pass kinds of one step
                extra["gs1024"][dt] = {"value": sg.dof / (msg * 1e-3), "unit": "DOF-steps/s", "ms_per_step": msg,
                                       "model_words_per_dof_step": words,
                                       "model_frac_of_" + peak_kind: words * sg.dof * es / (msg * 1e-3) / 1e9 / peak,
                                       "gpu_launches_per_step": sg.kernels_per_step}
                if args.gs_err_steps > 0:
                    finals[dt] = sg.run(gu0.cuda(), nsteps=args.gs_err_steps).double()
                del sg
                torch.cuda.empty_cache()
            if len(finals) == 2:
                extra["gs1024"]["fp32_vs_fp64_rel_l2"] = {
                    "value": float(torch.linalg.vector_norm(finals["f32"] - finals["f64"]) /
                                   torch.linalg.vector_norm(finals["f64"])),
                    "steps": args.gs_err_steps, "whole_run": args.gs_err_steps == gcfg["nsteps"]}
        except Exception as exc:   # keep the headline line whatever happens here
            extra["gs1024"]["error"] = "%s: %s" % (type(exc).__name__, exc)
        finals = None
        torch.cuda.empty_cache()

    # the 2D FitzHugh-Nagumo workload (65^2 Neumann nodes, its 200 steps), FP64 and FP32: a small grid whose
    # step is bound by launch latency rather than HBM; reported for completeness, errors kept in the record
    if rank == 0 and args.fhn_steps > 0:
        fcfg = W.config("fhn64")
        extra["fhn64"] = {"workload": "2D fractional FitzHugh-Nagumo, Neumann (DCT-I), N=64 (65^2 nodes), "
                                      "alpha=1.5, kappa=(1,0), dt=0.1", "steps": args.fhn_steps}
        for dt in ("f64", "f32"):
            try:
                sfhn = sf.Solver(fcfg, dtype=dt)
                sfhn.load(torch.as_tensor(np.stack(W.initial_fields(fcfg))), 0.0)
                sfhn.advance(3)
                torch.cuda.synchronize()
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                f0.record(sfhn.stream)
                sfhn.advance(args.fhn_steps)
                f1.record(sfhn.stream)
                torch.cuda.synchronize()
                msf = f0.elapsed_time(f1)
                extra["fhn64"][dt] = {"value": sfhn.dof * args.fhn_steps / (msf * 1e-3), "unit": "DOF-steps/s",
                                      "ms_per_step": msf / args.fhn_steps,
                                      "gpu_launches_per_step": sfhn.kernels_per_step}
                del sfhn
            except Exception as exc:   # keep the headline line whatever happens here
                extra["fhn64"][dt] = {"error": "%s: %s" % (type(exc).__name__, exc)}

    # the discrete adjoint on its workload (2D FitzHugh-Nagumo, 257^2 Neumann nodes, FP64, checkpoints every
    # 50 steps): one checkpointed forward run and one reverse sweep (with recomputation), timed by events
    if rank == 0 and args.adjoint_steps > 0:
        try:
            acfg = W.config("fhn256_adjoint")
            n, K = args.adjoint_steps, acfg["checkpoint_every"]
            sa = sf.Solver(acfg, dtype="f64")
            u0a = np.stack(W.initial_fields(acfg))
            tgt = torch.as_tensor(np.stack(W.initial_fields(acfg, seed=acfg["target"]["seed"])),
                                  device="cuda", dtype=torch.float64)
            for timed in (False, True):            # the first pass allocates the checkpoint buffer
                a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                torch.cuda.synchronize()
                a0.record(sa.stream)
                uT = sa.run_checkpointed(u0a, 0.0, n, K)
                a1.record(sa.stream)
                grads = sa.adjoint(uT - tgt, 0.0, n, K)
                a2.record(sa.stream)
                torch.cuda.synchronize()
            fwd, rev = a0.elapsed_time(a1), a1.elapsed_time(a2)
            extra["adjoint"] = {"value": sa.dof * n / ((fwd + rev) * 1e-3),
                                "unit": "DOF-steps/s (checkpointed forward + reverse sweep)",
                                "forward_ms": fwd, "reverse_ms": rev, "steps": n, "checkpoint_every": K,
                                "dtype": "f64", "dL_dalpha": grads[1], "dL_dkappa": grads[2],
                                "dL_dparams": list(grads[3][:1]),
                                "workload": "2D fractional FitzHugh-Nagumo, Neumann, N=256 (257^2 nodes), "
                                            "loss 0.5||u_T - target||^2"}
            del sa
            # the same forward run and reverse sweep in FP32 (FP64 coefficients), its errors against FP64
            s32 = sf.Solver(acfg, dtype="f32")
            uT32 = s32.run_checkpointed(u0a, 0.0, n, K)
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            uT32 = s32.run_checkpointed(u0a, 0.0, n, K)
            b0.record(s32.stream)
            g32 = s32.adjoint(uT32 - tgt.float(), 0.0, n, K)
            b1.record(s32.stream)
            torch.cuda.synchronize()

            def rel(a, b):
                return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)

            d64, d32 = grads[0].double(), g32[0].double()
            extra["adjoint"]["f32"] = {
                "reverse_ms": b0.elapsed_time(b1),
                "uT_rel_l2_vs_f64": float((uT32.double() - uT).norm() / uT.norm()),
                "dL_du0_rel_l2_vs_f64": float((d32 - d64).norm() / d64.norm()),
                "dL_dalpha_rel_vs_f64": rel(g32[1][0], grads[1][0]),
                "dL_dkappa_rel_vs_f64": rel(g32[2][0], grads[2][0]),
                "dL_dparams_rel_vs_f64": rel(g32[3][0], grads[3][0])}
            del s32
        except Exception as exc:
            extra["adjoint"] = {"error": "%s: %s" % (type(exc).__name__, exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "DOF-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": workload_desc(cfg), "grid_intervals": list(cfg["N"]),
                           "unknowns": list(solver.shape), "dof": dof, "parallelism": "replicas",
                           "l2": "inputs larger than L2 (resident state + stored spectra + coefficients "
                                 "%.2f GB > 126 MB)" % (solver.info.workspace_bytes / 1e9),
                           "timed": "sfrd_advance (captured CUDA graph), one ETDRK4-P13 step per bench step"},
                "gpu_launches": solver.kernels_per_step * args.steps,
                "roofline": roof, "step_roofline": step_roof, "kernels": per_kind, "repeats": repeats,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
