"""Builds libsfrd.so in this directory from csrc/*.cu with nvcc for sm_103a.

Each translation unit (or each part of one, for the sources split by SFRD_TU_PART) is
compiled in parallel, then linked into one shared
library with the CUDA runtime linked statically.  Usage: python -m
paper_2003_13569_gb300.build  (or call build()).
"""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libsfrd.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE]


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libsfrd.so)")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _newest_header():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max(os.path.getmtime(h) for h in hdrs)


def _parts(src):
    """Objects a source compiles to: one, or one per SFRD_TU_PART value it tests (0..k)."""
    with open(src) as f:
        found = [int(k) for k in re.findall(r"SFRD_TU_PART == (\d+)", f.read())]
    return list(range(max(found) + 1)) if found else [None]


def _cost_key(job):
    """Longest compiles first: register-FFT lengths by length, FP32 before FP64, then the rest."""
    name = os.path.basename(job[0])
    m = re.match(r"sfrd_(v2|batch)_f(32|64)_(\d+)", name)
    if not m:
        return (1, 0, name)
    kind, bits, n = m.groups()
    return (0, -(int(n) * (2 if bits == "32" else 1) * (2 if kind == "v2" else 1)), name)


def build(verbose=False, extra=()):
    """Compile every translation unit (in parallel, one job per core, longest first) and link
    libsfrd.so.  With SFRD_BUILD_INCREMENTAL=1 an object newer than its source and every header is
    reused (a local convenience; a fresh checkout always compiles everything)."""
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)
    incremental = os.environ.get("SFRD_BUILD_INCREMENTAL") == "1"
    newest_hdr = _newest_header() if incremental else 0.0
    jobs = []
    objs = []
    for src in sources():
        for part in _parts(src):
            stem = os.path.basename(src)[:-3] + ("" if part is None else "_p%d" % part)
            obj = os.path.join(BUILD_DIR, stem + ".o")
            objs.append(obj)
            if incremental and os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), newest_hdr):
                continue
            define = [] if part is None else ["-DSFRD_TU_PART=%d" % part]
            jobs.append((src, [nvcc, *ARCH, *FLAGS, *define, *extra, "-c", src, "-o", obj]))
    jobs.sort(key=_cost_key)

    def run(job):
        if verbose:
            print(" ".join(job[1]), flush=True)
        r = subprocess.run(job[1], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        return job[0], r.returncode, r.stdout.decode(errors="replace")

    failed = []
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        for src, rc, out in ex.map(run, jobs):
            if rc != 0:
                failed.append((src, out))
            elif verbose and out:
                print(out, flush=True)
    if failed:
        msg = "\n".join("%s:\n%s" % f for f in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, extra=[a for a in sys.argv[1:] if a != "-v"])
    print(LIB)
