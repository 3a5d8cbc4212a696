"""Build libme.so in-tree for sm_103a.

Steps: run the process generator (gen/) to emit one CUDA translation unit per
process plus the registry into _build/gen/, compile every unit with nvcc in
parallel (one -gencode: compute_103a / sm_103a), link the shared library
_build/libme.so.  No cmake; the generated sources are rebuilt whenever the
generator or a header changes.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.environ.get("ME_BUILD_DIR") or os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj")
LIB = os.path.join(BUILD, "libme.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v", "-I", INCLUDE, "-I", CSRC]

STATIC_SOURCES = ["me_abi.cu", "rambo.cu", "serve.cu"]
# processes compiled into the library (build option ME_BUILD_PROCESSES: a
# comma-separated subset, for quicker builds of kernel variants)
ALL_PROCESSES = ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg", "uux_epem", "uux_epemg", "uux_epemgg",
                 "uux_epemggg")
PROCESSES = tuple(p for p in os.environ.get("ME_BUILD_PROCESSES", ",".join(ALL_PROCESSES)).split(",")
                  if p in ALL_PROCESSES) or ALL_PROCESSES


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()


def _inputs():
    out = []
    for d in (CSRC, os.path.join(HERE, "gen"), INCLUDE):
        for fn in os.listdir(d):
            if fn.endswith((".cu", ".cuh", ".h", ".py")):
                out.append(os.path.join(d, fn))
    return out


def generate(processes=None) -> list:
    sys.path.insert(0, ROOT)
    from paper_2507_21039_gb300.gen import emit

    processes = processes or PROCESSES
    os.makedirs(GEN, exist_ok=True)
    srcs, metas = [], {}
    for p in processes:
        src, meta = emit.emit_process(p)
        path = os.path.join(GEN, f"proc_{p}.cu")
        if not os.path.exists(path) or open(path).read() != src:
            with open(path, "w") as f:
                f.write(src)
        srcs.append(path)
        metas[p] = meta
    reg = os.path.join(GEN, "registry.cu")
    rsrc = emit.emit_registry(processes)
    for fn in os.listdir(GEN):  # drop units of processes no longer built
        if fn.startswith("proc_") and fn[5:-3] not in processes:
            os.remove(os.path.join(GEN, fn))
    if not os.path.exists(reg) or open(reg).read() != rsrc:
        with open(reg, "w") as f:
            f.write(rsrc)
    srcs.append(reg)
    with open(os.path.join(GEN, "processes.json"), "w") as f:
        json.dump(metas, f, indent=1, default=str)
    return srcs


def _extra_flags() -> list:
    """Build option ME_NVCC_EXTRA: additional preprocessor definitions (-DNAME=V),
    used to compare kernel tuning parameters."""
    return [f for f in os.environ.get("ME_NVCC_EXTRA", "").split() if f.startswith("-D")]


def _compile(src: str, obj: str) -> tuple[str, str]:
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + _extra_flags() + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-4000:]}")
    return src, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OBJ, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = (_digest(_inputs()) + ",".join(PROCESSES) + os.environ.get("ME_GEN_KERNEL", "") + " ".join(_extra_flags())
           + os.environ.get("ME_INTERP_CONST", "") + os.environ.get("ME_SCALAR_MIN_CTAS", ""))
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    gen_srcs = generate()
    srcs = [os.path.join(CSRC, s) for s in STATIC_SOURCES] + gen_srcs
    objs = [os.path.join(OBJ, os.path.basename(s).replace(".cu", ".o")) for s in srcs]
    # biggest units first so the long pole starts early
    order = sorted(range(len(srcs)), key=lambda i: -os.path.getsize(srcs[i]))
    logs = {}
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_compile, srcs[i], objs[i]) for i in order]
        for f in cf.as_completed(futs):
            src, log = f.result()
            logs[os.path.basename(src)] = log
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for k in sorted(logs):
            f.write(f"== {k}\n{logs[k]}\n")
    if verbose:
        print(open(os.path.join(BUILD, "ptxas.log")).read())
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import time

    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv), f"{time.time() - t:.1f}s")
