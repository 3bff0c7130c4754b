"""Builds libpt.so (CUDA, sm_103a) in-tree: paper_2211_05458_gb300/_build/libpt.so.

Every .cu under csrc/ is compiled by nvcc in parallel and linked into one
shared library with the C ABI of include/pt.h.  Run ``python -m
paper_2211_05458_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libpt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
# extra nvcc flags for tuning builds, e.g. PT_NVCC_EXTRA="-DPT_PUSH_MINB=4"
FLAGS += os.environ.get("PT_NVCC_EXTRA", "").split()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libpt cannot be built")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  [os.path.join(ROOT, "include", "pt.h")])


def _digest(path, hdr_digest):
    h = hashlib.sha256(hdr_digest.encode())
    with open(path, "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hh = hashlib.sha256()
    for p in _headers():
        with open(p, "rb") as f:
            hh.update(f.read())
    hdr = hh.hexdigest()
    objs, todo = [], []
    for src in _sources():
        name = os.path.splitext(os.path.basename(src))[0]
        obj = os.path.join(BUILD, f"{name}.{_digest(src, hdr)}.o")
        objs.append(obj)
        if force or not os.path.exists(obj):
            todo.append((src, obj))

    def compile_one(item):
        src, obj = item
        tmp = obj + f".{os.getpid()}.tmp.o"
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr[-4000:]}")
        os.replace(tmp, obj)
        return src

    if todo:
        jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(jobs) as ex:
            for src in ex.map(compile_one, todo):
                if verbose:
                    print("compiled", os.path.basename(src), file=sys.stderr)
    stamp = os.path.join(BUILD, "libpt.objs")
    want = "\n".join(objs)
    have = open(stamp).read() if os.path.exists(stamp) else ""
    if todo or have != want or not os.path.exists(SO):
        tmp = SO + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, SO)
        with open(stamp, "w") as f:
            f.write(want)
    # drop stale objects
    keep = set(objs)
    for o in glob.glob(os.path.join(BUILD, "*.o")):
        if o not in keep:
            try:
                os.remove(o)
            except OSError:
                pass
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
