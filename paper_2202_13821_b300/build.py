"""Build libdghgks.so (CUDA, sm_103a) in-tree with nvcc."""
from __future__ import annotations

import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libdghgks.so")
SOURCES = [os.path.join(HERE, "csrc", "dghgks_api.cu"), os.path.join(HERE, "csrc", "dghgks_static.cu"),
           os.path.join(HERE, "csrc", "dghgks_adjoint.cu"), os.path.join(HERE, "csrc", "dghgks_peaks.cu")]
# extra device-compiler options per source (see the header of dghgks_adjoint.cu)
EXTRA = {"dghgks_adjoint.cu": ["-Xptxas", "-O1"]}
DEPS = [os.path.abspath(__file__)] + SOURCES + [os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc")) if f.endswith((".cu", ".cuh"))] + [
    os.path.join(ROOT, "include", "dghgks.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


OPCOUNT_JSON = os.path.join(HERE, "opcount.json")


def build_opcount(force: bool = False) -> str:
    """Compile and run the host operation counter; writes opcount.json."""
    src = os.path.join(HERE, "csrc", "opcount.cpp")
    deps = [src, os.path.join(HERE, "csrc", "gks_point.cuh")]
    if not force and os.path.exists(OPCOUNT_JSON) and os.path.getmtime(OPCOUNT_JSON) >= max(map(os.path.getmtime, deps)):
        return OPCOUNT_JSON
    exe = os.path.join(HERE, "opcount.bin")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "include")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wno-unknown-pragmas", "-I", cuda_inc, "-I", "/usr/local/cuda/include",
                    "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = [json.loads(l) for l in out.splitlines() if l.strip()]
    with open(OPCOUNT_JSON + ".tmp", "w") as f:
        json.dump(rows, f, indent=1)
    os.replace(OPCOUNT_JSON + ".tmp", OPCOUNT_JSON)
    os.remove(exe)
    return OPCOUNT_JSON


def opcounts(order: int, n_q: int, pr_fix: bool) -> dict:
    build_opcount()
    for r in json.load(open(OPCOUNT_JSON)):
        if r["order"] == order and r["n_q"] == n_q and r["pr_fix"] == pr_fix:
            return r
    raise KeyError((order, n_q, pr_fix))


def build(force: bool = False, verbose: bool = False) -> str:
    build_opcount(force)
    newest = max(os.path.getmtime(f) for f in DEPS if os.path.exists(f))
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = [f for f in NVCC_FLAGS if f != "-shared"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc(), *flags, *EXTRA.get(os.path.basename(src), []), "-I", os.path.join(ROOT, "include"), "-c",
               "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    for pr in procs:
        if pr.wait() != 0:
            raise subprocess.CalledProcessError(pr.returncode, "nvcc")
    link = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC", "-o", SO + ".tmp",
            *objs, "-lcudart"]
    subprocess.run(link, check=True)
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(SO)
