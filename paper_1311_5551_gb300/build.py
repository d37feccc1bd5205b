"""Build the CUDA library in-tree: nvcc for sm_103a (``-gencode arch=compute_103a,code=sm_103a``),
g++ for the host table builder, translation units compiled in parallel, one shared object."""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libqedmc.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return sorted(hs + [os.path.join(INCLUDE, "qed.h")])


def extra_defines() -> list[str]:
    """Launch-shape tunables of the step kernel for sweeps, e.g. QED_NVCC_DEFINES="-DQED_STAGES=4"
    (only -D flags are taken; the defaults are the measured best)."""
    return [f for f in os.environ.get("QED_NVCC_DEFINES", "").split() if f.startswith("-D")]


def _digest():
    h = hashlib.sha256()
    for p in _sources() + _headers() + [os.path.abspath(__file__)]:
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    h.update(" ".join(extra_defines()).encode())
    return h.hexdigest()[:16]


def lib_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "stamp")
    dig = _digest()
    if not force and os.path.exists(lib_path()) and os.path.exists(stamp) and open(stamp).read() == dig:
        return lib_path()
    nvcc = os.environ.get("NVCC", "nvcc")
    objs, cmds = [], []
    units = []
    for src in _sources():
        if os.path.basename(src) == "qed_kernels.cu":
            # three parts compiled in parallel (see QED_KERNELS_PART in the file)
            units += [(src, [f"-DQED_KERNELS_PART={k}"], f".{k}") for k in (1, 2, 3)]
        else:
            units.append((src, [], ""))
    for src, part, tag in units:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + tag + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            # --fmad=false: no implicit multiply-add contraction, so the step computes the same
            # bits in every kernel that inlines it (single scenario, batch, diagnostics); the hot
            # expressions use explicit fma() instead
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler",
                   "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
            if os.environ.get("QED_PTXAS_VERBOSE"):
                cmd.insert(1, "-Xptxas=-v")
            cmd[1:1] = extra_defines() + part
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-pthread",
                   "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        cmds.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for cmd, r in ex.map(run, cmds):
            if verbose or r.returncode != 0 or os.environ.get("QED_PTXAS_VERBOSE"):
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"compilation failed: {cmd[-3]}")
    tmp = lib_path() + f".{os.getpid()}.tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, lib_path())
    with open(stamp, "w") as f:
        f.write(dig)
    return lib_path()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
