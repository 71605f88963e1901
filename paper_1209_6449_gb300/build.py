"""Build the sm_103a CUDA library in-tree: paper_1209_6449_gb300/lib/libepsm.so."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB_DIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIB_DIR, "libepsm.so")
# a test build whose single-search filters pass every start (verification alone decides)
LIB_SOUND = os.path.join(LIB_DIR, "libepsm_sound.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh", ".inc")))


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, soundness: bool = False) -> str:
    lib = LIB_SOUND if soundness else LIB
    if not force and not needs_build(lib):
        return lib
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", f"-I{INCLUDE}",
           "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-pthread",
           "-o", tmp, os.path.join(CSRC, "epsm.cu")]
    if soundness:
        cmd.insert(1, "-DEPSM_FILTER_SOUNDNESS=1")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                soundness="--soundness" in sys.argv))
