"""In-tree build of the CUDA library (libcore_als.so) for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libcore_als.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def _sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + [INCLUDE / "core_als.h"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcore_als.so")
    return exe


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile each csrc/*.cu in parallel and link one shared library, unless
    the library is newer than every source."""
    OUT_DIR.mkdir(parents=True, exist_ok=True)
    if LIB.exists() and not force:
        newest = max(p.stat().st_mtime for p in _sources())
        if LIB.stat().st_mtime >= newest:
            return LIB
    tus = sorted(CSRC.glob("*.cu"))
    compile_flags = [f for f in FLAGS if f != "-shared"]
    procs = []
    for tu in tus:
        obj = OUT_DIR / (tu.stem + ".o")
        cmd = [nvcc(), *ARCH, *compile_flags, "-I", str(INCLUDE), "-I", str(CSRC), "-c", str(tu), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((tu, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    objs = []
    for tu, obj, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"nvcc failed on {tu.name}:\n" + out + err)
        if verbose:
            print(err)
        objs.append(str(obj))
    tmp = str(LIB) + ".tmp"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
