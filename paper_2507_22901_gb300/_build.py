"""Build libcvsearch.so in-tree for sm_103a (nvcc + g++, no cmake).

The library is written to paper_2507_22901_gb300/_build/libcvsearch.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG / "_build"
LIB = BUILD / "libcvsearch.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> Path:
    env = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if env:
        return Path(env)
    nvcc = shutil.which("nvcc")
    if nvcc:
        return Path(nvcc).resolve().parent.parent
    return Path("/usr/local/cuda")


def _sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cpp"))


def _deps():
    return _sources() + sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh")) + \
        sorted(INCLUDE.glob("*.h")) + [Path(__file__)]


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile every translation unit (in parallel) and link libcvsearch.so."""
    if not force and up_to_date():
        return LIB
    BUILD.mkdir(exist_ok=True)
    cuda = _cuda_home()
    nvcc = str(cuda / "bin" / "nvcc")
    objs, procs = [], []
    for src in _sources():
        obj = BUILD / (src.stem + ".o")
        objs.append(obj)
        if src.suffix == ".cu":
            extra = os.environ.get("CVS_NVCC_FLAGS", "").split()
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-v" if verbose else "-O3", "-I", str(INCLUDE), *extra, "-c",
                   str(src), "-o", str(obj)]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", str(cuda / "include"),
                   "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + out.decode())
        if verbose and out:
            print(out.decode())
    tmp = BUILD / f"libcvsearch.{os.getpid()}.tmp.so"
    link = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout.decode())
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
