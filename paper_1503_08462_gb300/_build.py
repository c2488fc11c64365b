"""In-tree native builds: the host AMG setup library and the CUDA solve library.

Both are compiled from source on the machine that runs them (x86 here, Arm on
the GPU host) and written next to the package sources; nothing is installed.
"""
from __future__ import annotations

import fcntl
import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
REPO = PKG.parent
SETUP_SRC = PKG / "inputs" / "csrc" / "amg_setup.cpp"
SETUP_LIB = PKG / "inputs" / "libamgsetup.so"
CUDA_DIR = PKG / "csrc"
CUDA_LIB = PKG / "libamgeig.so"
INCLUDE = REPO / "include"

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _locked(fn):
    def wrapper(*args, **kwargs):
        lock = PKG / ".build.lock"
        with open(lock, "w") as fh:
            fcntl.flock(fh, fcntl.LOCK_EX)
            try:
                return fn(*args, **kwargs)
            finally:
                fcntl.flock(fh, fcntl.LOCK_UN)
    return wrapper


@_locked
def build_setup_lib(force: bool = False) -> Path:
    """Compile the host AMG setup library with g++ (portable C++17)."""
    if force or _stale(SETUP_LIB, [SETUP_SRC]):
        tmp = SETUP_LIB.with_suffix(".so.tmp")
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", str(tmp), str(SETUP_SRC)],
                       check=True)
        os.replace(tmp, SETUP_LIB)
    return SETUP_LIB


def cuda_sources():
    # the CUDA translation units, and the host setup library's C/F splitting (used by the device setup)
    return sorted(CUDA_DIR.glob("*.cu")) + [SETUP_SRC]


def cuda_headers():
    return sorted(CUDA_DIR.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


@_locked
def build_cuda_lib(force: bool = False, jobs: int | None = None) -> Path:
    """Compile every CUDA translation unit for sm_103a and link libamgeig.so."""
    srcs = cuda_sources()
    deps = srcs + cuda_headers()
    if not (force or _stale(CUDA_LIB, deps)):
        return CUDA_LIB
    objdir = PKG / "_build"
    objdir.mkdir(exist_ok=True)
    flags = NVCC_ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE),
                         "-I", str(CUDA_DIR), "--expt-relaxed-constexpr"]
    procs = []
    objs = []
    for s in srcs:
        o = objdir / (s.stem + ".o")
        objs.append(o)
        if s.suffix == ".cpp":
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", str(s), "-o", str(o)]
        else:
            cmd = ["nvcc", *flags, "-c", str(s), "-o", str(o)]
        procs.append(subprocess.Popen(cmd))
        if jobs and len([p for p in procs if p.poll() is None]) >= jobs:
            procs[0].wait()
    rc = [p.wait() for p in procs]
    if any(rc):
        raise RuntimeError(f"nvcc failed for {[str(s) for s, r in zip(srcs, rc) if r]}")
    tmp = CUDA_LIB.with_suffix(".so.tmp")
    subprocess.run(["nvcc", *NVCC_ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"], check=True)
    os.replace(tmp, CUDA_LIB)
    return CUDA_LIB
