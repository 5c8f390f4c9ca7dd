"""Build libmss.so (CUDA, sm_103a) in-tree with nvcc.

Every translation unit is compiled in parallel; the two set-up units whose
floating point feeds index decisions (scaling, AMG set-up) are compiled with
FMA contraction disabled. The result is cached on a hash of the sources and
flags.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "libmss.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]
NO_FMA = {"setup_scale.cu", "amg_setup.cu"}
SOURCES = ["util.cu", "setup_scale.cu", "amg_setup.cu", "amg_cycle.cu", "bilu.cu", "spmv.cu", "krylov.cu",
           "residual.cu", "noalloc.cu", "condense.cu", "api.cu", "batch.cu", "fused.cu", "gnn.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmss")


def _digest(extra: list[str]) -> str:
    h = hashlib.sha256()
    for f in sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + [INCLUDE / "mss.h"]):
        h.update(f.name.encode())
        h.update(f.read_bytes())
    h.update(" ".join(ARCH + COMMON + extra).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    """Compile and link libmss.so next to this file; returns its path."""
    extra = list(extra or [])
    BUILD.mkdir(exist_ok=True)
    stamp = BUILD / "stamp"
    digest = _digest(extra)
    if not force and LIB.exists() and stamp.exists() and stamp.read_text() == digest:
        return LIB
    nvcc = _nvcc()

    def compile_one(src: str) -> Path:
        obj = BUILD / (src + ".o")
        flags = ARCH + COMMON + extra + (["-fmad=false"] if src in NO_FMA else [])
        cmd = [nvcc, *flags, "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return obj

    workers = min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = PKG / f"libmss.{os.getpid()}.so"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *map(str, objs), "-o", str(tmp)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    stamp.write_text(digest)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
