"""Build the oracle's shared library with gcc (FP64, FMA contraction off).

The oracle is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg load it.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
SRC = HERE / "mss_oracle.c"
OUT_DIR = HERE / "_build"
LIB = OUT_DIR / "libmss_oracle.so"

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-Wall", "-Wno-unused-function"]


def build_oracle(force: bool = False) -> Path:
    """Compile ``mss_oracle.c`` into ``_build/libmss_oracle.so`` if stale."""
    OUT_DIR.mkdir(exist_ok=True)
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = OUT_DIR / f"libmss_oracle.{os.getpid()}.so"
    cmd = ["gcc", *CFLAGS, str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
