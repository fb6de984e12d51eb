"""Builds the oracle's shared libraries (plain C, gcc) into oracle/_build/.

TEST INFRASTRUCTURE ONLY: the libraries built here are loaded by the test suite, the smoke
check and the CPU-baseline leg of the benchmark, never by the product path.
Compiled with -ffp-contract=off so that every product and sum is rounded on its own, the
same way on x86-64 and AArch64 hosts.

libpk_oracle.so is the sequential parity oracle.  libpk_oracle_omp.so is the OpenMP timing
copy of its pipelined CG (the CPU baseline's multi-threaded leg); it is built separately so
that a compiler without OpenMP leaves the parity oracle untouched.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
SOURCES = [HERE / "pk_oracle.c"]
OUT = HERE / "_build" / "libpk_oracle.so"
OMP_SOURCES = [HERE / "pk_oracle_omp.c"]
OMP_OUT = HERE / "_build" / "libpk_oracle_omp.so"
FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall"]


def _compile(sources, out: Path, extra, force: bool) -> Path:
    out.parent.mkdir(exist_ok=True)
    newest = max(s.stat().st_mtime for s in sources + [Path(__file__)])
    if not force and out.exists() and out.stat().st_mtime >= newest:
        return out
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc"] + FLAGS + extra + ["-o", str(tmp)] + [str(s) for s in sources] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> Path:
    out = _compile(SOURCES, OUT, [], force)
    try:
        build_omp(force)
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP: the CPU baseline reports its single-threaded leg only
    return out


def build_omp(force: bool = False) -> Path:
    return _compile(OMP_SOURCES, OMP_OUT, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_omp(force=True))
