"""Builds the oracle's shared library (plain C, gcc) into oracle/_build/.

TEST INFRASTRUCTURE ONLY: the library built here is loaded by the test suite, the smoke
check and the CPU-baseline leg of the benchmark, never by the product path.
Compiled with -ffp-contract=off so that every product and sum is rounded on its own, the
same way on x86-64 and AArch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
SOURCES = [HERE / "pk_oracle.c"]
OUT = HERE / "_build" / "libpk_oracle.so"


def build(force: bool = False) -> Path:
    OUT.parent.mkdir(exist_ok=True)
    newest = max(s.stat().st_mtime for s in SOURCES)
    if not force and OUT.exists() and OUT.stat().st_mtime >= newest:
        return OUT
    tmp = OUT.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", str(tmp)] + [str(s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
