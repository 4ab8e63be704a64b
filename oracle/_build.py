"""Build liboracle.so (the CPU oracle) with gcc.

Test infrastructure: only the tests, the smoke check and the CPU-baseline leg of
the benchmark use the library this produces.

The flags matter for the oracle's exactness claims: -ffp-contract=off forbids
fused multiply-add, -fno-fast-math keeps IEEE semantics, and no -march flag is
given, so the same source gives the same results on x86-64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fvisibility=hidden", "-Wall", "-Wextra"]


def _openmp_works() -> bool:
    probe = subprocess.run(["gcc", "-fopenmp", "-x", "c", "-", "-o", os.devnull],
                           input=b"#include <omp.h>\nint main(void){return omp_get_max_threads()<0;}\n",
                           capture_output=True)
    return probe.returncode == 0


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so when missing or older than the source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    flags = list(CFLAGS)
    if _openmp_works():
        flags.append("-fopenmp")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *flags, SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
