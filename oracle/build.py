"""Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, no cmake).

TEST INFRASTRUCTURE ONLY: the oracle is built here so the tests, the smoke
check and the CPU-baseline leg of the benchmark can load it.

``-ffp-contract=off`` keeps every double expression rounded step by step (no
fused multiply-add), so the acceptance tables come out the same whatever the
host architecture's default contraction is.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ("philox.c", "embed.c", "anneal.c", "decode.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}.{threading.get_ident()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", tmp]
    cmd += [os.path.join(HERE, s) for s in SOURCES]
    cmd += ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
