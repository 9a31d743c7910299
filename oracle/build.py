"""Compile the C oracle into a shared library under oracle/_build/.

TEST INFRASTRUCTURE ONLY. Plain gcc, no fast-math and no FMA contraction, so
the oracle computes the same bits on x86_64 and aarch64.
"""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
FLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-fno-fast-math",
         "-Wall", "-Wno-unused-function"]


def _sources():
    return sorted(glob.glob(os.path.join(HERE, "*.c")) + glob.glob(os.path.join(HERE, "*.h")))


def build(force: bool = False) -> str:
    srcs = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *FLAGS, "-o", tmp, *[s for s in srcs if s.endswith(".c")], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
