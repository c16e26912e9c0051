"""Builds the oracle's C library (TEST INFRASTRUCTURE).

Plain gcc, no CUDA; the GPU library is built separately and shares nothing
with this one.
"""

from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "rpq_oracle.c")
OUT = os.path.join(_HERE, "librpq_oracle.so")


def build_library(force: bool = False) -> str:
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(SRC)):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
           "-fvisibility=hidden", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build_library(force=True))
