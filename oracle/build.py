"""Build step for the CPU oracle (test infrastructure): plain gcc, OpenMP.

``-ffp-contract=off`` keeps gcc from fusing multiply-adds on aarch64 so the
oracle rounds the same way on x86_64 and on Arm hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bsolve_oracle.c")


def lib_path() -> str:
    return os.path.join(HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
