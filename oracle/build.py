"""Build the oracle's plain-C direct sum (test infrastructure only).

``build()`` compiles ``direct_sum.c`` with gcc into ``oracle/_build/`` and
returns the path of the shared object.  No product code links it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SO_PATH = os.path.join(BUILD_DIR, "liboracle_direct.so")
SRC = os.path.join(HERE, "direct_sum.c")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(SO_PATH)
            and os.path.getmtime(SO_PATH) >= os.path.getmtime(SRC)):
        return SO_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = SO_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, SO_PATH)
    return SO_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
