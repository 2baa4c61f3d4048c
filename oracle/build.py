"""Compile the FP64 CPU oracle (oracle.c) into oracle/liboracle.so.

Test infrastructure only.  OpenMP is used when the compiler supports it; the
oracle's arithmetic is the same either way (threads only split independent
sites and blocks).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", SRC, "-lm"]
    tmp = OUT + ".tmp%d" % os.getpid()
    for extra in (["-fopenmp"], []):
        cmd = base[:2] + extra + base[2:] + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), r.returncode, r.stderr, file=sys.stderr)
        if r.returncode == 0:
            os.replace(tmp, OUT)
            return OUT
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
