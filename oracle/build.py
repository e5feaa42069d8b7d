"""Builds the CPU oracle (test infrastructure) from ``awo_oracle.c``.

Two shared objects come from the one source: ``liboracle_f32.so`` (FP32, the
parity oracle) and ``liboracle_f64.so`` (FP64, for closed-form pins).  Both are
compiled with ``-ffp-contract=off`` so that no multiply-add is fused: every
arithmetic operation in the oracle is one IEEE-754 rounding in the order the
source writes it.  Plain gcc, no architecture flags, so the same results come
out on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "awo_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")

FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
         "-fno-strict-aliasing", "-Wall", "-Wno-unused-function"]


def lib_path(precision: str) -> str:
    if precision not in ("f32", "f64"):
        raise ValueError(precision)
    return os.path.join(OUT_DIR, f"liboracle_{precision}.so")


def build(force: bool = False) -> list[str]:
    os.makedirs(OUT_DIR, exist_ok=True)
    outs = []
    procs = []
    for prec, real in (("f32", "float"), ("f64", "double")):
        out = lib_path(prec)
        outs.append(out)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", *FLAGS, f"-DORC_REAL={real}", "-o", tmp, SRC, "-lm"]
        procs.append((subprocess.Popen(cmd), tmp, out, cmd))
    for p, tmp, out, cmd in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed: " + " ".join(cmd))
        os.replace(tmp, out)
    return outs


if __name__ == "__main__":
    for o in build(force="--force" in sys.argv):
        print(o)
