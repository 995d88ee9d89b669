"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liblbm_oracle.so.

Plain gcc, strict IEEE double arithmetic (no FMA contraction, no fast-math) so
that the oracle gives the same numbers on x86-64 and AArch64 hosts.  OpenMP
(when the compiler has it) spreads each pass's cell loop over threads; no pass
reduces across cells, so the numbers do not depend on the thread count.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
    r = subprocess.run(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:   # a compiler without OpenMP: plain serial loops
        subprocess.check_call(base + [SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
