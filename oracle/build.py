"""Build the plain FP64 CPU oracle (test infrastructure) as oracle/liboracle.so.

Compiled with gcc, OpenMP over spatial cells, no fast-math and no FMA contraction, so that
results do not depend on the host architecture's contraction rules.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, "mm_oracle.c"), os.path.join(HERE, "mm_oracle1d.c")]
    hdr = os.path.join(HERE, "mm_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in srcs + [hdr])):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
