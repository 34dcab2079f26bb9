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


def build_variant(outdir: str, replace) -> str:
    """Build a copy of the oracle in outdir with textual edits applied to its sources (used by
    tests that plant a mistake in the oracle and check that a pin catches it).  replace maps a
    source file name to a list of (old, new) pairs; each old must occur exactly once."""
    os.makedirs(outdir, exist_ok=True)
    srcs = []
    for name in ("mm_oracle.c", "mm_oracle1d.c", "mm_oracle.h"):
        with open(os.path.join(HERE, name)) as f:
            text = f.read()
        for old, new in replace.get(name, []):
            if text.count(old) != 1:
                raise ValueError("edit %r matches %d times in %s" % (old, text.count(old), name))
            text = text.replace(old, new)
        dst = os.path.join(outdir, name)
        with open(dst, "w") as f:
            f.write(text)
        if name.endswith(".c"):
            srcs.append(dst)
    out = os.path.join(outdir, "liboracle_variant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-o", out] + srcs + ["-lm"])
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
