"""Compile the CPU oracle (test infrastructure) into oracle/lib/liboracle.so.

Two builds of one source: ``REAL = double`` (the oracle) and ``REAL = long
double`` (a higher-precision copy used only to bound the double build's
rounding error).  No fused multiply-add contraction and no fast-math, so the
oracle's arithmetic is the source's arithmetic, in source order.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hawkes_oracle.c")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "liboracle.so")

CFLAGS = ["-O2", "-fPIC", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11"]


def compile_oracle(src=SRC, out=LIB, extra=()):
    """Compile ``src`` (both REAL builds) into the shared library ``out``."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    objs = []
    for tag, defs in (("f64", []), ("ld", ["-DORACLE_LONG"])):
        obj = out + "." + tag + ".o"
        subprocess.check_call(["gcc", *CFLAGS, *defs, *extra, "-c", src, "-o", obj])
        objs.append(obj)
    subprocess.check_call(["gcc", "-shared", "-fopenmp", "-o", out, *objs, "-lm"])
    for o in objs:
        os.remove(o)
    return out


def build(force=False):
    """Build liboracle.so unless it is newer than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    return compile_oracle()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
