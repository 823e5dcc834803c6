"""Build the C part of the oracle (liboracle.so) with gcc.

Test infrastructure only: the oracle is the independent CPU reference that the
test-suite, the smoke check and the CPU-baseline leg of bench.py compare the
CUDA library with.  It is never linked into, or called by, the library.

-ffp-contract=off keeps the delay-table arithmetic free of fused multiply-adds
on every host (gcc contracts by default on aarch64), so the table is the same
IEEE double computation on x86_64 and on Arm.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


# -O3 lets gcc vectorise the plain inner loops (the time loop of the
# dedispersion sum); no fast-math, so every floating-point result keeps its
# IEEE meaning.
CFLAGS = ["-O3", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared"]


def build_oracle(force: bool = False) -> str:
    newest = max(os.path.getmtime(SRC), os.path.getmtime(os.path.abspath(__file__)))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc"] + CFLAGS + [SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
