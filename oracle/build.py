"""Compile the CPU oracle (plain C, gcc) into oracle/liboracle.so.

The oracle is test infrastructure: it is built next to the CUDA library so
that the test-suite, the smoke check and the benchmark's CPU-baseline leg can
load it, but the library's product path never links or calls it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build_oracle(force=False):
    """Compile liboracle.so if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
