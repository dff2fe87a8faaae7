"""Compile the CPU oracle (plain C, FP64) into ``oracle/liboracle.so``.

Test infrastructure only: the GPU library never links or loads it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("fmm_oracle.c", "helmholtz_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("fmm_oracle.h", "oracle_tree.h")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its sources."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           *SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
