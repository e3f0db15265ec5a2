"""Compile the C oracle into ``oracle/liboracle.so`` with plain gcc.

Test infrastructure: the oracle is a checker, built beside the product but
never linked into it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmv_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    # OpenMP only spreads the rows of the timing-only parallel product over
    # the host cores; without it that product runs on one thread
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
