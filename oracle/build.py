"""Compile the CPU oracle (plain C, gcc) into oracle/libea_oracle.so.

Test infrastructure: the oracle is only loaded by the tests, the smoke check and
the CPU-baseline leg of the benchmark.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ea_oracle.c")
LIB = os.path.join(HERE, "libea_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # -ffp-contract=off keeps exp/ldexp/floor of the thresholds free of fused
    # operations; the arithmetic is otherwise integer.
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
