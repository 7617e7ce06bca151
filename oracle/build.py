"""Build the CPU oracle library (plain C, no CUDA).

Test infrastructure: compiles ``ds_oracle.c`` into ``libds_oracle.so`` beside
it with ``-O2 -ffp-contract=off`` so that every float/double operation is a
single IEEE-754 round-to-nearest operation on both x86-64 and aarch64 (GCC
contracts a*b+c into an FMA by default on aarch64, which would change the
rounding the oracle is meant to pin).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ds_oracle.c")
LIB = os.path.join(HERE, "libds_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
