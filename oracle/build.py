"""Compile the C oracle into a shared library next to its source.

Test infrastructure only: the oracle checks the CUDA path and is never part of
it.  Plain ``gcc -O2``, no architecture flags, so the same source builds on the
x86 build host and on an Arm GPU host.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sgagg_oracle.c")
LIB = os.path.join(HERE, "libsgagg_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-Wall", "-Wextra", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
