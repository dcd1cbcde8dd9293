"""Compile the CPU oracle (oracle/ctqr_oracle.c) into oracle/libctqr_oracle.so.

Test infrastructure only.  -ffp-contract=off keeps every multiply and add a
separately rounded IEEE double operation (no FMA contraction), which the
bit-exact Siddon comparison relies on.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ctqr_oracle.c")
LIB = os.path.join(HERE, "libctqr_oracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into the shared library `out`."""
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    return compile_source(SRC, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
