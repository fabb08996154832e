"""Build the C part of the oracle (plain gcc, OpenMP) in place.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library; nothing on the
product path may load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ewald_ref.c")
LIB = os.path.join(HERE, "libibpme_oracle.so")


def build(force: bool = False) -> str:
    """Compile ewald_ref.c into libibpme_oracle.so (portable flags only)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
