"""Compile the CPU oracle (plain C, FP64) into oracle/libns_oracle.so.

Test infrastructure: the oracle is the slow reference the CUDA path is
checked against.  Building it is part of ``__graft_entry__.build()``;
running it is reserved to the tests, the smoke check and the benchmark's
CPU-baseline leg.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ns_oracle.c")
LIB = os.path.join(HERE, "libns_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(HERE, "ns_oracle.h"))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
