"""Build liboracle.so (plain C, gcc) next to this file.

Test infrastructure only: the oracle is loaded by tests/, by
__graft_entry__.smoke() and by bench.py's CPU-baseline / reference arm.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c")]
HEADERS = [os.path.join(HERE, "heart_oracle.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SOURCES + HEADERS)


def build(force=False):
    """Compile the oracle (FP contraction off so x86 and Arm give the same bits)."""
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wno-unused-function", "-o", tmp] + SOURCES + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
