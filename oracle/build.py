"""Build the plain-C oracle into a shared library next to this file.

Test infrastructure only: the oracle may be built, loaded and run by the
test-suite, the smoke check and the CPU-baseline leg of the benchmark, and by
nothing in the product path.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hetal_oracle.c")
LIB = os.path.join(HERE, "_hetal_oracle.so")


def build(force: bool = False) -> str:
    """Compile hetal_oracle.c with gcc (-O2, POSIX threads, no target-specific flags) if stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-pthread", "-fPIC", "-shared", "-Wall", "-Wno-unused-function", "-Wno-maybe-uninitialized",
           SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
