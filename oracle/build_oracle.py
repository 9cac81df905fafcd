"""Compile the FP64 CPU oracle into a shared library beside its source.

Test infrastructure: the oracle is built on whichever machine runs the tests
(x86_64 here, aarch64 on a GPU host), with plain gcc and no machine-specific
flags, so its results do not depend on the host's vector units.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hubbard_oracle.c")
LIB = os.path.join(HERE, "libhubbard_oracle.so")


def build(force: bool = False) -> str:
    """Build ``libhubbard_oracle.so`` if it is missing or older than its source."""
    hdr = os.path.join(HERE, "hubbard_oracle.h")
    newest = max(os.path.getmtime(SRC), os.path.getmtime(hdr))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
