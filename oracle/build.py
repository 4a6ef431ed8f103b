"""Compiles the C oracle (ntt_oracle.c, plus the O(N log N) CPU baseline
ntt_radix2.c) into oracle/_build/liboracle.so.

Test infrastructure only (see oracle/__init__.py).  Plain gcc, no CUDA, so the
same source gives the same results on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "ntt_oracle.c"), os.path.join(HERE, "ntt_radix2.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Builds the oracle library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           "-Wall", "-Wextra", "-o", tmp] + SRCS
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
