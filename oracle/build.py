"""Builds the oracle's shared library with the host C compiler.

Test infrastructure: compiled by ``__graft_entry__.build()`` so that the checker
exists on every machine; nothing in the product path links or loads it.
``-ffp-contract=off`` keeps every product and sum separately rounded on x86
and Arm alike (GCC contracts to FMA by default on aarch64).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "tetm_oracle.c"), os.path.join(HERE, "tetm_rz_oracle.c")]
BUILD_DIR = os.path.join(HERE, "_build")


def library_path():
    return os.path.join(BUILD_DIR, "liboracle.so")


def build_oracle(verbose=False):
    os.makedirs(BUILD_DIR, exist_ok=True)
    out = library_path()
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + SRCS + ["-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(verbose=True))
