"""Compile the CPU oracle (test infrastructure only) into shared libraries.

Two builds of the same source: libhamr_oracle.so (double) and
libhamr_oracle_count.so (the flop-counting scalar type). Plain g++, no
architecture-specific flags, so the same source builds on x86_64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hamr_oracle.cpp")
FLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17", "-Wall"]


def _build_one(out, extra):
    cmd = ["g++", *FLAGS, *extra, SRC, "-o", out]
    subprocess.check_call(cmd, cwd=HERE)


def build(force=False):
    targets = [(os.path.join(HERE, "libhamr_oracle.so"), []),
               (os.path.join(HERE, "libhamr_oracle_count.so"), ["-DORA_COUNT_FLOPS"])]
    deps = [SRC, os.path.join(HERE, "hamr_oracle.h"), os.path.join(HERE, "ora_real.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    for out, extra in targets:
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            _build_one(out, extra)
    return [t[0] for t in targets]


if __name__ == "__main__":
    build(force="--force" in sys.argv)
