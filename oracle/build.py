"""Compile the CPU oracle (oracle/ckks_oracle.c) into oracle/libckks_oracle.so.

Test infrastructure: the oracle is the checker for the CUDA library, never part of its path.
Plain gcc, -O2, OpenMP when the compiler has it; no architecture-specific flags, so the
same source builds on x86-64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ckks_oracle.c")
LIB = os.path.join(HERE, "libckks_oracle.so")


def _compile(flags):
    cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", *flags, SRC, "-o", LIB, "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force=False):
    """Build the oracle library if it is missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    r = _compile(["-fopenmp"])
    if r.returncode != 0:
        sys.stderr.write("oracle: building without OpenMP:\n" + r.stderr[-2000:])
        r = _compile([])
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
