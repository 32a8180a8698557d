"""Compile the oracle's C sweep into ``oracle/_oracle_sweep.so`` (test infrastructure)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "oracle_sweep.c")
LIB = os.path.join(HERE, "_oracle_sweep.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    # -ffp-contract=off keeps the same IEEE rounding on x86-64 and aarch64 hosts.
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
