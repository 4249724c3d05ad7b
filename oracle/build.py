"""Compile the C oracle into oracle/_build/libtinylu_oracle.so.

TEST INFRASTRUCTURE ONLY: building the checker is not using it.  The flags
fix the arithmetic: -ffp-contract=off (every fused multiply-add in the
oracle is an explicit fma() call), no fast-math, portable (no -march).
OpenMP is used only to run independent systems on several host cores.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tinylu_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtinylu_oracle.so")

BASE_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False, extra_flags=(), out=None, quiet=True) -> str:
    """Build the oracle shared library (with OpenMP when gcc supports it).

    Returns the path of the library.  `extra_flags` and `out` let tests build
    variants (e.g. with a planted mistake) next to the real one.
    """
    out = out or LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC) and not extra_flags:
        return out
    cc = os.environ.get("CC", "gcc")
    tmp = out + f".tmp{os.getpid()}"
    for omp in (["-fopenmp"], []):
        cmd = [cc, *BASE_FLAGS, *omp, *extra_flags, SRC, "-o", tmp, "-lm"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode == 0:
            os.replace(tmp, out)
            return out
        if not quiet:
            sys.stderr.write(res.stderr)
    raise RuntimeError(f"oracle build failed:\n{' '.join(cmd)}\n{res.stderr}")


if __name__ == "__main__":
    print(build(force=True, quiet=False))
