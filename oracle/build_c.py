"""Compiles the oracle's plain-C helpers with gcc into oracle/_liboracle.so.
Portable flags only (the same source builds on x86_64 and aarch64)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "c", "oracle_dirac.c")]
OUT = os.path.join(HERE, "_liboracle.so")


def build_oracle_c(force: bool = False) -> str:
    newest = max(os.path.getmtime(s) for s in SRC)
    if force or not os.path.exists(OUT) or os.path.getmtime(OUT) < newest:
        tmp = OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c99", "-fcx-limited-range", "-fPIC", "-shared", "-o", tmp] + SRC + ["-lm", "-lpthread"])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build_oracle_c(force=True))
