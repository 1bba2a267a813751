"""Compile the C oracle into ``oracle/liboracle.so`` (gcc, C11, OpenMP)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def compile_shared(src: str, out: str) -> str:
    """gcc a C oracle source (its header beside it) into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "gsicp_oracle.c")
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "gsicp_oracle.h"))):
        return out
    return compile_shared(src, out)


if __name__ == "__main__":
    print(build(force=True))
