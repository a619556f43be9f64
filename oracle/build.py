"""Compile the oracle's plain C source into ``oracle/_build/liborc.so`` with gcc.

Test infrastructure only (see ``oracle/__init__.py``).  Flags keep the
arithmetic identical on x86-64 and aarch64 hosts: no ``-march``, no fast-math,
and ``-ffp-contract=off`` so that no multiply-add is fused unless the source
calls ``fma`` itself.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rmge_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into the shared library `out`, with the flags above."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
