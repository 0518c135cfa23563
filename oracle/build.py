"""Builds the oracle's C part (test infrastructure only) with the host gcc.

``build()`` writes ``oracle/_build/liboracle.so``.  ``build_variant`` compiles
the same source with extra ``-D`` flags into a caller-chosen directory; the
mutation tests use it to plant a mistake in a private copy of the oracle and
check that the pins catch it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build_variant(out_path, defines=()):
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", out_path, SRC]
    cmd[1:1] = ["-D" + d for d in defines]
    subprocess.run(cmd, check=True)
    return out_path


def build(force=False):
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    build_variant(tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
