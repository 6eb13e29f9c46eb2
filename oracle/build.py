"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qds_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_EXT = os.path.join(HERE, "liboracle_ext.so")  # long double build


def _build_one(lib, extra, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", *extra,
           "-o", lib + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


def build(force: bool = False, extended: bool = False) -> str:
    if extended:
        return _build_one(LIB_EXT, ["-DORA_EXTENDED"], force)
    return _build_one(LIB, [], force)


def build_all(force: bool = False):
    build(force)
    build(force, extended=True)


if __name__ == "__main__":
    build_all(force=True)
    print(LIB, LIB_EXT)
