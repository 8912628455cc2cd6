"""Compile the FP64 CPU oracle (plain C, gcc) into oracle/_build/liboracle.so.

Test infrastructure: building the checker is not using it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = [os.path.join(HERE, "pin_oracle.c")]
HDR = [os.path.join(HERE, "pin_oracle.h")]


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SRC + HDR)


def command():
    return ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-o", LIB] + SRC + ["-lm"]


def build(force=False):
    """Returns a started Popen (or None when up to date)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and not needs_build():
        return None
    return subprocess.Popen(command(), stdout=subprocess.PIPE, stderr=subprocess.STDOUT)


if __name__ == "__main__":
    p = build(force=True)
    if p is not None:
        out, _ = p.communicate()
        print(out.decode())
        raise SystemExit(p.returncode)
