"""In-tree build of the native libraries.

  _build/libpin.so     CUDA path for sm_103a (nvcc), C-ABI in include/pin.h
  _build/libpin_ic.so  seeded input generator (gcc), C-ABI in include/pin_ic.h

Both are compiled in parallel; nothing is installed outside the tree.
"""
import glob
import os
import shlex
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIBPIN = os.path.join(OUT_DIR, "libpin.so")
LIBIC = os.path.join(OUT_DIR, "libpin_ic.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources_pin():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")))


def _deps_pin():
    return (_sources_pin() + glob.glob(os.path.join(PKG, "csrc", "*.cuh"))
            + glob.glob(os.path.join(PKG, "csrc", "*.h")) + [os.path.join(INC, "pin.h")]
            + [IC_SRC, os.path.join(INC, "pin_ic.h")])


IC_SRC = os.path.join(PKG, "ic", "pin_ic.c")
IC_OBJ = os.path.join(OUT_DIR, "pin_ic_in_libpin.o")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


OBJ_DIR = os.path.join(OUT_DIR, "obj")


def cmd_pin(extra=()):
    """libpin links the seeded generator's host part (amplitude, key) for
    pin_set_ic_seed: pin_ic.c compiled by gcc with the flags of libpin_ic, and
    each CUDA source compiled by nvcc, all at once (one process each), then
    linked into the shared library."""
    ic = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-ffp-contract=off", "-I", INC,
          "-c", "-o", IC_OBJ, IC_SRC]
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Werror", "cross-execution-space-call",
                    "-Xcompiler", "-fPIC", "-I", INC, "-I", os.path.join(PKG, "csrc")] + list(extra)
    objs, steps = [], [shlex.join(ic) + " & pids=$!"]
    for src in _sources_pin():
        obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        steps.append(shlex.join([NVCC] + flags + ["-c", "-o", obj, src]) + ' & pids="$pids $!"')
    link = [NVCC] + ARCH + ["-shared", "-o", LIBPIN] + objs + [IC_OBJ, "-lm"]
    script = ["set -e", "mkdir -p " + shlex.quote(OBJ_DIR)] + steps + \
        ["for p in $pids; do wait $p; done", shlex.join(link)]
    return ["sh", "-c", "\n".join(script)]


def cmd_ic():
    src = os.path.join(PKG, "ic", "pin_ic.c")
    return ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-I", INC, "-o", LIBIC, src, "-lm"]


def _run(procs):
    errs = []
    for name, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append("%s build failed:\n%s" % (name, out.decode(errors="replace")))
    if errs:
        raise RuntimeError("\n".join(errs))


def start(force=False, which=("pin", "ic")):
    os.makedirs(OUT_DIR, exist_ok=True)
    procs = []
    if "ic" in which and (force or _stale(LIBIC, [os.path.join(PKG, "ic", "pin_ic.c"),
                                                  os.path.join(INC, "pin_ic.h")])):
        procs.append(("libpin_ic", subprocess.Popen(cmd_ic(), stdout=subprocess.PIPE,
                                                    stderr=subprocess.STDOUT)))
    if "pin" in which and _sources_pin() and (force or _stale(LIBPIN, _deps_pin())):
        procs.append(("libpin", subprocess.Popen(cmd_pin(), stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT)))
    return procs


def build_all(force=False):
    _run(start(force=force))


def ensure_ic():
    if _stale(LIBIC, [os.path.join(PKG, "ic", "pin_ic.c"), os.path.join(INC, "pin_ic.h")]):
        _run(start(which=("ic",)))
    return LIBIC


def ensure_pin():
    if _stale(LIBPIN, _deps_pin()):
        _run(start(which=("pin",)))
    return LIBPIN


if __name__ == "__main__":
    build_all(force=True)
    print("built", LIBPIN, LIBIC)
