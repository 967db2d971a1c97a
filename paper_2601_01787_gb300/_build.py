"""Builds libmsz.so (the C ABI of include/msz.h) for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library with the static CUDA runtime.  The result goes to ``_build/`` inside
the package (git-ignored) and is rebuilt when a source, a header or the flags
change.
"""
from __future__ import annotations

import hashlib
import re
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libmsz.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
# The correction kernels must keep every float operation a single IEEE
# round-to-nearest step (bit-exact Jacobi sweeps): no FMA contraction, no
# flush-to-zero, IEEE division / square root.
EXACT = ["-fmad=false", "-ftz=false", "-prec-div=true", "-prec-sqrt=true"]

# (source, extra flags)
UNITS = [
    ("msz_correct.cu", EXACT),
    ("msz_segment.cu", EXACT),
    ("msz_static.cu", EXACT),
    ("msz_batch.cu", EXACT),
    ("msz_relaxed.cu", EXACT),
    ("msz_learned.cu", []),
    ("msz_edits.cu", []),
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsz.so")


def source_hash() -> str:
    """Hash of the CUDA sources, the public header and the compile flags
    (machine independent): identifies the kernels a profile was taken of."""
    h = hashlib.sha256()
    files = sorted(os.listdir(CSRC)) + ["../../include/msz.h"]
    for name in files:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    h.update(repr(([c for c in COMMON if not c.startswith("/")], UNITS)).encode())
    return h.hexdigest()[:16]


def _code_only(text: bytes) -> bytes:
    """Source text without C/C++ comments and with whitespace collapsed."""
    t = re.sub(rb"/\*.*?\*/", b" ", text, flags=re.S)
    t = re.sub(rb"//[^\n]*", b" ", t)
    return re.sub(rb"\s+", b" ", t).strip()


def unit_hash(unit: str) -> str:
    """Hash of the code (comments and layout ignored) of one translation
    unit, every header it can include and its flags: identifies the kernels
    of that unit a profile was taken of (a change to another unit, or to a
    comment, leaves it unchanged)."""
    h = hashlib.sha256()
    names = [unit] + sorted(n for n in os.listdir(CSRC) if n.endswith((".cuh", ".h"))) + ["../../include/msz.h"]
    for name in names:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            with open(p, "rb") as fh:
                h.update(_code_only(fh.read()))
    flags = [u for u in UNITS if (u[0] if isinstance(u, (tuple, list)) else u) == unit]
    h.update(repr(([c for c in COMMON if not c.startswith("/")], flags)).encode())
    return h.hexdigest()[:16]


def _stamp() -> str:
    return source_hash() + "-" + os.uname().machine


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libmsz.so when missing or stale; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp_path = os.path.join(OUT_DIR, "libmsz.stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            if fh.read().strip() == stamp:
                return LIB
    nvcc = _nvcc()
    procs = []
    objs = []
    for src, extra in UNITS:
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    with open(stamp_path, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
