"""Build the C-ABI library libbitpic.so (sm_103a) in-tree.

Each CUDA translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3``; every unit except the
FP32 mover is compiled with ``-fmad=false`` so that the FP64 form rounds each multiply
and add separately.  The shared library lands in ``paper_2404_10270_gb300/_native/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_native")
LIB = os.path.join(OUT, "libbitpic.so")
# the bounds-checked device build (-DPIC_CHECKED): every index a kernel computes is
# checked and a violation latches a status bit; for tests, not for speed
LIB_CHECKED = os.path.join(OUT, "libbitpic_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "mover_f32.cu": [],
    "mover_f64.cu": ["-fmad=false"],
    "events.cu": ["-fmad=false"],
    "field.cu": ["-fmad=false"],
    "sort.cu": ["-fmad=false"],
    "io.cu": ["-fmad=false"],
    "engine.cu": ["-fmad=false"],
    "noalloc.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    files.append(os.path.join(ROOT, "include", "pic.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(lib: str) -> bool:
    if not os.path.exists(lib) or os.environ.get("BITPIC_NVCC_EXTRA"):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(unit: str, extra, verbose: bool, outdir: str = OUT) -> str:
    obj = os.path.join(outdir, unit.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
           "-c", os.path.join(SRC, unit), "-o", obj, *extra]
    cmd += os.environ.get("BITPIC_NVCC_EXTRA", "").split()
    if verbose:
        cmd.append("-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, r.stdout, r.stderr))
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def source_key(files=("mover.cuh", "common.cuh", "mover_f32.cu", "mover_f64.cu"), read=None) -> str:
    """SHA-256 of the code of the given sources with comments and blank space removed: the
    key under which measurements of the compiled kernels (ncu traffic) are kept, so that an
    edit of a comment does not disown them."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        text = read(f) if read else open(os.path.join(SRC, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link libbitpic.so (checked=True: libbitpic_checked.so, the
    bounds-checked device build) if any source is newer than the library."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    outdir = os.path.join(OUT, "checked") if checked else OUT
    os.makedirs(outdir, exist_ok=True)
    extra = ["-DPIC_CHECKED"] if checked else []
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1] + extra, verbose, outdir),
                           UNITS.items()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
