"""Builds libadjwt.so (the C-ABI library) in-tree for sm_103a with nvcc.

Every translation unit under csrc/ is compiled in parallel into _build/ and
linked as a shared library next to this file.  Run by __graft_entry__.build()
(and by `python -m paper_1707_02018_gb300.build_ext`); the Python binding does
not build: it raises when the library is missing.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build", "adjwt")
LIB = os.path.join(HERE, "libadjwt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libadjwt")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


CHECKED_LIB = os.path.join(ROOT, "_build", "checked", "libadjwt_checked.so")


def build(verbose=False, extra=(), checked=False):
    """Build libadjwt.so in-tree; checked=True builds the bounds-checked
    variant (-DADJWT_BOUNDS_CHECK) into _build/checked/ instead."""
    global BUILD, LIB
    if checked:
        saved = BUILD, LIB
        BUILD, LIB = os.path.join(ROOT, "_build", "checked", "obj"), CHECKED_LIB
        try:
            return build(verbose, tuple(extra) + ("-DADJWT_BOUNDS_CHECK",), False)
        finally:
            BUILD, LIB = saved
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, extra=sys.argv[1:]))
