"""Compile libdcflow.so (sm_103a) in-tree with nvcc.

Run as ``python -m paper_2501_17529_b300.csrc.build`` or call ``build()``.
Every source compiles to its own object under ``_build/`` (in parallel), with
a dependency list written by nvcc beside it; an object is rebuilt when its
source or a header it includes is newer than it, and the library is relinked
when any object was rebuilt.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libdcflow.so")
OBJ = os.path.join(ROOT, "_build", "obj")
SOURCES = ["api.cu", "dense64.cu", "setup.cu", "solve.cu", "n1_launch.cu", "n1_launch_tc.cu", "noalloc.cu", "mlp.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers_mtime():
    hs = [os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith(".cuh")]
    hs.append(os.path.join(ROOT, "include", "dcflow.h"))
    return max(os.path.getmtime(h) for h in hs)


def _obj(src):
    return os.path.join(OBJ, os.path.splitext(src)[0] + ".o")


def _deps(src):
    """Files the object of `src` was built from (nvcc's dependency list), or None."""
    d = _obj(src) + ".d"
    if not os.path.exists(d):
        return None
    text = open(d).read().replace("\\\n", " ")
    out = []
    for line in text.splitlines():
        if ":" in line:
            out += line.split(":", 1)[1].split()
    return [x for x in out if x.startswith(HERE) or x.startswith(os.path.join(ROOT, "include"))]


def _stale(src, hdr_t):
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    deps = _deps(src)
    if deps is None:
        return os.path.getmtime(os.path.join(HERE, src)) > t or hdr_t > t
    return any(not os.path.exists(x) or os.path.getmtime(x) > t for x in deps + [os.path.join(HERE, src)])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    hdr_t = _headers_mtime()
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    return any(os.path.getmtime(s) > t for s in srcs) or hdr_t > t


def build(force: bool = False, verbose: bool = False, extra=()):
    if not force and not needs_build():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    hdr_t = _headers_mtime()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "-I" + os.path.join(ROOT, "include"), "-I" + HERE] + list(extra)
    todo = [s for s in SOURCES if force or _stale(s, hdr_t)]

    def compile_one(src):
        cmd = [_nvcc()] + flags + ["-MD", "-MF", _obj(src) + ".d", "-c", os.path.join(HERE, src),
                                   "-o", _obj(src) + ".tmp"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.stdout or r.stderr:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise subprocess.CalledProcessError(r.returncode, cmd)
        os.replace(_obj(src) + ".tmp", _obj(src))

    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
        list(ex.map(compile_one, todo))
    cmd = [_nvcc(), ARCH, "-shared", "-o", LIB + ".tmp"] + [_obj(s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
