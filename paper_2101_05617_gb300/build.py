"""Build libswepi.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel into _build/, then linked into
paper_2101_05617_gb300/libswepi.so.  Called by __graft_entry__.build().
build(checked=True) makes the bounds-checked variant (-DSW_CHECK) instead:
objects in _build_check/, library libswepi_check.so (loaded by the binding
when SWEPI_CHECKED=1)."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libswepi.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libswepi_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
SOURCES = ["geom.cpp", "dfr.cu", "krylov.cu", "kiops.cu", "kiops_graph.cu", "capi.cu", "noalloc.cu", "dfr_split.cu", "dfr_tile.cu", "mlp.cu", "diag.cu", "ensemble.cu"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def _compile(src, extra, build_dir):
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-I", os.path.join(HERE, "..", "include"), "-c",
                                             os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def build(verbose=False, extra=(), checked=False):
    build_dir, lib = (BUILD_CHECK, LIB_CHECK) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    extra = list(extra) + (["-DSW_CHECK"] if checked else [])
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, build_dir), SOURCES))
    objs = []
    for src, obj, rc, out in results:
        if rc != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out}")
        if verbose and out.strip():
            print(out, file=sys.stderr)
        objs.append(obj)
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, extra=sys.argv[1:]))
