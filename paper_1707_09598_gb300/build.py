"""Build the CUDA library libsgiga.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into
paper_1707_09598_gb300/_lib/libsgiga.so. Usage: python -m paper_1707_09598_gb300.build
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libsgiga.so")
# the checked build (-DSGIGA_CHECKED): bounds checks in the hot kernels
OUT_CHECKED = os.path.join(HERE, "_lib_checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libsgiga.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            return cand
        raise RuntimeError("nvcc not found")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(src, extra, out=OUT):
    obj = os.path.join(out, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(verbose=False, extra=(), checked=False):
    out = OUT_CHECKED if checked else OUT
    lib = LIB_CHECKED if checked else LIB
    extra = list(extra) + (["-DSGIGA_CHECKED"] if checked else [])
    os.makedirs(out, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    objs = [o for o, _ in res]
    if verbose:
        for (o, err) in res:
            if err.strip():
                print(os.path.basename(o), err)
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(verbose=v or bool(extra), extra=extra, checked="--checked" in sys.argv))
