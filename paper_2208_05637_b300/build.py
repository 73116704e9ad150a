"""Build the CUDA library in-tree: paper_2208_05637_b300/_nqs.so for sm_103a.

    python paper_2208_05637_b300/build.py [--force]   (run by path: importing the package
                                                       needs the library this builds)

One nvcc invocation compiles every .cu/.cpp under csrc/ into a shared library with the C ABI of
include/nqs.h.  A stamp of the source hashes and flags skips rebuilds when nothing changed.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "_nqs.so")
STAMP = os.path.join(PKG, "_nqs.stamp")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "-shared", "--cudart", "shared",
         "-Xptxas", "-O3"]


def sources():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")) +
                  glob.glob(os.path.join(PKG, "csrc", "*.cpp")))


def _digest(extra):
    h = hashlib.sha256()
    for p in sources() + sorted(glob.glob(os.path.join(PKG, "csrc", "*.h")) +
                                glob.glob(os.path.join(PKG, "csrc", "*.cuh"))) + \
            [os.path.join(ROOT, "include", "nqs.h")]:
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + extra).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    extra = list(extra)
    dig = _digest(extra)
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    compile_flags = [f for f in FLAGS if f != "-shared"]

    def one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + compile_flags + extra + ["-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, res

    objs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        for src, obj, res in ex.map(one, sources()):
            if res.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n" + res.stdout + res.stderr)
            if verbose and (res.stdout or res.stderr):
                print(res.stdout + res.stderr)
            objs.append(obj)
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "--cudart", "shared", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
