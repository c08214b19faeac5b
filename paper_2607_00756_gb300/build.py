"""Builds libbip.so (the C-ABI library) in-tree for sm_103a.

CUDA sources are compiled by nvcc with one -gencode (compute_103a/sm_103a),
host sources by g++, in parallel; objects go to _build/ and the library to
this package directory.  A source is recompiled when it (or any header) is
newer than its object.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbip.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "bip.h"))
    return hs


def _stale(src, obj, newest_header):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def build(verbose=False, force=False):
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    newest_header = max(os.path.getmtime(h) for h in _headers())
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include")]
    jobs = []
    for f in sorted(os.listdir(CSRC)):
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        if f.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   *(["-Xptxas", "-v"] if verbose else []), *inc, "-c", src, "-o", obj]
        elif f.endswith(".cpp"):
            cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-Wall", *inc, "-c", src, "-o", obj]
        else:
            continue
        jobs.append((src, obj, cmd))

    def run(job):
        src, obj, cmd = job
        if not force and not _stale(src, obj, newest_header):
            return None
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr if verbose else None

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        for msg in ex.map(run, jobs):
            if msg:
                sys.stderr.write(msg)
    objs = [o for _, o, _ in jobs]
    newest_obj = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest_obj:
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, force="-f" in sys.argv)
    print(LIB)
