"""Build libsho.so for sm_103a with nvcc (one object per translation unit, compiled in parallel).

Usage: ``python -m paper_1905_00480_gb300.build`` or ``paper_1905_00480_gb300.build.build()``.
The library lands in ``paper_1905_00480_gb300/lib/`` (kept out of version control).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(HERE, "lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libsho.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the SHO library needs the CUDA toolkit to build")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return sorted(hs)


def _digest(path: str, extra: bytes = b"") -> str:
    h = hashlib.sha1(extra)
    with open(path, "rb") as f:
        h.update(f.read())
    for hp in headers():
        with open(hp, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def _compile(nvcc: str, src: str, verbose: bool) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(OBJ_DIR, f"{base}.{_digest(src)}.o")
    if os.path.exists(obj):
        return obj
    for old in os.listdir(OBJ_DIR):  # objects of earlier versions of this source
        if old.startswith(base + ".") and old.endswith(".o"):
            try:
                os.remove(os.path.join(OBJ_DIR, old))
            except OSError:
                pass
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int = None) -> str:
    """Compile every CUDA source for sm_103a and link libsho.so; returns its path."""
    nvcc = nvcc_path()
    os.makedirs(OBJ_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, verbose), srcs))
    lib = os.path.join(LIB_DIR, LIB_NAME)
    key = hashlib.sha1("".join(objs).encode()).hexdigest()[:16]
    stamp = lib + ".stamp"
    if os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read() == key:
                return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(key)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
