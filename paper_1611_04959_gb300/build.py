"""Build libdaq.so (the C ABI of include/daq.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libdaq.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs() -> list:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ (in parallel, one -gencode, -lineinfo) and
    link them into one shared library."""
    if not force and not stale():
        return LIB
    import concurrent.futures as cf
    obj_dir = os.path.join(PKG, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    base = [nvcc(), "-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    if verbose:
        base.insert(1, "-Xptxas=-v")

    def compile_one(src: str):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + f".{os.getpid()}.o")
        r = subprocess.run(base + ["-c", "-o", obj, src], capture_output=True, text=True)
        return src, obj, r

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, sources()))
    failed = [(src, r) for src, _, r in results if r.returncode != 0]
    if verbose:
        for _, _, r in results:
            sys.stderr.write(r.stderr)
    if failed:
        for src, r in failed:
            sys.stderr.write(f"--- {src}\n" + r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libdaq.so")
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *[o for _, o, _ in results]], capture_output=True,
                       text=True)
    for _, o, _ in results:
        try:
            os.remove(o)
        except OSError:
            pass
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libdaq.so")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
