"""Build the CUDA library ``_build/libswgpu.so`` in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD, "libswgpu.so")

SOURCES = ["sw_engine.cu", "sw_server.cu", "sw_noalloc.cu", "sw_potts.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source (in parallel) and link one shared library."""
    from concurrent.futures import ThreadPoolExecutor

    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        if os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(f) for f in _inputs()):
            return LIB_PATH
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = f".tmp{os.getpid()}"
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if verbose:
        common.append("-Xptxas=-v")

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + tag + ".o")
        subprocess.run(common + ["-c", "-o", obj, os.path.join(CSRC, src)], check=True)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + tag
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
