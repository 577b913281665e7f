"""Compile the CUDA/C++ sources under csrc/ into the in-tree shared library libspiir.so
for sm_103a (nvcc cross-compiles; no GPU is needed to build)."""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libspiir.so")

SOURCES = ["common.cu", "bank.cu", "coherent.cu", "coherent_tmem.cu", "xi2.cu", "candidates.cu", "frontend.cu", "pipeline.cu", "search.cu", "adjoint.cu", "batch.cu", "sky_tables.cpp"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
                "-I" + INCLUDE]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "spiir.h"))
    return files


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False, out: str = None) -> str:
    """checked=True defines SPIIR_CHECKED: kernels verify their indices against the buffer sizes
    they were given, record violations in the device status word and skip the access, and the
    batched path synchronises after every stage.  A debugging build, written to ``out``."""
    lib_path = out or LIB_PATH
    if not force and not checked and not _stale(lib_path):
        return lib_path
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + (".checked.o" if checked else ".o"))
        cmd = [NVCC] + FLAGS + (["-DSPIIR_CHECKED"] if checked else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    os.makedirs(os.path.dirname(os.path.abspath(lib_path)), exist_ok=True)
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    if "--checked" in sys.argv:
        print(build(force=True, checked=True, out=sys.argv[sys.argv.index("--checked") + 1]))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
