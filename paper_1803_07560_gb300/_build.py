"""Builds the CUDA library libbfi.so in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled in parallel into an object, then the
objects are linked into one shared library with the C ABI of include/bfi.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build", platform.machine())  # per host architecture
LIB = os.path.join(OUT_DIR, "libbfi.so")
CLI_SRC = os.path.join(PKG, "cli", "bfi_cli.cpp")
CLI = os.path.join(OUT_DIR, "bfi_cli")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbfi.so")
    return cand


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "bfi.h"), CLI_SRC, __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(CLI):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(CLI))
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile the library.  BFI_NVCC_EXTRA (environment) adds nvcc flags,
    e.g. -DBFI_INTEGRAND_MIN_BLOCKS=1 to compile for one CTA per SM."""
    extra_env = os.environ.get("BFI_NVCC_EXTRA", "").split()
    if extra_env:
        force = True
    if not force and not ptxas_info and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + extra_env

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, _sources()))
    logs = []
    for obj, log in results:
        objs.append(obj)
        logs.append(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    _build_cli()
    if verbose or ptxas_info:
        print("\n".join(logs))
    return LIB


def _build_cli() -> None:
    """The line-protocol integrand program, linked against libbfi.so (found
    beside it at run time)."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("no C++ compiler found for bfi_cli")
    tmp = CLI + f".tmp{os.getpid()}"
    cmd = [cxx, "-O2", "-std=c++17", "-Wall", f"-I{INCLUDE}", CLI_SRC, "-o", tmp, f"-L{OUT_DIR}", "-lbfi",
           "-Wl,-rpath,$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"bfi_cli build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CLI)


if __name__ == "__main__":
    import sys
    build(force=True, ptxas_info="-v" in sys.argv)
    print(LIB)
