"""Compile libhz (the CUDA kernels, the solver and its C ABI) for sm_103a, in-tree."""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libhz.so")
SOURCES = ["hz_kernels.cu", "hz_kernels32.cu", "hz_kernels_ff.cu", "hz_fci_tail32.cu",
           "hz_arnoldi_ff.cu", "hz_case_two.cu", "hz_api.cu", "hz_setup.cpp", "hz_noalloc.cu",
           "hz_conv.cu", "hz_net.cu", "hz_coop64.cu", "hz_ilu.cu", "hz_fft.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libhz needs the CUDA toolkit to build")


STAMP = LIB + ".sha256"


def _fingerprint(nvcc: str, deps) -> str:
    """sha256 over the compiler path, the flags and the content of every source and header."""
    h = hashlib.sha256()
    h.update(" ".join([nvcc, *ARCH, *FLAGS, *SOURCES]).encode())
    for d in deps:
        h.update(os.path.basename(d).encode())
        with open(d, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    """Build _build/libhz.so unless the library there was built from exactly these sources and
    flags (a content hash kept beside it; file times are not trusted); returns its path."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                     if f.endswith((".h", ".cuh")))
    deps = srcs + headers + [os.path.join(INCLUDE, "hz.h")]
    nvcc = _nvcc()
    fp = _fingerprint(nvcc, deps)
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as fh:
            if fh.read().strip() == fp:
                return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    # objects of sources that are no longer part of the library
    keep = {os.path.basename(s) + ".o" for s in SOURCES}
    for f in os.listdir(OUT_DIR):
        if f.endswith(".o") and f not in keep:
            os.remove(os.path.join(OUT_DIR, f))
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(fp + "\n")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force=True))
