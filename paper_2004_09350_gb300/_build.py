"""Builds libms.so (the CUDA library behind include/morphstore.h) in-tree with nvcc.

Translation units compile in parallel for sm_103a only; the shared object lands next
to this file.  No CMake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libms.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["ms_host.cu", "ms_ops.cu", "ms_noalloc.cu", "ms_consume.cu", "ms_place.cu", "ms_map_codec.cu",
           "ms_select_packed.cu",
           "ms_map_project.cu", "ms_map_calc.cu", "ms_map_emit.cu", "ms_mlp.cu",
           "ms_batch.cu", "ms_batch_d2.cu", "ms_batch_d3.cu", "ms_batch_d4.cu",
           "ms_batch_static.cu", "ms_rle.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "morphstore.h"))
    return max(os.path.getmtime(f) for f in files)


STAMP = LIB + ".defines"  # the tuning definitions the library was built with


def _defines():
    # MS_NVCC_DEFINES: extra -D definitions for a tuning build (space separated)
    return [d for d in os.environ.get("MS_NVCC_DEFINES", "").split() if d]


def _stamp_matches(defines) -> bool:
    try:
        with open(STAMP) as f:
            return f.read() == " ".join(defines)
    except OSError:
        return not defines


def build(force: bool = False, verbose: bool = False) -> str:
    defines = _defines()
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps()
            and _stamp_matches(defines)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    common += [f"-D{d}" for d in defines]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(" ".join(defines))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
