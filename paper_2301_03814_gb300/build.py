"""Build libswkb.so in-tree with nvcc for sm_103a (no cmake, no torch).

Each translation unit under csrc/ is compiled in parallel to _build/, then
linked into paper_2301_03814_gb300/libswkb.so.  The CUDA runtime is linked
statically so the library only needs the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libswkb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswkb.so")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(verbose: bool = False, extra=(), checked: bool = False) -> str:
    """checked=True builds libswkb_checked.so with -DSWKB_BOUNDS_CHECK: device
    indices are checked against their buffers (a violation is clamped and
    reported as an error), the substitute for a memory sanitizer."""
    build_dir = BUILD + ("_checked" if checked else "")
    lib_path = LIB.replace("libswkb.so", "libswkb_checked.so") if checked else LIB
    if checked:
        extra = (*extra, "-DSWKB_BOUNDS_CHECK")
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    # FP32 denormals never occur on this path (deviation variables are >= 1e-12),
    # and every FP32 quotient that must be exact is a power of two done by scalbn
    common = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-ftz=true", "-prec-div=false",
              "-prec-sqrt=false", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]

    def compile_one(src):
        obj = os.path.join(build_dir, src[:-3] + ".o")
        cmd = [cc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, len(sources()))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib_path + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=[a for a in sys.argv[1:] if a != "-v"]))
