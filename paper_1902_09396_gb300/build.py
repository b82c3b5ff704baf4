"""In-tree build of the product library libhmlfc.so for sm_103a (GB300).

CUDA sources go through nvcc with ``-gencode arch=compute_103a,code=sm_103a``;
host sources through g++; everything links into one shared object with the
CUDA runtime linked statically.  Translation units compile in parallel.

``build(check=True)`` makes the bounds-checked variant (``-DHMLFC_CHECK``:
every kernel read of a stream array is checked against the array's length
and reported through the stream's status word) in ``_build_check/``; load it
by pointing the environment variable HMLFC_LIB at CHECK_LIB.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libhmlfc.so"
CHECK_DIR = PKG / "_build_check"
CHECK_LIB = CHECK_DIR / "libhmlfc.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hmlfc_kernels.cu", "hmlfc_encode_gpu.cu", "hmlfc_host.cpp", "hmlfc_encode.cpp", "hmlfc_touched.cpp"]


def _cuda_home() -> Path:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return Path(nvcc).resolve().parent.parent
    return Path(os.environ.get("CUDA_HOME", "/usr/local/cuda"))


def _stale(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + [ROOT / "include" / "hmlfc.h", Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> Path:
    out_dir, lib = (CHECK_DIR, CHECK_LIB) if check else (OUT_DIR, LIB)
    if not force and not _stale(lib):
        return lib
    if check:
        build(verbose=verbose)        # the checks live in the kernels; the other objects are the normal build's
    out_dir.mkdir(parents=True, exist_ok=True)
    cuda = _cuda_home()
    nvcc = str(cuda / "bin" / "nvcc")
    inc = ["-I", str(ROOT / "include"), "-I", str(CSRC)]
    procs = []
    objs = []
    for src in SOURCES:
        if check and src != "hmlfc_kernels.cu":
            objs.append(OUT_DIR / (src + ".o"))
            continue
        obj = out_dir / (src + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                   *(["-DHMLFC_CHECK"] if check else []), "-c", str(CSRC / src), "-o", str(obj)]
        else:
            cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall", *inc,
                   "-I", str(cuda / "include"), "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out}")
        elif verbose and out:
            print(out)
    if errors:
        raise RuntimeError("building libhmlfc failed:\n" + "\n".join(errors))
    tmp = out_dir / f"libhmlfc.{os.getpid()}.so"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-pthread",
            "-o", str(tmp), *map(str, objs)]
    if verbose:
        print(" ".join(link))
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("linking libhmlfc failed:\n" + r.stdout)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
