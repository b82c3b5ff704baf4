"""In-tree build of the product library libhmlfc.so for sm_103a (GB300).

CUDA sources go through nvcc with ``-gencode arch=compute_103a,code=sm_103a``;
host sources through g++; everything links into one shared object with the
CUDA runtime linked statically.  Translation units compile in parallel.
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
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hmlfc_kernels.cu", "hmlfc_encode_gpu.cu", "hmlfc_host.cpp", "hmlfc_encode.cpp", "hmlfc_touched.cpp"]


def _cuda_home() -> Path:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return Path(nvcc).resolve().parent.parent
    return Path(os.environ.get("CUDA_HOME", "/usr/local/cuda"))


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + [ROOT / "include" / "hmlfc.h", Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not _stale():
        return LIB
    OUT_DIR.mkdir(parents=True, exist_ok=True)
    cuda = _cuda_home()
    nvcc = str(cuda / "bin" / "nvcc")
    inc = ["-I", str(ROOT / "include"), "-I", str(CSRC)]
    procs = []
    objs = []
    for src in SOURCES:
        obj = OUT_DIR / (src + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                   "-c", str(CSRC / src), "-o", str(obj)]
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
    tmp = OUT_DIR / f"libhmlfc.{os.getpid()}.so"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-pthread",
            "-o", str(tmp), *map(str, objs)]
    if verbose:
        print(" ".join(link))
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("linking libhmlfc failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
