"""Builds libgfh.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked with cuFFT.  Host code is compiled with
-ffp-contract=off: the fixed-point tables must round every double expression as written.
"""
from __future__ import annotations

import concurrent.futures
import os
import pathlib
import shutil
import subprocess
import sys

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = ROOT / "_build"
LIB = PKG / "libgfh.so"
SOURCES = ["gfh_host.cpp", "gfh_hough.cu", "gfh_peakmap.cu", "gfh_cnn.cu", "gfh_squares.cu",
           "gfh_followup.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgfh")
    return cand


def _flags() -> list[str]:
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", str(ROOT / "include"),
                   "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-Xptxas", "-O3"]


def _compile(src: str, verbose: bool) -> pathlib.Path:
    obj = BUILD / (src + ".o")
    cmd = [_nvcc(), "-c", str(CSRC / src), "-o", str(obj)] + _flags()
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, force: bool = False) -> pathlib.Path:
    """Compile and link libgfh.so; skipped when it is newer than every source and header."""
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list((ROOT / "include").glob("*.h"))
    if (not force and LIB.exists()
            and LIB.stat().st_mtime > max(p.stat().st_mtime for p in deps)):
        return LIB
    BUILD.mkdir(exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [_nvcc(), "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
