"""In-tree build of libdof.so: one nvcc job per .cu file (in parallel), then a shared
link.  sm_103a only (GB300)."""

from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
LIB_DIR = PKG / "_lib"
LIB = LIB_DIR / "libdof.so"
SOURCES = ["api.cu", "bvh.cu", "trace.cu", "post.cu", "temporal.cu", "recon.cu", "noalloc.cu", "raster.cu"]
HEADERS_EXTRA = ["batch.cuh", "geometry.cuh"]
HEADERS = ["dof_internal.cuh", "filters.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    return "nvcc"


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                   "--expt-relaxed-constexpr", "-I", str(PKG.parent / "include")]


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = [CSRC / s for s in SOURCES + HEADERS + HEADERS_EXTRA] + [PKG.parent / "include" / "dof.h", Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not _stale():
        return LIB
    obj_dir = LIB_DIR / "obj"
    obj_dir.mkdir(parents=True, exist_ok=True)
    nv = nvcc()

    def compile_one(src):
        obj = obj_dir / (Path(src).stem + ".o")
        cmd = [nv, "-c", str(CSRC / src), "-o", str(obj)] + _flags()
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        (obj_dir / (Path(src).stem + ".ptxas.txt")).write_text(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [nv, "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for s in SOURCES:
            print((obj_dir / (Path(s).stem + ".ptxas.txt")).read_text())
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
