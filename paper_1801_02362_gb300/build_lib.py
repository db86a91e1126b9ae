"""Build the CUDA library libpcv.so in-tree (nvcc, sm_103a only).

The translation units are compiled in parallel and linked into
``paper_1801_02362_gb300/_build/libpcv.so``.  No CMake, no torch extension machinery:
the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libpcv.so"
SOURCES = ["k_pair.cu", "k_aux.cu", "k_adjoint.cu", "pcv_api.cu", "k_noalloc.cu", "k_tile.cu", "k_mma.cu", "k_shard.cu", "k_stream.cu", "k_nl.cu", "k_metad.cu", "k_xmma.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[Path]:
    return [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + [ROOT / "include" / "pcv.h"]


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    if not force and up_to_date():
        return LIB
    BUILD.mkdir(exist_ok=True)
    # CUDA 13 deprecates double4 in favour of types with a stated alignment; the library uses
    # it only with its 16-byte layout, which double4 keeps
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                    "-Xcompiler", "-Wno-deprecated-declarations", "-diag-suppress", "1444",
                    "--expt-relaxed-constexpr", "-I", str(ROOT / "include")] + (extra or [])
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs = []

    def compile_one(src: str):
        obj = BUILD / (src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", str(CSRC / src), "-o", str(obj)] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = BUILD / f"libpcv.{os.getpid()}.so"
    cmd = [nvcc(), "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
