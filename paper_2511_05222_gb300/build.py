"""Build libvmcf.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel and linked into
paper_2511_05222_gb300/_build/libvmcf.so. A rebuild happens only when a source is newer
than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
SRC = PKG / "csrc"
INC = PKG.parent / "include"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libvmcf.so"
UNITS = ["vmcf_api.cu", "k_fp64.cu", "k_fp32.cu", "k_fp64_jb.cu", "k_fp32_jb.cu", "k_small_fp64.cu", "k_small_fp32.cu",
         "k_small_fp64_jb.cu", "k_small_fp32_jb.cu",
         "k_reduce.cu", "k_probe.cu", "noalloc.cu", "k_tc_sumprod.cu", "k_batch.cu", "k_batch_fp64.cu", "k_batch_jb.cu",
         "k_batch_fp64_jb.cu", "batch_api.cu", "checkpoint.cu", "k_tc_rows.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvmcf")


def _sources():
    return [SRC / u for u in UNITS] + sorted(SRC.glob("*.cuh")) + sorted(SRC.glob("*.h")) + sorted(INC.glob("*.h"))


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _sources())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> Path:
    if not force and up_to_date():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INC)] + (extra_flags or [])
    tag = f"{os.getpid()}"

    def compile_unit(u: str) -> Path:
        obj = OUT_DIR / (Path(u).stem + f".{tag}.o")
        cmd = [cc, *flags, "-c", str(SRC / u), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    objs = [OUT_DIR / (Path(u).stem + f".{tag}.o") for u in UNITS]
    tmp = OUT_DIR / f"libvmcf.{tag}.so"
    try:
        with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
            list(ex.map(compile_unit, UNITS))
        r = subprocess.run([cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    finally:  # no objects or partial library are left behind, whether or not the build succeeded
        for o in objs + [tmp]:
            o.unlink(missing_ok=True)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
