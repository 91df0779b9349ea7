"""Compile the package's native libraries in-tree.

Two shared libraries are produced under ``paper_2511_14955_gb300/_lib``:

* ``libsynth.so``      - the seeded corpus generator (host C, gcc);
* ``libintergrams.so`` - the sm_103a kernels and the C ABI (nvcc).

Builds are incremental: a library is rebuilt when any of its sources is newer
than the library. No cmake; one ``-gencode`` (sm_103a); translation units are
compiled in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
LIB = PKG / "_lib"
INCLUDE = PKG.parent / "include"

CUDA_HOME = Path(os.environ.get("CUDA_HOME", "/usr/local/cuda"))
NVCC = str(CUDA_HOME / "bin" / "nvcc") if (CUDA_HOME / "bin" / "nvcc").exists() else "nvcc"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SYNTH_SOURCES = [CSRC / "synth.c"]
CUDA_SOURCES = sorted(CSRC.glob("*.cu"))
CUDA_HEADERS = sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(map(str, cmd)) + "\n" + r.stdout)
    return r.stdout


def build_synth(force: bool = False) -> Path:
    LIB.mkdir(exist_ok=True)
    out = LIB / "libsynth.so"
    if force or _stale(out, SYNTH_SOURCES):
        tmp = out.with_suffix(".so.tmp")
        _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", str(tmp),
              *map(str, SYNTH_SOURCES), "-lm", "-lpthread"])
        os.replace(tmp, out)
    return out


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> Path:
    LIB.mkdir(exist_ok=True)
    out = LIB / "libintergrams.so"
    deps = CUDA_SOURCES + CUDA_HEADERS
    if not (force or _stale(out, deps)):
        return out
    objdir = LIB / "obj"
    objdir.mkdir(exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
             "-I", str(INCLUDE), "-I", str(CSRC), "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def compile_one(src: Path) -> Path:
        obj = objdir / (src.stem + ".o")
        if force or _stale(obj, [src] + CUDA_HEADERS):
            _run([NVCC, "-c", *flags, "-o", str(obj), str(src)])
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, CUDA_SOURCES))
    tmp = out.with_suffix(".so.tmp")
    _run([NVCC, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lcudart"])
    os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> None:
    build_synth(force)
    if shutil.which(NVCC) or Path(NVCC).exists():
        build_cuda(force)
    else:
        raise RuntimeError("nvcc not found; the CUDA library cannot be built")
