"""Compile the CUDA library (sm_103a) in-tree: csrc/*.cu -> _lib/libbtrt.so.

Translation units compile in parallel with nvcc; the shared object is linked
with nvcc as well.  A build is skipped when a stamp beside the library records
the same digest of every source, header and flag, on the same architecture.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "_lib"
LIB = OUT / "libbtrt.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit contraction of a*b + c into an FMA.  The hot paths
# write their FMAs explicitly, so every kernel form (plain, TMA-staged, batched)
# rounds each node's arithmetic identically and their results agree bitwise.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", str(ROOT / "include")] + ARCH


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbtrt")


def _sources():
    return sorted(CSRC.glob("*.cu"))


def _deps():
    return list(CSRC.glob("*")) + list((ROOT / "include").glob("*.h")) + [Path(__file__)]


def _stamp(extra) -> str:
    """Digest of everything the library is built from (sources, headers, this
    script, the extra flags) and of the machine: a copied tree whose file times
    say nothing, or a library built on another architecture, is rebuilt."""
    import hashlib
    import platform
    h = hashlib.sha256()
    for p in sorted(_deps()):
        h.update(p.name.encode())
        h.update(p.read_bytes())
    h.update(" ".join(list(extra or [])).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _stamp_path(lib: Path) -> Path:
    return Path(str(lib) + ".stamp")


def up_to_date(lib: Path = LIB, extra=None) -> bool:
    if not lib.exists() or not _stamp_path(lib).exists():
        return False
    return _stamp_path(lib).read_text().strip() == _stamp(extra)


def build(force: bool = False, verbose: bool = False, extra=None, lib: Path = LIB) -> Path:
    """Compile every csrc/*.cu and link `lib`.  `extra` adds nvcc flags (for example
    -DBTRT_DEBUG_BOUNDS for the index-checked build, linked to another path)."""
    lib = Path(lib)
    if not force and up_to_date(lib, extra):
        return lib
    lib.parent.mkdir(parents=True, exist_ok=True)
    objdir = lib.parent / "obj"
    objdir.mkdir(exist_ok=True)
    flags = NVCC_FLAGS + list(extra or [])

    def compile_one(src: Path):
        obj = objdir / (src.stem + ".o")
        cmd = [nvcc(), "-c", str(src), "-o", str(obj)] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = str(lib) + ".tmp"
    # --no-undefined: a missing template instantiation fails the build, not the first dlopen
    cmd = [nvcc(), "-shared", "-o", tmp] + [str(o) for o in objs] + ARCH + ["-lcudart", "-Xlinker", "--no-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    _stamp_path(lib).write_text(_stamp(extra) + "\n")
    return lib


DEBUG_LIB = OUT / "debug" / "libbtrt.so"


def build_debug(force: bool = False) -> Path:
    """The index-checked build (every global access of the sweeps checks its index
    and raises flag bit 3 instead of faulting), for tests on tiny grids."""
    return build(force=force, extra=["-DBTRT_DEBUG_BOUNDS"], lib=DEBUG_LIB)


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
