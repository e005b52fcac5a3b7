"""Build libpond.so, the PonD CUDA library, for sm_103a (GB300).

Each .cu under csrc/ is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -lineinfo -O3) and linked into
paper_1806_05089_gb300/libpond.so (in-tree; static CUDA runtime).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libpond.so")
BUILD_DIR = os.path.join(HERE, "_build")
# debug build: the staged kernel's index checks compiled in (POND_DEBUG)
DEBUG_LIB = os.path.join(HERE, "libpond_debug.so")
DEBUG_BUILD_DIR = os.path.join(HERE, "_build_debug")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the PonD CUDA library cannot be built")
    return cand


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "pond.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), out: str | None = None,
          build_dir: str | None = None, debug: bool = False) -> str:
    """Compile and link; ``extra_flags``/``out``/``build_dir`` build a variant
    library elsewhere (tuning experiments) without touching the default one;
    ``debug`` builds libpond_debug.so with the index checks (POND_DEBUG)."""
    if debug:
        extra_flags = tuple(extra_flags) + ("-DPOND_DEBUG",)
        out = out or DEBUG_LIB
        build_dir = build_dir or DEBUG_BUILD_DIR
        if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
                os.path.getmtime(d) for d in sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
                + [os.path.join(INCLUDE, "pond.h")]):
            return out
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    nvcc = _nvcc()
    bdir = build_dir or BUILD_DIR
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(f) for f in failed))
    fd, tmp = tempfile.mkstemp(prefix="libpond.", suffix=".so", dir=os.path.dirname(lib))
    os.close(fd)
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lrt", "-lpthread", "-ldl"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
