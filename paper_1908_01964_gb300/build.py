"""Build the CUDA shared library (sm_103a) in-tree with nvcc.

    python -m paper_1908_01964_gb300.build        # or build() from Python
    python -m paper_1908_01964_gb300.build --debug   # the index-checking build

Translation units compile in parallel into ``_build/`` and link into
``paper_1908_01964_gb300/librcscm.so`` (CUDA runtime linked statically, so the
library only needs the NVIDIA driver at load time).  ``build(debug=True)``
compiles with RCSCM_DEBUG (row, slot and shape checks in every kernel that set
RCSCM_EBOUNDS instead of touching memory out of range) into ``_build_debug/``
and ``librcscm_debug.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "librcscm.so")
LIB_DEBUG = os.path.join(PKG, "librcscm_debug.so")
SOURCES = ["api.cu", "setup.cu", "iterate.cu", "naive.cu", "extract.cu", "objective.cu", "host.cu", "noalloc.cu", "adjoint.cu", "accel1.cu", "ilrma.cu", "probe.cu", "frontend.cu"]
# (threads per row, slots per thread) shapes of the accelerated kernels: iterate_inst.cu
# is compiled once per shape so that the large unrolled kernels build in parallel.
INSTANCES = [(32, 4), (32, 8), (64, 4), (64, 8), (128, 4), (128, 8), (256, 4), (256, 8), (512, 4), (512, 8),
             (1024, 4)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librcscm.so")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES + ["iterate_inst.cu"]]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def up_to_date(lib: str = None) -> bool:
    lib = lib or LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=None, debug: bool = False) -> str:
    """Compile every translation unit for sm_103a and link librcscm.so (or, with
    debug, librcscm_debug.so); returns its path."""
    lib = LIB_DEBUG if debug else LIB
    build_dir = BUILD_DIR + "_debug" if debug else BUILD_DIR
    if not force and up_to_date(lib):
        return lib
    nvcc = nvcc_path()
    os.makedirs(build_dir, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DRCSCM_DEBUG"] if debug else [])
    procs = []
    objs = []
    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    units += [("iterate_inst.cu", f"iterate_b{b}_s{t}.o", [f"-DRCSCM_INST_BLOCK={b}", f"-DRCSCM_INST_SPT={t}"])
              for b, t in INSTANCES]
    for src, objname, defs in units:
        obj = os.path.join(build_dir, objname)
        cmd = [nvcc, *ARCH, *flags, *defs, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
