"""In-tree build of libnbgpu.so (sm_103a) with nvcc.

Each translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into a
shared library next to this file.  The CUDA runtime is linked statically, so the
library needs only the driver at run time.  Rebuilds happen when a source or header
is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnbgpu.so")
OBJDIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# per-file extra flags: the mixed kernels flush FP32 denormals (no distinct particles are
# 1e-19 apart) so that rsqrtf is a single hardware instruction; the integrator and the array
# corrector keep the plain definition's FP64 operation order (no FMA contraction), and the
# irregular force shares its per-row code with the integrator's fused step, so it is compiled
# with the same flags (the two give the same bits for a row)
EXTRA = {"force_mixed.cu": ["-ftz=true"], "adjoint.cu": ["-ftz=true"], "irregular.cu": ["-ftz=true", "-fmad=false"],
         "ac.cu": ["-ftz=true", "-fmad=false"], "hermite.cu": ["-fmad=false"]}
SOURCES = ["nb_api.cu", "predict.cu", "force_mixed.cu", "force_fp64.cu", "neighbours.cu", "adjoint.cu",
           "noalloc.cu", "irregular.cu", "sched.cu", "ac.cu", "roworder.cu",
           "hermite.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnbgpu.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "nbgpu.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def needs_build() -> bool:
    return not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest_input()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libnbgpu.so."""
    if not force and not needs_build():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(OBJDIR, s.replace(".cu", ".o")) for s in srcs]

    def compile_one(src, obj):
        cmd = [nvcc, *ARCH, *COMMON, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return r.stderr

    workers = min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        logs = list(ex.map(compile_one, srcs, objs))
    if verbose or ptxas_info:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"--- {s}\n{log}")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
