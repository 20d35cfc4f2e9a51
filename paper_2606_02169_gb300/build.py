"""Build libhm.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
paper_2606_02169_gb300/_build/libhm.so against the shared CUDA runtime, so
the library shares torch's runtime (and its streams) inside one process.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhm.so")
SOURCES = ["capi.cpp", "plan.cpp", "tile_plan.cpp", "apply.cu", "apply_f32.cu", "apply_df64.cu", "apply_f64.cu",
           "tile_f32.cu", "tile_df64.cu", "adjoint.cu", "lanczos.cu", "grad_static.cu", "sector.cu", "sector_blk.cu",
           "stream_f32.cu", "stream_df64.cu", "stream_f64.cu", "apply_pf_f32.cu", "apply_pf_df64.cu",
           "apply_pf_f64.cu", "apply_v2_f32.cu", "apply_v4_f32.cu", "apply_v_df64.cu",
           "apply_batch_f32.cu", "apply_batch_df64.cu", "apply_vi_df64.cu", "apply_vi_f32.cu",
           "apply_pf_vi_df64.cu", "apply_pf_vi_f32.cu", "apply_cx_f32.cu", "apply_cx_df64.cu", "apply_cx_f64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc):
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _stale(srcs, out):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "hm.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    if not force and not _stale(srcs, LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + _cuda_lib_dir(nvcc)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
