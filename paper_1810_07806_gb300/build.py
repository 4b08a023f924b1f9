"""Build libwcns.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the shared library is linked
against the CUDA runtime.  Usage: python -m paper_1810_07806_gb300.build
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwcns.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr"]
# The FP32 sweep may use approximate division/sqrt and flush denormals; the
# FP64 units keep IEEE division and square root (always the case for double).
# No multiply-add contraction where FP32 arithmetic runs: the code writes
# every fused multiply-add it wants as fmaf, so each kernel instance (single
# grid, batched, any tile shape) rounds identically.
NO_CONTRACT = ["-fmad=false"]
FP32_FLAGS = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"] + NO_CONTRACT
EXTRA = {"sweep_fp32.cu": FP32_FLAGS, "sweep_fp32_cfg1.cu": FP32_FLAGS, "sweep_fp32_cfg2.cu": FP32_FLAGS,
         "sweep_batch_fp32.cu": FP32_FLAGS, "sweep_fp32_weights.cu": FP32_FLAGS,
         "sweep_fp32_weights_lin.cu": FP32_FLAGS, "sweep_fp32_weights_z.cu": FP32_FLAGS,
         "wcns_rk.cu": NO_CONTRACT, "wcns_batch.cu": NO_CONTRACT}
SOURCES = ["wcns_api.cu", "wcns_rk.cu", "sweep_fp64.cu", "sweep_fp32.cu", "sweep_fp32_cfg1.cu",
           "sweep_fp32_cfg2.cu", "wcns_noalloc.cu",
           "wcns_batch.cu", "sweep_batch_fp64.cu", "sweep_batch_fp32.cu", "wcns_serve.cu",
           "wcns_scalar.cu", "sweep_fp32_weights.cu", "sweep_fp32_weights_lin.cu", "sweep_fp32_weights_z.cu",
           "wcns_probe.cu"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _needs(src, obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + deps)


def build(force=False, verbose=False, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(CSRC, "sweep_fp32.cu"))   # included by the other configurations
    deps.append(os.path.join(CSRC, "sweep_fp32_weights.cu"))   # included by the other weights
    deps.append(os.path.join(HERE, "..", "include", "wcns.h"))
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        if force or _needs(src, obj, deps):
            cmd = [nvcc()] + ARCH + COMMON + EXTRA.get(s, []) + (["-Xptxas", "-v"] if ptxas_info else []) \
                + ["-c", src, "-o", obj]
            jobs.append((s, cmd))
    def run(job):
        name, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
        return name, r.stderr
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for name, err in ex.map(run, jobs):
            if verbose or ptxas_info:
                print("== %s\n%s" % (name, err))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
